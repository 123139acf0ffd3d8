"""Minimal nested-sampling driver over the batch API (Sect. 3.2).

The paper couples MultiNest to its forward model.  This driver keeps what
touches the GPU and replaces MultiNest's ellipsoidal proposals by the
simplest valid stand-in:

* N live points are drawn from the prior (a box; parameters with lo == hi
  are fixed) and scored with forward_model_batch + log_likelihood_batch;
* each round draws a batch of candidates uniformly from the bounding box of
  the live points, widened by ``enlarge`` x its span on each side and clipped
  to the prior, scores them in one batch, and hands them to hr2_ns_absorb,
  which replaces the lowest live point by every candidate that beats it, in
  order, and accumulates ln Z and the information H in FP64 on the device
  (X_i = exp(-i/N));
* the run stops when the live points can add at most ``dlogz`` to ln Z
  (ln(Z + L_max X) - ln Z < dlogz); hr2_ns_finalize adds them.

A candidate drawn from a box that held the whole constrained region
{L > L*} stays a uniform draw from every later, smaller region, so one
batch serves many replacements.  With a GPU backend the box and the
candidates are made on the device (hr2_ns_propose, SplitMix64 deviates), so
per round the host reads only the small state struct; a backend without
that call gets the live points and draws the candidates on the host.
"""
from __future__ import annotations

import math
import time
from typing import Dict, Optional

import numpy as np

from . import hr2


class GpuBackend:
    """Live set, dead points and evidence state on one GPU; likelihoods from the library."""

    def __init__(self, ctx, setups, setup_index: int = 0, n_live: int = 400, dead_cap: Optional[int] = None,
                 device: int = 0, stream=None):
        import torch
        self.torch = torch
        self.ctx = ctx
        self.setups = list(setups)
        self.g = int(setup_index)
        self.n_live = int(n_live)
        self.dev = torch.device("cuda", device)
        self.stream = stream
        cap = int(dead_cap or 200 * n_live)
        f = dict(dtype=torch.float64, device=self.dev)
        self.live_lnl = torch.empty(n_live, **f)
        self.live_theta = torch.empty((n_live, hr2.HR2_NPARAM), **f)
        self.dead_lnl = torch.empty(cap, **f)
        self.dead_logw = torch.empty(cap, **f)
        self.dead_theta = torch.empty((cap, hr2.HR2_NPARAM), **f)
        self.state = torch.empty(hr2.NS_STATE_DOUBLES, **f)
        self.out = torch.empty(2, **f)
        nb = max(hr2.hr2_setup_info(s)[0] for s in self.setups)
        self._nb = nb
        self._bins = None
        hr2.hr2_ns_state_init(ctx, self.state, stream)

    def _score(self, theta_dev):
        torch = self.torch
        m = theta_dev.shape[0]
        if self._bins is None or self._bins.shape[0] < m:
            self._bins = torch.empty((m, self._nb), dtype=torch.float32, device=self.dev)
            self._lnl = torch.empty(m, dtype=torch.float64, device=self.dev)
            self._sid = torch.full((m,), self.g, dtype=torch.int32, device=self.dev)
        bins, lnl, sid = self._bins[:m], self._lnl[:m], self._sid[:m]
        hr2.forward_model_batch(self.ctx, self.setups, sid, theta_dev, bins, None, None, self.stream)
        hr2.log_likelihood_batch(self.ctx, self.setups, sid, bins, lnl, None, self.stream)
        return lnl

    def init_live(self, theta: np.ndarray) -> None:
        with self._on_stream():
            th = self.torch.as_tensor(theta, device=self.dev)
            self.live_theta.copy_(th)
            self.live_lnl.copy_(self._score(self.live_theta))

    def live_theta_host(self) -> np.ndarray:
        return self._read(lambda t: t.cpu().numpy(), self.live_theta)

    def _on_stream(self):
        """Copies made by torch go to the backend's stream (or the current one)."""
        torch = self.torch
        s = self.stream
        if s is None:
            s = torch.cuda.current_stream(self.dev)
        elif isinstance(s, int):
            s = torch.cuda.ExternalStream(s, device=self.dev)
        return torch.cuda.stream(s)

    def _read(self, fn, *args):
        """fn(*args) reading device results, after the backend's stream is done."""
        with self._on_stream():
            return fn(*args)

    def step(self, cand: np.ndarray) -> Dict:
        with self._on_stream():
            th = self.torch.as_tensor(np.ascontiguousarray(cand), device=self.dev)
        lnl = self._score(th)
        hr2.hr2_ns_absorb(self.ctx, self.live_lnl, self.live_theta, lnl, th, self.state, self.dead_lnl,
                          self.dead_logw, self.dead_theta, self.stream)
        return self._read(hr2.ns_state_read, self.state)

    def step_device(self, n: int, lo: np.ndarray, hi: np.ndarray, enlarge: float, seed: int, counter: int) -> Dict:
        """One round with the candidates drawn on the device (hr2_ns_propose):
        no host copy of the live set or of the candidates."""
        torch = self.torch
        with self._on_stream():
            if getattr(self, "_prior", None) is None or not (np.array_equal(self._prior[0], lo) and
                                                             np.array_equal(self._prior[1], hi)):
                self._prior = (np.array(lo, dtype=np.float64), np.array(hi, dtype=np.float64))
                self._prior_dev = (torch.as_tensor(self._prior[0], device=self.dev),
                                   torch.as_tensor(self._prior[1], device=self.dev))
                self._box = torch.empty((hr2.HR2_NPARAM, 2), dtype=torch.float64, device=self.dev)
            if getattr(self, "_cand", None) is None or self._cand.shape[0] != n:
                self._cand = torch.empty((n, hr2.HR2_NPARAM), dtype=torch.float64, device=self.dev)
        th = self._cand
        hr2.hr2_ns_propose(self.ctx, self.live_theta, self._prior_dev[0], self._prior_dev[1], enlarge, self._box, th,
                           seed, counter, self.stream)
        lnl = self._score(th)
        hr2.hr2_ns_absorb(self.ctx, self.live_lnl, self.live_theta, lnl, th, self.state, self.dead_lnl,
                          self.dead_logw, self.dead_theta, self.stream)
        return self._read(hr2.ns_state_read, self.state)

    def finalize(self):
        hr2.hr2_ns_finalize(self.ctx, self.live_lnl, self.state, self.out, self.stream)
        o = self._read(lambda t: t.cpu().numpy(), self.out)
        return float(o[0]), float(o[1])

    def dead(self, n: int):
        return self._read(lambda: (self.dead_lnl[:n].cpu().numpy(), self.dead_logw[:n].cpu().numpy(),
                                   self.dead_theta[:n].cpu().numpy()))


def log_add(a: float, b: float) -> float:
    if a == -math.inf:
        return b
    if b == -math.inf:
        return a
    m = max(a, b)
    return m + math.log(math.exp(a - m) + math.exp(b - m))


class NestedSampler:
    """lo, hi: prior box per parameter ([HR2_NPARAM] each; lo == hi fixes a parameter)."""

    def __init__(self, backend, lo, hi, batch: int = 1024, enlarge: float = 0.25, seed: int = 0,
                 device_proposals: bool = True):
        self.b = backend
        self.device_proposals = bool(device_proposals)
        self.lo = np.asarray(lo, dtype=np.float64)
        self.hi = np.asarray(hi, dtype=np.float64)
        self.free = self.hi > self.lo
        self.batch = int(batch)
        self.enlarge = float(enlarge)
        self.rng = np.random.default_rng([seed, 11])

    def _draw(self, n: int, lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
        th = np.repeat(self.lo[None, :], n, axis=0)
        f = self.free
        th[:, f] = self.rng.uniform(lo[f], hi[f], (n, int(f.sum())))
        return th

    def run(self, dlogz: float = 0.5, max_rounds: int = 1000) -> Dict:
        t0 = time.perf_counter()
        n_live = self.b.n_live
        self.b.init_live(self._draw(n_live, self.lo, self.hi))
        n_evals = n_live
        st = None
        rounds = 0
        device = self.device_proposals and hasattr(self.b, "step_device")
        seed = int(self.rng.integers(0, 2 ** 63)) if device else 0
        for rounds in range(1, max_rounds + 1):
            if device:
                st = self.b.step_device(self.batch, self.lo, self.hi, self.enlarge, seed,
                                        (rounds - 1) * self.batch * len(self.lo))
            else:
                live = self.b.live_theta_host()
                span = live.max(axis=0) - live.min(axis=0)
                blo = np.maximum(self.lo, live.min(axis=0) - self.enlarge * span)
                bhi = np.minimum(self.hi, live.max(axis=0) + self.enlarge * span)
                st = self.b.step(self._draw(self.batch, blo, bhi))
            n_evals += self.batch
            if st["log_z"] > -math.inf and log_add(st["log_z"], st["lnl_max"] + st["log_x"]) - st["log_z"] < dlogz:
                break
        log_z, info = self.b.finalize()
        secs = time.perf_counter() - t0
        return {"log_z": log_z, "log_z_err": math.sqrt(max(info, 0.0) / n_live), "info": info,
                "n_dead": int(st["n_dead"]), "n_evals": n_evals, "rounds": rounds,
                "acceptance": st["n_dead"] / max(n_evals - n_live, 1), "seconds": secs,
                "evals_per_s": n_evals / secs}
