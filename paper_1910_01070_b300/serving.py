"""Continuous-batching serving loop for forward-model + likelihood requests.

Concurrent retrievals (samplers) submit requests: a batch of parameter
vectors for one of the resident setups.  The server keeps tables, setups and
per-slot buffers on the device and runs an event loop:

* admission: a request is admitted when its device footprint fits the memory
  budget next to the requests already admitted (FIFO, no overtaking);
* batching: whenever a slot (a CUDA stream with its own pinned staging
  buffers and workspace) is free, the admitted requests waiting at that moment
  are packed, in arrival order, into one mixed-setup batch of at most
  max_batch samples and launched: host-to-device copy, forward_model_batch,
  log_likelihood_batch, device-to-host copy of lnL, all asynchronous on the
  slot's stream, followed by an event;
* completion: finished slots are polled; each request gets its lnL and its
  latency (arrival to lnL on the host), and its memory is released.

Requests that arrive while other batches are on the GPU join the next batch
as soon as a slot and memory free up, and batches on different slots overlap
on the device.  A sample's result does not depend on the batch it lands in
(the kernels compute each sample independently).
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable, Deque, Dict, List, Optional, Sequence

import numpy as np

from . import hr2


@dataclasses.dataclass
class Request:
    rid: int
    stream: int
    setup: int                 # index into the server's setups
    params: np.ndarray         # [n, HR2_NPARAM] float64
    t_arrival: float = 0.0
    t_done: float = 0.0
    lnl: Optional[np.ndarray] = None

    @property
    def n(self) -> int:
        return int(self.params.shape[0])

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


def admit(pending: Deque, admitted: Deque, mem_in_use: int, budget: int, footprint: Callable) -> int:
    """Move requests from pending to admitted in arrival order while their footprints fit the budget
    (the head of the queue is never overtaken).  Returns the new memory in use."""
    while pending and mem_in_use + footprint(pending[0]) <= budget:
        r = pending.popleft()
        mem_in_use += footprint(r)
        admitted.append(r)
    return mem_in_use


def pack(admitted: Deque, max_batch: int) -> List[tuple]:
    """Take whole admitted requests, in order, while they fit max_batch samples: [(request, offset)]."""
    batch, m = [], 0
    while admitted and m + admitted[0].n <= max_batch:
        r = admitted.popleft()
        batch.append((r, m))
        m += r.n
    return batch


class _Slot:
    def __init__(self, device, max_batch: int, n_bins_max: int):
        import torch
        self.stream = torch.cuda.Stream(device=device)
        self.h_params = torch.empty((max_batch, hr2.HR2_NPARAM), dtype=torch.float64).pin_memory()
        self.h_sid = torch.empty(max_batch, dtype=torch.int32).pin_memory()
        self.h_lnl = torch.empty(max_batch, dtype=torch.float64).pin_memory()
        self.d_params = torch.empty((max_batch, hr2.HR2_NPARAM), dtype=torch.float64, device=device)
        self.d_sid = torch.empty(max_batch, dtype=torch.int32, device=device)
        self.d_bins = torch.empty((max_batch, n_bins_max), dtype=torch.float32, device=device)
        self.d_lnl = torch.empty(max_batch, dtype=torch.float64, device=device)
        self.event = torch.cuda.Event()
        self.busy: List[tuple] = []     # (request, offset)
        self.n = 0


class Server:
    """Continuous-batching server over one context's resident setups.

    setups:        handles, indexed by Request.setup
    setup_shapes:  per setup (n_bins, n_nu, n_levels) for the footprint
    mem_budget:    bytes of device memory that admitted requests may occupy
    """

    def __init__(self, ctx, setups: Sequence, setup_shapes: Sequence[tuple], device: int = 0, slots: int = 3,
                 max_batch: int = 2048, mem_budget: int = 1 << 30, clock: Callable[[], float] = time.perf_counter):
        import torch
        self.ctx = ctx
        self.setups = list(setups)
        self.shapes = list(setup_shapes)
        self.max_batch = int(max_batch)
        self.mem_budget = int(mem_budget)
        self.clock = clock
        dev = torch.device("cuda", device)
        nb = max(s[0] for s in self.shapes)
        nn = max(s[1] for s in self.shapes)
        self.nb = nb
        self.slots = [_Slot(dev, self.max_batch, nb) for _ in range(slots)]
        for sl in self.slots:          # size every slot's library workspace up front
            hr2.hr2_reserve(ctx, self.max_batch, nn, sl.stream)
        self.pending: Deque[Request] = collections.deque()
        self.admitted: Deque[Request] = collections.deque()
        self.mem_in_use = 0
        self.done: List[Request] = []
        self.batches = 0
        self.samples = 0

    # ------------------------------------------------------------ accounting
    def footprint(self, req: Request) -> int:
        """Device bytes a request occupies while admitted: its inputs, bins, lnL, and its share of
        the per-sample records and F+ scratch of the workspace."""
        nb, nn, nl = self.shapes[req.setup]
        per_sample = hr2.HR2_NPARAM * 8 + 4 + nb * 4 + 8 + nl * 64 + nn * 4 + 160
        return req.n * per_sample

    def submit(self, req: Request) -> None:
        if req.n > self.max_batch:
            raise ValueError("request of %d samples exceeds max_batch %d" % (req.n, self.max_batch))
        if self.footprint(req) > self.mem_budget:
            raise ValueError("request needs %d bytes, more than the whole budget" % self.footprint(req))
        self.pending.append(req)

    def _admit(self) -> None:
        self.mem_in_use = admit(self.pending, self.admitted, self.mem_in_use, self.mem_budget, self.footprint)

    # ------------------------------------------------------------ event loop
    def _poll(self) -> int:
        finished = 0
        for sl in self.slots:
            if sl.busy and sl.event.query():
                now = self.clock()
                lnl = sl.h_lnl.numpy()
                for req, off in sl.busy:
                    req.lnl = lnl[off:off + req.n].copy()
                    req.t_done = now
                    self.mem_in_use -= self.footprint(req)
                    self.done.append(req)
                    finished += 1
                sl.busy = []
        return finished

    def _launch(self, sl: _Slot) -> bool:
        batch = pack(self.admitted, self.max_batch)
        if not batch:
            return False
        m = batch[-1][1] + batch[-1][0].n
        hp = sl.h_params.numpy()
        hs = sl.h_sid.numpy()
        for r, off in batch:
            hp[off:off + r.n] = r.params
            hs[off:off + r.n] = r.setup
        import torch
        with torch.cuda.stream(sl.stream):
            sl.d_params[:m].copy_(sl.h_params[:m], non_blocking=True)
            sl.d_sid[:m].copy_(sl.h_sid[:m], non_blocking=True)
            hr2.forward_model_batch(self.ctx, self.setups, sl.d_sid[:m], sl.d_params[:m], sl.d_bins[:m], None, None,
                                    sl.stream)
            hr2.log_likelihood_batch(self.ctx, self.setups, sl.d_sid[:m], sl.d_bins[:m], sl.d_lnl[:m], None,
                                     sl.stream)
            sl.h_lnl[:m].copy_(sl.d_lnl[:m], non_blocking=True)
            sl.event.record(sl.stream)
        sl.busy = batch
        sl.n = m
        self.batches += 1
        self.samples += m
        return True

    def step(self) -> int:
        """One pass of the loop: collect finished slots, admit, launch on free slots."""
        finished = self._poll()
        self._admit()
        for sl in self.slots:
            if not sl.busy and self.admitted:
                self._launch(sl)
        return finished

    def idle(self) -> bool:
        return not self.pending and not self.admitted and all(not sl.busy for sl in self.slots)

    def drain(self) -> None:
        while not self.idle():
            self.step()


# ---------------------------------------------------------------- workload
@dataclasses.dataclass
class RetrievalStream:
    """A seeded nested-sampling-like client: batches of 32-512 parameter vectors drawn from a box
    that contracts around the best sample returned so far, issued at Poisson arrival times."""
    sid: int
    setup: int
    lo: np.ndarray
    hi: np.ndarray
    rate: float                 # requests per second
    seed: int
    shrink: float = 0.97

    def __post_init__(self):
        self.rng = np.random.default_rng([self.seed, 7])
        self.center = 0.5 * (self.lo + self.hi)
        self.width = self.hi - self.lo
        self.best = -np.inf
        self.next_t = self.rng.exponential(1.0 / self.rate)

    def make_request(self, rid: int, template: np.ndarray) -> Request:
        n = int(self.rng.integers(32, 513))
        lo = np.maximum(self.lo, self.center - 0.5 * self.width)
        hi = np.minimum(self.hi, self.center + 0.5 * self.width)
        th = np.repeat(template[None, :], n, axis=0)
        free = self.hi > self.lo
        th[:, free] = self.rng.uniform(lo[free], hi[free], (n, int(free.sum())))
        self.next_t += self.rng.exponential(1.0 / self.rate)
        return Request(rid=rid, stream=self.sid, setup=self.setup, params=th)

    def feedback(self, req: Request) -> None:
        i = int(np.argmax(req.lnl))
        if req.lnl[i] > self.best:
            self.best = float(req.lnl[i])
            self.center = req.params[i].copy()
        self.width = self.width * self.shrink


def run_open_loop(server: Server, streams: Sequence[RetrievalStream], templates: Sequence[np.ndarray],
                  duration: float) -> Dict:
    """Feed the streams' Poisson arrivals for `duration` seconds, then drain; returns statistics."""
    t0 = server.clock()
    rid = 0
    by_stream = {s.sid: s for s in streams}
    while True:
        now = server.clock() - t0
        if now >= duration:
            break
        for s in streams:
            while s.next_t <= now:
                t_arr = t0 + s.next_t
                req = s.make_request(rid, templates[s.sid])
                req.t_arrival = t_arr
                rid += 1
                server.submit(req)
        n_before = len(server.done)
        server.step()
        for req in server.done[n_before:]:
            by_stream[req.stream].feedback(req)
    server.drain()
    t_end = server.clock()
    lat = np.array([r.latency for r in server.done])
    n_samples = sum(r.n for r in server.done)
    return {"requests": len(server.done), "samples": n_samples, "seconds": t_end - t0,
            "throughput_models_per_s": n_samples / (t_end - t0),
            "p50_ms": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
            "batches": server.batches, "mean_batch": server.samples / max(server.batches, 1)}
