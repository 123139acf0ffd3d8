"""Continuous-batching serving loop for forward-model + likelihood requests.

Concurrent retrievals (samplers) submit requests: a batch of parameter
vectors for one of the resident setups.  The server keeps tables, setups and
per-slot buffers on the device and runs an event loop:

* memory: the server works inside a device-memory budget that counts
  everything it relies on: the context's own allocations as hr2_ctx_memory
  reports them (opacity tables, setups with their level-gridded operands,
  the per-stream workspaces it reserves) plus its own slot buffers and
  captured-graph buffers.  All of it is allocated when the server is built;
  the serving path allocates nothing.  A budget that cannot hold the slots
  is an error at construction.
* admission: a request is admitted, in arrival order (the head of the queue
  is never overtaken), when the device bytes it occupies while in flight
  (its samples' share of the reserved workspace and slot buffers, measured
  from the context's accounting) fit the reserved pool next to the requests
  already admitted or running;
* overload: a request that would take the queue (pending and admitted
  samples) beyond queue_limit is rejected at once, so that overload sheds
  work instead of growing the queue without bound;
* batching: whenever a slot (a CUDA stream with pinned staging buffers, its
  workspace and CUDA graphs captured for batch buckets) is free, the admitted
  requests waiting at that moment are packed, in arrival order, into one
  mixed-setup batch of at most max_batch samples; the smallest captured
  bucket that holds it is replayed (prep, plan, forward, bins, lnL), padding
  samples carrying setup -1, between an asynchronous host-to-device copy of
  the inputs and a device-to-host copy of lnL, then an event;
* completion: finished slots are polled; each request gets its lnL and its
  latency (arrival to lnL on the host) and its bytes are released; a
  request's callback runs then, and an exception it raises is recorded on
  that request only.  A request still pending or admitted can be cancelled.

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

DONE, REJECTED, CANCELLED, FAILED = "done", "rejected", "cancelled", "failed"


@dataclasses.dataclass
class Request:
    rid: int
    stream: int
    setup: int                 # index into the server's setups
    params: np.ndarray         # [n, HR2_NPARAM] float64
    t_arrival: float = 0.0
    t_done: float = 0.0
    lnl: Optional[np.ndarray] = None
    callback: Optional[Callable[["Request"], None]] = None
    status: str = ""
    error: Optional[BaseException] = None

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


def over_queue_limit(queued_samples: int, req_n: int, queue_limit: int) -> bool:
    """Whether admitting req_n more samples to the queue would exceed its bound."""
    return queued_samples + req_n > queue_limit


def cancel_from(queues: Sequence[Deque], rid: int) -> Optional[Request]:
    """Remove request rid from the first queue holding it; None if none does."""
    for q in queues:
        for r in q:
            if r.rid == rid:
                q.remove(r)
                return r
    return None


def bucket_sizes(max_batch: int, smallest: int = 64) -> List[int]:
    """Powers of two from `smallest` up, the last one max_batch itself."""
    out, n = [], smallest
    while n < max_batch:
        out.append(n)
        n *= 2
    out.append(max_batch)
    return out


def pick_bucket(sizes: Sequence[int], m: int) -> int:
    for n in sizes:
        if n >= m:
            return n
    raise ValueError("batch of %d exceeds the largest bucket %d" % (m, sizes[-1]))


class _Slot:
    """One CUDA stream with pinned staging buffers and, per bucket size, static device buffers
    and the captured graph of forward + likelihood for that size (or eager launches)."""

    def __init__(self, ctx, setups, device, sizes: Sequence[int], n_bins_max: int, n_nu_max: int,
                 graphs: bool):
        import torch
        self.ctx = ctx
        self.setups = list(setups)
        self.stream = torch.cuda.Stream(device=device)
        mb = sizes[-1]
        self.h_params = torch.empty((mb, hr2.HR2_NPARAM), dtype=torch.float64).pin_memory()
        self.h_sid = torch.full((mb,), -1, dtype=torch.int32).pin_memory()
        self.h_lnl = torch.empty(mb, dtype=torch.float64).pin_memory()
        hr2.hr2_reserve(ctx, mb, n_nu_max, self.stream)
        self.bufs: Dict[int, tuple] = {}
        self.graphs: Dict[int, object] = {}
        self.device_bytes = 0
        for n in sizes:
            b = (torch.zeros((n, hr2.HR2_NPARAM), dtype=torch.float64, device=device),
                 torch.full((n,), -1, dtype=torch.int32, device=device),
                 torch.zeros((n, n_bins_max), dtype=torch.float32, device=device),
                 torch.zeros(n, dtype=torch.float64, device=device))
            self.bufs[n] = b
            self.device_bytes += sum(t.numel() * t.element_size() for t in b)
        if graphs:
            with torch.cuda.stream(self.stream):
                for n in sizes:                # loads the kernels; the workspace is already sized
                    self._launch(n)
            self.stream.synchronize()
            for n in sizes:
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=self.stream):
                    self._launch(n)
                self.graphs[n] = g
            self.stream.synchronize()
        self.event = torch.cuda.Event()
        self.busy: List[tuple] = []     # (request, offset)
        self.n = 0

    def _launch(self, n: int):
        par, sid, bins, lnl = self.bufs[n]
        hr2.forward_model_batch(self.ctx, self.setups, sid, par, bins, None, None, self.stream)
        hr2.log_likelihood_batch(self.ctx, self.setups, sid, bins, lnl, None, self.stream)

    def run(self, n: int, m: int) -> None:
        """Copy m staged samples (the rest of bucket n padded with setup -1), evaluate the bucket,
        copy lnL back and record the slot's event, all asynchronously on the slot's stream."""
        import torch
        par, sid, bins, lnl = self.bufs[n]
        with torch.cuda.stream(self.stream):
            par[:m].copy_(self.h_params[:m], non_blocking=True)
            sid.copy_(self.h_sid[:n], non_blocking=True)
            if n in self.graphs:
                self.graphs[n].replay()
            else:
                self._launch(n)
            self.h_lnl[:m].copy_(lnl[:m], non_blocking=True)
            self.event.record(self.stream)


class Server:
    """Continuous-batching server over one context's resident setups.

    setups:        handles, indexed by Request.setup
    setup_shapes:  per setup (n_bins, n_nu, n_levels)
    mem_budget:    device bytes for everything the server relies on: the context's allocations
                   (hr2_ctx_memory: tables, setups, workspaces) plus the server's buffers
    queue_limit:   most samples that may wait (pending + admitted); default 2 x slots x max_batch
    graphs:        replay captured CUDA graphs (True) or launch eagerly
    """

    def __init__(self, ctx, setups: Sequence, setup_shapes: Sequence[tuple], device: int = 0, slots: int = 2,
                 max_batch: int = 1024, mem_budget: int = 8 << 30, queue_limit: Optional[int] = None,
                 graphs: bool = True, clock: Callable[[], float] = time.perf_counter):
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
        self.sizes = bucket_sizes(self.max_batch)
        used0 = hr2.hr2_ctx_memory(ctx)[0]
        self.slots: List[_Slot] = []
        for _ in range(slots):
            sl = _Slot(ctx, self.setups, dev, self.sizes, nb, nn, graphs)
            self.slots.append(sl)
        ctx_used = hr2.hr2_ctx_memory(ctx)[0]
        own = sum(sl.device_bytes for sl in self.slots)
        #: device bytes the server relies on: the context's (tables, setups, workspaces) and its own
        self.device_bytes = ctx_used + own
        if self.device_bytes > self.mem_budget:
            raise ValueError("the server needs %d device bytes (context %d, slot buffers %d), more than the "
                             "budget %d" % (self.device_bytes, ctx_used, own, self.mem_budget))
        # the in-flight pool: what the slots reserved for their samples (workspaces and buffers),
        # per sample of batch capacity
        pool = (ctx_used - used0) + own
        self.bytes_per_sample = max(1, pool // (slots * self.max_batch))
        self.pool_bytes = self.bytes_per_sample * slots * self.max_batch
        self.queue_limit = int(queue_limit) if queue_limit is not None else 2 * slots * self.max_batch
        self.pending: Deque[Request] = collections.deque()
        self.admitted: Deque[Request] = collections.deque()
        self.mem_in_use = 0
        self.done: List[Request] = []
        self.rejected: List[Request] = []
        self.cancelled: List[Request] = []
        self.batches = 0
        self.samples = 0

    def reset(self) -> None:
        """Forget finished, rejected and cancelled requests and the batch counters (the server must
        be idle); the slots, graphs and reserved memory stay."""
        if not self.idle():
            raise RuntimeError("reset of a busy server")
        self.mem_in_use = 0
        self.done, self.rejected, self.cancelled = [], [], []
        self.batches = 0
        self.samples = 0

    # ------------------------------------------------------------ accounting
    def footprint(self, req: Request) -> int:
        """Device bytes a request occupies while admitted or running: its samples' share of the
        reserved pool (workspace records, F+ scratch and slot buffers)."""
        return req.n * self.bytes_per_sample

    def queued_samples(self) -> int:
        return sum(r.n for r in self.pending) + sum(r.n for r in self.admitted)

    def submit(self, req: Request) -> bool:
        """Queue a request; returns False (and marks it rejected) when the queue is full."""
        if req.n > self.max_batch:
            raise ValueError("request of %d samples exceeds max_batch %d" % (req.n, self.max_batch))
        if over_queue_limit(self.queued_samples(), req.n, self.queue_limit):
            req.status = REJECTED
            req.t_done = self.clock()
            self.rejected.append(req)
            return False
        self.pending.append(req)
        return True

    def cancel(self, rid: int) -> bool:
        """Withdraw a request that has not been launched; its bytes are released."""
        r = cancel_from([self.pending], rid)
        if r is None:
            r = cancel_from([self.admitted], rid)
            if r is not None:
                self.mem_in_use -= self.footprint(r)
        if r is None:
            return False
        r.status = CANCELLED
        r.t_done = self.clock()
        self.cancelled.append(r)
        return True

    def _admit(self) -> None:
        self.mem_in_use = admit(self.pending, self.admitted, self.mem_in_use, self.pool_bytes, self.footprint)

    # ------------------------------------------------------------ event loop
    def _poll(self) -> int:
        finished: List[Request] = []
        for sl in self.slots:
            if sl.busy and sl.event.query():
                now = self.clock()
                lnl = sl.h_lnl.numpy()
                for req, off in sl.busy:
                    req.lnl = lnl[off:off + req.n].copy()
                    req.t_done = now
                    req.status = DONE
                    self.mem_in_use -= self.footprint(req)
                    self.done.append(req)
                    finished.append(req)
                sl.busy = []
        self._callbacks(finished)
        return len(finished)

    def _callbacks(self, reqs: Sequence[Request]) -> None:
        for req in reqs:
            if req.callback is None:
                continue
            try:
                req.callback(req)
            except Exception as e:          # a failing consumer affects its own request only
                req.error = e
                req.status = FAILED

    def _launch(self, sl: _Slot) -> bool:
        batch = pack(self.admitted, self.max_batch)
        if not batch:
            return False
        m = batch[-1][1] + batch[-1][0].n
        n = pick_bucket(self.sizes, m)
        hp = sl.h_params.numpy()
        hs = sl.h_sid.numpy()
        for r, off in batch:
            hp[off:off + r.n] = r.params
            hs[off:off + r.n] = r.setup
        hs[m:n] = -1
        sl.run(n, m)
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
    """Feed the streams' Poisson arrivals for `duration` seconds, then drain; returns statistics
    (latency over the served requests; rejected requests counted separately)."""
    t0 = server.clock()
    rid = 0
    by_stream = {s.sid: s for s in streams}
    offered = 0
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
                offered += req.n
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
            "offered_samples": offered,
            "rejected_requests": len(server.rejected), "rejected_samples": sum(r.n for r in server.rejected),
            "p50_ms": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
            "max_ms": float(lat.max() * 1e3) if len(lat) else None,
            "batches": server.batches, "mean_batch": server.samples / max(server.batches, 1),
            "slots": len(server.slots), "max_batch": server.max_batch, "graphs": bool(server.slots[0].graphs),
            "queue_limit_samples": server.queue_limit, "device_bytes": server.device_bytes}
