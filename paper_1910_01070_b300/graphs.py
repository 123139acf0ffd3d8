"""CUDA-graph-captured evaluation of fixed-size batches.

A captured batch owns static device buffers for one batch size (a "bucket"):
parameters, setup indices, model bins and lnL.  The forward model and the
likelihood (prep, planner, persistent forward kernel, conv+binning, lnL) are
captured once into a CUDA graph on a private stream; each evaluation copies
its inputs into the static buffers and replays the graph, removing the
per-launch CPU cost that dominates small serving batches.  Batches smaller
than the bucket are padded with samples whose setup index is -1: the planner
drops them, so padding costs no forward work (their lnL is -inf).

The library's workspace for the capture stream is reserved before capture
(hr2_reserve), so nothing is allocated while capturing.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence

import numpy as np

from . import hr2


class CapturedBatch:
    def __init__(self, ctx, setups: Sequence, n: int, n_bins_max: int, n_nu_max: int, device: int = 0,
                 warmup: int = 2):
        import torch
        self.ctx = ctx
        self.setups = list(setups)
        self.n = int(n)
        self.nb = int(n_bins_max)
        dev = torch.device("cuda", device)
        self.stream = torch.cuda.Stream(device=dev)
        self.params = torch.zeros((self.n, hr2.HR2_NPARAM), dtype=torch.float64, device=dev)
        self.sid = torch.full((self.n,), -1, dtype=torch.int32, device=dev)
        self.bins = torch.zeros((self.n, self.nb), dtype=torch.float32, device=dev)
        self.lnl = torch.zeros(self.n, dtype=torch.float64, device=dev)
        hr2.hr2_reserve(ctx, self.n, n_nu_max, self.stream)
        with torch.cuda.stream(self.stream):
            for _ in range(warmup):          # loads the kernels, sizes everything
                self._launch()
        self.stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self._launch()
        self.stream.synchronize()

    def _launch(self):
        hr2.forward_model_batch(self.ctx, self.setups, self.sid, self.params, self.bins, None, None, self.stream)
        hr2.log_likelihood_batch(self.ctx, self.setups, self.sid, self.bins, self.lnl, None, self.stream)

    def run(self, params, setup_of_sample, sync: bool = True):
        """Evaluate up to n samples: params [m, HR2_NPARAM], setup_of_sample [m] (torch tensors, any device,
        or numpy).  Returns (lnL [m], bins [m, n_bins_max]) views of the static buffers."""
        import torch
        m = int(params.shape[0])
        if m > self.n:
            raise ValueError("batch of %d exceeds the captured bucket %d" % (m, self.n))
        p = torch.as_tensor(params)
        s = torch.as_tensor(setup_of_sample)
        with torch.cuda.stream(self.stream):
            self.params[:m].copy_(p, non_blocking=True)
            self.sid[:m].copy_(s, non_blocking=True)
            if m < self.n:
                self.sid[m:].fill_(-1)
            self.graph.replay()
        if sync:
            self.stream.synchronize()
        return self.lnl[:m], self.bins[:m]


class GraphPool:
    """Captured batches for power-of-two buckets between min_n and max_n."""

    def __init__(self, ctx, setups: Sequence, n_bins_max: int, n_nu_max: int, min_n: int = 32, max_n: int = 2048,
                 device: int = 0):
        self.buckets: Dict[int, CapturedBatch] = {}
        n = min_n
        while n <= max_n:
            self.buckets[n] = CapturedBatch(ctx, setups, n, n_bins_max, n_nu_max, device)
            n *= 2
        self.sizes = sorted(self.buckets)

    def bucket_for(self, m: int) -> CapturedBatch:
        for n in self.sizes:
            if n >= m:
                return self.buckets[n]
        raise ValueError("batch of %d exceeds the largest bucket %d" % (m, self.sizes[-1]))

    def run(self, params, setup_of_sample, sync: bool = True):
        return self.bucket_for(int(params.shape[0])).run(params, setup_of_sample, sync)
