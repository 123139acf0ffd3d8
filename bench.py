#!/usr/bin/env python
"""Throughput benchmark of the Helios-r2 forward model + likelihood on B300.

One step = forward_model_batch + log_likelihood_batch over one batch of
synthetic parameter samples (FP16-offset tables, FP32 solve, FP64 lnL) on
the 1024-sample, 100-layer, 6-absorber, 8501-wavenumber workload (4 Gauss
nodes, R = 300, 300 bins).  Inputs are resident in HBM; L2 is flushed (a
256 MB write) between timed steps, outside the timed events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hr2|reference]

Under torchrun (N > 1) every rank runs the same per-GPU workload on its own
GPU with its own samples (weak scaling, no data-path collective); rank 0
prints one JSON line with the whole-job throughput over the slowest rank.
``--impl reference`` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
from typing import Optional

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "forward models/sec and HBM-roofline fraction at 1e-4 rel. flux error; p50/p99 latency"
WORKLOAD = "batch1024_l100_k6_nu8501"
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
PROFILE_TRAFFIC_UNEVEN = os.path.join(ROOT, "profiles", "traffic_uneven.json")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="hr2", choices=["hr2", "reference"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU comparison")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-samples", type=int, default=64)
    p.add_argument("--no-extras", action="store_true",
                   help="skip the uneven three-setup batch and the serving-loop measurements")
    p.add_argument("--uneven-only", action="store_true",
                   help="of the extra records, run only the uneven batch (counter captures of its launch)")
    p.add_argument("--serving-seconds", type=float, default=4.0)
    p.add_argument("--sweep-large", action="store_true",
                   help="instead of the main line: batch sweep on the 290001-point, 12-absorber tables")
    p.add_argument("--sweep-nu", type=int, default=290001, help="wavenumber points of the swept tables")
    p.add_argument("--sweep-modes", default="direct,cached,stream")
    p.add_argument("--sweep-batches", default="1,2,4,8,16,32,64,128,256")
    p.add_argument("--sweep-reps", type=int, default=0,
                   help="timed launches per sweep point (0: about 0.3 s worth, at least 3)")
    p.add_argument("--no-large", action="store_true",
                   help="skip the 290001-point, 12-absorber table measurements (batch 1 and 256)")
    p.add_argument("--peaks", action="store_true",
                   help="instead of the main line: microbenchmarks of the special-function unit (ex2, rcp) and "
                        "the FMA pipe, with the SM clock sampled during each")
    return p.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ helpers
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def method_work_per_model(setup, n_cia: int) -> dict:
    """Special-function and FP32 work the method needs per model (the algorithmic
    count, independent of how the kernel issues it).  Per wavenumber:
      ex2: one 10^x per absorber and per CIA pair present on every level, one
           Planck exponential per level, one transmission factor e^{-tau/mu} per
           layer and angle node: (L+1)(K + n_cia + 1) + L N_mu;
      rcp: one 1/dtau per layer (shared by the nodes) and one 1/(e^x - 1) per
           level: L + (L+1);
      fp32: per level 2 per absorber and CIA pair (the T interpolation and the
           abundance-weighted sum), 3 for the Planck function (x, e^x - 1 and the
           product), 5 for the layer (trapezoid, source difference, slope,
           cumulative tau), and 3 per angle node (exponent, difference of the
           transmissions, accumulation): (L+1)(2(K + n_cia) + 8) + 3 L N_mu."""
    L = setup.n_layers
    K = len(setup.species)
    nu = float(setup.n_nu)
    return {"ex2": nu * ((L + 1) * (K + n_cia + 1) + L * setup.n_mu),
            "rcp": nu * (L + (L + 1)),
            "fp32": nu * ((L + 1) * (2 * (K + n_cia) + 8) + 3 * L * setup.n_mu)}


def mufu_ops_per_model(setup, n_cia: int) -> float:
    """Exponentials the method needs per model (see method_work_per_model)."""
    return method_work_per_model(setup, n_cia)["ex2"]


def unit_peaks(rates: dict, n_sm: int) -> dict:
    """Peak rates at the maximum SM clock from the measured operations per SM clock:
    ex2 and rcp of the special-function unit and scalar FP32 FMA."""
    f = SM_MAX_MHZ * 1e6
    return {"ex2_per_s": rates["ex2"]["ops_per_clk_sm"] * n_sm * f,
            "rcp_per_s": rates["rcp"]["ops_per_clk_sm"] * n_sm * f,
            "fp32_per_s": rates["ffma"]["ops_per_clk_sm"] * n_sm * f,
            "ops_per_clk_sm": {k: rates[k]["ops_per_clk_sm"] for k in ("ex2", "rcp", "ex2_rcp", "ffma", "ffma2")},
            "ex2_rcp_share_one_unit": rates["ex2_rcp"].get("mix_over_shared_prediction"),
            "sm_mhz": SM_MAX_MHZ}


def roofline_of(work: dict, kernel_ms: float, peaks: dict, counters: Optional[dict]) -> dict:
    """The forward kernel against its roofs.  MUFU: the special-function time the method
    needs (ex2 / ex2 rate + rcp / rcp rate) over the kernel time, reported as
    ex2-equivalents per second (rcp weighted by the ratio of the rates).  FMA: the
    method's FP32 operations over the FMA rate.  DRAM and L2: the ncu counters of the
    same kernel source (committed under profiles/), else null.  binding = the largest."""
    t = kernel_ms / 1e3
    t_mufu = work["ex2"] / peaks["ex2_per_s"] + work["rcp"] / peaks["rcp_per_s"]
    ex2_eq = work["ex2"] + work["rcp"] * peaks["ex2_per_s"] / peaks["rcp_per_s"]
    fr = {"mufu": t_mufu / t, "fma": work["fp32"] / peaks["fp32_per_s"] / t}
    hbm_peak, hbm_src = _hbm_peak()
    if counters:
        fr["dram"] = counters["dram_bytes"] / t / 1e9 / hbm_peak
        if counters.get("l2_frac") is not None:
            fr["l2"] = counters["l2_frac"] * counters.get("kernel_ms_ncu", kernel_ms) / kernel_ms
    return {"bound": "alu", "achieved": ex2_eq / t / 1e12, "peak": peaks["ex2_per_s"] / 1e12,
            "unit": "Tex2-eq/s", "frac": fr["mufu"],
            "binding": max(fr.values()), "binding_unit": max(fr, key=fr.get), "fractions": fr,
            "work_per_launch": work, "peak_source": "hr2_measure_unit_rate in this run (ops per SM clock) x SMs "
                                                     "x %d MHz" % SM_MAX_MHZ}


def cpu_baseline(wl, n_samples: int):
    """The FP64 oracle, as it stands, on the host cores over a bounded sample."""
    import oracle
    from paper_1910_01070_b300 import workloads as W
    oracle.build()
    tabs = W.make_tables(wl.table)
    om = oracle.Model(tabs, wl.setups[0].as_dict())
    theta, _ = wl.params(n_samples, seed_offset=99)
    om.forward_batch(theta[:2], n_threads=0)          # warm-up (page-in)
    t0 = time.perf_counter()
    om.forward_batch(theta, n_threads=0)
    dt = time.perf_counter() - t0
    return {"value": n_samples / dt, "unit": "models/s", "cores": int(om.last_threads), "kind": "oracle",
            "sample": "%d samples of %s (full spectra + bins), FP64, OpenMP over samples, %.1f s wall"
                      % (n_samples, wl.name, dt)}


# ------------------------------------------------------------------ reference arm
def run_reference(args, world, rank):
    if rank != 0:
        return
    from paper_1910_01070_b300 import workloads as W
    import oracle
    wl = W.WORKLOADS[args.workload]()
    oracle.build()
    tabs = W.make_tables(wl.table)
    om = oracle.Model(tabs, wl.setups[0].as_dict())
    # one sample per host core per step: each step is about one model's worth
    # of CPU time, so --steps K ends within a few minutes for K of a few hundred
    per_step = max(1, os.cpu_count() or 1)
    times = []
    for k in range(args.warmup + args.steps):
        theta, _ = wl.params(per_step, seed_offset=1000 + k)
        t0 = time.perf_counter()
        om.forward_batch(theta, n_threads=0)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = per_step * len(times) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "models/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "samples_per_step": per_step,
                       "note": "each step a bounded sample of the workload's batch"},
            "cpu_baseline": {"value": value, "unit": "models/s", "cores": int(om.last_threads), "kind": "oracle",
                             "sample": "%d samples per step of %s" % (per_step, wl.name)},
            "e2e": {"value": value, "unit": "models/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ hr2 arm
def run_hr2(args, world, rank, local):
    import torch

    from paper_1910_01070_b300 import hr2
    from paper_1910_01070_b300 import workloads as W
    from paper_1910_01070_b300.build import build
    from paper_1910_01070_b300.engine import Engine

    build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = W.WORKLOADS[args.workload]()
    setup = wl.setups[0]
    n = wl.n_samples
    tabs = W.make_tables(wl.table)
    eng = Engine(local)
    t16 = eng.add_tables(wl.table, "fp16", tabs)
    s16 = eng.add_setup(t16, setup)
    stream = torch.cuda.current_stream()

    # mock observation: the model at a fixed "true" sample plus seeded noise
    truth = torch.as_tensor(wl.truth(0)[None, :], device=dev)
    sid1 = torch.zeros(1, dtype=torch.int32, device=dev)
    tb = eng.forward([s16], sid1, truth)
    D, sig = W.mock_observation(tb.double().cpu().numpy()[0], wl.seed)
    eng.set_observation(s16, D, sig)

    # a pool of distinct parameter batches resident in HBM (per-rank seeds)
    pool = []
    for p in range(4):
        th, sid = wl.params(n, seed_offset=17 * rank + p)
        pool.append((torch.as_tensor(th, device=dev), torch.as_tensor(sid, device=dev)))
    bins = torch.empty((n, setup.n_bins), dtype=torch.float32, device=dev)
    lnl = torch.empty(n, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(k, setups):
        th, sid = pool[k % len(pool)]
        hr2.forward_model_batch(eng.ctx, setups, sid, th, bins, None, None, stream)
        hr2.log_likelihood_batch(eng.ctx, setups, sid, bins, lnl, None, stream)

    def timed(setups, steps, warmup):
        for k in range(warmup):
            step(k, setups)
        torch.cuda.synchronize()
        hr2.hr2_profile_read(eng.ctx, True)
        hr2.hr2_profile_enable(eng.ctx, True)
        evs = []
        barrier(world)
        torch.cuda.synchronize()
        for k in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(k, setups)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        barrier(world)
        hr2.hr2_profile_enable(eng.ctx, False)
        kms, launches = hr2.hr2_profile_read(eng.ctx, True)
        times = [a.elapsed_time(b) for a, b in evs]
        return times, kms, launches

    # the special-function and FMA rates of this GPU, measured before the timed region
    props = torch.cuda.get_device_properties(local)
    rates = measure_unit_rates(local, clocks=False)
    peaks = unit_peaks(rates, props.multi_processor_count)

    clocks = ClockSampler(local)
    clocks.start()
    times, kms, launches = timed([s16], args.steps, args.warmup)
    clk = clocks.stop()
    total_ms = max_over_ranks(world, sum(times))
    ms_step = total_ms / args.steps
    value = world * n * args.steps / (total_ms / 1e3)
    lat = np.asarray(times)
    n_cia = int(wl.table.cia) * 2
    work = {k: v * n for k, v in method_work_per_model(setup, n_cia).items()}
    kernel_ms = kms / max(launches, 1)
    counters = committed_counters()
    roofline = roofline_of(work, kernel_ms, peaks, counters)
    roofline.update({"traffic": counters["dram_bytes"] if counters else None, "kernel": "k_forward32",
                     "kernel_ms": kernel_ms, "counters": counters["source"] if counters else None})
    hbm_peak, hbm_src = _hbm_peak()
    hbm = None
    if counters:
        gbs = counters["dram_bytes"] / (kernel_ms / 1e3) / 1e9
        hbm = {"achieved_gbs": gbs, "peak_gbs": hbm_peak, "frac": gbs / hbm_peak, "peak_source": hbm_src,
               "traffic_bytes_per_launch": counters["dram_bytes"]}

    # end to end through the host-buffer entry point (pinned buffers)
    h_par = [torch.as_tensor(p[0].cpu().numpy()).pin_memory() for p in pool]
    h_sid = [torch.as_tensor(p[1].cpu().numpy()).pin_memory() for p in pool]
    h_out = torch.empty(n, dtype=torch.float64).pin_memory()
    for k in range(2):
        hr2.hr2_evaluate_host(eng.ctx, [s16], h_sid[k % 4], h_par[k % 4], h_out, None, None, stream)
    e2e_t = []
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hr2.hr2_evaluate_host(eng.ctx, [s16], h_sid[k % 4], h_par[k % 4], h_out, None, None, stream)
        e2e_t.append(time.perf_counter() - t0)
    e2e_total = max_over_ranks(world, sum(e2e_t))
    # copied per step: parameters and setup indices in; lnL and the library's status word out
    e2e = {"value": world * n * args.steps / e2e_total, "unit": "models/s",
           "h2d_bytes_per_step": n * (8 * hr2.HR2_NPARAM + 4), "d2h_bytes_per_step": n * 8 + 8,
           "ms_per_step": 1e3 * e2e_total / args.steps, "api": "hr2_evaluate_host (pinned host buffers)"}

    graph = None
    if rank == 0 and world == 1 and not args.no_extras and not args.uneven_only:
        graph = graph_replay_timing(eng, [s16], pool, n, setup.n_bins, setup.n_nu, flush, local)

    fp64 = None
    if not args.no_fp64:
        t64 = eng.add_tables(wl.table, "fp64", tabs)
        s64 = eng.add_setup(t64, setup)
        eng.set_observation(s64, D, sig)
        k64 = min(args.steps, 5)
        t64s, kms64, l64 = timed([s64], k64, 3)
        tot64 = max_over_ranks(world, sum(t64s))
        fp64 = {"value": world * n * k64 / (tot64 / 1e3), "unit": "models/s", "steps": k64,
                "p50_ms": float(np.percentile(t64s, 50)), "p99_ms": float(np.percentile(t64s, 99)),
                "kernel_ms": kms64 / max(l64, 1), "tables": "fp64"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, args.cpu_samples)

    extras = None
    if rank == 0 and world == 1 and not args.no_extras:
        extras = run_extras(args, local, flush)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "models/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": wl.name, "samples_per_gpu": n, "layers": setup.n_layers,
                           "absorbers": len(setup.species), "wavenumbers": setup.n_nu, "gauss_nodes": setup.n_mu,
                           "bins": setup.n_bins, "resolving_power": setup.resolving_power,
                           "tables": "FP16 log10 sigma - integer offset per species",
                           "l2": "flushed between timed steps (256 MB write outside the events)",
                           "launch": list(hr2.hr2_get_launch_config(eng.ctx))},
                "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
                "fp64_path": fp64, "e2e": e2e, "roofline": roofline, "hbm": hbm,
                "effective_streaming": effective_streaming(setup, value),
                "cpu_baseline": cpu, "clocks": clk,
                "gpu_launches": 5 * args.steps}
        if graph:
            line["graph_replay"] = graph
        if extras:
            line.update(extras)
        if fp64:
            line["speedup_vs_fp64_path"] = value / fp64["value"]
        print(json.dumps(line), flush=True)
    eng.close()


def effective_streaming(setup, models_per_s: float) -> dict:
    """Models/s times the table bytes one model interpolates from, (L+1) levels x 4 corners
    x N_nu points x (K absorbers + 1/2 for the two CIA rows) x 2 bytes of FP16: the rate a
    design without on-chip reuse would have to stream; above the HBM peak by the reuse."""
    per_model = (setup.n_layers + 1) * 4 * setup.n_nu * (len(setup.species) + 0.5) * 2
    return {"gbs": models_per_s * per_model / 1e9, "bytes_per_model": per_model,
            "label": "effective streaming bandwidth (models/s x per-model algorithmic table bytes; "
                     "not DRAM traffic, which is in hbm)"}


def graph_replay_timing(eng, setups, pool, n, n_bins, n_nu, flush, local, reps=60):
    """The step (forward_model_batch + log_likelihood_batch) captured once as a CUDA graph
    and replayed: before each replay the next parameter batch of the pool is copied into the
    graph's static buffers and L2 is flushed, both on the capture stream and outside the
    events; each replay is event-timed on that stream.  Median and p99 over the replays."""
    import torch

    from paper_1910_01070_b300 import graphs
    cb = graphs.CapturedBatch(eng.ctx, setups, n, n_bins, n_nu, device=local)
    evs = []
    for k in range(3 + reps):
        th, sd = pool[k % len(pool)]
        with torch.cuda.stream(cb.stream):
            cb.params.copy_(th, non_blocking=True)
            cb.sid.copy_(sd, non_blocking=True)
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(cb.stream)
            cb.graph.replay()
            e1.record(cb.stream)
        if k >= 3:
            evs.append((e0, e1))
    cb.stream.synchronize()
    t = np.asarray([a.elapsed_time(b) for a, b in evs])
    med = float(np.percentile(t, 50))
    return {"replays": reps, "p50_ms": med, "p99_ms": float(np.percentile(t, 99)),
            "models_per_s_at_p50": n / (med / 1e3), "launches_per_replay": 5,
            "api": "graphs.CapturedBatch: the step captured once, replayed per batch"}


def _gpu_workload(wl, eng, dev, seed_offset=0):
    """Tables and setups of a workload on the engine with a mock observation per setup
    (the GPU model of the setup's true sample plus seeded noise)."""
    import torch
    from paper_1910_01070_b300 import workloads as W
    t = eng.add_tables(wl.table, "fp16", W.make_tables(wl.table))
    setups = [eng.add_setup(t, s) for s in wl.setups]
    for g, (h, s) in enumerate(zip(setups, wl.setups)):
        tb = eng.forward(setups, torch.full((1,), g, dtype=torch.int32, device=dev),
                         torch.as_tensor(wl.truth(g)[None, :], device=dev))
        D, sig = W.mock_observation(tb.double().cpu().numpy()[0, : s.n_bins], wl.seed + g)
        eng.set_observation(h, D, sig)
    return setups


def run_extras(args, local, flush):
    """The uneven three-setup batch (one persistent launch over 2048 samples of 12 setup
    variants, launch shape autotuned on the batch) and the continuous-batching serving
    loop on those setups."""
    import torch

    from paper_1910_01070_b300 import autotune, hr2, serving
    from paper_1910_01070_b300 import workloads as W
    from paper_1910_01070_b300.engine import Engine

    dev = torch.device("cuda", local)
    wl = W.uneven2048_3setups()
    out = {}
    with Engine(local) as eng:
        setups = _gpu_workload(wl, eng, dev)
        n = wl.n_samples
        nb = max(s.n_bins for s in wl.setups)
        pool = []
        for p in range(3):
            th, sid = wl.params(n, seed_offset=31 + p)
            pool.append((torch.as_tensor(th, device=dev), torch.as_tensor(sid, device=dev), sid))
        bins = torch.empty((n, nb), dtype=torch.float32, device=dev)
        lnl = torch.empty(n, dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream()
        for k in range(3):
            hr2.forward_model_batch(eng.ctx, setups, pool[k][1], pool[k][0], bins, None, None, stream)
        torch.cuda.synchronize()
        # the launch shape tuned on this batch (timed candidates, no cache)
        best, tried = autotune.tune(eng.ctx, setups, pool[0][1], pool[0][0], bins,
                                    [autotune.setup_info_from_spec(s) for s in wl.setups], use_cache=False)
        steps = max(3, min(args.steps, 40))
        evs = []
        hr2.hr2_profile_read(eng.ctx, True)
        hr2.hr2_profile_enable(eng.ctx, True)
        torch.cuda.nvtx.range_push("uneven_batch_timed")     # ncu filters on this range
        for k in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            th, sd, _ = pool[k % 3]
            e0.record(stream)
            hr2.forward_model_batch(eng.ctx, setups, sd, th, bins, None, None, stream)
            hr2.log_likelihood_batch(eng.ctx, setups, sd, bins, lnl, None, stream)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        hr2.hr2_profile_enable(eng.ctx, False)
        kms, nl = hr2.hr2_profile_read(eng.ctx, True)
        times = [a.elapsed_time(b) for a, b in evs]
        cap = n * steps / (sum(times) / 1e3)
        work = {"ex2": 0.0, "rcp": 0.0, "fp32": 0.0}
        for p in range(3):
            for g, s in enumerate(wl.setups):
                for k, v in method_work_per_model(s, 2).items():
                    work[k] += float(np.sum(pool[p][2] == g)) * v / 3
        props = torch.cuda.get_device_properties(local)
        peaks = unit_peaks(measure_unit_rates(local, clocks=False), props.multi_processor_count)
        ctr = committed_counters(PROFILE_TRAFFIC_UNEVEN)
        rl = roofline_of(work, kms / max(nl, 1), peaks, ctr)
        out["uneven_batch"] = {"workload": wl.name, "samples": n, "setups": len(wl.setups),
                               "value": cap, "unit": "models/s", "ms_per_step": float(np.mean(times)),
                               "p99_ms": float(np.percentile(times, 99)),
                               "kernel_ms": kms / max(nl, 1),
                               "mufu_frac": rl["fractions"]["mufu"], "fma_frac": rl["fractions"]["fma"],
                               "binding": rl["binding"], "binding_unit": rl["binding_unit"],
                               "fractions": rl["fractions"],
                               "traffic": ctr["dram_bytes"] if ctr else None,
                               "counters": ctr["source"] if ctr else None,
                               "launch": list(hr2.hr2_get_launch_config(eng.ctx)),
                               "autotuned": {"candidates": len(tried), "best": list(best),
                                             "shape": "(warps per CTA, CTAs per SM, 128-point tiles per item, "
                                                      "stages; 0 = by batch shape)",
                                             "tiles_per_item_tried": sorted({c[2] for c in tried}),
                                             "fastest_ms": min(tried.values()) if tried else None,
                                             "default_ms": tried.get(autotune.DEFAULT_SHAPE)}}
        if args.uneven_only:
            return out
        # serving: 16 nested-sampling-like streams over the 12 setups, Poisson arrivals
        shapes = [(s.n_bins, s.n_nu, s.n_layers + 1) for s in wl.setups]
        res = []
        servers = {}
        for load, graphs in ((0.5, True), (0.8, True), (1.2, True), (0.8, False)):
            if graphs not in servers:
                servers[graphs] = serving.Server(eng.ctx, setups, shapes, device=local, slots=2, max_batch=512,
                                                 mem_budget=32 << 30, graphs=graphs)
            srv = servers[graphs]
            srv.reset()
            streams, templates = [], []
            for k in range(16):
                g = k % len(wl.setups)
                t = wl.truth(g)
                lo, hi = t.copy(), t.copy()
                lo[0], hi[0] = 4.0, 5.5
                lo[1], hi[1] = 0.5, 2.0
                nt = wl.setups[g].n_tnodes
                lo[3:3 + nt], hi[3:3 + nt] = 0.7 * t[3:3 + nt], 1.3 * t[3:3 + nt]
                nsp = len(wl.setups[g].species)
                lo[19:19 + nsp], hi[19:19 + nsp] = -8.0, -2.0
                rate = load * cap / (16 * 272.0)
                streams.append(serving.RetrievalStream(k, g, lo, hi, rate=rate, seed=100 + k))
                templates.append(t)
            st = serving.run_open_loop(srv, streams, templates, duration=args.serving_seconds)
            st["offered_load"] = load
            st["offered_models_per_s"] = load * cap
            res.append(st)
        out["serving"] = {"streams": 16, "request_sizes": "32-512", "capacity_models_per_s": cap,
                          "latency": "arrival to lnL on the host (served requests; rejected ones counted)",
                          "loads": res}
    if not args.no_large:
        out["large_tables"] = large_table_sweep(local, modes=("direct", "cached", "stream"), batches=(1, 64, 256))
    out["linear_sigma_option"] = run_linear_option(args, local, flush)
    out["parabolic_source_option"] = run_linear_option(args, local, flush, sc="parabolic")
    out["nested_sampling"] = run_nested(args, local)
    return out


def run_nested(args, local):
    """A bounded nested-sampling run on the benchmark setup and its mock observation:
    the driver's loop (host proposals, forward + lnL batch, device-side absorb) timed
    end to end; likelihood evaluations per second is the figure."""
    import torch

    from paper_1910_01070_b300 import hr2
    from paper_1910_01070_b300 import workloads as W
    from paper_1910_01070_b300.engine import Engine
    from paper_1910_01070_b300.nested import GpuBackend, NestedSampler

    dev = torch.device("cuda", local)
    wl = W.WORKLOADS[args.workload]()
    spec = wl.setups[0]
    with Engine(local) as eng:
        t = eng.add_tables(wl.table, "fp16", W.make_tables(wl.table))
        s = eng.add_setup(t, spec)
        truth = wl.truth(0)
        tb = eng.forward([s], torch.zeros(1, dtype=torch.int32, device=dev), torch.as_tensor(truth[None, :], device=dev))
        D, sig = W.mock_observation(tb.double().cpu().numpy()[0, : spec.n_bins], wl.seed)
        eng.set_observation(s, D, sig)
        lo, hi = truth.copy(), truth.copy()
        lo[0], hi[0] = 4.0, 5.5
        lo[1], hi[1] = 0.5, 2.0
        nt = spec.n_tnodes
        lo[3:3 + nt], hi[3:3 + nt] = 300.0, 3000.0
        nsp = len(spec.species)
        lo[19:19 + nsp], hi[19:19 + nsp] = -8.0, -2.0
        n_live, batch = 1024, 4096
        be = GpuBackend(eng.ctx, [s], 0, n_live=n_live)
        res = NestedSampler(be, lo, hi, batch=batch, seed=1).run(dlogz=0.5, max_rounds=10)
        res.update({"workload": wl.name, "n_live": n_live, "batch": batch, "free_parameters": int(np.sum(hi > lo)),
                    "note": "bounded run (10 rounds): throughput of the sampling loop, not a converged evidence"})
        return res


def run_linear_option(args, local, flush, **option):
    """The benchmark workload with a setup option changed (the opacity tables
    interpolated in sigma instead of log10 sigma by default, or the parabolic source);
    a different model, so not the headline: forward + lnL per step, same batch, same
    L2 flush."""
    import dataclasses

    import torch

    from paper_1910_01070_b300 import hr2
    from paper_1910_01070_b300 import workloads as W
    from paper_1910_01070_b300.engine import Engine

    dev = torch.device("cuda", local)
    wl = W.WORKLOADS[args.workload]()
    option = option or {"interp": "linear"}
    spec = dataclasses.replace(wl.setups[0], **option)
    with Engine(local) as eng:
        t = eng.add_tables(wl.table, "fp16", W.make_tables(wl.table))
        s = eng.add_setup(t, spec)
        tb = eng.forward([s], torch.zeros(1, dtype=torch.int32, device=dev),
                         torch.as_tensor(wl.truth(0)[None, :], device=dev))
        D, sig = W.mock_observation(tb.double().cpu().numpy()[0, : spec.n_bins], wl.seed)
        eng.set_observation(s, D, sig)
        n = wl.n_samples
        th, sid = wl.params(n, seed_offset=7)
        th, sid = torch.as_tensor(th, device=dev), torch.as_tensor(sid, device=dev)
        bins = torch.empty((n, spec.n_bins), dtype=torch.float32, device=dev)
        lnl = torch.empty(n, dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream()
        for _ in range(3):
            hr2.forward_model_batch(eng.ctx, [s], sid, th, bins, None, None, stream)
        torch.cuda.synchronize()
        steps = max(3, min(args.steps, 40))
        evs = []
        hr2.hr2_profile_read(eng.ctx, True)
        hr2.hr2_profile_enable(eng.ctx, True)
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            hr2.forward_model_batch(eng.ctx, [s], sid, th, bins, None, None, stream)
            hr2.log_likelihood_batch(eng.ctx, [s], sid, bins, lnl, None, stream)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        hr2.hr2_profile_enable(eng.ctx, False)
        kms, nl = hr2.hr2_profile_read(eng.ctx, True)
        times = [a.elapsed_time(b) for a, b in evs]
        return {"workload": wl.name, "option": option, "samples": n, "value": n * steps / (sum(times) / 1e3),
                "unit": "models/s", "ms_per_step": float(np.mean(times)), "kernel_ms": kms / max(nl, 1)}


PROFILE_TRAFFIC_LARGE = os.path.join(ROOT, "profiles", "traffic_large.json")


def large_counters() -> Optional[dict]:
    """DRAM bytes per launch of the forward kernel on the 290001-point tables (from a
    capture on a slice of the wavenumbers, scaled by the tile count), per mode and batch,
    if they belong to the current kernel source."""
    if not os.path.exists(PROFILE_TRAFFIC_LARGE):
        return None
    with open(PROFILE_TRAFFIC_LARGE) as f:
        tr = json.load(f)
    if tr.get("kernel_source_hash") != _kernel_hash():
        return None
    return tr


def large_table_sweep(local, n_nu=290001, modes=("direct", "cached"), batches=(1, 256), print_lines=False,
                      target_s=0.3, fixed_reps=0):
    """Batch sweep on the 290001-point, 12-absorber FP16 tables (2.09 GB): the direct FP16
    interpolation and the level-gridded operand, event-timed kernel per (mode, batch) with the
    SM clock sampled during each, to show where HBM binds (small batches) and where the ALU
    does.  Each point repeats its launch for about target_s seconds (at least 3 times)."""
    import torch

    from paper_1910_01070_b300 import hr2
    from paper_1910_01070_b300 import workloads as W
    from paper_1910_01070_b300.build import build
    from paper_1910_01070_b300.engine import Engine

    build()
    dev = torch.device("cuda", local)
    wl = W.large_l100_k12_nu290001_b256(n_nu)
    s = wl.setups[0]
    res = []
    hbm_peak, hbm_src = _hbm_peak()
    counters = large_counters() if n_nu == 290001 else None
    with Engine(local) as eng:
        t = eng.add_tables(wl.table, "fp16")
        # "direct": the FP16 tables read in place (batches up to the context's split_max_batch
        # in two passes), "direct1": the same in one pass always, "cached": the level-gridded
        # operand, "stream": that operand built per call and group of tiles into a ring
        # (batches of 32 and more; smaller ones read the tables directly, so they are skipped)
        setups = {m: eng.add_setup(t, s, level_cache="stream" if m == "stream" else (m == "cached"))
                  for m in modes}
        cfg0 = hr2.hr2_get_launch_config(eng.ctx)
        th_all, _ = wl.params(max(batches))
        # algorithmic bytes one model reads: on the direct path the FP16 corners (4 per level
        # and point for each of the K absorbers, 2 for each of the two CIA pairs), the
        # per-model count of the scope table; on the level-gridded path the operand blocks,
        # (K + 2) rows of value and T difference (8 B per point) per level over the setup's
        # 128-point tiles
        n_tiles = (s.nu_first + s.n_nu - 1) // 128 - s.nu_first // 128 + 1
        algo = {"direct": (s.n_layers + 1) * 4 * s.n_nu * (len(s.species) + 1) * 2,
                "cached": (s.n_layers + 1) * n_tiles * 128 * (len(s.species) + 2) * 8}
        algo["direct1"] = algo["direct"]
        algo["stream"] = algo["cached"]
        for mode, h in setups.items():
            per_model_bytes = algo[mode]
            hr2.hr2_set_launch_config(eng.ctx, *cfg0[:4], 0 if mode == "direct1" else cfg0[4])
            for b in batches:
                if mode == "stream" and b < 32:
                    continue
                th = torch.as_tensor(th_all[:b], device=dev)
                sd = torch.zeros(b, dtype=torch.int32, device=dev)
                bins = torch.empty((b, s.n_bins), dtype=torch.float32, device=dev)
                torch.cuda.synchronize()
                m0 = hr2.hr2_ctx_memory(eng.ctx)[0]
                eng.forward([h], sd, th, bins)
                torch.cuda.synchronize()
                ring_bytes = hr2.hr2_ctx_memory(eng.ctx)[0] - m0   # the streamed path's ring and views
                t0 = time.perf_counter()
                eng.forward([h], sd, th, bins)
                torch.cuda.synchronize()
                reps = fixed_reps or int(min(200, max(3, target_s / max(time.perf_counter() - t0, 1e-5))))
                cs = ClockSampler(local)
                cs.start()
                hr2.hr2_profile_read(eng.ctx, True)
                hr2.hr2_profile_enable(eng.ctx, True)
                for _ in range(reps):
                    eng.forward([h], sd, th, bins)
                torch.cuda.synchronize()
                hr2.hr2_profile_enable(eng.ctx, False)
                clk = cs.stop()
                ms, n = hr2.hr2_profile_read(eng.ctx, True)
                ms /= max(n, 1)
                passes = 2 if mode not in ("cached", "stream") and b <= hr2.hr2_get_launch_config(eng.ctx)[4] else 1
                line = {"workload": wl.name, "mode": mode, "batch": b, "passes": passes, "kernel_ms": ms, "reps": reps,
                        "models_per_s": b / (ms / 1e3),
                        "algorithmic_bytes_per_model": per_model_bytes,
                        "algorithmic_gbs": b * per_model_bytes / (ms / 1e3) / 1e9,
                        "algorithmic_hbm_frac": b * per_model_bytes / (ms / 1e3) / 1e9 / hbm_peak,
                        "clocks": clk}
                # counters per path: "direct2" the two-pass direct path, "direct" the one-pass one
                key = "%s_b%d" % ("cached" if mode == "cached" else ("direct2" if passes == 2 else "direct"), b)
                line["operand_bytes"] = hr2.hr2_setup_memory(h)[1]
                if mode == "stream":
                    # the operand every call writes (all T cells of every level and tile) and
                    # its rate over the whole call
                    build_b = (s.n_layers + 1) * n_tiles * 128 * (len(s.species) + 2) * 8 * (len(wl.table.T_grid) - 1)
                    line.update({"ring_bytes": ring_bytes, "operand_build_bytes_per_call": build_b,
                                 "operand_build_gbs_over_call": build_b / (ms / 1e3) / 1e9})
                if counters and mode != "stream" and key in counters.get("dram_bytes_per_launch", {}):
                    dram = counters["dram_bytes_per_launch"][key]
                    line.update({"dram_bytes_per_launch": dram, "dram_gbs": dram / (ms / 1e3) / 1e9,
                                 "dram_hbm_frac": dram / (ms / 1e3) / 1e9 / hbm_peak,
                                 "dram_source": counters.get("source")})
                res.append(line)
                if print_lines:
                    print(json.dumps(line), flush=True)
    return {"lines": res, "hbm_peak_gbs": hbm_peak, "hbm_peak_source": hbm_src}


def run_sweep_large(args, local):
    modes = tuple(m for m in args.sweep_modes.split(",") if m)
    batches = tuple(int(b) for b in args.sweep_batches.split(",") if b)
    return large_table_sweep(local, args.sweep_nu, modes, batches, print_lines=True, fixed_reps=args.sweep_reps)


UNIT_KINDS = (("ex2_rcp", 0), ("rcp", 1), ("ex2", 2), ("ffma", 3), ("ffma2", 4))


def measure_unit_rates(local, iters=20000, clocks=True):
    """Throughput of the special-function unit and the FMA pipe (hr2_measure_unit_rate),
    per kind: operations per clock per SM at the clock the kernel ran at.  The
    interleaved ex2/rcp kind is compared with what one shared unit would give."""
    from paper_1910_01070_b300 import hr2
    from paper_1910_01070_b300.build import build
    build()
    out = {}
    for name, kind in UNIT_KINDS:
        cs = ClockSampler(local) if clocks else None
        if cs:
            cs.start()
        r = hr2.hr2_measure_unit_rate(local, kind, iters)
        if cs:
            r["clocks"] = cs.stop()
        out[name] = r
    # the interleaved chains tell whether ex2 and rcp share one unit: if they do,
    # a mixed op takes the mean of the two single-kind times
    t_mix = 1.0 / out["ex2_rcp"]["ops_per_clk_sm"]
    t_shared = 0.5 / out["ex2"]["ops_per_clk_sm"] + 0.5 / out["rcp"]["ops_per_clk_sm"]
    out["ex2_rcp"]["shared_unit_prediction_ops_per_clk_sm"] = 1.0 / t_shared
    out["ex2_rcp"]["mix_over_shared_prediction"] = t_shared / t_mix
    return out


def run_peaks(args, local):
    rates = measure_unit_rates(local)
    line = {"peaks": "arithmetic units", "sm_max_mhz": SM_MAX_MHZ, "rates": rates,
            "note": "ops_per_clk_sm: operations per SM per clock at the clock the kernel ran at (clock64 over "
                    "the global timer); 8 CTAs x 256 threads per SM, 16 independent chains per thread"}
    print(json.dumps(line), flush=True)
    return line


SM_MAX_MHZ = 2032.0


def committed_counters(path: str = PROFILE_TRAFFIC) -> Optional[dict]:
    """ncu counters of the forward kernel committed under profiles/ (DRAM bytes per launch
    and L2 throughput as a fraction of peak), if they belong to the current kernel source."""
    if not os.path.exists(path):
        return None
    with open(path) as f:
        tr = json.load(f)
    if tr.get("kernel_source_hash") != _kernel_hash():
        return None
    return {"dram_bytes": tr.get("bytes_per_launch"), "l2_frac": tr.get("l2_throughput_frac"),
            "kernel_ms_ncu": tr.get("kernel_ms_ncu"), "source": tr.get("source")}


def _hbm_peak():
    """Measured copy bandwidth of this machine's B300 (GB/s), else the recipe's fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


def _code_only(src: str) -> str:
    """C++ source without comments and whitespace (what the compiler sees as tokens)."""
    import re
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return re.sub(r"\s+", "", src)


def _kernel_hash() -> str:
    """Hash of the forward kernel's code (comments and whitespace ignored), to tell whether
    the committed DRAM counters still belong to it."""
    import hashlib
    h = hashlib.sha256()
    for f in ("kern_forward.cu", "kern_forward32.cuh", "hr2_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1910_01070_b300", "csrc", f)) as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.sweep_large:
        if rank == 0:
            run_sweep_large(args, local)
    elif args.peaks:
        if rank == 0:
            run_peaks(args, local)
    else:
        run_hr2(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
