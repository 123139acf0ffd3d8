"""Autotuner for the launch shape of the persistent forward kernel.

The forward kernel's tile is fixed (128 wavenumbers, two packed pairs per
lane); what is tuned is how many samples share one work item (warps per CTA,
which also sets the per-CTA shared-memory pipeline size) and how many
persistent CTAs run per SM.  For a batch shape the tuner times every candidate with the
library's kernel-event instrumentation (hr2_profile_*) on the caller's real
inputs, keeps the fastest, and caches the choice in a JSON file keyed by the
shape, so later runs (and the serving loop) reuse it without re-timing.
"""
from __future__ import annotations

import json
import os
import threading
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

from . import hr2

DEFAULT_CANDIDATES: Tuple[Tuple[int, int], ...] = (
    (1, 16), (2, 6), (2, 8), (4, 2), (4, 3), (4, 4), (4, 6), (8, 1), (8, 2), (8, 3), (16, 1))
_LOCK = threading.Lock()


def cache_path() -> str:
    return os.environ.get("HR2_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "hr2", "autotune.json"))


def shape_key(setups_info: Sequence[Dict], n: int) -> str:
    """Key of a batch shape: per-setup (K, L, N_mu, n_nu bucket, cached) and the batch-size bucket."""
    parts = []
    for s in sorted(setups_info, key=lambda d: (d["K"], d["L"], d["n_mu"], d["n_nu"])):
        nu_bucket = 1 << max(0, int(s["n_nu"]) - 1).bit_length()
        parts.append("K%dL%dM%dN%dC%d" % (s["K"], s["L"], s["n_mu"], nu_bucket, int(s.get("cached", 1))))
    n_bucket = 1 << max(0, n - 1).bit_length()
    return "n%d|%s" % (n_bucket, "+".join(parts))


def load_cache(path: Optional[str] = None) -> Dict[str, List[int]]:
    path = path or cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
        return {k: list(v) for k, v in data.items()}
    except (OSError, ValueError):
        return {}


def save_cache(cache: Dict[str, List[int]], path: Optional[str] = None) -> None:
    path = path or cache_path()
    with _LOCK:
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        tmp = path + ".tmp.%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def pick_best(timings: Dict[Tuple[int, int], float]) -> Tuple[int, int]:
    """Fastest candidate; ties go to fewer warps, then fewer CTAs (smaller shared-memory footprint)."""
    return min(timings, key=lambda c: (round(timings[c], 6), c[0], c[1]))


def tune(ctx, setups: Sequence, setup_of_sample, params, out_bins, setups_info: Sequence[Dict],
         candidates: Iterable[Tuple[int, int]] = DEFAULT_CANDIDATES, reps: int = 3, use_cache: bool = True,
         path: Optional[str] = None, stream=None) -> Tuple[Tuple[int, int], Dict[Tuple[int, int], float]]:
    """Time each (warps_per_cta, ctas_per_sm) candidate on this batch and set the best on ctx.

    Returns (best, {candidate: ms per forward-kernel launch}).  With use_cache a cached
    choice for the same shape key is applied without timing.
    """
    import torch
    key = shape_key(setups_info, int(params.shape[0]))
    cache = load_cache(path) if use_cache else {}
    if use_cache and key in cache:
        best = tuple(cache[key])
        hr2.hr2_set_launch_config(ctx, *best)
        return best, {}
    timings = {}
    for w, c in candidates:
        hr2.hr2_set_launch_config(ctx, w, c)
        hr2.forward_model_batch(ctx, setups, setup_of_sample, params, out_bins, None, None, stream)  # warm-up
        torch.cuda.synchronize()
        hr2.hr2_profile_read(ctx, True)
        hr2.hr2_profile_enable(ctx, True)
        for _ in range(reps):
            hr2.forward_model_batch(ctx, setups, setup_of_sample, params, out_bins, None, None, stream)
        torch.cuda.synchronize()
        hr2.hr2_profile_enable(ctx, False)
        ms, n = hr2.hr2_profile_read(ctx, True)
        timings[(w, c)] = ms / max(n, 1)
    best = pick_best(timings)
    hr2.hr2_set_launch_config(ctx, *best)
    if use_cache:
        cache = load_cache(path)
        cache[key] = list(best)
        save_cache(cache, path)
    return best, timings


def setup_info_from_spec(spec, cached: bool = True) -> Dict:
    return {"K": len(spec.species), "L": int(spec.n_layers), "n_mu": int(spec.n_mu), "n_nu": int(spec.n_nu),
            "cached": int(bool(cached))}
