"""Shared helpers of the test-suite: the storage rule applied on the oracle's
side (numpy), oracle construction, and the comparison metrics.

Nothing here calls the CUDA path; the GPU tests call it through the C ABI
binding and compare with what these helpers compute from the oracle.
"""
import numpy as np

import oracle
from paper_1910_01070_b300 import workloads as W

FLUX_RTOL = 1e-4          # max relative flux error per spectrum
LNL_ATOL = 1e-3           # |delta lnL| near the data
FP64_RTOL = 2e-7          # plain FP64 GPU path vs the FP64 oracle (FP32 outputs)


def fp16_offset_dequantise(v):
    """The FP16-offset storage rule, written independently of the library:
    off = rint((min+max)/2); stored = binary16(v - off) (round to nearest
    even); value seen by the kernels = stored + off."""
    v = np.asarray(v, dtype=np.float64)
    off = np.rint(0.5 * (v.min() + v.max()))
    return (v - off).astype(np.float16).astype(np.float64) + off


def tables_as_stored(tabs, storage):
    """Table arrays with the values the device holds (for the oracle)."""
    if storage == "fp64":
        return tabs
    out = dict(tabs)
    out["log10_sigma"] = np.stack([fp16_offset_dequantise(s) for s in tabs["log10_sigma"]])
    for key in ("log10_cia_h2h2", "log10_cia_h2he"):
        if tabs.get(key) is not None:
            out[key] = fp16_offset_dequantise(tabs[key])
    return out


def oracle_model(tabs_stored, setup):
    return oracle.Model(tabs_stored, setup.as_dict())


def rel_flux_err(F, Fref):
    """Per spectrum: max_i |F - Fref| / max(|Fref|, 1e-6 max|Fref|)."""
    F = np.asarray(F, dtype=np.float64)
    Fref = np.asarray(Fref, dtype=np.float64)
    floor = 1e-6 * np.max(np.abs(Fref))
    return float(np.max(np.abs(F - Fref) / np.maximum(np.abs(Fref), floor)))
