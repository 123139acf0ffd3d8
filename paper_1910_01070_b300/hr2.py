"""ctypes binding of libhr2.so (include/hr2.h).

Argument marshalling only: every step of the forward model and the
likelihood runs in the library's CUDA kernels.  Functions keep the C names.
Device buffers are torch CUDA tensors (their ``data_ptr()`` is passed);
streams default to torch's current stream.  Loading fails loudly if the
library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# HR2_LIBRARY selects another build of the same library (the bounds-checked one)
LIB_PATH = os.environ.get("HR2_LIBRARY") or os.path.join(_HERE, "libhr2.so")

HR2_OK, HR2_EINVAL, HR2_ENOMEM, HR2_ECUDA, HR2_ETIMEDOUT, HR2_EBUSY, HR2_EBOUNDS = 0, -1, -2, -3, -4, -5, -6
HR2_SAMPLE_BAD_T, HR2_SAMPLE_BAD_ABUND, HR2_SAMPLE_BAD_SCALE, HR2_SAMPLE_BAD_SETUP = 1, 2, 4, 8
HR2_SAMPLE_BAD_CLOUD = 16
HR2_MAX_TNODES, HR2_MAX_SPECIES, HR2_MAX_MU, HR2_MAX_LEVELS, HR2_MAX_SETUPS = 16, 16, 8, 256, 32
HR2_P_LOGG, HR2_P_F, HR2_P_DIST, HR2_P_T0, HR2_P_X0, HR2_P_CLOUD, HR2_NPARAM = 0, 1, 2, 3, 19, 35, 38
HR2_STORE_FP16_OFFSET, HR2_STORE_FP64 = 1, 2
HR2_INTERP_LOG10, HR2_INTERP_LINEAR = 0, 1
HR2_LEVEL_CACHE_AUTO = 2
HR2_LEVEL_CACHE_STREAM = 3
INTERP = {"log10": HR2_INTERP_LOG10, "linear": HR2_INTERP_LINEAR}
HR2_PROFILE_FE, HR2_PROFILE_MILNE = 0, 1
PROFILE = {"fe": HR2_PROFILE_FE, "milne": HR2_PROFILE_MILNE}
HR2_SC_LINEAR, HR2_SC_PARABOLIC = 0, 1
SC = {"linear": HR2_SC_LINEAR, "parabolic": HR2_SC_PARABOLIC}

EXPORTED = [
    "hr2_ctx_create", "hr2_ctx_destroy", "hr2_last_error", "hr2_ctx_memory", "hr2_set_launch_config",
    "hr2_get_launch_config", "hr2_reserve", "create_opacity_tables", "hr2_tables_upload_species",
    "hr2_tables_info", "hr2_tables_destroy", "hr2_setup_create", "hr2_setup_set_observation", "hr2_setup_info",
    "hr2_setup_destroy", "forward_model_batch", "forward_model_batch_noalloc", "log_likelihood_batch",
    "hr2_evaluate_host", "hr2_profile_enable",
    "hr2_profile_read", "hr2_stream_check", "hr2_nodes_from_b", "hr2_version",
    "hr2_ns_state_init", "hr2_ns_absorb", "hr2_ns_propose", "hr2_ns_finalize", "hr2_effective_temperature",
    "hr2_measure_unit_rate", "hr2_noalloc_check", "hr2_set_wait_limit", "hr2_get_wait_limit",
    "hr2_set_wait_fault", "hr2_setup_memory", "hr2_set_stream_group",
]


class Hr2Error(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("hr2 error %d: %s" % (code, msg))
        self.code = code


class TableDesc(C.Structure):
    _fields_ = [("n_species", C.c_int), ("n_T", C.c_int), ("T_grid", C.POINTER(C.c_double)), ("n_p", C.c_int),
                ("log10p_grid", C.POINTER(C.c_double)), ("nu0", C.c_double), ("dnu", C.c_double), ("n_nu", C.c_int),
                ("species_mass", C.POINTER(C.c_double)), ("has_cia_h2h2", C.c_int), ("has_cia_h2he", C.c_int)]


class SetupDesc(C.Structure):
    _fields_ = [("nu_first", C.c_int), ("n_nu", C.c_int), ("n_layers", C.c_int), ("p_top", C.c_double),
                ("p_bot", C.c_double), ("n_species", C.c_int), ("species", C.POINTER(C.c_int)), ("n_mu", C.c_int),
                ("fe_elements", C.c_int), ("fe_order", C.c_int), ("resolving_power", C.c_double),
                ("n_bins", C.c_int), ("bin_edges", C.POINTER(C.c_double)), ("obs_flux", C.POINTER(C.c_double)),
                ("obs_sigma", C.POINTER(C.c_double)), ("r_he", C.c_double), ("radius_cm", C.c_double),
                ("level_cache", C.c_int), ("interp", C.c_int), ("profile", C.c_int), ("cloud", C.c_int),
                ("sc", C.c_int)]


class UnitRate(C.Structure):
    _fields_ = [("ms", C.c_double), ("ops", C.c_double), ("ops_per_s", C.c_double), ("sm_ghz", C.c_double),
                ("ops_per_clk_sm", C.c_double), ("n_sm", C.c_int)]


HR2_UNIT_EX2_RCP, HR2_UNIT_RCP, HR2_UNIT_EX2, HR2_UNIT_FFMA, HR2_UNIT_FFMA2, HR2_UNIT_KINDS = 0, 1, 2, 3, 4, 5


class LaunchCfg(C.Structure):
    _fields_ = [("warps_per_cta", C.c_int), ("ctas_per_sm", C.c_int), ("tiles_per_item", C.c_int),
                ("stages", C.c_int), ("split_max_batch", C.c_int)]


class NsState(C.Structure):
    _fields_ = [("n_dead", C.c_longlong), ("n_seen", C.c_longlong), ("log_z", C.c_double), ("info", C.c_double),
                ("log_x", C.c_double), ("lnl_min", C.c_double), ("lnl_max", C.c_double),
                ("reserved", C.c_double)]


_LIB = None
_LOCK = threading.Lock()
_VP, _DP, _IP, _FP = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_float)


def lib():
    """Load libhr2.so (raises if it is missing: there is no fallback)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libhr2.so not built: run python -m paper_1910_01070_b300.build")
            L = C.CDLL(LIB_PATH)
            sig = {
                "hr2_ctx_create": (C.c_int, [C.c_int, C.c_size_t, C.POINTER(_VP)]),
                "hr2_ctx_destroy": (C.c_int, [_VP]),
                "hr2_last_error": (C.c_char_p, [_VP]),
                "hr2_ctx_memory": (C.c_int, [_VP, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
                "hr2_set_launch_config": (C.c_int, [_VP, C.POINTER(LaunchCfg)]),
                "hr2_get_launch_config": (C.c_int, [_VP, C.POINTER(LaunchCfg)]),
                "hr2_set_stream_group": (C.c_int, [_VP, C.c_int]),
                "hr2_reserve": (C.c_int, [_VP, _VP, C.c_int, C.c_int]),
                "create_opacity_tables": (C.c_int, [_VP, C.POINTER(TableDesc), _DP, _DP, _DP, C.c_int,
                                                    C.POINTER(_VP)]),
                "hr2_tables_upload_species": (C.c_int, [_VP, _VP, C.c_int, _DP]),
                "hr2_tables_info": (C.c_int, [_VP, _DP, C.POINTER(C.c_size_t)]),
                "hr2_tables_destroy": (C.c_int, [_VP, _VP]),
                "hr2_setup_create": (C.c_int, [_VP, _VP, C.POINTER(SetupDesc), C.POINTER(_VP)]),
                "hr2_setup_set_observation": (C.c_int, [_VP, _VP, _DP, _DP]),
                "hr2_setup_info": (C.c_int, [_VP, _IP, _IP, C.POINTER(C.c_longlong)]),
                "hr2_setup_destroy": (C.c_int, [_VP, _VP]),
                "forward_model_batch": (C.c_int, [_VP, C.c_int, C.POINTER(_VP), _VP, _VP, C.c_int, _VP, C.c_int,
                                                  _VP, C.c_int, _VP, _VP]),
                "forward_model_batch_noalloc": (C.c_int, [_VP, C.c_int, C.POINTER(_VP), _VP, _VP, C.c_int, _VP,
                                                          C.c_int, _VP, C.c_int, _VP, _VP]),
                "log_likelihood_batch": (C.c_int, [_VP, C.c_int, C.POINTER(_VP), _VP, _VP, C.c_int, _VP, C.c_int,
                                                   _VP, _VP]),
                "hr2_evaluate_host": (C.c_int, [_VP, C.c_int, C.POINTER(_VP), _VP, _VP, _VP, C.c_int, _VP, _VP,
                                                C.c_int, _VP]),
                "hr2_profile_enable": (C.c_int, [_VP, C.c_int]),
                "hr2_profile_read": (C.c_int, [_VP, C.c_int, _DP, _IP]),
                "hr2_stream_check": (C.c_int, [_VP, _VP]),
                "hr2_nodes_from_b": (C.c_int, [C.c_int, C.c_double, _DP, _DP]),
                "hr2_version": (C.c_char_p, []),
                "hr2_ns_state_init": (C.c_int, [_VP, _VP, _VP]),
                "hr2_effective_temperature": (C.c_int, [_VP, C.c_int, C.POINTER(_VP), _VP, _VP, C.c_int, C.c_int,
                                                        _VP, _VP]),
                "hr2_ns_absorb": (C.c_int, [_VP, C.c_int, _VP, _VP, C.c_int, _VP, _VP, _VP, _VP, _VP, _VP,
                                            C.c_longlong, _VP]),
                "hr2_ns_propose": (C.c_int, [_VP, C.c_int, _VP, _VP, _VP, C.c_double, C.c_int, _VP, _VP,
                                             C.c_ulonglong, C.c_ulonglong, _VP]),
                "hr2_ns_finalize": (C.c_int, [_VP, C.c_int, _VP, _VP, _VP, _VP]),
                "hr2_measure_unit_rate": (C.c_int, [C.c_int, C.c_int, C.c_longlong, C.POINTER(UnitRate)]),
                "hr2_noalloc_check": (C.c_int, [_VP, _VP]),
                "hr2_set_wait_limit": (C.c_int, [_VP, C.c_longlong]),
                "hr2_get_wait_limit": (C.c_int, [_VP, C.POINTER(C.c_longlong)]),
                "hr2_set_wait_fault": (C.c_int, [_VP, C.c_int]),
                "hr2_setup_memory": (C.c_int, [_VP, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t), _IP]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = L
    return _LIB


def _check(rc: int, ctx=None):
    if rc != HR2_OK:
        raise Hr2Error(rc, lib().hr2_last_error(ctx).decode())


def _dptr(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_DP)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _tensor_ptr(t, dtype, name, shape=None):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape[: len(shape)]) != tuple(shape):
        raise ValueError("%s has shape %s, expected leading %s" % (name, tuple(t.shape), shape))
    return t.data_ptr()


def _setup_array(setups):
    arr = (_VP * len(setups))(*[s.handle if hasattr(s, "handle") else s for s in setups])
    return arr


# ------------------------------------------------------------------ raw ABI
def hr2_version() -> str:
    return lib().hr2_version().decode()


def hr2_ctx_create(device: int = 0, mem_budget_bytes: int = 0):
    h = _VP()
    _check(lib().hr2_ctx_create(device, mem_budget_bytes, C.byref(h)))
    return h


def hr2_ctx_destroy(ctx):
    _check(lib().hr2_ctx_destroy(ctx))


def hr2_last_error(ctx=None) -> str:
    return lib().hr2_last_error(ctx).decode()


def hr2_ctx_memory(ctx):
    u, b = C.c_size_t(), C.c_size_t()
    _check(lib().hr2_ctx_memory(ctx, C.byref(u), C.byref(b)), ctx)
    return u.value, b.value


def hr2_set_launch_config(ctx, warps_per_cta: int, ctas_per_sm: int, tiles_per_item: int = 1, stages: int = 0,
                          split_max_batch: int = 2):
    cfg = LaunchCfg(warps_per_cta, ctas_per_sm, tiles_per_item, stages, split_max_batch)
    _check(lib().hr2_set_launch_config(ctx, C.byref(cfg)), ctx)


def hr2_set_stream_group(ctx, tiles: int):
    """Tiles per group of the streamed operand for later calls (0: sized by the batch)."""
    _check(lib().hr2_set_stream_group(ctx, int(tiles)), ctx)


def hr2_get_launch_config(ctx):
    """(warps_per_cta, ctas_per_sm, tiles_per_item, stages, split_max_batch)."""
    cfg = LaunchCfg()
    _check(lib().hr2_get_launch_config(ctx, C.byref(cfg)), ctx)
    return cfg.warps_per_cta, cfg.ctas_per_sm, cfg.tiles_per_item, cfg.stages, cfg.split_max_batch


def hr2_reserve(ctx, n: int, n_nu_max: int, stream=None):
    _check(lib().hr2_reserve(ctx, _stream_ptr(stream), n, n_nu_max), ctx)


def create_opacity_tables(ctx, T_grid, log10p_grid, nu0, dnu, n_nu, species_mass, log10_sigma=None,
                          log10_cia_h2h2=None, log10_cia_h2he=None, storage=HR2_STORE_FP16_OFFSET):
    T_grid, pT = _dptr(T_grid)
    log10p_grid, pp = _dptr(log10p_grid)
    mass, pm = _dptr(species_mass)
    d = TableDesc(len(mass), len(T_grid), pT, len(log10p_grid), pp, float(nu0), float(dnu), int(n_nu), pm,
                  int(log10_cia_h2h2 is not None), int(log10_cia_h2he is not None))
    keep = []

    def opt(a, shape):
        if a is None:
            return _DP()
        a = np.ascontiguousarray(a, dtype=np.float64)
        assert a.shape == shape, (a.shape, shape)
        keep.append(a)
        return a.ctypes.data_as(_DP)

    K, nT, nP = len(mass), len(T_grid), len(log10p_grid)
    ps = opt(log10_sigma, (K, nT, nP, int(n_nu)))
    c0 = opt(log10_cia_h2h2, (nT, int(n_nu)))
    c1 = opt(log10_cia_h2he, (nT, int(n_nu)))
    h = _VP()
    _check(lib().create_opacity_tables(ctx, C.byref(d), ps, c0, c1, int(storage), C.byref(h)), ctx)
    return h


def hr2_tables_upload_species(ctx, tables, s: int, log10_sigma_s):
    a, p = _dptr(log10_sigma_s)
    _check(lib().hr2_tables_upload_species(ctx, tables, int(s), p), ctx)


def hr2_tables_info(tables, n_species: int):
    off = np.zeros(n_species + 2)
    b = C.c_size_t()
    _check(lib().hr2_tables_info(tables, off.ctypes.data_as(_DP), C.byref(b)))
    return off, b.value


def hr2_tables_destroy(ctx, tables):
    _check(lib().hr2_tables_destroy(ctx, tables), ctx)


def hr2_setup_create(ctx, tables, nu_first, n_nu, n_layers, species, n_mu, fe_elements, fe_order,
                     resolving_power, bin_edges, p_top=1e-4, p_bot=100.0, r_he=0.17, radius_cm=7.1492e9,
                     obs_flux=None, obs_sigma=None, level_cache=True, interp="log10", profile="fe", cloud=False,
                     sc="linear"):
    """interp: "log10" (HR2_INTERP_LOG10) or "linear" (HR2_INTERP_LINEAR);
    profile: "fe" (HR2_PROFILE_FE) or "milne" (HR2_PROFILE_MILNE);
    cloud: add the gray cloud layer of parameters HR2_P_CLOUD..;
    sc: "linear" (HR2_SC_LINEAR) or "parabolic" (HR2_SC_PARABOLIC) source interpolation."""
    sp = np.ascontiguousarray(np.asarray(species, dtype=np.int32))
    edges, pe = _dptr(bin_edges)
    keep = [sp, edges]
    if obs_flux is not None:
        of, pf = _dptr(obs_flux)
        os_, ps = _dptr(obs_sigma)
        keep += [of, os_]
    else:
        pf, ps = _DP(), _DP()
    d = SetupDesc(int(nu_first), int(n_nu), int(n_layers), float(p_top), float(p_bot), len(sp),
                  sp.ctypes.data_as(_IP), int(n_mu), int(fe_elements), int(fe_order), float(resolving_power),
                  len(edges) - 1, pe, pf, ps, float(r_he), float(radius_cm), _level_cache_arg(level_cache),
                  INTERP[interp], PROFILE[profile], int(bool(cloud)), SC[sc])
    h = _VP()
    _check(lib().hr2_setup_create(ctx, tables, C.byref(d), C.byref(h)), ctx)
    return h


def hr2_setup_set_observation(ctx, setup, obs_flux, obs_sigma):
    f, pf = _dptr(obs_flux)
    s, ps = _dptr(obs_sigma)
    _check(lib().hr2_setup_set_observation(ctx, setup, pf, ps), ctx)


def hr2_setup_info(setup):
    nb, nn, nnz = C.c_int(), C.c_int(), C.c_longlong()
    _check(lib().hr2_setup_info(setup, C.byref(nb), C.byref(nn), C.byref(nnz)))
    return nb.value, nn.value, nnz.value


def hr2_setup_memory(setup):
    """(device bytes of the setup, bytes of its level-gridded operand, whether the operand was built)."""
    b, ob, lg = C.c_size_t(), C.c_size_t(), C.c_int()
    _check(lib().hr2_setup_memory(setup, C.byref(b), C.byref(ob), C.byref(lg)))
    return b.value, ob.value, lg.value == 1


def hr2_setup_streamed(setup) -> bool:
    """Whether the setup builds its operand per call (level_cache="stream")."""
    b, ob, lg = C.c_size_t(), C.c_size_t(), C.c_int()
    _check(lib().hr2_setup_memory(setup, C.byref(b), C.byref(ob), C.byref(lg)))
    return lg.value == HR2_LEVEL_CACHE_STREAM


def _level_cache_arg(v) -> int:
    """level_cache as the ABI takes it: True/False, "auto" (HR2_LEVEL_CACHE_AUTO) or
    "stream" (HR2_LEVEL_CACHE_STREAM)."""
    if isinstance(v, str):
        if v not in ("auto", "stream"):
            raise ValueError("level_cache must be a bool, 'auto' or 'stream'")
        return HR2_LEVEL_CACHE_AUTO if v == "auto" else HR2_LEVEL_CACHE_STREAM
    return int(bool(v))


def hr2_setup_destroy(ctx, setup):
    _check(lib().hr2_setup_destroy(ctx, setup), ctx)


def forward_model_batch(ctx, setups: Sequence, setup_of_sample, params, out_bins, out_highres=None,
                        out_status=None, stream=None):
    """Device tensors: setup_of_sample int32 [n], params float64 [n, HR2_NPARAM], out_bins float32 [n, ld],
    out_highres float32 [n, ld2] or None, out_status int32 [n] or None."""
    import torch
    n = int(params.shape[0]) if params is not None else 0
    arr = _setup_array(setups)
    p_sos = _tensor_ptr(setup_of_sample, torch.int32, "setup_of_sample", (n,))
    p_par = _tensor_ptr(params, torch.float64, "params", (n, HR2_NPARAM))
    p_bins = _tensor_ptr(out_bins, torch.float32, "out_bins", (n,))
    p_hr = _tensor_ptr(out_highres, torch.float32, "out_highres", (n,))
    p_st = _tensor_ptr(out_status, torch.int32, "out_status", (n,))
    rc = lib().forward_model_batch(ctx, len(setups), arr, p_sos, p_par, n, p_bins, int(out_bins.shape[1]),
                                   p_hr, int(out_highres.shape[1]) if out_highres is not None else 0, p_st,
                                   _stream_ptr(stream))
    _check(rc, ctx)


HR2_NOALLOC_SCRATCH_BYTES = 8 << 20


def forward_model_batch_noalloc(ctx, setups: Sequence, setup_of_sample, params, out_bins, out_highres,
                                out_status=None, stream=None):
    """forward_model_batch without any device allocation (FP16 tables; out_highres required).
    Its scratch is one static device array shared by all calls: do not overlap calls on the GPU."""
    import torch
    n = int(params.shape[0])
    arr = _setup_array(setups)
    rc = lib().forward_model_batch_noalloc(
        ctx, len(setups), arr, _tensor_ptr(setup_of_sample, torch.int32, "setup_of_sample", (n,)),
        _tensor_ptr(params, torch.float64, "params", (n, HR2_NPARAM)), n,
        _tensor_ptr(out_bins, torch.float32, "out_bins", (n,)), int(out_bins.shape[1]),
        _tensor_ptr(out_highres, torch.float32, "out_highres", (n,)), int(out_highres.shape[1]),
        _tensor_ptr(out_status, torch.int32, "out_status", (n,)), _stream_ptr(stream))
    _check(rc, ctx)


def log_likelihood_batch(ctx, setups: Sequence, setup_of_sample, model_bins, out_lnL, log_eps=None, stream=None):
    import torch
    n = int(model_bins.shape[0])
    arr = _setup_array(setups)
    rc = lib().log_likelihood_batch(
        ctx, len(setups), arr, _tensor_ptr(setup_of_sample, torch.int32, "setup_of_sample", (n,)),
        _tensor_ptr(model_bins, torch.float32, "model_bins", (n,)), int(model_bins.shape[1]),
        _tensor_ptr(log_eps, torch.float64, "log_eps", (n,)), n,
        _tensor_ptr(out_lnL, torch.float64, "out_lnL", (n,)), _stream_ptr(stream))
    _check(rc, ctx)


def hr2_evaluate_host(ctx, setups: Sequence, setup_of_sample, params, out_lnL, log_eps=None, out_bins=None,
                      stream=None):
    """Host numpy buffers (pinned torch CPU tensors also accepted): int32 [n], float64 [n, HR2_NPARAM],
    float64 [n] out, optional float64 [n], optional float32 [n, ld] out.  Synchronous."""

    def hp(a, dtype, name):
        if a is None:
            return None
        if hasattr(a, "data_ptr"):  # torch CPU tensor (pinned or not)
            if a.is_cuda or not a.is_contiguous():
                raise ValueError("%s must be a contiguous host tensor" % name)
            return a.data_ptr()
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("%s must be C-contiguous %s" % (name, dtype))
        return a.ctypes.data

    n = int(params.shape[0])
    arr = _setup_array(setups)
    rc = lib().hr2_evaluate_host(ctx, len(setups), arr, hp(setup_of_sample, np.int32, "setup_of_sample"),
                                 hp(params, np.float64, "params"), hp(log_eps, np.float64, "log_eps"), n,
                                 hp(out_lnL, np.float64, "out_lnL"), hp(out_bins, np.float32, "out_bins"),
                                 int(out_bins.shape[1]) if out_bins is not None else 0, _stream_ptr(stream))
    _check(rc, ctx)


def hr2_profile_enable(ctx, on: bool = True):
    _check(lib().hr2_profile_enable(ctx, int(bool(on))), ctx)


def hr2_profile_read(ctx, reset: bool = True):
    """(summed ms of the main forward kernel, launches) since the last reset."""
    ms, n = C.c_double(), C.c_int()
    _check(lib().hr2_profile_read(ctx, int(bool(reset)), C.byref(ms), C.byref(n)), ctx)
    return ms.value, n.value


def hr2_effective_temperature(ctx, setups: Sequence, setup_of_sample, highres, out_teff, stream=None):
    """CUDA tensors: int32 [n], float32 [n, ld] (F+ from forward_model_batch), float64 [n] out."""
    import torch
    n = int(highres.shape[0])
    rc = lib().hr2_effective_temperature(
        ctx, len(setups), _setup_array(setups), _tensor_ptr(setup_of_sample, torch.int32, "setup_of_sample", (n,)),
        _tensor_ptr(highres, torch.float32, "highres", (n,)), int(highres.shape[1]), n,
        _tensor_ptr(out_teff, torch.float64, "out_teff", (n,)), _stream_ptr(stream))
    _check(rc, ctx)


# ------------------------------------------------------------ nested sampling
NS_STATE_DOUBLES = C.sizeof(NsState) // 8


def hr2_ns_state_init(ctx, state, stream=None):
    """state: CUDA float64 tensor of NS_STATE_DOUBLES elements holding an hr2_ns_state."""
    import torch
    _check(lib().hr2_ns_state_init(ctx, _tensor_ptr(state, torch.float64, "state", (NS_STATE_DOUBLES,)),
                                   _stream_ptr(stream)), ctx)


def hr2_ns_absorb(ctx, live_lnl, live_theta, cand_lnl, cand_theta, state, dead_lnl, dead_logw, dead_theta,
                  stream=None):
    """CUDA float64 tensors: live [N], [N, HR2_NPARAM] (updated), candidates [m], [m, HR2_NPARAM], the state,
    dead [cap], [cap], [cap, HR2_NPARAM] (dead point k at row k)."""
    import torch
    n, m, cap = int(live_lnl.shape[0]), int(cand_lnl.shape[0]), int(dead_lnl.shape[0])
    f = torch.float64
    rc = lib().hr2_ns_absorb(
        ctx, n, _tensor_ptr(live_lnl, f, "live_lnl"), _tensor_ptr(live_theta, f, "live_theta", (n, HR2_NPARAM)), m,
        _tensor_ptr(cand_lnl, f, "cand_lnl"), _tensor_ptr(cand_theta, f, "cand_theta", (m, HR2_NPARAM)),
        _tensor_ptr(state, f, "state", (NS_STATE_DOUBLES,)), _tensor_ptr(dead_lnl, f, "dead_lnl"),
        _tensor_ptr(dead_logw, f, "dead_logw", (cap,)), _tensor_ptr(dead_theta, f, "dead_theta", (cap, HR2_NPARAM)),
        cap, _stream_ptr(stream))
    _check(rc, ctx)


def hr2_ns_propose(ctx, live_theta, prior_lo, prior_hi, enlarge, box, out_theta, seed, counter, stream=None):
    """CUDA float64 tensors: live [N, HR2_NPARAM], prior box [HR2_NPARAM] each, box [HR2_NPARAM, 2] (written),
    candidates [n, HR2_NPARAM] (written).  Uses n * HR2_NPARAM counter values from `counter` on."""
    import torch
    f = torch.float64
    n_live, n = int(live_theta.shape[0]), int(out_theta.shape[0])
    _check(lib().hr2_ns_propose(
        ctx, n_live, _tensor_ptr(live_theta, f, "live_theta", (n_live, HR2_NPARAM)),
        _tensor_ptr(prior_lo, f, "prior_lo", (HR2_NPARAM,)), _tensor_ptr(prior_hi, f, "prior_hi", (HR2_NPARAM,)),
        float(enlarge), n, _tensor_ptr(box, f, "box", (HR2_NPARAM, 2)),
        _tensor_ptr(out_theta, f, "out_theta", (n, HR2_NPARAM)), int(seed) & (2 ** 64 - 1),
        int(counter) & (2 ** 64 - 1), _stream_ptr(stream)), ctx)


def hr2_ns_finalize(ctx, live_lnl, state, out, stream=None):
    """out: CUDA float64 tensor [2] <- (ln Z, H) with the live points added."""
    import torch
    f = torch.float64
    _check(lib().hr2_ns_finalize(ctx, int(live_lnl.shape[0]), _tensor_ptr(live_lnl, f, "live_lnl"),
                                 _tensor_ptr(state, f, "state", (NS_STATE_DOUBLES,)), _tensor_ptr(out, f, "out", (2,)),
                                 _stream_ptr(stream)), ctx)


def ns_state_read(state) -> dict:
    """The hr2_ns_state in a (device) float64 tensor, as a dict (synchronises)."""
    raw = state.detach().cpu().numpy().tobytes()
    st = NsState.from_buffer_copy(raw)
    return {name: getattr(st, name) for name, _ in NsState._fields_ if name != "reserved"}


def hr2_noalloc_check(ctx, stream=None):
    _check(lib().hr2_noalloc_check(ctx, _stream_ptr(stream)), ctx)


def hr2_set_wait_limit(ctx, cycles: int):
    _check(lib().hr2_set_wait_limit(ctx, int(cycles)), ctx)


def hr2_set_wait_fault(ctx, on: bool):
    _check(lib().hr2_set_wait_fault(ctx, 1 if on else 0), ctx)


def hr2_get_wait_limit(ctx) -> int:
    v = C.c_longlong()
    _check(lib().hr2_get_wait_limit(ctx, C.byref(v)), ctx)
    return v.value


def hr2_stream_check(ctx, stream=None):
    """Synchronise the stream; raises Hr2Error(HR2_ETIMEDOUT) if a bounded device wait gave up."""
    _check(lib().hr2_stream_check(ctx, _stream_ptr(stream)), ctx)


def hr2_nodes_from_b(T1: float, b) -> np.ndarray:
    b, pb = _dptr(b)
    out = np.zeros(len(b) + 1)
    _check(lib().hr2_nodes_from_b(len(out), float(T1), pb, out.ctypes.data_as(_DP)))
    return out


def hr2_measure_unit_rate(device: int, kind: int, iters: int) -> dict:
    """Microbenchmark of one arithmetic unit (HR2_UNIT_*): time, operations, rate and the SM clock."""
    r = UnitRate()
    rc = lib().hr2_measure_unit_rate(device, kind, iters, C.byref(r))
    if rc != HR2_OK:
        raise Hr2Error(rc, "hr2_measure_unit_rate(kind=%d) failed" % kind)
    return {"ms": r.ms, "ops": r.ops, "ops_per_s": r.ops_per_s, "sm_ghz": r.sm_ghz,
            "ops_per_clk_sm": r.ops_per_clk_sm, "n_sm": r.n_sm}
