"""Plain double-precision CPU oracle of the Helios-r2 emission forward model.

TEST INFRASTRUCTURE ONLY.  The oracle is the independent reference that the
CUDA library is checked against (Kitzmann et al. 2020, Sects. 2-3).  Only the
test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA path: the C
source ``hr2_oracle.c`` is compiled on its own with gcc (no fast-math, no FMA
contraction) and loaded here through ctypes.

Functions and the readings of the paper they follow are documented in the C
source.  This module only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hr2_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_LOCK = threading.Lock()
_LIB = None

NPARAM = 38
P_LOGG, P_F, P_DIST, P_T0, P_X0 = 0, 1, 2, 3, 19


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class _Model(C.Structure):
    _fields_ = [
        ("n_species_tab", C.c_int), ("n_T", C.c_int), ("n_p", C.c_int), ("n_nu_tab", C.c_int),
        ("T_grid", C.POINTER(C.c_double)), ("log10p_grid", C.POINTER(C.c_double)),
        ("nu0", C.c_double), ("dnu", C.c_double),
        ("log10_sigma", C.POINTER(C.c_double)),
        ("log10_cia_h2h2", C.POINTER(C.c_double)), ("log10_cia_h2he", C.POINTER(C.c_double)),
        ("species_mass", C.POINTER(C.c_double)),
        ("nu_first", C.c_int), ("n_nu", C.c_int), ("n_layers", C.c_int),
        ("p_top", C.c_double), ("p_bot", C.c_double),
        ("n_used", C.c_int), ("species", C.POINTER(C.c_int)),
        ("n_mu", C.c_int), ("fe_elements", C.c_int), ("fe_order", C.c_int),
        ("resolving_power", C.c_double), ("n_bins", C.c_int), ("bin_edges", C.POINTER(C.c_double)),
        ("r_he", C.c_double), ("radius_cm", C.c_double), ("interp", C.c_int),
        ("profile", C.c_int), ("n_hopf", C.c_int), ("hopf_tau", C.POINTER(C.c_double)),
        ("hopf_q", C.POINTER(C.c_double)), ("cloud", C.c_int), ("sc_order", C.c_int),
    ]

# short-characteristics source interpolation (Sect. 2.1)
SC_ORDER = {"linear": 1, "parabolic": 2}

# temperature profile of the setup (Sect. 2.5)
PROFILE = {"fe": 0, "milne": 1}

# interpolation space of the opacity tables (a setup option)
INTERP = {"log10": 0, "linear": 1}


_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int)


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = C.CDLL(build())
            M = C.POINTER(_Model)
            sig = {
                "or_gauss_legendre01": (C.c_int, [C.c_int, _DP, _DP]),
                "or_gauss_lobatto01": (C.c_int, [C.c_int, _DP]),
                "or_lagrange": (C.c_double, [C.c_int, _DP, C.c_int, C.c_double]),
                "or_fe_temperature": (C.c_double, [C.c_int, C.c_int, _DP, C.c_double]),
                "or_nodes_from_b": (None, [C.c_int, C.c_double, _DP, _DP]),
                "or_planck": (C.c_double, [C.c_double, C.c_double]),
                "or_sc_intensity": (C.c_double, [C.c_int, _DP, _DP, C.c_double, C.c_double]),
                "or_sc_flux": (C.c_double, [C.c_int, _DP, _DP, C.c_double, C.c_int]),
                "or_sc_intensity_parabolic": (C.c_double, [C.c_int, _DP, _DP, C.c_double, C.c_double]),
                "or_log10_sigma": (C.c_double, [M, C.c_int, C.c_double, C.c_double, C.c_int]),
                "or_sigma": (C.c_double, [M, C.c_int, C.c_double, C.c_double, C.c_int]),
                "or_cia_coeff": (C.c_double, [M, _DP, C.c_double, C.c_int]),
                "or_hopf": (C.c_double, [M, C.c_double]),
                "or_effective_temperature": (C.c_double, [M, _DP]),
                "or_convolve": (None, [M, _DP, _DP]),
                "or_bin": (C.c_int, [M, _DP, _DP]),
                "or_forward": (C.c_int, [M, _DP, _DP, _DP]),
                "or_top_flux_at": (C.c_int, [M, _DP, C.c_int, _IP, _DP]),
                "or_bins_at": (C.c_int, [M, _DP, C.c_int, _IP, _DP]),
                "or_lnL": (C.c_double, [C.c_int, _DP, _DP, _DP, C.c_double]),
                "or_forward_batch": (C.c_int, [M, C.c_int, _DP, _DP, _DP, _IP, C.c_int]),
                "or_level_temperatures": (C.c_int, [M, _DP, _DP]),
                "or_layer_dtau": (C.c_int, [M, _DP, C.c_int, _DP]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = lib
    return _LIB


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_DP)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_IP)


# ---------------------------------------------------------------- quadratures
def gauss_legendre01(n: int):
    mu, w = np.zeros(n), np.zeros(n)
    if _lib().or_gauss_legendre01(n, mu.ctypes.data_as(_DP), w.ctypes.data_as(_DP)) != 0:
        raise ValueError("node count out of range")
    return mu, w


def gauss_lobatto01(npts: int):
    xi = np.zeros(npts)
    if _lib().or_gauss_lobatto01(npts, xi.ctypes.data_as(_DP)) != 0:
        raise ValueError("point count out of range")
    return xi


def lagrange(xi, i: int, x: float) -> float:
    xi, p = _d(xi)
    return _lib().or_lagrange(len(xi), p, i, float(x))


def fe_temperature(n_elements: int, order: int, nodes, x: float) -> float:
    nodes, p = _d(nodes)
    return _lib().or_fe_temperature(n_elements, order, p, float(x))


def nodes_from_b(T1: float, b):
    b, pb = _d(b)
    out = np.zeros(len(b) + 1)
    _lib().or_nodes_from_b(len(out), float(T1), pb, out.ctypes.data_as(_DP))
    return out


def planck(nu, T):
    """Planck function per unit wavenumber (vectorised by a Python loop)."""
    nu_b, T_b = np.broadcast_arrays(np.asarray(nu, float), np.asarray(T, float))
    out = np.empty(nu_b.shape)
    f = _lib().or_planck
    for idx in np.ndindex(nu_b.shape):
        out[idx] = f(float(nu_b[idx]), float(T_b[idx]))
    return out if out.shape else float(out)


def sc_intensity(dtau, S, I_bottom: float, mu: float) -> float:
    dtau, pd = _d(dtau)
    S, ps = _d(S)
    assert len(S) == len(dtau) + 1
    return _lib().or_sc_intensity(len(dtau), pd, ps, float(I_bottom), float(mu))


def sc_intensity_parabolic(dtau, S, I_bottom: float, mu: float) -> float:
    dtau, pd = _d(dtau)
    S, ps = _d(S)
    assert len(S) == len(dtau) + 1
    return _lib().or_sc_intensity_parabolic(len(dtau), pd, ps, float(I_bottom), float(mu))


def sc_flux(dtau, S, I_bottom: float, n_mu: int) -> float:
    dtau, pd = _d(dtau)
    S, ps = _d(S)
    assert len(S) == len(dtau) + 1
    return _lib().or_sc_flux(len(dtau), pd, ps, float(I_bottom), int(n_mu))


def lnL(D, sigma, Dm, log_eps: float = float("nan")) -> float:
    D, pD = _d(D)
    sigma, ps = _d(sigma)
    Dm, pm = _d(Dm)
    return _lib().or_lnL(len(D), pD, ps, pm, float(log_eps))


# ---------------------------------------------------------------- the model
class Model:
    """One spectral/atmospheric setup over one set of (dequantised) tables.

    ``tables`` is a dict with T_grid, log10p_grid, nu0, dnu, log10_sigma
    [K][nT][np][nnu] (float64, already the values the CUDA path stores),
    optional log10_cia_h2h2 / log10_cia_h2he [nT][nnu], species_mass [K].
    ``setup`` is a dict with nu_first, n_nu, n_layers, p_top, p_bot, species,
    n_mu, fe_elements, fe_order, resolving_power, bin_edges, r_he, radius_cm,
    and optionally interp ("log10", the default, or "linear"), profile ("fe", the
    default, or "milne": parameters 3 and 4 are Tbar_eff and log10 kappa_R) and
    cloud (True: a gray cloud layer from parameters 35..37) and sc ("linear", the
    default, or "parabolic" source interpolation in the short characteristics).
    """

    def __init__(self, tables: dict, setup: dict):
        self._keep = []
        m = _Model()

        def keepd(a):
            a, p = _d(a)
            self._keep.append(a)
            return p

        def keepi(a):
            a, p = _i(a)
            self._keep.append(a)
            return p

        sig = np.asarray(tables["log10_sigma"])
        m.n_species_tab, m.n_T, m.n_p, m.n_nu_tab = sig.shape
        m.T_grid = keepd(tables["T_grid"])
        m.log10p_grid = keepd(tables["log10p_grid"])
        m.nu0 = float(tables["nu0"])
        m.dnu = float(tables["dnu"])
        m.log10_sigma = keepd(sig)
        for key in ("log10_cia_h2h2", "log10_cia_h2he"):
            v = tables.get(key)
            setattr(m, key, keepd(v) if v is not None else _DP())
        m.species_mass = keepd(tables["species_mass"])
        m.nu_first = int(setup["nu_first"])
        m.n_nu = int(setup["n_nu"])
        m.n_layers = int(setup["n_layers"])
        m.p_top = float(setup["p_top"])
        m.p_bot = float(setup["p_bot"])
        sp = np.asarray(setup["species"], dtype=np.int32)
        m.n_used = len(sp)
        m.species = keepi(sp)
        m.n_mu = int(setup["n_mu"])
        m.fe_elements = int(setup["fe_elements"])
        m.fe_order = int(setup["fe_order"])
        m.resolving_power = float(setup["resolving_power"])
        edges = np.asarray(setup["bin_edges"], dtype=np.float64)
        m.n_bins = len(edges) - 1
        m.bin_edges = keepd(edges)
        m.r_he = float(setup["r_he"])
        m.radius_cm = float(setup["radius_cm"])
        m.interp = INTERP[setup.get("interp", "log10")]
        m.profile = PROFILE[setup.get("profile", "fe")]
        m.cloud = int(bool(setup.get("cloud", False)))
        m.sc_order = SC_ORDER[setup.get("sc", "linear")]
        if m.profile == PROFILE["milne"]:
            from . import hopf
            ht, hq = hopf.hopf_table()
            m.n_hopf = len(ht)
            m.hopf_tau = keepd(ht)
            m.hopf_q = keepd(hq)
        self.m = m
        self._cia = {key: m_ptr for key, m_ptr in (("h2h2", m.log10_cia_h2h2), ("h2he", m.log10_cia_h2he))}
        self.ref = C.byref(m)
        self.n_bins = m.n_bins
        self.n_nu = m.n_nu
        self.n_layers = m.n_layers
        first = m.nu_first
        self.nu = float(m.nu0) + np.arange(first, first + m.n_nu, dtype=np.float64) * float(m.dnu)

    # single-sample evaluations -------------------------------------------
    def forward(self, theta, want_top: bool = False):
        theta, pt = _d(theta)
        assert theta.shape == (NPARAM,)
        bins = np.zeros(self.n_bins)
        top = np.zeros(self.n_nu) if want_top else None
        ok = _lib().or_forward(self.ref, pt, bins.ctypes.data_as(_DP),
                               top.ctypes.data_as(_DP) if want_top else _DP())
        return (bins, top, bool(ok)) if want_top else (bins, bool(ok))

    def forward_batch(self, theta, want_top: bool = False, n_threads: int = 0):
        theta, pt = _d(theta)
        n = theta.shape[0]
        assert theta.shape == (n, NPARAM)
        bins = np.zeros((n, self.n_bins))
        top = np.zeros((n, self.n_nu)) if want_top else None
        valid = np.zeros(n, dtype=np.int32)
        used = _lib().or_forward_batch(self.ref, n, pt, bins.ctypes.data_as(_DP),
                                       top.ctypes.data_as(_DP) if want_top else _DP(),
                                       valid.ctypes.data_as(_IP), int(n_threads))
        self.last_threads = used
        return bins, top, valid.astype(bool)

    def top_flux_at(self, theta, idx):
        theta, pt = _d(theta)
        idx, pi = _i(idx)
        out = np.zeros(len(idx))
        ok = _lib().or_top_flux_at(self.ref, pt, len(idx), pi, out.ctypes.data_as(_DP))
        return out, bool(ok)

    def bins_at(self, theta, sel):
        theta, pt = _d(theta)
        sel, ps = _i(sel)
        out = np.zeros(len(sel))
        ok = _lib().or_bins_at(self.ref, pt, len(sel), ps, out.ctypes.data_as(_DP))
        return out, bool(ok)

    def level_temperatures(self, theta):
        theta, pt = _d(theta)
        out = np.zeros(self.n_layers + 1)
        ok = _lib().or_level_temperatures(self.ref, pt, out.ctypes.data_as(_DP))
        return out, bool(ok)

    def layer_dtau(self, theta, k: int):
        theta, pt = _d(theta)
        out = np.zeros(self.n_layers)
        ok = _lib().or_layer_dtau(self.ref, pt, int(k), out.ctypes.data_as(_DP))
        return out, bool(ok)

    def log10_sigma(self, s: int, T: float, log10p: float, inu: int) -> float:
        return _lib().or_log10_sigma(self.ref, int(s), float(T), float(log10p), int(inu))

    def hopf(self, tau: float) -> float:
        """q(tau) as the Milne profile uses it (Milne setups only)."""
        assert self.m.profile == PROFILE["milne"]
        return _lib().or_hopf(self.ref, float(tau))

    def effective_temperature(self, theta) -> float:
        """T_eff from F+ integrated over the setup's wavenumbers (Sect. 2.6)."""
        _, top, ok = self.forward(theta, want_top=True)
        top, pt = _d(top)
        return _lib().or_effective_temperature(self.ref, pt) if ok else float("nan")

    def sigma(self, s: int, T: float, log10p: float, inu: int) -> float:
        """Cross-section in the setup's interpolation space."""
        return _lib().or_sigma(self.ref, int(s), float(T), float(log10p), int(inu))

    def cia_coeff(self, pair: str, T: float, inu: int) -> float:
        """CIA coefficient (pair "h2h2" or "h2he") in the setup's interpolation space."""
        return _lib().or_cia_coeff(self.ref, self._cia[pair], float(T), int(inu))

    def convolve(self, F):
        F, pF = _d(F)
        assert F.shape == (self.n_nu,)
        out = np.zeros(self.n_nu)
        _lib().or_convolve(self.ref, pF, out.ctypes.data_as(_DP))
        return out

    def bin(self, F):
        F, pF = _d(F)
        assert F.shape == (self.n_nu,)
        out = np.zeros(self.n_bins)
        _lib().or_bin(self.ref, pF, out.ctypes.data_as(_DP))
        return out
