"""Seeded synthetic inputs shaped like the Helios-r2 brown-dwarf workloads.

This module only draws inputs: opacity tables, collision-induced absorption
tables, level/spectral setups, parameter vectors from prior boxes and the
noise of mock observations.  It holds none of the forward model's arithmetic,
so both the CUDA path and the oracle consume exactly the same inputs from it.

Recipe (the paper's line-list tables, SpeX/ISAAC spectra and MultiNest live
points are not available; these stand in for them):

* Cross-section tables, per absorber s, on a T grid linear in T and a grid
  uniform in log10 p:  log10 sigma_s(T_a, p_b, nu) = -22 + 2 z_s(nu)
  + alpha_s ln(T_a / 1000 K) + beta_s log10(p_b / bar) + 0.3 z_{s,a,b}(nu),
  with z unit-variance white noise smoothed along nu by a Gaussian of FWHM
  5 cm^-1, alpha_s ~ U(0.5, 2), beta_s ~ U(0, 0.3).  z_{s,a,b} is a random
  unit-norm mix of four smoothed basis rows of the absorber, so every (T, p)
  row differs while generation stays cheap at 290001 wavenumbers.
* CIA tables (H2-H2, H2-He): log10 k(T, nu) = c0 + 0.5 ln(T / 1000 K)
  - ((nu - nu_c) / (0.6 W))^2 in cm^5, nu_c the band centre, W its width.
* Parameters: log g, log10 VMRs, calibration factor f uniform in the prior
  box; the finite-element temperatures from T_1 ~ U(1000, 3000) K and
  b_i ~ U(0.3, 0.95) (Table 1), or independent random control points.
* Mock observations: D = D_m(theta_true) + N(0, s^2), s = 0.2 x median(D_m)
  (Sect. 4.1), D_m computed by whichever side consumes the observation.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional

import numpy as np

NPARAM = 38
P_LOGG, P_F, P_DIST, P_T0, P_X0, P_CLOUD = 0, 1, 2, 3, 19, 35
MAX_TNODES = 16
MAX_SPECIES = 16

R_JUPITER_CM = 7.1492e9
BASE_SEED = 1910010700

# Molecular masses (u) of the absorbers named in Sect. 2.3, used in order.
ABSORBER_MASSES = [18.015, 16.043, 28.010, 44.009, 17.031, 34.081, 39.098, 22.990,
                   18.015, 16.043, 28.010, 44.009, 17.031, 34.081, 39.098, 22.990]


@dataclasses.dataclass
class TableSpec:
    n_species: int
    T_grid: np.ndarray          # K, ascending
    log10p_grid: np.ndarray     # log10(p / bar), ascending
    nu0: float                  # cm^-1
    dnu: float                  # cm^-1
    n_nu: int
    seed: int
    cia: bool = True

    @property
    def nu(self) -> np.ndarray:
        return self.nu0 + np.arange(self.n_nu, dtype=np.float64) * self.dnu

    @property
    def masses(self) -> np.ndarray:
        return np.asarray(ABSORBER_MASSES[: self.n_species], dtype=np.float64)


@dataclasses.dataclass
class SetupSpec:
    nu_first: int               # first table index used
    n_nu: int                   # number of wavenumber points
    n_layers: int               # L layers, L+1 levels
    species: List[int]          # table indices of the absorbers used
    n_mu: int                   # Gauss angle nodes
    fe_elements: int
    fe_order: int
    resolving_power: float      # <= 0: no instrument profile
    bin_edges: np.ndarray       # cm^-1, n_bins+1
    p_top: float = 1e-4         # bar
    p_bot: float = 100.0        # bar
    r_he: float = 0.17          # n_He / n_H2
    radius_cm: float = R_JUPITER_CM
    interp: str = "log10"       # opacity interpolation space: "log10" or "linear"
    profile: str = "fe"         # temperature profile: "fe" (finite elements) or "milne"
    cloud: bool = False         # gray cloud layer from parameters 35..37
    sc: str = "linear"          # short characteristics: "linear" or "parabolic" source

    @property
    def n_bins(self) -> int:
        return len(self.bin_edges) - 1

    @property
    def n_tnodes(self) -> int:
        """Temperature parameters: the FE nodes, or (Tbar_eff, log10 kappa_R) for Milne's profile."""
        return 2 if self.profile == "milne" else self.fe_elements * self.fe_order + 1

    def as_dict(self) -> Dict:
        return dataclasses.asdict(self)


def _smooth_rows(rng: np.random.Generator, n_rows: int, n: int, fwhm_pts: float) -> np.ndarray:
    """Unit-variance white noise smoothed along the last axis (FFT, periodic)."""
    sig = fwhm_pts / 2.3548200450309493
    white = rng.standard_normal((n_rows, n))
    freq = np.fft.rfftfreq(n)
    kern = np.exp(-2.0 * (np.pi * freq * sig) ** 2)
    sm = np.fft.irfft(np.fft.rfft(white, axis=-1) * kern, n=n, axis=-1)
    sm -= sm.mean(axis=-1, keepdims=True)
    sm /= sm.std(axis=-1, keepdims=True)
    return sm


def species_table(spec: TableSpec, s: int) -> np.ndarray:
    """log10 cross-section table of absorber s, shape [n_T][n_p][n_nu] float64."""
    rng = np.random.default_rng([spec.seed, 1, s])
    fwhm_pts = 5.0 / spec.dnu
    base = _smooth_rows(rng, 5, spec.n_nu, fwhm_pts)     # z_s and four basis rows
    alpha = rng.uniform(0.5, 2.0)
    beta = rng.uniform(0.0, 0.3)
    nT, nP = len(spec.T_grid), len(spec.log10p_grid)
    mix = rng.standard_normal((nT, nP, 4))
    mix /= np.linalg.norm(mix, axis=-1, keepdims=True)
    out = np.empty((nT, nP, spec.n_nu))
    for a in range(nT):
        for b in range(nP):
            row = mix[a, b] @ base[1:]
            out[a, b] = (-22.0 + 2.0 * base[0] + alpha * np.log(spec.T_grid[a] / 1000.0)
                         + beta * spec.log10p_grid[b] + 0.3 * row)
    return out


def cia_tables(spec: TableSpec):
    """(H2-H2, H2-He) log10 CIA tables [n_T][n_nu] in cm^5, or (None, None)."""
    if not spec.cia:
        return None, None
    nu = spec.nu
    width = max(nu[-1] - nu[0], spec.dnu)
    out = []
    for c0, centre_frac in ((-46.0, 0.35), (-46.5, 0.55)):
        nuc = nu[0] + centre_frac * width
        lt = 0.5 * np.log(spec.T_grid / 1000.0)
        out.append(c0 + lt[:, None] - ((nu[None, :] - nuc) / (0.6 * width)) ** 2)
    return out[0], out[1]


def make_tables(spec: TableSpec) -> Dict:
    """All tables as float64 arrays (the unquantised values)."""
    sig = np.stack([species_table(spec, s) for s in range(spec.n_species)])
    h2h2, h2he = cia_tables(spec)
    return dict(T_grid=np.asarray(spec.T_grid, float), log10p_grid=np.asarray(spec.log10p_grid, float),
                nu0=spec.nu0, dnu=spec.dnu, log10_sigma=sig, log10_cia_h2h2=h2h2,
                log10_cia_h2he=h2he, species_mass=spec.masses)


def log_uniform_edges(nu_lo: float, nu_hi: float, n_bins: int) -> np.ndarray:
    """Observational bin edges uniform in ln(nu) spanning [nu_lo, nu_hi]."""
    e = np.exp(np.linspace(np.log(nu_lo), np.log(nu_hi), n_bins + 1))
    e[0], e[-1] = nu_lo, nu_hi
    return e


def make_setup(spec: TableSpec, nu_lo: float, nu_hi: float, n_layers: int, species, n_mu: int,
               fe_elements: int, fe_order: int, resolving_power: float, n_bins: int) -> SetupSpec:
    first = int(round((nu_lo - spec.nu0) / spec.dnu))
    last = int(round((nu_hi - spec.nu0) / spec.dnu))
    n = last - first + 1
    lo = spec.nu0 + first * spec.dnu
    hi = spec.nu0 + last * spec.dnu
    return SetupSpec(nu_first=first, n_nu=n, n_layers=n_layers, species=list(species), n_mu=n_mu,
                     fe_elements=fe_elements, fe_order=fe_order, resolving_power=resolving_power,
                     bin_edges=log_uniform_edges(lo, hi, n_bins))


@dataclasses.dataclass
class Prior:
    log_g: tuple = (4.0, 5.5)
    log_x: tuple = (-8.0, -2.0)
    f: tuple = (0.5, 2.0)
    T1: tuple = (1000.0, 3000.0)
    b: tuple = (0.3, 0.95)
    dist_pc: float = 10.0
    free_nodes: Optional[tuple] = None   # (Tmin, Tmax): independent control points instead of (T1, b)
    t_bar: tuple = (400.0, 2000.0)       # Milne profile: Tbar_eff, K
    log_kappa: tuple = (-4.0, 0.0)       # Milne profile: log10 kappa_R, cm^2 g^-1
    log_tau_cloud: tuple = (-2.0, 1.0)   # gray cloud: log10 optical depth
    log_p_cloud: tuple = (-3.0, 1.0)     # gray cloud: log10 top pressure, bar
    log_f_cloud: tuple = (-1.5, 0.0)     # gray cloud: log10 (top / bottom pressure)


def draw_params(setup: SetupSpec, n: int, seed: int, prior: Prior = Prior()) -> np.ndarray:
    """Parameter vectors [n][NPARAM] drawn uniformly from the prior box."""
    rng = np.random.default_rng([seed, 2])
    th = np.zeros((n, NPARAM))
    th[:, P_LOGG] = rng.uniform(*prior.log_g, n)
    th[:, P_F] = rng.uniform(*prior.f, n)
    th[:, P_DIST] = prior.dist_pc
    nt = setup.n_tnodes
    if setup.profile == "milne":
        th[:, P_T0] = rng.uniform(*prior.t_bar, n)
        th[:, P_T0 + 1] = rng.uniform(*prior.log_kappa, n)
    elif prior.free_nodes is not None:
        th[:, P_T0:P_T0 + nt] = rng.uniform(*prior.free_nodes, (n, nt))
    else:
        T1 = rng.uniform(*prior.T1, n)
        b = rng.uniform(*prior.b, (n, nt - 1))
        nodes = np.empty((n, nt))
        nodes[:, 0] = T1
        for i in range(1, nt):
            nodes[:, i] = nodes[:, i - 1] * b[:, i - 1]
        th[:, P_T0:P_T0 + nt] = nodes
    k = len(setup.species)
    th[:, P_X0:P_X0 + k] = rng.uniform(*prior.log_x, (n, k))
    if setup.cloud:
        th[:, P_CLOUD] = rng.uniform(*prior.log_tau_cloud, n)
        th[:, P_CLOUD + 1] = rng.uniform(*prior.log_p_cloud, n)
        th[:, P_CLOUD + 2] = rng.uniform(*prior.log_f_cloud, n)
    return th


def noise_draws(n_bins: int, seed: int) -> np.ndarray:
    """Standard-normal draws for the mock observation of one setup."""
    return np.random.default_rng([seed, 3]).standard_normal(n_bins)


def mock_observation(model_bins: np.ndarray, seed: int, noise_frac: float = 0.2):
    """(D, sigma): model bins plus Gaussian noise of sd noise_frac x median (Sect. 4.1)."""
    model_bins = np.asarray(model_bins, dtype=np.float64)
    s = noise_frac * float(np.median(model_bins))
    sigma = np.full(model_bins.shape, s)
    return model_bins + s * noise_draws(len(model_bins), seed), sigma


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    table: TableSpec
    setups: List[SetupSpec]
    n_samples: int
    prior: Prior
    seed: int
    storage: str = "fp16"          # "fp16" or "fp64"
    setup_weights: Optional[List[float]] = None

    def params(self, n: Optional[int] = None, seed_offset: int = 0):
        """(theta [n][NPARAM], setup index per sample) for a batch."""
        n = self.n_samples if n is None else n
        rng = np.random.default_rng([self.seed + seed_offset, 4])
        if len(self.setups) == 1:
            sid = np.zeros(n, dtype=np.int32)
        else:
            w = np.asarray(self.setup_weights or [1.0] * len(self.setups), float)
            sid = rng.choice(len(self.setups), size=n, p=w / w.sum()).astype(np.int32)
        theta = np.zeros((n, NPARAM))
        for g, st in enumerate(self.setups):
            idx = np.nonzero(sid == g)[0]
            if len(idx):
                theta[idx] = draw_params(st, len(idx), self.seed + seed_offset * 131 + g, self.prior)
        return theta, sid

    def truth(self, g: int = 0) -> np.ndarray:
        """The "true" parameter vector of setup g for the mock observation: a
        late-T-dwarf-like atmosphere as in the paper's test case (Sect. 4:
        log g = 4.75, f = 1, d = 10 pc), a monotonic profile from 2200 K at the
        bottom to 500 K at the top, and log10 mixing ratios of -3.5.  A workload
        whose prior fixes nodes independently draws them from that prior."""
        st = self.setups[g]
        if self.prior.free_nodes is not None:
            return draw_params(st, 1, self.seed + 7919 + g, self.prior)[0]
        th = np.zeros(NPARAM)
        th[P_LOGG], th[P_F], th[P_DIST] = 4.75, 1.0, self.prior.dist_pc
        nt = st.n_tnodes
        th[P_T0:P_T0 + nt] = 2200.0 * (500.0 / 2200.0) ** (np.arange(nt) / (nt - 1))
        th[P_X0:P_X0 + len(st.species)] = -3.5
        return th


def _grid_T(n: int) -> np.ndarray:
    return np.linspace(200.0, 3000.0, n)


def _grid_logp(n: int) -> np.ndarray:
    return np.linspace(-4.0, 2.0, n)


def single_l50_k1_nu6001() -> Workload:
    """One model: 50 layers, 1 absorber, 6001 points 4000-10000 cm^-1, R=200, 150 bins."""
    seed = BASE_SEED + 0
    t = TableSpec(1, _grid_T(12), _grid_logp(8), 4000.0, 1.0, 6001, seed)
    s = make_setup(t, 4000.0, 10000.0, 50, [0], 3, 4, 1, 200.0, 150)
    prior = Prior(log_g=(4.75, 4.75), log_x=(-3.0, -3.0), f=(1.0, 1.0), free_nodes=(500.0, 2000.0))
    return Workload("single_l50_k1_nu6001", t, [s], 1, prior, seed, storage="fp64")


def batch1024_l100_k6_nu8501(storage: str = "fp16") -> Workload:
    """1024 samples: 100 layers, 6 absorbers, 8501 points 4000-12500 cm^-1, 4 nodes, R=300, 300 bins."""
    seed = BASE_SEED + 1
    t = TableSpec(6, _grid_T(20), _grid_logp(15), 4000.0, 1.0, 8501, seed)
    s = make_setup(t, 4000.0, 12500.0, 100, range(6), 4, 3, 2, 300.0, 300)
    return Workload("batch1024_l100_k6_nu8501", t, [s], 1024, Prior(), seed, storage=storage)


def uneven2048_3setups() -> Workload:
    """2048 samples over three spectral setups (4000-12500 R=300, 1500-6000 R=100,
    6000-16000 R=1000), 80-120 layers and 6-10 absorbers varying per setup variant."""
    seed = BASE_SEED + 2
    t = TableSpec(10, _grid_T(20), _grid_logp(15), 1500.0, 1.0, 14501, seed)
    rng = np.random.default_rng([seed, 5])
    setups = []
    for (lo, hi, R, nb) in ((4000.0, 12500.0, 300.0, 300), (1500.0, 6000.0, 100.0, 139),
                            (6000.0, 16000.0, 1000.0, 981)):
        for _ in range(4):
            L = int(rng.integers(80, 121))
            K = int(rng.integers(6, 11))
            sp = sorted(rng.choice(10, size=K, replace=False).tolist())
            setups.append(make_setup(t, lo, hi, L, sp, 4, 3, 2, R, nb))
    return Workload("uneven2048_3setups", t, setups, 2048, Prior(), seed)


def large_l100_k12_nu290001_b256(n_nu: int = 290001) -> Workload:
    """256 samples on 0.1 cm^-1 tables over 1000-30000 cm^-1 (290001 points), 12 absorbers,
    100 layers, 8 nodes, R=1000, 2000 bins.  A smaller n_nu keeps the same grid from
    1000 cm^-1 up (for captures that must hold only a few GB)."""
    seed = BASE_SEED + 4
    t = TableSpec(12, _grid_T(20), _grid_logp(15), 1000.0, 0.1, n_nu, seed)
    s = make_setup(t, 1000.0, 1000.0 + 0.1 * (n_nu - 1), 100, range(12), 8, 3, 2, 1000.0, 2000)
    name = "large_l100_k12_nu%d_b256" % n_nu
    return Workload(name, t, [s], 256, Prior(), seed)


def tiny(n_nu: int = 16, n_layers: int = 3, n_species: int = 2, n_T: int = 3, n_p: int = 3,
         n_mu: int = 2, resolving_power: float = 0.0, n_bins: int = 4, seed: int = 11) -> Workload:
    """A tiny grid for brute-force comparisons and ragged-tail cases."""
    t = TableSpec(n_species, np.linspace(300.0, 2500.0, n_T), np.linspace(-4.0, 2.0, n_p),
                  5000.0, 1.0, n_nu, BASE_SEED + 100 + seed)
    s = make_setup(t, 5000.0, 5000.0 + n_nu - 1, n_layers, range(n_species), n_mu, 2, 1,
                   resolving_power, n_bins)
    return Workload("tiny", t, [s], 4, Prior(), BASE_SEED + 100 + seed)


WORKLOADS = {
    "single_l50_k1_nu6001": single_l50_k1_nu6001,
    "batch1024_l100_k6_nu8501": batch1024_l100_k6_nu8501,
    "uneven2048_3setups": uneven2048_3setups,
    "large_l100_k12_nu290001_b256": large_l100_k12_nu290001_b256,
}
