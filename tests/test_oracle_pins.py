"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, textbook/library routines (numpy Gauss quadrature, scipy E_n and
normal log-pdf, scipy physical constants), invariants, and brute-force
integration of the formal solution on tiny grids.  The choice is such that a
dropped term, a wrong sign or index, or a transposed operand in any step
fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.constants as sc
import scipy.integrate as si
import scipy.special as ss
import scipy.stats as sst

import oracle
from paper_1910_01070_b300 import workloads as W

# Independent cgs constants (scipy's SI CODATA values, converted here).
H = sc.h * 1e7
CL = sc.c * 1e2
KB = sc.k * 1e7
AMU = sc.atomic_mass * 1e3                   # CODATA 2022 here; the oracle uses 2018 (1.4e-9 apart)
SIGMA_SB = sc.Stefan_Boltzmann * 1e3          # erg s^-1 cm^-2 K^-4
PARSEC = sc.parsec * 1e2


def planck_indep(nu, T):
    return 2 * H * CL ** 2 * nu ** 3 / np.expm1(H * CL * nu / (KB * T))


# ------------------------------------------------------------ quadratures
def test_gauss_legendre_two_nodes_closed_form(oracle_lib):
    mu, w = oracle.gauss_legendre01(2)
    assert np.allclose(mu, [0.5 - math.sqrt(3) / 6, 0.5 + math.sqrt(3) / 6], rtol=0, atol=1e-15)
    assert np.allclose(w, [0.5, 0.5], rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", list(range(1, 17)))
def test_gauss_legendre_matches_numpy_and_is_exact(oracle_lib, n):
    mu, w = oracle.gauss_legendre01(n)
    x, wx = np.polynomial.legendre.leggauss(n)
    assert np.allclose(mu, (x + 1) / 2, rtol=0, atol=1e-14)
    assert np.allclose(w, wx / 2, rtol=0, atol=1e-14)
    for k in range(2 * n):                       # exact for degree <= 2n-1
        assert abs(np.sum(w * mu ** k) - 1.0 / (k + 1)) < 1e-13


def test_gauss_lobatto_closed_forms(oracle_lib):
    assert np.allclose(oracle.gauss_lobatto01(2), [0, 1], atol=1e-15)
    assert np.allclose(oracle.gauss_lobatto01(3), [0, 0.5, 1], atol=1e-15)
    a = 1 / math.sqrt(5)
    assert np.allclose(oracle.gauss_lobatto01(4), [0, (1 - a) / 2, (1 + a) / 2, 1], atol=1e-15)
    b = math.sqrt(3 / 7)
    assert np.allclose(oracle.gauss_lobatto01(5), [0, (1 - b) / 2, 0.5, (1 + b) / 2, 1], atol=1e-15)


@pytest.mark.parametrize("npts", [6, 7, 9, 12])
def test_gauss_lobatto_interior_are_roots_of_dP(oracle_lib, npts):
    xi = oracle.gauss_lobatto01(npts)
    N = npts - 1
    c = np.zeros(N + 1)
    c[N] = 1
    roots = np.sort(np.polynomial.legendre.legroots(np.polynomial.legendre.legder(c)))
    assert np.allclose(xi[1:-1], (roots + 1) / 2, atol=1e-13)


def test_lagrange_cardinal_and_partition_of_unity(oracle_lib):
    xi = oracle.gauss_lobatto01(4)
    for i in range(4):
        for j in range(4):
            assert abs(oracle.lagrange(xi, i, xi[j]) - (1.0 if i == j else 0.0)) < 1e-14
    for x in np.linspace(0, 1, 11):
        assert abs(sum(oracle.lagrange(xi, i, x) for i in range(4)) - 1) < 1e-13


# ------------------------------------------------------------ T profile
def _node_positions(Ke, q):
    xi = oracle.gauss_lobatto01(q + 1)
    pos = [0.0]
    for k in range(Ke):
        for i in range(1, q + 1):
            pos.append((k + xi[i]) / Ke)
    return np.array(pos)


@pytest.mark.parametrize("Ke,q", [(1, 1), (4, 1), (3, 2), (2, 3), (4, 4), (6, 1)])
def test_fe_reproduces_polynomials_up_to_order_q(oracle_lib, Ke, q):
    rng = np.random.default_rng(Ke * 10 + q)
    coef = rng.normal(size=q + 1)
    pos = _node_positions(Ke, q)
    assert len(pos) == Ke * q + 1                 # Eq. (16)
    nodes = np.polyval(coef, pos)
    for x in rng.uniform(0, 1, 25):
        assert abs(oracle.fe_temperature(Ke, q, nodes, x) - np.polyval(coef, x)) < 1e-12
    # one degree more is not reproduced (the test would otherwise be vacuous)
    coef2 = np.concatenate([[1.0], np.zeros(q + 1)])
    nodes2 = np.polyval(coef2, pos)
    errs = [abs(oracle.fe_temperature(Ke, q, nodes2, x) - np.polyval(coef2, x)) for x in np.linspace(0.01, 0.99, 50)]
    assert max(errs) > 1e-6


def test_fe_first_order_is_piecewise_linear(oracle_lib):
    nodes = np.array([1800.0, 1400.0, 900.0, 1100.0, 600.0])
    pos = np.linspace(0, 1, 5)
    for x in np.linspace(0, 1, 37):
        assert abs(oracle.fe_temperature(4, 1, nodes, x) - np.interp(x, pos, nodes)) < 1e-10


@pytest.mark.parametrize("Ke,q", [(3, 2), (4, 3)])
def test_fe_continuous_across_elements(oracle_lib, Ke, q):
    rng = np.random.default_rng(5)
    nodes = rng.uniform(500, 2000, Ke * q + 1)
    pos = _node_positions(Ke, q)
    for x, T in zip(pos, nodes):                  # interpolates its nodes
        assert abs(oracle.fe_temperature(Ke, q, nodes, x) - T) < 1e-9
    for k in range(1, Ke):
        xb = k / Ke
        lo = oracle.fe_temperature(Ke, q, nodes, xb - 1e-12)
        hi = oracle.fe_temperature(Ke, q, nodes, xb + 1e-12)
        assert abs(lo - hi) < 1e-6


def test_nodes_from_b(oracle_lib):
    out = oracle.nodes_from_b(2000.0, [0.9, 0.5, 0.8])
    assert np.allclose(out, [2000.0, 1800.0, 900.0, 720.0], rtol=1e-15)


# ------------------------------------------------------------ Planck
@pytest.mark.parametrize("T", [300.0, 1000.0, 2500.0])
def test_planck_integrates_to_stefan_boltzmann(oracle_lib, T):
    f = lambda nu: oracle.planck(nu, T)
    top = 60.0 * T                                # x = 86 at the upper end
    val, _ = si.quad(f, 1e-6, top, limit=400, epsrel=1e-12)
    assert abs(math.pi * val / (SIGMA_SB * T ** 4) - 1) < 1e-8


def test_planck_limits(oracle_lib):
    T = 1500.0
    nu = 1e-3                                     # Rayleigh-Jeans: B = 2 c k T nu^2
    assert abs(oracle.planck(nu, T) / (2 * CL * KB * T * nu ** 2) - 1) < 1e-5
    nu = 40000.0                                  # Wien: B = 2 h c^2 nu^3 e^{-x}
    x = H * CL * nu / (KB * T)
    assert abs(oracle.planck(nu, T) / (2 * H * CL ** 2 * nu ** 3 * math.exp(-x)) - 1) < 1e-12
    for nu in (1000.0, 5000.0, 20000.0):
        assert abs(oracle.planck(nu, T) / planck_indep(nu, T) - 1) < 1e-12


# ------------------------------------------------------------ short characteristics
def test_sc_isothermal_stays_at_planck(oracle_lib):
    rng = np.random.default_rng(1)
    dtau = 10 ** rng.uniform(-9, 3, 60)
    S = np.full(61, 3.7)
    for mu in (0.05, 0.3, 0.7, 1.0):
        assert abs(oracle.sc_intensity(dtau, S, 3.7, mu) - 3.7) < 1e-13
    assert abs(oracle.sc_flux(dtau, S, 3.7, 4) - math.pi * 3.7) < 1e-12


def test_sc_opacity_free_gives_bottom_intensity(oracle_lib):
    S = np.linspace(1, 9, 11)
    for mu in (0.2, 1.0):
        assert oracle.sc_intensity(np.zeros(10), S, 5.5, mu) == 5.5
    assert abs(oracle.sc_flux(np.zeros(10), S, 5.5, 3) - math.pi * 5.5) < 1e-13


@pytest.mark.parametrize("tau", [1e-4, 0.3, 2.0, 15.0])
def test_sc_single_slab_exact(oracle_lib, tau):
    Ib, S = 4.0, 1.5
    for mu in (0.1, 0.5, 1.0):
        t = tau / mu
        exact = Ib * math.exp(-t) + S * (-math.expm1(-t))
        assert abs(oracle.sc_intensity([tau], [S, S], Ib, mu) - exact) < 1e-14 * max(1, exact)
    # the angular integral converges to the E3 form (Eq. 8 exactly integrated)
    F_exact = math.pi * S + 2 * math.pi * (Ib - S) * ss.expn(3, tau)
    assert abs(oracle.sc_flux([tau], [S, S], Ib, 16) / F_exact - 1) < 2e-6


def test_sc_linear_source_exact(oracle_lib):
    rng = np.random.default_rng(2)
    dtau = 10 ** rng.uniform(-3, 0.5, 40)
    tau = np.concatenate([[0.0], np.cumsum(dtau)])
    a, b = 2.0, 0.7
    S = a + b * tau
    for mu in (0.15, 0.6, 1.0):
        Ib = a + b * (tau[-1] + mu)                # diffusion-like bottom intensity
        assert abs(oracle.sc_intensity(dtau, S, Ib, mu) - (a + b * mu)) < 1e-12
    # F = 2 pi int (a + b mu) mu dmu = pi (a + 2b/3): Gauss with n >= 2 is exact.
    # (the bottom intensity depends on mu, so build the flux from intensities)
    for n in (2, 3, 8):
        mu, w = oracle.gauss_legendre01(n)
        F = 2 * math.pi * sum(wk * mk * oracle.sc_intensity(dtau, S, a + b * (tau[-1] + mk), mk)
                              for mk, wk in zip(mu, w))
        assert abs(F - math.pi * (a + 2 * b / 3)) < 1e-11


def _brute_force_intensity(dtau, S, Ib, mu, nsub=20000):
    """Eq. (1) at tau=0 for a piecewise-linear S(tau), by composite Simpson."""
    total = 0.0
    t0 = 0.0
    for l, d in enumerate(dtau):
        t = np.linspace(0.0, d, nsub + 1)
        s = S[l] + (S[l + 1] - S[l]) * t / d
        y = s * np.exp(-(t0 + t) / mu) / mu
        total += si.simpson(y, x=t)
        t0 += d
    return total + Ib * math.exp(-t0 / mu)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sc_matches_brute_force_formal_solution(oracle_lib, seed):
    rng = np.random.default_rng(seed)
    L = int(rng.integers(2, 5))
    dtau = 10 ** rng.uniform(-2, 0.7, L)
    S = rng.uniform(0.5, 5.0, L + 1)
    Ib = rng.uniform(0.5, 5.0)
    for mu in (0.2, 0.55, 1.0):
        bf = _brute_force_intensity(dtau, S, Ib, mu)
        assert abs(oracle.sc_intensity(dtau, S, Ib, mu) - bf) < 1e-10 * max(1.0, bf)


def test_sc_flux_matches_schwarzschild_milne(oracle_lib):
    """Eq. (3): F = 2 pi int S E2 dt (+ 2 pi I_b E3(tau_L)) for piecewise-linear S."""
    rng = np.random.default_rng(3)
    dtau = 10 ** rng.uniform(-1.5, 0.3, 4)
    tau = np.concatenate([[0.0], np.cumsum(dtau)])
    S = rng.uniform(1.0, 4.0, 5)
    Ib = 4.5
    F_sm = 0.0
    for l in range(4):
        f = lambda t, l=l: (S[l] + (S[l + 1] - S[l]) * (t - tau[l]) / dtau[l]) * ss.expn(2, t)
        v, _ = si.quad(f, tau[l], tau[l + 1], epsabs=1e-13, epsrel=1e-12, limit=200)
        F_sm += 2 * math.pi * v
    F_sm += 2 * math.pi * Ib * ss.expn(3, tau[-1])
    assert abs(oracle.sc_flux(dtau, S, Ib, 16) / F_sm - 1) < 1e-4


# ------------------------------------------------------------ model-level pins
def _tiny_model(fill=None, cia=True, n_layers=4, n_mu=3, R=0.0, n_bins=4, n_nu=24, species=(0, 1), n_T=4, n_p=3):
    spec = W.TableSpec(2, np.linspace(400.0, 2400.0, n_T), np.linspace(-4.0, 2.0, n_p), 6000.0, 1.0, n_nu,
                       seed=99, cia=cia)
    tabs = W.make_tables(spec)
    if fill is not None:
        tabs["log10_sigma"] = fill(tabs)
    setup = W.make_setup(spec, 6000.0, 6000.0 + n_nu - 1, n_layers, list(species), n_mu, 2, 1, R, n_bins)
    return oracle.Model(tabs, setup.as_dict()), tabs, setup


def _theta(nodes, logg=4.75, f=1.0, d=10.0, logx=(-3.0, -3.5)):
    th = np.zeros(oracle.NPARAM)
    th[0], th[1], th[2] = logg, f, d
    th[3:3 + len(nodes)] = nodes
    th[19:19 + len(logx)] = logx
    return th


def test_interpolation_exact_at_nodes_and_for_bilinear_fields(oracle_lib):
    m, tabs, _ = _tiny_model()
    T, lp = tabs["T_grid"], tabs["log10p_grid"]
    sig = tabs["log10_sigma"]
    for a in range(len(T)):
        for b in range(len(lp)):
            assert m.log10_sigma(1, T[a], lp[b], 5) == pytest.approx(sig[1, a, b, 5], abs=1e-13)
    c = [-21.0, 1.3e-3, -0.4, 2.0e-4]
    field = lambda t, p: c[0] + c[1] * t + c[2] * p + c[3] * t * p
    m2, _, _ = _tiny_model(fill=lambda tb: np.broadcast_to(
        field(tb["T_grid"][:, None], tb["log10p_grid"][None, :])[None, :, :, None], tb["log10_sigma"].shape).copy())
    rng = np.random.default_rng(4)
    for _ in range(20):
        t, p = rng.uniform(T[0], T[-1]), rng.uniform(lp[0], lp[-1])
        assert m2.log10_sigma(0, t, p, 3) == pytest.approx(field(t, p), abs=1e-12)
    # clamped beyond the grid edges
    assert m2.log10_sigma(0, 50.0, -9.0, 3) == pytest.approx(field(T[0], lp[0]), abs=1e-12)
    assert m2.log10_sigma(0, 9000.0, 5.0, 3) == pytest.approx(field(T[-1], lp[-1]), abs=1e-12)


def test_optical_depth_closed_form_and_scalings(oracle_lib):
    sig0 = -23.0
    m, tabs, setup = _tiny_model(fill=lambda tb: np.full(tb["log10_sigma"].shape, sig0), cia=False,
                                 species=(0,), n_layers=6)
    x = 1e-3
    th = _theta([1500.0, 1200.0, 900.0], logx=(math.log10(x),))
    dtau, ok = m.layer_dtau(th, 3)
    assert ok
    g = 10 ** 4.75
    xh2 = (1 - x) / 1.17
    mmw = x * tabs["species_mass"][0] + xh2 * 2.01588 + 0.17 * xh2 * 4.002602
    p = 10 ** np.linspace(-4, 2, 7) * 1e6
    expect = x * 10 ** sig0 * np.diff(p) / (mmw * AMU * g)
    assert np.allclose(dtau, expect, rtol=1e-8)
    th2 = th.copy()
    th2[0] += math.log10(2.0)
    d2, _ = m.layer_dtau(th2, 3)
    assert np.allclose(d2, dtau / 2, rtol=1e-12)


@pytest.mark.parametrize("sc,cloud", [("linear", False), ("parabolic", False), ("linear", True)])
def test_forward_flux_is_the_composition_of_its_pinned_steps(oracle_lib, sc, cloud):
    """F+ of the forward model at every wavenumber (Eq. 8 over the short
    characteristics of Eqs. 4-7) equals the flux rebuilt here from its steps,
    each pinned on its own: the layer optical depths (closed forms above), the
    level temperatures (profile pins), the Planck source (Eq. 2) written here
    from the exact SI constants, the intensity along each ray (brute force and
    closed forms above), and numpy's Gauss-Legendre nodes mapped to [0, 1].
    A slip in how the forward model itself puts these together -- its own
    optical depth, source or bottom boundary -- fails here even where every
    step passes alone."""
    fill = lambda tb: tb["log10_sigma"] - 1.5                # a mix of thin and thick layers
    m, tabs, setup = _tiny_model(fill=fill, cia=True, n_layers=7, n_mu=4, n_nu=12)
    if sc != "linear" or cloud:
        setup.sc = sc
        setup.cloud = cloud
        m = oracle.Model(tabs, setup.as_dict())
    th = _theta([1700.0, 1250.0, 800.0])
    if cloud:
        th[35], th[36], th[37] = math.log10(2.5), math.log10(0.01), math.log10(0.1)
    _, top, ok = m.forward(th, want_top=True)
    assert ok
    T, _ = m.level_temperatures(th)
    x, w = np.polynomial.legendre.leggauss(setup.n_mu)
    mu, w = 0.5 * (x + 1.0), 0.5 * w
    intensity = oracle.sc_intensity if sc == "linear" else oracle.sc_intensity_parabolic
    saw_thin = saw_thick = False
    for k in range(setup.n_nu):
        dtau, _ = m.layer_dtau(th, k)
        saw_thin |= bool(np.any(dtau < 0.05))
        saw_thick |= bool(np.any(dtau > 1.0))
        nu = tabs["nu0"] + (setup.nu_first + k) * tabs["dnu"]
        S = planck_indep(nu, T)
        F = 2 * math.pi * sum(wk * mk * intensity(dtau, S, S[-1], mk) for wk, mk in zip(w, mu))
        assert top[k] == pytest.approx(F, rel=1e-10)
    assert saw_thin and saw_thick


def test_cia_enters_quadratically_in_h2(oracle_lib):
    m, tabs, _ = _tiny_model(fill=lambda tb: np.full(tb["log10_sigma"].shape, -300.0), cia=True, species=(0,))
    th = _theta([1500.0, 1200.0, 900.0], logx=(math.log10(0.5),))
    th_lo = _theta([1500.0, 1200.0, 900.0], logx=(-12.0,))
    d_half, _ = m.layer_dtau(th, 2)
    d_full, _ = m.layer_dtau(th_lo, 2)
    xh2_half, xh2_full = 0.5 / 1.17, 1.0 / 1.17
    mm = lambda xa, xh: xa * tabs["species_mass"][0] + xh * 2.01588 + 0.17 * xh * 4.002602
    ratio = (xh2_half / xh2_full) ** 2 * mm(1e-12, xh2_full) / mm(0.5, xh2_half)
    assert np.allclose(d_half / d_full, ratio, rtol=1e-7)


def test_isothermal_atmosphere_radiates_planck(oracle_lib):
    m, tabs, setup = _tiny_model(n_layers=8)
    th = _theta([1234.0, 1234.0, 1234.0])
    _, top, ok = m.forward(th, want_top=True)
    assert ok
    assert np.allclose(top, math.pi * planck_indep(m.nu, 1234.0), rtol=1e-12)


def test_opacity_free_atmosphere_shows_bottom(oracle_lib):
    m, tabs, setup = _tiny_model(fill=lambda tb: np.full(tb["log10_sigma"].shape, -300.0), cia=False)
    th = _theta([1900.0, 1200.0, 700.0])
    _, top, ok = m.forward(th, want_top=True)
    assert np.allclose(top, math.pi * planck_indep(m.nu, 1900.0), rtol=1e-12)


def test_optically_thick_isothermal_deep_layers(oracle_lib):
    """Very opaque table: the emergent flux comes from the top layers only."""
    m, tabs, setup = _tiny_model(fill=lambda tb: np.full(tb["log10_sigma"].shape, -15.0), cia=False, n_layers=10)
    th = _theta([2500.0, 700.0, 700.0])           # upper half isothermal at 700 K
    _, top, ok = m.forward(th, want_top=True)
    assert np.allclose(top, math.pi * planck_indep(m.nu, 700.0), rtol=1e-9)


def test_radius_distance_scaling(oracle_lib):
    m, tabs, setup = _tiny_model()
    th = _theta([1600.0, 1100.0, 800.0])
    b1, _ = m.forward(th)
    th2 = th.copy()
    th2[1], th2[2] = 2.5, 20.0
    b2, _ = m.forward(th2)
    assert np.allclose(b2 / b1, 2.5 / 4.0, rtol=1e-13)
    _, top, _ = m.forward(th, want_top=True)
    scale = (W.R_JUPITER_CM / (10.0 * PARSEC)) ** 2
    assert np.allclose(m.bin(top * scale), b1, rtol=1e-12)   # R <= 0: bins of scaled F+


def test_convolution_invariants(oracle_lib):
    m, _, _ = _tiny_model(R=800.0, n_nu=400, n_bins=10)
    nu = m.nu
    assert np.allclose(m.convolve(np.full(len(nu), 3.0)), 3.0, rtol=1e-14)
    lin = 2.0 + 1e-3 * (nu - nu[0])
    out = m.convolve(lin)
    sig = nu / (800.0 * 2 * math.sqrt(2 * math.log(2)))
    inner = (nu - 5 * sig > nu[0] + 1) & (nu + 5 * sig < nu[-1] - 1)
    assert inner.sum() > 100
    assert np.allclose(out[inner], lin[inner], rtol=1e-12)
    # Gaussian line of sd s0 -> sd sqrt(s0^2 + sigma^2) near the centre
    c = nu[200]
    s0 = 3.0
    line = np.exp(-0.5 * ((nu - c) / s0) ** 2)
    out = m.convolve(line)
    s_tot = math.sqrt(s0 ** 2 + sig[200] ** 2)
    assert out[200] == pytest.approx(s0 / s_tot, rel=2e-3)


def test_binning_means(oracle_lib):
    m, _, setup = _tiny_model(n_nu=24, n_bins=4)
    nu = m.nu
    F = nu.copy()
    bins = m.bin(F)
    e = setup.bin_edges
    for b in range(4):
        sel = (nu >= e[b]) & ((nu < e[b + 1]) if b < 3 else (nu <= e[b + 1]))
        assert bins[b] == pytest.approx(F[sel].mean(), rel=1e-15)
    assert np.isclose(np.sum([((nu >= e[b]) & (nu < e[b + 1])).sum() for b in range(3)]) +
                      ((nu >= e[3]) & (nu <= e[4])).sum(), len(nu))


def test_lnL_against_normal_logpdf(oracle_lib):
    rng = np.random.default_rng(6)
    Dm = rng.uniform(1, 2, 50)
    sigma = rng.uniform(0.05, 0.2, 50)
    D = Dm + sigma * rng.standard_normal(50)
    assert oracle.lnL(D, sigma, Dm) == pytest.approx(sst.norm.logpdf(D, Dm, sigma).sum(), rel=1e-13)
    eps = -2.3
    s = np.sqrt(sigma ** 2 + 10 ** eps)
    assert oracle.lnL(D, sigma, Dm, eps) == pytest.approx(sst.norm.logpdf(D, Dm, s).sum(), rel=1e-13)
    assert oracle.lnL(Dm, sigma, Dm) == pytest.approx(-0.5 * np.sum(np.log(2 * np.pi * sigma ** 2)), rel=1e-14)
    c = 0.01
    assert oracle.lnL(Dm + c, sigma, Dm) == pytest.approx(
        -c * c * np.sum(1 / (2 * sigma ** 2)) - 0.5 * np.sum(np.log(2 * np.pi * sigma ** 2)), rel=1e-13)
    bad = Dm.copy()
    bad[3] = np.nan
    assert oracle.lnL(D, sigma, bad) == -np.inf


def test_invalid_samples_flagged(oracle_lib):
    m, _, _ = _tiny_model()
    for th in (_theta([1500.0, -5.0, 800.0]), _theta([1500.0, 1000.0, 800.0], f=0.0),
               _theta([1500.0, 1000.0, 800.0], logx=(-0.1, -0.2))):
        bins, ok = m.forward(th)
        assert not ok and np.all(np.isnan(bins))


def test_level_count_convergence(oracle_lib):
    """More levels than ~70 change the spectrum little (Sect. 2)."""
    spec = W.TableSpec(1, np.linspace(200, 3000, 12), np.linspace(-4, 2, 8), 4000.0, 1.0, 301, seed=3)
    tabs = W.make_tables(spec)
    th = _theta([2000.0, 1600.0, 1100.0, 900.0, 700.0], logx=(-3.0,))
    out = []
    for L in (69, 139, 278):
        s = W.make_setup(spec, 4000.0, 4300.0, L, [0], 2, 4, 1, 0.0, 10)
        out.append(oracle.Model(tabs, s.as_dict()).forward(th)[0])
    d1 = np.max(np.abs(out[1] / out[0] - 1))
    d2 = np.max(np.abs(out[2] / out[1] - 1))
    assert d1 < 2e-2 and d2 < d1 / 2               # converging with level count


def test_generators_are_seeded(oracle_lib):
    wl = W.batch1024_l100_k6_nu8501()
    a, sa = wl.params(16)
    b, sb = wl.params(16)
    assert np.array_equal(a, b) and np.array_equal(sa, sb)
    t1 = W.species_table(W.tiny().table, 1)
    t2 = W.species_table(W.tiny().table, 1)
    assert np.array_equal(t1, t2)


def test_level_temperatures_follow_profile_direction(oracle_lib):
    """Level 0 is the top (p_top), level L the bottom; the first node is the bottom T."""
    m, tabs, setup = _tiny_model(n_layers=10)
    nodes = [2000.0, 1500.0, 800.0]               # 2 linear elements, bottom first
    T, ok = m.level_temperatures(_theta(nodes))
    assert ok
    logp = np.linspace(-4.0, 2.0, 11)             # levels equidistant in log p, top first
    x = (2.0 - logp) / 6.0                        # 0 at the bottom, 1 at the top
    assert np.allclose(T, np.interp(x, [0, 0.5, 1], nodes), rtol=1e-13)
    assert T[0] == pytest.approx(800.0) and T[-1] == pytest.approx(2000.0)


def test_optical_depth_is_trapezoid_of_level_coefficients(oracle_lib):
    c = [-24.0, 4e-4, 0.35]                       # log10 sigma linear in T and log10 p
    field = lambda t, p: c[0] + c[1] * t + c[2] * p
    m, tabs, setup = _tiny_model(fill=lambda tb: np.broadcast_to(
        field(tb["T_grid"][:, None], tb["log10p_grid"][None, :])[None, :, :, None], tb["log10_sigma"].shape).copy(),
        cia=False, species=(0,), n_layers=7)
    x = 10 ** -2.5
    th = _theta([2000.0, 1300.0, 900.0], logx=(math.log10(x),))
    dtau, _ = m.layer_dtau(th, 4)
    T, _ = m.level_temperatures(th)
    logp = np.linspace(-4.0, 2.0, 8)
    chi = x * 10 ** field(T, logp)
    xh2 = (1 - x) / 1.17
    mmw = x * tabs["species_mass"][0] + xh2 * 2.01588 + 0.17 * xh2 * 4.002602
    p = 10 ** logp * 1e6
    expect = 0.5 * (chi[:-1] + chi[1:]) * np.diff(p) / (mmw * AMU * 10 ** 4.75)
    assert np.allclose(dtau, expect, rtol=1e-8)


@pytest.mark.parametrize("which", ["h2h2", "h2he"])
def test_each_cia_pair_closed_form(oracle_lib, which):
    spec = W.TableSpec(1, np.linspace(400.0, 2400.0, 4), np.linspace(-4.0, 2.0, 3), 6000.0, 1.0, 8, seed=5)
    tabs = W.make_tables(spec)
    tabs["log10_sigma"] = np.full(tabs["log10_sigma"].shape, -300.0)
    k0 = -45.0
    tabs["log10_cia_h2h2"] = np.full((4, 8), k0) if which == "h2h2" else None
    tabs["log10_cia_h2he"] = np.full((4, 8), k0) if which == "h2he" else None
    setup = W.make_setup(spec, 6000.0, 6007.0, 5, [0], 2, 1, 1, 0.0, 2)
    m = oracle.Model(tabs, setup.as_dict())
    x = 1e-3
    Tiso = 1100.0
    th = _theta([Tiso, Tiso], logx=(math.log10(x),))
    dtau, _ = m.layer_dtau(th, 3)
    xh2 = (1 - x) / 1.17
    xhe = 0.17 * xh2
    pair = xh2 * xh2 if which == "h2h2" else xh2 * xhe
    mmw = x * tabs["species_mass"][0] + xh2 * 2.01588 + xhe * 4.002602
    p = 10 ** np.linspace(-4.0, 2.0, 6) * 1e6
    chi = pair * (p / (KB * Tiso)) * 10 ** k0
    expect = 0.5 * (chi[:-1] + chi[1:]) * np.diff(p) / (mmw * AMU * 10 ** 4.75)
    assert np.allclose(dtau, expect, rtol=1e-8)


def test_several_absorbers_through_a_species_map_closed_form(oracle_lib):
    """Sects. 2.3, 2.8: chi is the sum over the setup's absorbers of x_s times
    the cross-section of the TABLE species the setup maps s to, and the mean
    molecular weight sums x_s times that table species' mass.  Three table
    species with different constant cross-sections and masses, used through
    the non-identity map [2, 0]; abundances large and unequal, so that using
    one absorber's x for all, the setup index instead of the table index (for
    sigma or for the mass), or dropping an absorber changes dtau far beyond
    1e-8."""
    spec = W.TableSpec(3, np.linspace(400.0, 2400.0, 4), np.linspace(-4.0, 2.0, 3), 6000.0, 1.0, 8, seed=5,
                       cia=False)
    tabs = W.make_tables(spec)
    lsig = np.array([-22.0, -25.0, -23.5])
    tabs["log10_sigma"] = np.broadcast_to(lsig[:, None, None, None], tabs["log10_sigma"].shape).copy()
    tabs["species_mass"] = np.array([10.0, 60.0, 250.0])
    setup = W.make_setup(spec, 6000.0, 6007.0, 5, [2, 0], 2, 1, 1, 0.0, 2)
    m = oracle.Model(tabs, setup.as_dict())
    x = np.array([0.04, 0.15])                    # setup absorbers 0 (table 2) and 1 (table 0)
    th = _theta([1300.0, 900.0], logx=tuple(np.log10(x)))
    dtau, ok = m.layer_dtau(th, 3)
    assert ok
    xh2 = (1 - x.sum()) / 1.17
    mmw = x[0] * 250.0 + x[1] * 10.0 + xh2 * 2.01588 + 0.17 * xh2 * 4.002602
    chi = x[0] * 10 ** lsig[2] + x[1] * 10 ** lsig[0]
    p = 10 ** np.linspace(-4.0, 2.0, 6) * 1e6
    expect = chi * np.diff(p) / (mmw * AMU * 10 ** 4.75)
    assert np.allclose(dtau, expect, rtol=1e-8)


def test_abundances_and_gravity_scaled_together_leave_the_spectrum(oracle_lib):
    """Sects. 2.3, 2.8 with hydrostatic columns: dtau is proportional to
    x_s / (mmw g).  When every absorber has the mass of the H2/He fill,
    mmw does not depend on the abundances, so scaling all x_s and g by the
    same factor leaves every layer's optical depth, and so the spectrum,
    unchanged (no CIA, whose x_H2^2 term would break it)."""
    spec = W.TableSpec(3, np.linspace(400.0, 2400.0, 4), np.linspace(-4.0, 2.0, 3), 6000.0, 1.0, 24, seed=8,
                       cia=False)
    tabs = W.make_tables(spec)
    m_fill = (2.01588 + 0.17 * 4.002602) / 1.17
    tabs["species_mass"] = np.full(3, m_fill)
    setup = W.make_setup(spec, 6000.0, 6023.0, 6, [1, 2, 0], 3, 2, 1, 0.0, 4)
    m = oracle.Model(tabs, setup.as_dict())
    logx = (-3.1, -4.4, -2.6)
    th = _theta([1900.0, 1400.0, 800.0], logx=logx)
    th2 = _theta([1900.0, 1400.0, 800.0], logg=4.75 + math.log10(3.0), logx=tuple(v + math.log10(3.0) for v in logx))
    _, top, ok = m.forward(th, want_top=True)
    _, top2, ok2 = m.forward(th2, want_top=True)
    assert ok and ok2
    assert np.allclose(top2, top, rtol=1e-12)
    d1, _ = m.layer_dtau(th, 7)
    d2, _ = m.layer_dtau(th2, 7)
    assert np.allclose(d2, d1, rtol=1e-12)
    # the same scaling of one absorber only does change the optical depth
    th3 = th.copy()
    th3[19] += math.log10(3.0)
    d3, _ = m.layer_dtau(th3, 7)
    assert not np.allclose(d3, d1, rtol=1e-3)


def test_log10_cia_interpolated_linearly_in_temperature(oracle_lib):
    """Sect. 2.8, reading R3 applied to CIA: log10 k is interpolated linearly
    in T.  Tables with log10 k(T) = a + b T (different for the two pairs) are
    then reproduced exactly between the T nodes, so on a profile whose levels
    fall between nodes, dtau is the trapezoid of
    x_H2^2 n 10^(a0 + b0 T) + x_H2 x_He n 10^(a1 + b1 T); swapped cell
    weights or swapped pairs fail."""
    spec = W.TableSpec(1, np.linspace(400.0, 2400.0, 5), np.linspace(-4.0, 2.0, 3), 6000.0, 1.0, 8, seed=5)
    tabs = W.make_tables(spec)
    tabs["log10_sigma"] = np.full(tabs["log10_sigma"].shape, -300.0)
    Tg = spec.T_grid
    a0, b0, a1, b1 = -46.0, 6.0e-4, -45.2, -3.5e-4
    tabs["log10_cia_h2h2"] = np.broadcast_to((a0 + b0 * Tg)[:, None], (5, 8)).copy()
    tabs["log10_cia_h2he"] = np.broadcast_to((a1 + b1 * Tg)[:, None], (5, 8)).copy()
    setup = W.make_setup(spec, 6000.0, 6007.0, 6, [0], 2, 2, 1, 0.0, 2)
    m = oracle.Model(tabs, setup.as_dict())
    x = 1e-3
    th = _theta([2230.0, 1610.0, 720.0], logx=(math.log10(x),))
    T, _ = m.level_temperatures(th)
    assert np.all(np.min(np.abs(T[:, None] - Tg[None, :]), axis=1) > 20.0)   # no level on a node
    assert m.cia_coeff("h2h2", T[3], 2) == pytest.approx(10 ** (a0 + b0 * T[3]), rel=1e-12)
    assert m.cia_coeff("h2he", T[3], 2) == pytest.approx(10 ** (a1 + b1 * T[3]), rel=1e-12)
    dtau, ok = m.layer_dtau(th, 3)
    assert ok
    xh2 = (1 - x) / 1.17
    xhe = 0.17 * xh2
    mmw = x * tabs["species_mass"][0] + xh2 * 2.01588 + xhe * 4.002602
    p = 10 ** np.linspace(-4.0, 2.0, 7) * 1e6
    n = p / (KB * T)
    chi = xh2 * xh2 * n * 10 ** (a0 + b0 * T) + xh2 * xhe * n * 10 ** (a1 + b1 * T)
    expect = 0.5 * (chi[:-1] + chi[1:]) * np.diff(p) / (mmw * AMU * 10 ** 4.75)
    assert np.allclose(dtau, expect, rtol=1e-8)


def test_wavenumber_offset_indexes_the_table(oracle_lib):
    """Setup point k reads table column nu_first + k."""
    spec = W.TableSpec(1, np.linspace(400.0, 2400.0, 4), np.linspace(-4.0, 2.0, 3), 6000.0, 1.0, 40, seed=5,
                       cia=False)
    tabs = W.make_tables(spec)
    tabs["log10_sigma"] = np.broadcast_to((-25.0 + 0.01 * np.arange(40))[None, None, None, :], (1, 4, 3, 40)).copy()
    setup = W.make_setup(spec, 6007.0, 6030.0, 3, [0], 2, 1, 1, 0.0, 2)
    assert setup.nu_first == 7
    m = oracle.Model(tabs, setup.as_dict())
    th = _theta([1000.0, 1000.0], logx=(-3.0,))
    d0, _ = m.layer_dtau(th, 0)
    d5, _ = m.layer_dtau(th, 5)
    assert np.allclose(d5 / d0, 10 ** 0.05, rtol=1e-12)
    _, top, _ = m.forward(th, want_top=True)
    assert np.allclose(top, math.pi * planck_indep(6007.0 + np.arange(24), 1000.0), rtol=1e-12)


def test_convolution_truncates_at_five_sigma(oracle_lib):
    m, _, _ = _tiny_model(R=2000.0, n_nu=200, n_bins=5)
    nu = m.nu
    c = 100
    delta = np.zeros(len(nu))
    delta[c] = 1.0
    out = m.convolve(delta)
    sig = nu / (2000.0 * 2 * math.sqrt(2 * math.log(2)))
    reach = np.abs(nu[c] - nu) <= 5 * sig
    assert np.all(out[reach] > 0) and np.all(out[~reach] == 0)
    assert reach.sum() < len(nu)


# ------------------------------------------------------------ linear-sigma interpolation option
def _linear_model(fill=None, cia=True, cia_fill=None, species=(0, 1), n_layers=4):
    spec = W.TableSpec(2, np.linspace(400.0, 2400.0, 4), np.linspace(-4.0, 2.0, 3), 6000.0, 1.0, 24, seed=99,
                       cia=cia)
    tabs = W.make_tables(spec)
    if fill is not None:
        tabs["log10_sigma"] = fill(tabs)
    if cia_fill is not None:
        tabs["log10_cia_h2h2"] = cia_fill(tabs)
    setup = W.make_setup(spec, 6000.0, 6023.0, n_layers, list(species), 3, 2, 1, 0.0, 4)
    setup.interp = "linear"
    return oracle.Model(tabs, setup.as_dict()), tabs, setup


def test_linear_interpolation_exact_at_nodes_and_for_bilinear_cross_sections(oracle_lib):
    """With the linear option the cross-section itself is interpolated: exact
    at the grid nodes and for any sigma bilinear in (T, log10 p); the log10
    option is not exact for such a field (it interpolates geometrically)."""
    m, tabs, setup = _linear_model()
    T, lp, sig = tabs["T_grid"], tabs["log10p_grid"], tabs["log10_sigma"]
    for a in range(len(T)):
        for b in range(len(lp)):
            assert m.sigma(1, T[a], lp[b], 5) == pytest.approx(10 ** sig[1, a, b, 5], rel=1e-13)
    c = [2.0e-22, 3.0e-25, 4.0e-23, 1.0e-25]
    field = lambda t, p: c[0] + c[1] * t + c[2] * (p + 4.0) + c[3] * t * (p + 4.0)
    fill = lambda tb: np.broadcast_to(np.log10(field(tb["T_grid"][:, None], tb["log10p_grid"][None, :]))[None, :, :, None],
                                      tb["log10_sigma"].shape).copy()
    m2, t2, s2 = _linear_model(fill=fill)
    mlog = oracle.Model(t2, dict(s2.as_dict(), interp="log10"))
    rng = np.random.default_rng(8)
    worst_log = 0.0
    for _ in range(20):
        t, p = rng.uniform(T[0], T[-1]), rng.uniform(lp[0], lp[-1])
        assert m2.sigma(0, t, p, 3) == pytest.approx(field(t, p), rel=1e-12)
        worst_log = max(worst_log, abs(mlog.sigma(0, t, p, 3) / field(t, p) - 1.0))
    assert worst_log > 1e-3
    assert m2.sigma(0, 50.0, -9.0, 3) == pytest.approx(field(T[0], lp[0]), rel=1e-12)   # clamped


def test_linear_interpolation_bounds_the_log_interpolation(oracle_lib):
    """Weighted AM-GM: sum w_i 10^l_i >= 10^(sum w_i l_i), equal where the
    corners agree; so the linear option never gives less than the log10 one."""
    m, tabs, setup = _linear_model()
    mlog = oracle.Model(tabs, dict(setup.as_dict(), interp="log10"))
    rng = np.random.default_rng(9)
    T, lp = tabs["T_grid"], tabs["log10p_grid"]
    for _ in range(50):
        t, p, inu = rng.uniform(T[0], T[-1]), rng.uniform(lp[0], lp[-1]), int(rng.integers(0, 24))
        assert m.sigma(1, t, p, inu) >= mlog.sigma(1, t, p, inu) * (1 - 1e-14)
    flat = lambda tb: np.full(tb["log10_sigma"].shape, -22.5)
    m3, t3, s3 = _linear_model(fill=flat)
    assert m3.sigma(0, 1234.0, -1.3, 2) == pytest.approx(10 ** -22.5, rel=1e-13)


def test_linear_option_cia_and_optical_depth_closed_form(oracle_lib):
    """CIA coefficient linear in T is reproduced exactly between nodes, and on
    an isothermal atmosphere the layer optical depth is the trapezoid of
    x sigma(T) + x_H2^2 n k(T) with those exact values."""
    sa, sb = 1.0e-22, 2.0e-25          # sigma(T) = sa + sb (T - 400), constant in p
    ka, kb = 1.0e-45, 3.0e-48          # k_H2H2(T) = ka + kb (T - 400)
    fill = lambda tb: np.broadcast_to(np.log10(sa + sb * (tb["T_grid"] - 400.0))[None, :, None, None],
                                      tb["log10_sigma"].shape).copy()
    cia_fill = lambda tb: np.broadcast_to(np.log10(ka + kb * (tb["T_grid"] - 400.0))[:, None],
                                          (len(tb["T_grid"]), 24)).copy()
    m, tabs, setup = _linear_model(fill=fill, cia_fill=cia_fill, species=(0,), n_layers=5)
    tabs["log10_cia_h2he"] = None
    m = oracle.Model(dict(tabs, log10_cia_h2he=None), setup.as_dict())
    Tiso = 1111.0
    assert m.cia_coeff("h2h2", Tiso, 4) == pytest.approx(ka + kb * (Tiso - 400.0), rel=1e-12)
    x = 2e-4
    th = _theta([Tiso, Tiso, Tiso], logx=(math.log10(x),))
    dtau, ok = m.layer_dtau(th, 4)
    assert ok
    xh2 = (1 - x) / 1.17
    mmw = x * tabs["species_mass"][0] + xh2 * 2.01588 + 0.17 * xh2 * 4.002602
    p = 10 ** np.linspace(-4.0, 2.0, 6) * 1e6
    chi = x * (sa + sb * (Tiso - 400.0)) + xh2 * xh2 * (p / (KB * Tiso)) * (ka + kb * (Tiso - 400.0))
    expect = 0.5 * (chi[:-1] + chi[1:]) * np.diff(p) / (mmw * AMU * 10 ** 4.75)
    assert np.allclose(dtau, expect, rtol=1e-8)
