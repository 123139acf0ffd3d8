"""Pins of the oracle's Milne profile (Sect. 2.5, exact Hopf function) and of
its effective-temperature post-processing (Sect. 2.6)."""
import math

import numpy as np
import pytest
import scipy.constants as sc
from scipy import integrate
from scipy.special import expn

import oracle
from oracle import hopf
from paper_1910_01070_b300 import workloads as W

H_ = sc.h * 1e7
CL = sc.c * 1e2
KB = sc.k * 1e7
SIGMA_SB = sc.Stefan_Boltzmann * 1e3


def _ln_1m_tcot(th):
    if th < 0.05:
        t2 = th * th
        return math.log(t2 / 3.0) + math.log1p(t2 / 15.0 + 2.0 * t2 * t2 / 315.0)
    return math.log(1.0 - th / math.tan(th))


def h_function(mu):
    """Chandrasekhar's H for conservative isotropic scattering, by its integral representation."""
    v, _ = integrate.quad(lambda th: _ln_1m_tcot(th) / (math.cos(th) ** 2 + mu * mu * math.sin(th) ** 2),
                          0.0, math.pi / 2, limit=400, epsabs=1e-13)
    return math.exp(-mu / math.pi * v)


def test_hopf_end_values():
    """q(0) = 1/sqrt(3) and q(inf) = 1/sqrt(3) + (1/(2 sqrt 3)) int_0^1 dmu / (H (a^2 + (pi mu/2)^2)),
    a = 1 - (mu/2) ln((1+mu)/(1-mu)) (the Hopf constant 0.710446...)."""
    assert hopf.hopf(0.0) == pytest.approx(1 / math.sqrt(3), abs=1e-8)

    tail, _ = integrate.quad(_g, 0.0, 1.0, limit=400, epsabs=1e-12)
    q_inf = 1 / math.sqrt(3) + tail / (2 * math.sqrt(3))
    assert q_inf == pytest.approx(0.7104460896, abs=1e-9)
    assert hopf.hopf(40.0) == pytest.approx(q_inf, abs=2e-8)



def _g(mu):
    a = 1.0 - 0.5 * mu * math.log((1 + mu) / (1 - mu))
    return 1.0 / (h_function(mu) * (a * a + (math.pi * mu / 2) ** 2))


@pytest.mark.parametrize("tau", [0.01, 0.3, 0.8, 2.5])
def test_hopf_function_matches_chandrasekhars_closed_form(tau):
    """Between the ends: q(tau) = 1/sqrt(3) + (1/(2 sqrt 3)) int_0^1 g(mu) (1 - e^{-tau/mu}) dmu
    with g = 1 / (H (a^2 + (pi mu/2)^2)) (Chandrasekhar's solution of Milne's problem),
    an independent route to the function the integral-equation solve tabulates."""
    v, _ = integrate.quad(lambda mu: _g(mu) * -math.expm1(-tau / mu), 0.0, 1.0, limit=400, epsabs=1e-12)
    assert hopf.hopf(tau) == pytest.approx(1 / math.sqrt(3) + v / (2 * math.sqrt(3)), abs=2e-8)

@pytest.mark.parametrize("tau", [0.0, 0.2, 1.0, 4.0])
def test_milne_flux_is_constant(tau):
    """Radiative equilibrium: with S = t + q(t) the flux 2 int_tau^inf S E2(t - tau) dt -
    2 int_0^tau S E2(tau - t) dt equals 4/3 at every depth (Schwarzschild-Milne, Eq. 3)."""
    S = lambda t: t + hopf.hopf(t)
    up, _ = integrate.quad(lambda t: S(t) * expn(2, t - tau), tau, tau + 60.0, limit=400, points=[tau + 1.0])
    dn = 0.0
    if tau > 0:
        dn, _ = integrate.quad(lambda t: S(t) * expn(2, tau - t), 0.0, tau, limit=400)
    assert 2 * up - 2 * dn == pytest.approx(4.0 / 3.0, abs=2e-8)


@pytest.mark.parametrize("mu", [0.2, 0.6, 1.0])
def test_milne_emergent_intensity_is_the_h_function(mu):
    """I(0, mu) = int_0^inf (t + q(t)) e^{-t/mu} dt / mu = H(mu) / sqrt(3)."""
    v, _ = integrate.quad(lambda t: hopf.hopf(t) * math.exp(-t / mu) / mu, 0.0, 60.0 * mu, limit=400)
    assert mu + v == pytest.approx(h_function(mu) / math.sqrt(3), abs=1e-8)


def _milne_model(n_layers=30):
    spec = W.TableSpec(1, np.linspace(300.0, 3000.0, 4), np.linspace(-4.0, 2.0, 3), 6000.0, 1.0, 16, seed=4)
    tabs = W.make_tables(spec)
    setup = W.make_setup(spec, 6000.0, 6015.0, n_layers, [0], 2, 1, 1, 0.0, 2)
    setup.profile = "milne"
    return oracle.Model(tabs, setup.as_dict()), setup


def test_milne_profile_surface_and_depth():
    m, setup = _milne_model()
    th = np.zeros(oracle.NPARAM)
    th[0], th[1], th[2], th[3], th[19] = 4.5, 1.0, 10.0, 1200.0, -4.0
    th[4] = -14.0                                   # kappa_R tiny: tau_R ~ 0 at every level
    T, ok = m.level_temperatures(th)
    assert ok
    assert np.allclose(T, (math.sqrt(3) / 4) ** 0.25 * 1200.0, rtol=1e-6)   # T_0 = 0.8112 Tbar
    th[4] = 1.0                                     # kappa_R = 10 cm^2/g: deep levels at tau >> 1
    T, ok = m.level_temperatures(th)
    p = 10 ** np.linspace(-4.0, 2.0, setup.n_layers + 1) * 1e6
    tau = 10.0 * p / 10 ** 4.5
    deep = tau > 40.0
    assert deep.sum() > 3
    assert np.allclose(T[deep] ** 4, 0.75 * 1200.0 ** 4 * (tau[deep] + 0.7104460896), rtol=1e-6)
    assert np.all(np.diff(T) > 0)                   # temperature rises inward


def _planck_band(nu1, nu2, T):
    """int_nu1^nu2 pi B_nu dnu by the series int_a^inf x^3/(e^x-1) dx = sum_n e^{-na}(a^3/n + 3a^2/n^2 + 6a/n^3 + 6/n^4)."""
    def tail(a):
        return math.fsum(math.exp(-n * a) * (a ** 3 / n + 3 * a * a / n ** 2 + 6 * a / n ** 3 + 6 / n ** 4)
                         for n in range(1, 4000))
    c = H_ * CL / (KB * T)
    return math.pi * 2 * H_ * CL ** 2 * (1 / c) ** 4 * (tail(c * nu1) - tail(c * nu2))


@pytest.mark.parametrize("T,nu1,nu2", [(1200.0, 500.0, 10000.0), (300.0, 1.0, 8000.0)])
def test_effective_temperature_of_an_isothermal_atmosphere(T, nu1, nu2):
    """F+ = pi B(T) for an isothermal atmosphere, so T_eff = (int pi B dnu / sigma)^(1/4) over the
    setup's band (-> T itself when the band holds the whole Planck curve)."""
    n = int(nu2 - nu1) + 1
    spec = W.TableSpec(1, np.linspace(200.0, 3000.0, 3), np.linspace(-4.0, 2.0, 2), nu1, 1.0, n, seed=9, cia=False)
    tabs = W.make_tables(spec)
    setup = W.make_setup(spec, nu1, nu2, 2, [0], 2, 1, 1, 0.0, 1)
    m = oracle.Model(tabs, setup.as_dict())
    th = np.zeros(oracle.NPARAM)
    th[0], th[1], th[2], th[3], th[4], th[19] = 4.5, 1.0, 10.0, T, T, -4.0
    teff = m.effective_temperature(th)
    ref = (_planck_band(nu1, nu2, T) / SIGMA_SB) ** 0.25
    assert teff == pytest.approx(ref, rel=1e-6)
    if T == 300.0:
        assert teff == pytest.approx(T, rel=2e-4)
