"""Pins of the oracle's parabolic short characteristics (Sect. 2.1, higher-
order source interpolants)."""
import math

import numpy as np
import pytest

import oracle
from paper_1910_01070_b300 import workloads as W


def _quadratic_case(mu, seed=0, L=40):
    """S(tau) = a + b tau + c tau^2 on an irregular grid with a very thin top layer; the exact
    emergent intensity is a + b mu + 2 c mu^2 for the bottom intensity
    I(tau_L) = a + b (tau_L + mu) + c (tau_L^2 + 2 mu tau_L + 2 mu^2)."""
    rng = np.random.default_rng(seed)
    dtau = rng.uniform(0.05, 0.6, L)
    dtau[0] = 1e-5
    tau = np.concatenate([[0.0], np.cumsum(dtau)])
    a, b, c = 2.0, 1.5, 0.3
    S = a + b * tau + c * tau * tau
    tl = tau[-1]
    Ib = a + b * (tl + mu) + c * (tl * tl + 2 * mu * tl + 2 * mu * mu)
    return dtau, S, Ib, a + b * mu + 2 * c * mu * mu


@pytest.mark.parametrize("mu", [0.07, 0.35, 1.0])
def test_parabolic_is_exact_for_a_quadratic_source(oracle_lib, mu):
    dtau, S, Ib, exact = _quadratic_case(mu)
    # exact but for the linear top layer (c mu^2 D^3/6 ~ 1e-16) and rounding amplified by the thin layer
    assert oracle.sc_intensity_parabolic(dtau, S, Ib, mu) == pytest.approx(exact, rel=1e-11)
    assert abs(oracle.sc_intensity(dtau, S, Ib, mu) / exact - 1) > 1e-4   # the linear scheme is not


def test_parabolic_thin_and_thick_layers_stay_exact(oracle_lib):
    """Layers from 1e-9 to 30 optical depths (series and closed-form moments)."""
    rng = np.random.default_rng(3)
    dtau = 10 ** rng.uniform(-9, 1.5, 50)
    dtau[0] = 1e-9
    tau = np.concatenate([[0.0], np.cumsum(dtau)])
    S = 1.0 + 0.4 * tau + 0.01 * tau * tau
    mu = 0.6
    tl = tau[-1]
    Ib = 1.0 + 0.4 * (tl + mu) + 0.01 * (tl * tl + 2 * mu * tl + 2 * mu * mu)
    assert oracle.sc_intensity_parabolic(dtau, S, Ib, mu) == pytest.approx(1.0 + 0.4 * mu + 0.02 * mu * mu, rel=1e-11)


def _formal(tau, S_of, mu, n=200000):
    """Brute force: I(0) = int_0^tau_L S(t) e^{-t/mu} dt/mu + S(tau_L) e^{-tau_L/mu}."""
    t = np.linspace(0.0, tau[-1], n + 1)
    f = S_of(t) * np.exp(-t / mu) / mu
    return float(np.sum((f[1:] + f[:-1]) * np.diff(t) / 2)) + S_of(tau[-1]) * math.exp(-tau[-1] / mu)


def test_parabolic_converges_at_third_order(oracle_lib):
    """Smooth source on uniform grids: halving the layer thickness divides the parabolic
    error by ~8 (third order) and the linear error by ~4."""
    S_of = lambda t: np.exp(0.7 * np.asarray(t)) + np.sin(3.0 * np.asarray(t))
    mu = 0.5
    errs_p, errs_l = [], []
    for L in (8, 16, 32):
        tau = np.linspace(0.0, 6.0, L + 1)
        S = S_of(tau)
        ref = _formal(tau, S_of, mu)
        dt = np.diff(tau)
        errs_p.append(abs(oracle.sc_intensity_parabolic(dt, S, S[-1], mu) - ref))
        errs_l.append(abs(oracle.sc_intensity(dt, S, S[-1], mu) - ref))
    assert errs_l[1] / errs_l[2] == pytest.approx(4.0, rel=0.25)
    assert errs_p[1] / errs_p[2] > 6.0
    assert errs_p[2] < errs_l[2] / 3          # (the top layer is linear in both schemes)


def test_parabolic_model_keeps_isothermal_planck(oracle_lib):
    spec = W.TableSpec(2, np.linspace(300.0, 3000.0, 4), np.linspace(-4.0, 2.0, 3), 6000.0, 1.0, 8, seed=5)
    tabs = W.make_tables(spec)
    setup = W.make_setup(spec, 6000.0, 6007.0, 20, [0, 1], 4, 1, 1, 0.0, 2)
    setup.sc = "parabolic"
    m = oracle.Model(tabs, setup.as_dict())
    th = np.zeros(oracle.NPARAM)
    th[0], th[1], th[2], th[3], th[4], th[19], th[20] = 4.5, 1.0, 10.0, 1300.0, 1300.0, -3.0, -4.0
    _, top, ok = m.forward(th, want_top=True)
    nu = 6000.0 + np.arange(8)
    assert np.allclose(top, math.pi * oracle.planck(nu, 1300.0), rtol=1e-10)
