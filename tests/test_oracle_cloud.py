"""Pins of the oracle's gray cloud layer (Appendix, "Impact of a gray cloud
layer"; readings R16-R17): optical depth spread evenly in pressure over
[p_top, p_top / f_c], gray and absorbing."""
import math

import numpy as np
import pytest
import scipy.constants as sc

import oracle
from paper_1910_01070_b300 import workloads as W

H_, CL, KB = sc.h * 1e7, sc.c * 1e2, sc.k * 1e7


def _model(n_layers=12, gas=-300.0, cia=False):
    spec = W.TableSpec(1, np.linspace(300.0, 3000.0, 4), np.linspace(-4.0, 2.0, 3), 6000.0, 1.0, 8, seed=3, cia=cia)
    tabs = W.make_tables(spec)
    tabs["log10_sigma"] = np.full(tabs["log10_sigma"].shape, gas)
    setup = W.make_setup(spec, 6000.0, 6007.0, n_layers, [0], 4, 1, 1, 0.0, 2)
    setup.cloud = True
    return oracle.Model(tabs, setup.as_dict()), setup


def _theta(T_bottom, T_top, tau_c, p_top_bar, f_c):
    th = np.zeros(oracle.NPARAM)
    th[0], th[1], th[2], th[3], th[4], th[19] = 4.5, 1.0, 10.0, T_bottom, T_top, -4.0
    th[35], th[36], th[37] = math.log10(tau_c), math.log10(p_top_bar), math.log10(f_c)
    return th


def test_cloud_optical_depth_is_spread_evenly_in_pressure():
    m, setup = _model()
    th = _theta(1500.0, 800.0, 3.7, 0.02, 0.05)          # layer from 0.02 to 0.4 bar
    dtau, ok = m.layer_dtau(th, 2)
    assert ok
    p = 10 ** np.linspace(-4.0, 2.0, setup.n_layers + 1)  # bar
    assert dtau.sum() == pytest.approx(3.7, rel=1e-12)
    inside = (p[:-1] >= 0.02) & (p[1:] <= 0.4)
    outside = (p[1:] <= 0.02) | (p[:-1] >= 0.4)
    assert inside.sum() >= 1 and outside.sum() >= 6
    per_bar = dtau[inside] / np.diff(p)[inside]
    assert np.allclose(per_bar, 3.7 / (0.4 - 0.02), rtol=1e-12)
    assert np.all(dtau[outside] < 1e-250)                  # only the 1e-300 gas opacity


def test_cloud_keeps_an_isothermal_atmosphere_at_planck():
    m, _ = _model(gas=-22.0, cia=True)
    th = _theta(1100.0, 1100.0, 40.0, 0.05, 0.2)
    _, top, ok = m.forward(th, want_top=True)
    nu = 6000.0 + np.arange(8)
    planck = 2 * H_ * CL ** 2 * nu ** 3 / np.expm1(H_ * CL * nu / (KB * 1100.0))
    assert np.allclose(top, math.pi * planck, rtol=1e-9)


def test_opaque_cloud_filling_one_layer_shows_its_top_level():
    """No gas opacity: the atmosphere above is transparent, and an opaque cloud that fills
    exactly one model layer emits the Planck function of that layer's top level."""
    m, setup = _model(n_layers=12)
    p = 10 ** np.linspace(-4.0, 2.0, setup.n_layers + 1)
    j = 7
    th = _theta(1600.0, 700.0, 1e7, p[j], p[j] / p[j + 1])
    T, _ = m.level_temperatures(th)
    _, top, ok = m.forward(th, want_top=True)
    assert ok
    nu = 6000.0 + np.arange(8)
    planck = 2 * H_ * CL ** 2 * nu ** 3 / np.expm1(H_ * CL * nu / (KB * T[j]))
    assert np.allclose(top, math.pi * planck, rtol=1e-5)


def test_cloud_bottom_above_top_is_invalid():
    m, _ = _model()
    bins, ok = m.forward(_theta(1500.0, 800.0, 1.0, 0.1, 1.5))
    assert not ok
