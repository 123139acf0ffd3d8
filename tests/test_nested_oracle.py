"""Pins of the nested-sampling evidence bookkeeping of the oracle (Sect. 3.2,
after Skilling 2004) against closed forms and against brute-force sums."""
import decimal
import math

import numpy as np
import pytest

from oracle import nested as N


def test_shell_weights_telescope_to_the_whole_prior():
    """sum_{i<=n} (X_{i-1} - X_i) + X_n = 1 for X_i = exp(-i/N)."""
    for n_live in (1, 7, 400):
        for n in (1, 10, 3000):
            w = [math.exp(N.log_shell_weight(i, n_live)) for i in range(1, n + 1)]
            assert math.fsum(w) + math.exp(-n / n_live) == pytest.approx(1.0, abs=1e-13)
            # ln(1 - e^(-1/N)) to 40 digits
            with decimal.localcontext() as ctx:
                ctx.prec = 40
                ref = float((1 - (-1 / decimal.Decimal(n_live)).exp()).ln())
            assert N.log_shell_weight(1, n_live) == pytest.approx(ref, abs=1e-14)


def test_log_add_against_direct_sums():
    rng = np.random.default_rng(0)
    for _ in range(100):
        a, b = rng.uniform(-700, 700, 2)
        m = max(a, b)
        assert N.log_add(a, b) == pytest.approx(m + math.log1p(math.exp(-abs(a - b))), abs=1e-12)
    assert N.log_add(-math.inf, 3.5) == 3.5 and N.log_add(2.0, -math.inf) == 2.0
    assert N.log_add(-math.inf, -math.inf) == -math.inf


def test_running_sums_equal_the_definitions():
    """ln Z = ln sum e^(lnl + lnw) and H = sum p ln(L/Z), p = L w / Z, by fsum."""
    rng = np.random.default_rng(1)
    lnl = rng.normal(-50.0, 20.0, 300)
    lw = rng.normal(-5.0, 3.0, 300)
    lnl[7] = -math.inf
    s = N.State()
    for a, b in zip(lnl, lw):
        s.add(float(a), float(b))
    m = np.max(lnl + lw)
    terms = [math.exp(a + b - m) for a, b in zip(lnl, lw)]
    log_z = m + math.log(math.fsum(terms))
    assert s.log_z == pytest.approx(log_z, abs=1e-10)
    p = [math.exp(a + b - log_z) for a, b in zip(lnl, lw)]
    h = math.fsum(pi * (a - log_z) for pi, a in zip(p, lnl) if pi > 0)
    assert s.info == pytest.approx(h, rel=1e-9, abs=1e-9)


def test_constant_likelihood_gives_exactly_that_evidence():
    """Dead points at L = c over any number of shells plus the live remainder: Z = c."""
    for n_live, n_dead in ((5, 0), (5, 17), (64, 1000)):
        s = N.State()
        for i in range(1, n_dead + 1):
            s.add(-3.25, N.log_shell_weight(i, n_live))
        s.n_dead = n_dead
        log_z, info = N.finalize(np.full(n_live, -3.25), s)
        assert log_z == pytest.approx(-3.25, abs=1e-12)
        assert info == pytest.approx(0.0, abs=1e-10)


def test_absorb_replaces_the_worst_in_order_and_respects_the_cap():
    live = np.array([-1.0, -5.0, -3.0, -5.0])
    th = np.arange(4 * 3, dtype=float).reshape(4, 3)
    cand = np.array([-6.0, -4.0, -4.5, -0.5, -10.0])
    cth = 100.0 + np.arange(5 * 3, dtype=float).reshape(5, 3)
    s, dead = N.State(), []
    N.absorb(live, th, cand, cth, s, dead, dead_cap=10)
    # -6 rejected; -4 replaces index 1 (first -5); -4.5 replaces index 3 (-5); -0.5 replaces -4.5
    assert [d[0] for d in dead] == [-5.0, -5.0, -4.5]
    assert np.array_equal(dead[0][2], [3.0, 4.0, 5.0]) and np.array_equal(dead[1][2], [9.0, 10.0, 11.0])
    assert np.array_equal(live, [-1.0, -4.0, -3.0, -0.5])
    assert s.n_dead == 3 and s.n_seen == 5
    s2, dead2 = N.State(), []
    live2 = np.array([-1.0, -5.0, -3.0, -5.0])
    N.absorb(live2, th.copy(), cand, cth, s2, dead2, dead_cap=1)
    assert s2.n_dead == 1 and s2.n_seen == 2


def _sample_in_ball(rng, c, r, d):
    v = rng.normal(size=d)
    v /= np.linalg.norm(v)
    return c + v * r * rng.uniform() ** (1.0 / d)


def test_gaussian_evidence_and_information_closed_form():
    """L = exp(-|x - c|^2 / (2 s^2)) on the unit cube (d = 3, s = 0.04, so the cube holds
    the Gaussian): Z = (2 pi s^2)^(d/2) and H = -ln Z - d/2.  Replacement points are drawn
    exactly from the constrained prior (uniform in the likelihood ball), so the check is
    on the bookkeeping alone: ln Z within 4 sqrt(H/N) of the closed form."""
    d, sd, n_live = 3, 0.04, 300
    c = np.full(d, 0.5)
    lnl_of = lambda x: -np.sum((x - c) ** 2, axis=-1) / (2 * sd * sd)
    rng = np.random.default_rng(5)
    th = rng.uniform(size=(n_live, d))
    live = lnl_of(th)
    s, dead = N.State(), []
    while True:
        worst = N.argmin_first(live)
        r = math.sqrt(-2 * sd * sd * live[worst])
        x = _sample_in_ball(rng, c, min(r, 0.5), d)
        N.absorb(live, th, np.array([lnl_of(x)]), x[None, :], s, dead, dead_cap=10 ** 6)
        if np.max(live) + (-s.n_dead / n_live) - s.log_z < math.log(1e-4):
            break
    log_z, info = N.finalize(live, s)
    z_ref = 0.5 * d * math.log(2 * math.pi * sd * sd)
    h_ref = -z_ref - 0.5 * d
    err = math.sqrt(info / n_live)
    assert abs(log_z - z_ref) < 4 * err, (log_z, z_ref, err)
    assert abs(info - h_ref) < 0.5, (info, h_ref)
