"""Nested-sampling bookkeeping on the device against the oracle's, and the
driver running on the forward model."""
import math

import numpy as np
import pytest

import oracle
from oracle import nested as N
from paper_1910_01070_b300 import hr2
from paper_1910_01070_b300 import workloads as W
from paper_1910_01070_b300.engine import Engine
from paper_1910_01070_b300.nested import GpuBackend, NestedSampler
from tests.helpers import oracle_model, tables_as_stored

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def eng():
    from paper_1910_01070_b300 import build
    build.build()
    e = Engine(0)
    yield e
    e.close()


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("n_live,n_cand,cap", [(1, 50, 100), (37, 400, 10 ** 4), (300, 3000, 10 ** 4), (64, 500, 40),
                                               (4096, 700, 10 ** 4), (5000, 700, 10 ** 4)])
def test_absorb_and_finalize_match_the_oracle(eng, n_live, n_cand, cap):
    rng = np.random.default_rng(n_live + n_cand)
    live = np.round(rng.normal(-100.0, 30.0, n_live), 1)          # rounding makes ties
    if n_live > 5:
        live[3] = -np.inf
        live[4] = np.nan
    cand = np.round(rng.normal(-60.0, 40.0, n_cand), 1)
    cand[::17] = -np.inf
    cand[5::23] = np.nan
    lth = rng.normal(size=(n_live, hr2.HR2_NPARAM))
    cth = rng.normal(size=(n_cand, hr2.HR2_NPARAM))
    # oracle
    o_live, o_th = live.copy(), lth.copy()
    s, dead = N.State(), []
    half = n_cand // 2
    N.absorb(o_live, o_th, cand[:half], cth[:half], s, dead, cap)
    N.absorb(o_live, o_th, cand[half:], cth[half:], s, dead, cap)
    o_z, o_h = N.finalize(o_live, s)
    # device, in the same two calls
    d_live, d_th = _t(live), _t(lth)
    state = torch.empty(hr2.NS_STATE_DOUBLES, dtype=torch.float64, device="cuda")
    hr2.hr2_ns_state_init(eng.ctx, state)
    dl, dw, dt = (torch.full((cap,), 7.0, dtype=torch.float64, device="cuda"),
                  torch.full((cap,), 7.0, dtype=torch.float64, device="cuda"),
                  torch.zeros((cap, hr2.HR2_NPARAM), dtype=torch.float64, device="cuda"))
    hr2.hr2_ns_absorb(eng.ctx, d_live, d_th, _t(cand[:half]), _t(cth[:half]), state, dl, dw, dt)
    hr2.hr2_ns_absorb(eng.ctx, d_live, d_th, _t(cand[half:]), _t(cth[half:]), state, dl, dw, dt)
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    hr2.hr2_ns_finalize(eng.ctx, d_live, state, out)
    st = hr2.ns_state_read(state)
    nd = len(dead)
    assert st["n_dead"] == s.n_dead == nd and st["n_seen"] == s.n_seen
    assert np.array_equal(d_live.cpu().numpy(), o_live, equal_nan=True)
    assert np.array_equal(d_th.cpu().numpy(), o_th)
    assert np.array_equal(dl.cpu().numpy()[:nd], np.array([x[0] for x in dead]))
    assert np.allclose(dw.cpu().numpy()[:nd], [x[1] for x in dead], rtol=1e-14, atol=1e-14)
    assert np.array_equal(dt.cpu().numpy()[:nd], np.array([x[2] for x in dead]).reshape(nd, hr2.HR2_NPARAM))
    assert np.all(dl.cpu().numpy()[nd:] == 7.0)                    # nothing beyond the dead points
    if nd:
        assert st["log_z"] == pytest.approx(s.log_z, rel=1e-12, abs=1e-12)
        assert st["info"] == pytest.approx(s.info, rel=1e-10, abs=1e-10)
    assert st["log_x"] == pytest.approx(-nd / n_live, abs=1e-15)
    key = np.where(np.isnan(o_live), np.inf, o_live)
    assert st["lnl_min"] == key.min() and st["lnl_max"] == np.nanmax(o_live)
    o = out.cpu().numpy()
    assert math.isnan(o[0]) == math.isnan(o_z)                  # a NaN live point propagates on both sides
    if not math.isnan(o_z):
        assert o[0] == pytest.approx(o_z, rel=1e-12, abs=1e-12)
    if math.isfinite(o_h):
        assert o[1] == pytest.approx(o_h, rel=1e-10, abs=1e-10)


def test_driver_on_the_forward_model(eng):
    """A short run on a small setup with a mock observation: dead points leave in
    non-decreasing likelihood, and each one's lnL is what the oracle gives for it."""
    spec = W.TableSpec(2, np.linspace(300.0, 2500.0, 6), np.linspace(-4.0, 2.0, 5), 5000.0, 1.0, 400, seed=12)
    tabs = W.make_tables(spec)
    setup = W.make_setup(spec, 5000.0, 5399.0, 20, [0, 1], 3, 2, 1, 300.0, 12)
    t = eng.add_tables(spec, "fp16", tabs)
    s = eng.add_setup(t, setup)
    om = oracle_model(tables_as_stored(tabs, "fp16"), setup)
    truth = np.zeros(hr2.HR2_NPARAM)
    truth[0], truth[1], truth[2] = 4.75, 1.0, 10.0
    truth[3:6] = [1600.0, 1100.0, 700.0]
    truth[19:21] = [-3.5, -4.0]
    tb, ok = om.forward(truth)
    D, sig = W.mock_observation(tb, 77)
    eng.set_observation(s, D, sig)
    lo, hi = truth.copy(), truth.copy()
    lo[0], hi[0] = 4.0, 5.5
    lo[3:6], hi[3:6] = 400.0, 2400.0
    lo[19:21], hi[19:21] = -8.0, -2.0
    be = GpuBackend(eng.ctx, [s], 0, n_live=128)
    res = NestedSampler(be, lo, hi, batch=512, seed=4).run(dlogz=0.5, max_rounds=6)
    assert res["n_dead"] > 0 and math.isfinite(res["log_z"])
    dl, dw, dth = be.dead(res["n_dead"])
    assert np.all(np.diff(dl) >= 0)
    for k in np.linspace(0, res["n_dead"] - 1, 6).astype(int):
        ref = oracle.lnL(D, sig, om.forward(dth[k])[0])
        assert dl[k] == pytest.approx(ref, rel=1e-5, abs=1e-3)
    assert np.allclose(dw, [N.log_shell_weight(i, 128) for i in range(1, res["n_dead"] + 1)], rtol=1e-14, atol=1e-14)
    # the same run on a side stream of the backend's own gives the same dead points
    side = torch.cuda.Stream()
    be2 = GpuBackend(eng.ctx, [s], 0, n_live=128, stream=side)
    res2 = NestedSampler(be2, lo, hi, batch=512, seed=4).run(dlogz=0.5, max_rounds=6)
    assert res2["n_dead"] == res["n_dead"] and res2["log_z"] == res["log_z"]
    dl2, _, dth2 = be2.dead(res2["n_dead"])
    assert np.array_equal(dl2, dl) and np.array_equal(dth2, dth)
    # the host-drawn proposals (the path of a backend without hr2_ns_propose)
    be3 = GpuBackend(eng.ctx, [s], 0, n_live=128)
    res3 = NestedSampler(be3, lo, hi, batch=512, seed=4, device_proposals=False).run(dlogz=0.5, max_rounds=6)
    dl3, _, dth3 = be3.dead(res3["n_dead"])
    assert res3["n_dead"] > 0 and np.all(np.diff(dl3) >= 0)
    k = res3["n_dead"] - 1
    assert dl3[k] == pytest.approx(oracle.lnL(D, sig, om.forward(dth3[k])[0]), rel=1e-5, abs=1e-3)


def test_device_proposals_stay_in_the_box_and_are_reproducible(eng):
    """hr2_ns_propose: the box is the live points' range widened by enlarge x span
    and clipped to the prior; every draw lies in it, fixed parameters stay at
    their value, equal (seed, counter) give equal draws, row i uses counters
    counter + i HR2_NPARAM .. (so a shifted counter shifts the rows), and each
    free parameter's draws are uniform on its interval."""
    from scipy import stats
    rng = np.random.default_rng(5)
    P = hr2.HR2_NPARAM
    lo, hi = np.zeros(P), np.zeros(P)
    free = np.arange(P) % 3 != 2
    lo[free], hi[free] = -1.0 - rng.random(free.sum()), 1.0 + rng.random(free.sum())
    lo[~free] = hi[~free] = rng.normal(size=(~free).sum())
    live = np.repeat(lo[None, :], 300, axis=0)
    live[:, free] = rng.uniform(-0.5, 0.8, (300, free.sum()))
    live[0, 0] = lo[0]                                   # reaches the prior edge: the box is clipped there
    enlarge = 0.25
    span = live.max(0) - live.min(0)
    ref_lo = np.maximum(lo, live.min(0) - enlarge * span)
    ref_hi = np.minimum(hi, live.max(0) + enlarge * span)
    d_live, d_lo, d_hi = _t(live), _t(lo), _t(hi)
    box = torch.empty((P, 2), dtype=torch.float64, device="cuda")
    n = 4096

    def draw(n, seed, counter):
        out = torch.empty((n, P), dtype=torch.float64, device="cuda")
        hr2.hr2_ns_propose(eng.ctx, d_live, d_lo, d_hi, enlarge, box, out, seed, counter)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    a = draw(n, 11, 0)
    b = box.cpu().numpy()
    assert np.allclose(b[free, 0], ref_lo[free], rtol=1e-15, atol=1e-15)
    assert np.allclose(b[free, 1], ref_hi[free], rtol=1e-15, atol=1e-15)
    assert b[0, 0] == lo[0]
    assert np.all(a[:, free] >= b[free, 0]) and np.all(a[:, free] < b[free, 1])
    assert np.array_equal(a[:, ~free], np.repeat(lo[None, ~free], n, axis=0))
    assert np.array_equal(draw(n, 11, 0), a)
    assert np.array_equal(draw(n - 1, 11, P), a[1:])
    assert not np.array_equal(draw(n, 12, 0), a)
    u = (a[:, free] - b[free, 0]) / (b[free, 1] - b[free, 0])
    for col in u.T:
        assert stats.kstest(col, "uniform").pvalue > 1e-4
    assert abs(np.corrcoef(u[:, 0], u[:, 1])[0, 1]) < 0.06


def test_device_proposals_argument_errors(eng):
    P = hr2.HR2_NPARAM
    live = _t(np.zeros((4, P)))
    lo, hi = _t(np.zeros(P)), _t(np.ones(P))
    box = torch.empty((P, 2), dtype=torch.float64, device="cuda")
    out = torch.empty((8, P), dtype=torch.float64, device="cuda")
    with pytest.raises(hr2.Hr2Error):
        hr2.hr2_ns_propose(eng.ctx, live, lo, hi, -0.5, box, out, 1, 0)
    with pytest.raises(hr2.Hr2Error):
        hr2.hr2_ns_propose(eng.ctx, live[:0], lo, hi, 0.25, box, out, 1, 0)
