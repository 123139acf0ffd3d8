"""The streamed level-gridded operand (level_cache="stream") through the C ABI.

A streamed setup keeps no operand: a call with it alone and at least 32
samples builds the operand (the tables interpolated in p onto the levels,
FP32 arithmetic) one group of tiles at a time into a per-stream ring and
sweeps each group before building the next.  The oracle is the FP64 oracle on
the tables as stored; the operand's own rounding differs from the
level-gridded operand built once at creation (FP64 arithmetic), so the two
agree to FP32 rounding, not bit for bit.  Per tile the arithmetic does not
depend on how the tiles are grouped, so every grouping gives the same bits.
"""
import numpy as np
import pytest

from paper_1910_01070_b300 import hr2
from paper_1910_01070_b300 import workloads as W
from paper_1910_01070_b300.engine import Engine
from tests.helpers import FLUX_RTOL, oracle_model, rel_flux_err, tables_as_stored

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def eng():
    from paper_1910_01070_b300 import build
    build.build()
    e = Engine(0)
    yield e
    e.close()


def _case():
    # 8 tiles of 128 points (the last one ragged), 20 layers, 3 absorbers
    spec = W.TableSpec(3, np.linspace(300.0, 3000.0, 7), np.linspace(-4.0, 2.0, 6), 5000.0, 1.0, 1100, seed=71)
    setup = W.make_setup(spec, 5030.0, 5990.0, 20, [0, 1, 2], 4, 3, 2, 400.0, 24)
    return spec, W.make_tables(spec), setup


def _run(eng, s, setup, theta):
    n = len(theta)
    bins = torch.full((n, setup.n_bins), -1.0, dtype=torch.float32, device="cuda")
    hi = torch.full((n, setup.n_nu), -1.0, dtype=torch.float32, device="cuda")
    st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    sd = torch.zeros(n, dtype=torch.int32, device="cuda")
    th = torch.as_tensor(theta, device="cuda")
    hr2.forward_model_batch(eng.ctx, [s], sd, th, bins, hi, st)
    hr2.hr2_stream_check(eng.ctx)
    torch.cuda.synchronize()
    return bins.cpu().numpy(), hi.cpu().numpy(), st.cpu().numpy()


def test_streamed_setup_matches_oracle_over_several_groups(eng):
    spec, tabs, setup = _case()
    t = eng.add_tables(spec, "fp16", tabs)
    s = eng.add_setup(t, setup, level_cache="stream")
    assert hr2.hr2_setup_streamed(s)
    b_, ob, lg = hr2.hr2_setup_memory(s)
    assert ob == 0 and lg is False
    theta = W.draw_params(setup, 64, 5, W.Prior())
    hr2.hr2_set_stream_group(eng.ctx, 3)             # groups of 3, 3 and 2 tiles
    try:
        bins, hi, st = _run(eng, s, setup, theta)
    finally:
        hr2.hr2_set_stream_group(eng.ctx, 0)
    assert np.all(st == 0)
    om = oracle_model(tables_as_stored(tabs, "fp16"), setup)
    for i in range(0, 64, 5):
        ob_, otop, ok = om.forward(theta[i], want_top=True)
        assert ok
        assert rel_flux_err(hi[i], otop) <= FLUX_RTOL
        assert rel_flux_err(bins[i], ob_) <= FLUX_RTOL


def test_groupings_agree_bitwise_and_with_the_level_gridded_operand(eng):
    spec, tabs, setup = _case()
    t = eng.add_tables(spec, "fp16", tabs)
    s_str = eng.add_setup(t, setup, level_cache="stream")
    s_lvl = eng.add_setup(t, setup, level_cache=True)
    theta = W.draw_params(setup, 64, 6, W.Prior())
    out = {}
    for g in (1, 3, 8, 0):
        hr2.hr2_set_stream_group(eng.ctx, g)
        try:
            out[g] = _run(eng, s_str, setup, theta)
        finally:
            hr2.hr2_set_stream_group(eng.ctx, 0)
    for g in (1, 3, 8):
        assert np.array_equal(out[g][0], out[0][0])
        assert np.array_equal(out[g][1], out[0][1])
    bl, hl, stl = _run(eng, s_lvl, setup, theta)
    assert np.all(stl == 0) and np.all(out[0][2] == 0)
    # FP32 against FP64 arithmetic of the same operand: a few units of FP32 rounding
    for i in range(64):
        assert rel_flux_err(out[0][1][i], hl[i].astype(np.float64)) <= 2e-5
        assert rel_flux_err(out[0][0][i], bl[i].astype(np.float64)) <= 2e-5


def test_small_and_mixed_batches_read_the_tables_directly(eng):
    """Below 32 samples, or beside another setup, a streamed setup is evaluated like a
    setup without an operand: the same bits as one created with level_cache=False."""
    spec, tabs, setup = _case()
    t = eng.add_tables(spec, "fp16", tabs)
    s_str = eng.add_setup(t, setup, level_cache="stream")
    s_dir = eng.add_setup(t, setup, level_cache=False)
    theta = W.draw_params(setup, 12, 7, W.Prior())
    a = _run(eng, s_str, setup, theta)
    b = _run(eng, s_dir, setup, theta)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # mixed with a direct setup in one call (40 samples, alternating)
    theta = W.draw_params(setup, 40, 8, W.Prior())
    sid = (np.arange(40) % 2).astype(np.int32)
    n = 40
    bins = torch.empty((n, setup.n_bins), dtype=torch.float32, device="cuda")
    hi = torch.empty((n, setup.n_nu), dtype=torch.float32, device="cuda")
    hr2.forward_model_batch(eng.ctx, [s_str, s_dir], torch.as_tensor(sid, device="cuda"),
                            torch.as_tensor(theta, device="cuda"), bins, hi, None)
    torch.cuda.synchronize()
    h = hi.cpu().numpy()
    assert np.all(np.isfinite(h))
    b2 = _run(eng, s_dir, setup, theta)
    assert np.array_equal(h, b2[1])


def test_streamed_option_argument_errors(eng):
    spec, tabs, setup = _case()
    t64 = eng.add_tables(spec, "fp64", tabs)
    with pytest.raises(hr2.Hr2Error) as ei:
        eng.add_setup(t64, setup, level_cache="stream")
    assert ei.value.code == hr2.HR2_EINVAL
    t = eng.add_tables(spec, "fp16", tabs)
    setup.interp = "linear"
    with pytest.raises(hr2.Hr2Error) as ei:
        eng.add_setup(t, setup, level_cache="stream")
    assert ei.value.code == hr2.HR2_EINVAL
    with pytest.raises(hr2.Hr2Error) as ei:
        hr2.hr2_set_stream_group(eng.ctx, -1)
    assert ei.value.code == hr2.HR2_EINVAL


def test_streamed_batch_replayed_from_a_cuda_graph(eng):
    """graphs.CapturedBatch on a streamed setup: its eager warm-up calls allocate the
    capture stream's ring, the capture records every group's build, plan and sweep, and a
    replay gives the eager call's bits."""
    from paper_1910_01070_b300 import graphs
    spec, tabs, setup = _case()
    t = eng.add_tables(spec, "fp16", tabs)
    s = eng.add_setup(t, setup, level_cache="stream")
    theta = W.draw_params(setup, 64, 9, W.Prior())
    ref_b, _, st = _run(eng, s, setup, theta)
    assert np.all(st == 0)
    D, sig = W.mock_observation(ref_b[0].astype(np.float64), 9)
    eng.set_observation(s, D, sig)
    hr2.hr2_set_stream_group(eng.ctx, 3)
    try:
        cb = graphs.CapturedBatch(eng.ctx, [s], 64, setup.n_bins, setup.n_nu)
        lnl, bins = cb.run(torch.as_tensor(theta), torch.zeros(64, dtype=torch.int32))
        got = bins.cpu().numpy()
    finally:
        hr2.hr2_set_stream_group(eng.ctx, 0)
    assert np.array_equal(got[:, : setup.n_bins], ref_b)
    assert np.all(np.isfinite(lnl.cpu().numpy()))


def test_concentrated_batch_builds_only_the_cells_it_uses(eng):
    """64 samples within 1 % of one draw sit in few T cells per level, so most of the ring's
    blocks are not rebuilt for them and hold an earlier group's contents: the results still
    match the level-gridded operand (FP32 rounding) and do not depend on the grouping."""
    spec, tabs, setup = _case()
    t = eng.add_tables(spec, "fp16", tabs)
    s_str = eng.add_setup(t, setup, level_cache="stream")
    s_lvl = eng.add_setup(t, setup, level_cache=True)
    base = W.draw_params(setup, 1, 10, W.Prior())[0]
    rng = np.random.default_rng(10)
    theta = np.repeat(base[None, :], 64, axis=0)
    theta[:, 3:10] *= 1.0 + 0.01 * rng.standard_normal((64, 7))
    prior = W.draw_params(setup, 64, 11, W.Prior())
    out = {}
    for g in (2, 0):
        hr2.hr2_set_stream_group(eng.ctx, g)
        try:
            _run(eng, s_str, setup, prior)          # fills the ring with other cells first
            out[g] = _run(eng, s_str, setup, theta)
        finally:
            hr2.hr2_set_stream_group(eng.ctx, 0)
    assert np.array_equal(out[2][0], out[0][0]) and np.array_equal(out[2][1], out[0][1])
    bl, hl, _ = _run(eng, s_lvl, setup, theta)
    assert np.all(out[0][2] == 0)
    for i in range(64):
        assert rel_flux_err(out[0][1][i], hl[i].astype(np.float64)) <= 2e-5
        assert rel_flux_err(out[0][0][i], bl[i].astype(np.float64)) <= 2e-5


def test_several_streamed_setups_in_one_call(eng):
    """Three streamed setups (8, 4 and 5 tiles; 20, 16 and 24 layers; 3, 2 and 1 absorbers)
    mixed in one call stream together: per group each builds its own tiles into its section
    of the ring, and a setup whose tiles are all behind takes no work.  Against the same
    setups with the level-gridded operand (FP32 rounding), across groupings (bit for bit)
    and against the oracle."""
    spec, tabs, _ = _case()
    specs = [W.make_setup(spec, 5030.0, 5990.0, 20, [0, 1, 2], 4, 3, 2, 400.0, 24),
             W.make_setup(spec, 5000.0, 5400.0, 16, [0, 2], 4, 3, 2, 300.0, 10),
             W.make_setup(spec, 5500.0, 6090.0, 24, [1], 4, 3, 2, 500.0, 16)]
    t = eng.add_tables(spec, "fp16", tabs)
    s_str = [eng.add_setup(t, sp, level_cache="stream") for sp in specs]
    s_lvl = [eng.add_setup(t, sp, level_cache=True) for sp in specs]
    n = 96
    sid = (np.arange(n) % 3).astype(np.int32)
    theta = np.concatenate([W.draw_params(specs[g], 1, 100 + i, W.Prior()) for i, g in enumerate(sid)])
    nb = max(sp.n_bins for sp in specs)
    nn = max(sp.n_nu for sp in specs)

    def run(setups):
        bins = torch.full((n, nb), -1.0, dtype=torch.float32, device="cuda")
        hi = torch.full((n, nn), -1.0, dtype=torch.float32, device="cuda")
        st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        hr2.forward_model_batch(eng.ctx, setups, torch.as_tensor(sid, device="cuda"),
                                torch.as_tensor(theta, device="cuda"), bins, hi, st)
        hr2.hr2_stream_check(eng.ctx)
        torch.cuda.synchronize()
        return bins.cpu().numpy(), hi.cpu().numpy(), st.cpu().numpy()

    out = {}
    for g in (2, 0):
        hr2.hr2_set_stream_group(eng.ctx, g)
        try:
            out[g] = run(s_str)
        finally:
            hr2.hr2_set_stream_group(eng.ctx, 0)
    assert np.all(out[0][2] == 0)
    assert np.array_equal(out[2][0], out[0][0]) and np.array_equal(out[2][1], out[0][1])
    bl, hl, _ = run(s_lvl)
    stored = tables_as_stored(tabs, "fp16")
    for i in range(n):
        sp = specs[sid[i]]
        assert rel_flux_err(out[0][1][i, : sp.n_nu], hl[i, : sp.n_nu].astype(np.float64)) <= 2e-5
        assert rel_flux_err(out[0][0][i, : sp.n_bins], bl[i, : sp.n_bins].astype(np.float64)) <= 2e-5
    for i in (0, 1, 2, 50, 94, 95):
        sp = specs[sid[i]]
        ob, otop, ok = oracle_model(stored, sp).forward(theta[i], want_top=True)
        assert ok
        assert rel_flux_err(out[0][1][i, : sp.n_nu], otop) <= FLUX_RTOL
        assert rel_flux_err(out[0][0][i, : sp.n_bins], ob) <= FLUX_RTOL
