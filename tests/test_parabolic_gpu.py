"""The parabolic short-characteristics option through the C ABI against the
oracle (same gates as the linear source), and its argument rules."""
import dataclasses

import numpy as np
import pytest

from paper_1910_01070_b300 import hr2
from paper_1910_01070_b300 import workloads as W
from paper_1910_01070_b300.engine import Engine
from tests.helpers import FLUX_RTOL, FP64_RTOL, oracle_model, rel_flux_err, tables_as_stored

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def eng():
    from paper_1910_01070_b300 import build
    build.build()
    e = Engine(0)
    yield e
    e.close()


def _run(eng, setups, sid, theta, nn):
    n = len(sid)
    nb = max(hr2.hr2_setup_info(s)[0] for s in setups)
    bins = torch.empty((n, nb), dtype=torch.float32, device="cuda")
    hi = torch.full((n, nn), -7.0, dtype=torch.float32, device="cuda")
    st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    eng.forward(setups, torch.as_tensor(sid, dtype=torch.int32, device="cuda"), torch.as_tensor(theta, device="cuda"),
                bins, hi, st)
    torch.cuda.synchronize()
    return bins.cpu().numpy().astype(np.float64), hi.cpu().numpy().astype(np.float64), st.cpu().numpy()


CASES = [(300, 25, 3, 4, 400.0), (200, 60, 2, 3, 0.0), (129, 6, 1, 8, 900.0)]


@pytest.mark.parametrize("storage", ["fp16-level-gridded", "fp16-direct", "fp64"])
@pytest.mark.parametrize("case", CASES, ids=["nu%d_L%d_K%d_mu%d" % c[:4] for c in CASES])
def test_parabolic_matches_oracle(eng, storage, case):
    n_nu, L, K, nmu, R = case
    spec = W.TableSpec(K, np.linspace(300.0, 3000.0, 7), np.linspace(-4.0, 2.0, 6), 5000.0, 1.0, n_nu + 9,
                       seed=80 + L)
    tabs = W.make_tables(spec)
    setup = W.make_setup(spec, 5004.0, 5004.0 + n_nu - 1, L, range(K), nmu, 2, 2, R, 9)
    setup.sc = "parabolic"
    st_ = storage[:4]
    t = eng.add_tables(spec, st_, tabs)
    s = eng.add_setup(t, setup, level_cache=(storage == "fp16-level-gridded"))
    theta = W.draw_params(setup, 5, 31, W.Prior(b=(0.8, 0.97)))
    b, h, st = _run(eng, [s], np.zeros(5, np.int32), theta, n_nu)
    assert np.all(st == 0)
    om = oracle_model(tables_as_stored(tabs, st_), setup)
    om_lin = oracle_model(tables_as_stored(tabs, st_), dataclasses.replace(setup, sc="linear"))
    tol = FLUX_RTOL if st_ == "fp16" else FP64_RTOL
    worst_lin = 0.0
    for i in range(5):
        ob, otop, ok = om.forward(theta[i], want_top=True)
        assert ok
        assert rel_flux_err(h[i], otop) <= tol
        assert rel_flux_err(b[i], ob) <= tol
        worst_lin = max(worst_lin, rel_flux_err(om_lin.forward(theta[i], want_top=True)[1], otop))
    assert worst_lin > 1e-4          # the option changes the result


def test_parabolic_on_the_batch_setup(eng):
    wl = W.batch1024_l100_k6_nu8501()
    tabs = W.make_tables(wl.table)
    spec = dataclasses.replace(wl.setups[0], sc="parabolic")
    t = eng.add_tables(wl.table, "fp16", tabs)
    s = eng.add_setup(t, spec)
    theta, _ = wl.params(6, seed_offset=41)
    b, h, st = _run(eng, [s], np.zeros(6, np.int32), theta, spec.n_nu)
    om = oracle_model(tables_as_stored(tabs, "fp16"), spec)
    for i in range(6):
        ob, otop, ok = om.forward(theta[i], want_top=True)
        assert rel_flux_err(h[i], otop) <= FLUX_RTOL
        assert rel_flux_err(b[i], ob) <= FLUX_RTOL


def test_one_source_interpolation_per_batch(eng):
    spec = W.TableSpec(1, np.linspace(300.0, 3000.0, 3), np.linspace(-4.0, 2.0, 3), 5000.0, 1.0, 64, seed=2)
    t = eng.add_tables(spec, "fp16", W.make_tables(spec))
    lin = W.make_setup(spec, 5000.0, 5063.0, 4, [0], 2, 1, 1, 0.0, 2)
    par = dataclasses.replace(lin, sc="parabolic")
    s1, s2 = eng.add_setup(t, lin), eng.add_setup(t, par)
    theta = W.draw_params(lin, 2, 3, W.Prior(b=(0.8, 0.95)))
    with pytest.raises(hr2.Hr2Error):
        _run(eng, [s1, s2], np.array([0, 1], np.int32), theta, 64)


@pytest.mark.parametrize("ks", [(1, 2), (5, 6), (7, 10), (13, 16), (1, 6)], ids=lambda ks: "k" + "_".join(map(str, ks)))
def test_parabolic_absorber_bounds(eng, ks):
    """The parabolic source on the level-gridded operand runs the kernel compiled
    for the batch's even absorber bound (counts from K-4 to K, zero-weight
    padding) or, for a wider mix ((1, 6)), the runtime-count kernel.  Every
    sample matches the oracle of its setup, and a setup's samples come out
    bit-identical alone (its own bound) and in a mix with a 1-absorber setup
    (runtime count): padding adds exact zeros in the same summation order."""
    K = max(ks)
    spec = W.TableSpec(K, np.linspace(300.0, 2500.0, 5), np.linspace(-4.0, 2.0, 4), 5000.0, 1.0, 300, seed=60 + K)
    tabs = W.make_tables(spec)
    t = eng.add_tables(spec, "fp16", tabs)
    specs = [dataclasses.replace(W.make_setup(spec, 5000.0 + 5 * g, 5260.0 + 9 * g, 14 + 5 * g, range(k), 3, 2, 2,
                                              300.0, 5), sc="parabolic") for g, k in enumerate(ks)]
    setups = [eng.add_setup(t, sp) for sp in specs]
    n = 8
    sid = np.arange(n, dtype=np.int32) % len(ks)
    theta = np.concatenate([W.draw_params(specs[g], 1, 200 + i, W.Prior(b=(0.8, 0.97))) for i, g in enumerate(sid)])
    nn = max(sp.n_nu for sp in specs)
    b, h, st = _run(eng, setups, sid, theta, nn)
    assert np.all(st == 0)
    stored = tables_as_stored(tabs, "fp16")
    for g, sp in enumerate(specs):
        om = oracle_model(stored, sp)
        for i in np.nonzero(sid == g)[0]:
            ob, otop, ok = om.forward(theta[i], want_top=True)
            assert ok
            assert rel_flux_err(h[i, :sp.n_nu], otop) <= FLUX_RTOL
            assert rel_flux_err(b[i, :sp.n_bins], ob) <= FLUX_RTOL
    # the widest setup alone, then mixed with a 1-absorber setup (runtime count)
    one = dataclasses.replace(W.make_setup(spec, 5003.0, 5200.0, 20, range(1), 3, 2, 2, 300.0, 5), sc="parabolic")
    s_one = eng.add_setup(t, one)
    g = len(ks) - 1
    idx = np.nonzero(sid == g)[0]
    b_alone, h_alone, _ = _run(eng, [setups[g]], np.zeros(len(idx), np.int32), theta[idx], nn)
    th_one = W.draw_params(one, 3, 9, W.Prior(b=(0.8, 0.97)))
    mix_sid = np.concatenate([np.zeros(len(idx), np.int32), np.ones(3, np.int32)])
    b_mix, h_mix, st_mix = _run(eng, [setups[g], s_one], mix_sid, np.concatenate([theta[idx], th_one]), nn)
    assert np.all(st_mix == 0)
    ng = specs[g].n_nu
    assert np.array_equal(h_mix[:len(idx), :ng], h_alone[:, :ng])
    assert np.array_equal(b_mix[:len(idx), :specs[g].n_bins], b_alone[:, :specs[g].n_bins])
