"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Gates (written here, not derived from the CUDA path):
  * FP16-offset tables, FP32 solve: max relative flux error per spectrum
    <= 1e-4 on F+ and on the binned model, against the oracle run on the
    same dequantised tables (the tables the kernels actually read);
  * plain FP64 path with FP64 tables: <= 2e-7, the rounding of its FP32
    outputs (the ABI returns F+ and the bins as float);
  * log-likelihood: same model bins -> FP64 reduction agrees to 1e-9
    relative; end to end |delta lnL| < 1e-3 for samples near the data.
Sizes span several 128-point tiles with ragged heads and tails; the full
workload sizes run in the launch shape the benchmark times and are checked
on sampled outputs.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1910_01070_b300 import hr2
from paper_1910_01070_b300 import workloads as W
from paper_1910_01070_b300.engine import Engine
from tests.helpers import FLUX_RTOL, FP64_RTOL, LNL_ATOL, oracle_model, rel_flux_err, tables_as_stored

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def eng():
    from paper_1910_01070_b300 import build
    build.build()
    e = Engine(0)
    yield e
    e.close()


def _dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _run(eng, setups, sid, theta, highres_ld=None):
    n = len(sid)
    nb = max(hr2.hr2_setup_info(s)[0] for s in setups)
    nn = highres_ld or max(hr2.hr2_setup_info(s)[1] for s in setups)
    bins = torch.full((n, nb), -7.0, dtype=torch.float32, device="cuda")
    hi = torch.full((n, nn), -7.0, dtype=torch.float32, device="cuda")
    st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    eng.forward(setups, _dev(sid, torch.int32), _dev(theta, torch.float64), bins, hi, st)
    hr2.hr2_stream_check(eng.ctx)             # no bounded device wait gave up
    torch.cuda.synchronize()
    return bins.cpu().numpy().astype(np.float64), hi.cpu().numpy().astype(np.float64), st.cpu().numpy()


def _compare(om, theta, bins, hi, tol, n_nu):
    ob, otop, ok = om.forward(theta, want_top=True)
    assert ok
    e_hi = rel_flux_err(hi[:n_nu], otop)
    e_b = rel_flux_err(bins[: om.n_bins], ob)
    assert e_hi <= tol, e_hi
    assert e_b <= tol, e_b
    return e_hi, e_b


# ------------------------------------------------------------ tiny grids
TINY = [
    # n_nu, L, K, nT, nP, n_mu, R, bins, first_off, fe (Ke, q)
    (16, 3, 2, 3, 3, 2, 0.0, 4, 0, (2, 1)),
    (100, 7, 3, 4, 3, 3, 500.0, 5, 0, (3, 2)),
    (130, 12, 1, 5, 4, 8, 2000.0, 7, 5, (2, 3)),
    (65, 1, 2, 2, 2, 1, 0.0, 3, 63, (1, 1)),
    (257, 30, 4, 6, 5, 5, 800.0, 9, 17, (4, 2)),
]


@pytest.mark.parametrize("storage", ["fp16-level-gridded", "fp16-direct", "fp64"])
@pytest.mark.parametrize("case", TINY, ids=[f"nu{c[0]}_L{c[1]}_K{c[2]}_mu{c[5]}" for c in TINY])
def test_tiny_grids_match_oracle(eng, storage, case):
    n_nu, L, K, nT, nP, nmu, R, nb, off, (Ke, q) = case
    spec = W.TableSpec(K, np.linspace(300.0, 2500.0, nT), np.linspace(-4.0, 2.0, nP), 5000.0, 1.0,
                       n_nu + off + 3, seed=hash(case) % 1000)
    tabs = W.make_tables(spec)
    setup = W.make_setup(spec, 5000.0 + off, 5000.0 + off + n_nu - 1, L, range(K), nmu, Ke, q, R, nb)
    t = eng.add_tables(spec, storage[:4], tabs)
    s = eng.add_setup(t, setup, level_cache=(storage == "fp16-level-gridded"))
    storage = storage[:4]
    theta = W.draw_params(setup, 4, 17, W.Prior(T1=(900.0, 2400.0), b=(0.85, 0.99)))
    bins, hi, st = _run(eng, [s], np.zeros(4, np.int32), theta, highres_ld=n_nu + 64)
    assert np.all(st == 0)
    om = oracle_model(tables_as_stored(tabs, storage), setup)
    tol = FLUX_RTOL if storage == "fp16" else FP64_RTOL
    for i in range(4):
        _compare(om, theta[i], bins[i], hi[i], tol, n_nu)
    assert np.all(hi[:, n_nu:] == -7.0)      # nothing written past the setup's points


@pytest.mark.parametrize("storage", ["fp16-level-gridded", "fp64"])
def test_bins_scale_over_distances_and_flux_factors(eng, storage):
    """The bins carry f (R/d)^2 (Eq. 9): over distances from 1e-6 to 1e4 pc and flux
    factors from 1e-3 to 1e3 the scale spans ~1e-3 .. 1e-29, and every bin still
    matches the oracle to the flux tolerance (the FP32 path applies it as an FP32
    head and tail)."""
    spec = W.TableSpec(3, np.linspace(300.0, 2500.0, 4), np.linspace(-4.0, 2.0, 3), 5000.0, 1.0, 200, seed=12)
    tabs = W.make_tables(spec)
    setup = W.make_setup(spec, 5010.0, 5189.0, 20, range(3), 3, 2, 2, 500.0, 6)
    t = eng.add_tables(spec, storage[:4], tabs)
    s = eng.add_setup(t, setup, level_cache=(storage == "fp16-level-gridded"))
    dist_f = [(1e-6, 1e3), (1e-3, 1.0), (1.0, 1e-3), (10.0, 1.0), (1e3, 1e3), (1e4, 1e-3)]
    theta = W.draw_params(setup, len(dist_f), 23, W.Prior(b=(0.8, 0.97)))
    for i, (d, f) in enumerate(dist_f):
        theta[i, W.P_DIST] = d
        theta[i, W.P_F] = f
    bins, hi, st = _run(eng, [s], np.zeros(len(dist_f), np.int32), theta)
    assert np.all(st == 0)
    om = oracle_model(tables_as_stored(tabs, storage[:4]), setup)
    tol = FLUX_RTOL if storage.startswith("fp16") else FP64_RTOL
    scales = []
    for i in range(len(dist_f)):
        _compare(om, theta[i], bins[i], hi[i], tol, setup.n_nu)
        scales.append(np.median(bins[i, :setup.n_bins]))
    assert max(scales) / min(scales) > 1e20      # the scale really spans that range


def test_cia_only_setup(eng):
    spec = W.TableSpec(2, np.linspace(300.0, 2500.0, 4), np.linspace(-4.0, 2.0, 3), 5000.0, 1.0, 90, seed=3)
    tabs = W.make_tables(spec)
    setup = W.make_setup(spec, 5000.0, 5089.0, 9, [], 3, 2, 1, 300.0, 4)
    t = eng.add_tables(spec, "fp16", tabs)
    s = eng.add_setup(t, setup)
    theta = W.draw_params(setup, 2, 5, W.Prior(b=(0.8, 0.95)))
    bins, hi, st = _run(eng, [s], np.zeros(2, np.int32), theta)
    om = oracle_model(tables_as_stored(tabs, "fp16"), setup)
    for i in range(2):
        _compare(om, theta[i], bins[i], hi[i], FLUX_RTOL, 90)


@pytest.mark.parametrize("storage", ["fp16-level-gridded", "fp16-direct", "fp64"])
def test_low_wavenumbers_small_x_planck(eng, storage):
    """20-339 cm^-1 with a hot profile: hc nu / kT falls below 1/16 on the first
    tiles, where 1 - e^{-x} of the Planck function comes from its series (the
    FP32 kernel runs those items through its small-x sweep), and rises to ~2 on
    the last ones.  Every path matches the oracle at its tolerance."""
    spec = W.TableSpec(3, np.linspace(300.0, 4000.0, 8), np.linspace(-4.0, 2.0, 5), 20.0, 1.0, 320, seed=33)
    tabs = W.make_tables(spec)
    st, direct = ("fp16", storage == "fp16-direct") if storage.startswith("fp16") else ("fp64", False)
    setup = W.make_setup(spec, 20.0, 339.0, 30, range(3), 4, 2, 2, 100.0, 5)
    t = eng.add_tables(spec, st, tabs)
    s = eng.add_setup(t, setup, level_cache=not direct)
    theta = W.draw_params(setup, 6, 17, W.Prior(T1=(2500.0, 3800.0), b=(0.85, 0.97)))
    x_min = 1.4387768775039337 * 20.0 / theta[:, W.P_T0].max()
    assert x_min < 1.0 / 16.0
    bins, hi, status = _run(eng, [s], np.zeros(6, np.int32), theta)
    assert np.all(status == 0)
    om = oracle_model(tables_as_stored(tabs, st), setup)
    tol = FLUX_RTOL if st == "fp16" else FP64_RTOL
    for i in range(6):
        _compare(om, theta[i], bins[i], hi[i], tol, setup.n_nu)


def _absorber_spec(K, seed, with_cia=True):
    spec = W.TableSpec(K, np.linspace(300.0, 2500.0, 5), np.linspace(-4.0, 2.0, 4), 5000.0, 1.0, 300, seed=seed)
    tabs = W.make_tables(spec)
    if not with_cia:
        tabs = dict(tabs, log10_cia_h2h2=None, log10_cia_h2he=None)
    return spec, tabs


@pytest.mark.parametrize("K,with_cia", [(3, False), (5, False), (5, True), (6, False)])
def test_absorber_counts_level_gridded(eng, K, with_cia):
    """The level-gridded kernel is compiled for an even absorber bound; an odd
    count runs with one zero-weight absorber, whose shared-memory rows are the
    stage's next rows (the CIA rows, zero when the tables have no CIA)."""
    spec, tabs = _absorber_spec(K, 40 + K, with_cia)
    setup = W.make_setup(spec, 5000.0, 5299.0, 20, range(K), 4, 2, 2, 300.0, 6)
    t = eng.add_tables(spec, "fp16", tabs)
    s = eng.add_setup(t, setup)
    theta = W.draw_params(setup, 8, 23, W.Prior(b=(0.8, 0.97)))
    bins, hi, st = _run(eng, [s], np.zeros(8, np.int32), theta)
    assert np.all(st == 0)
    om = oracle_model(tables_as_stored(tabs, "fp16"), setup)
    for i in range(8):
        _compare(om, theta[i], bins[i], hi[i], FLUX_RTOL, 300)


@pytest.mark.parametrize("ks", [(5, 6), (4, 6), (6, 3, 5), (2, 6), (1, 6), (2, 7, 5), (8, 5, 7), (10, 6, 9, 7),
                                (12, 9), (16, 13, 12)])
def test_mixed_absorber_counts_in_one_batch(eng, ks):
    """Setups with different absorber counts in one batch: counts from K-4 to K
    share the even bound K (zero-weight padding, up to 4 padded absorbers
    reading the stage's other values; from a bound of 8 up each item runs its
    own setup's even bound), wider mixes ((1, 6), (2, 7, 5)) take the
    runtime-count kernel.  Every sample matches the oracle of its setup."""
    spec, tabs = _absorber_spec(max(ks), 77)
    t = eng.add_tables(spec, "fp16", tabs)
    specs = [W.make_setup(spec, 5000.0 + 7 * g, 5250.0 + 11 * g, 16 + 3 * g, range(k), 3, 2, 2, 300.0, 5)
             for g, k in enumerate(ks)]
    setups = [eng.add_setup(t, sp) for sp in specs]
    sid = np.arange(12, dtype=np.int32) % len(ks)
    theta = np.concatenate([W.draw_params(specs[g], 1, 100 + i, W.Prior(b=(0.8, 0.97))) for i, g in enumerate(sid)])
    bins, hi, st = _run(eng, setups, sid, theta)
    assert np.all(st == 0)
    stored = tables_as_stored(tabs, "fp16")
    for g, sp in enumerate(specs):
        om = oracle_model(stored, sp)
        for i in np.nonzero(sid == g)[0]:
            _compare(om, theta[i], bins[i], hi[i], FLUX_RTOL, sp.n_nu)


# ------------------------------------------------------------ the largest shapes the ABI accepts
@pytest.mark.parametrize("storage", ["fp16-level-gridded", "fp16-direct", "fp64"])
def test_maximum_sizes(eng, storage):
    """HR2_MAX_LEVELS - 1 layers, HR2_MAX_SPECIES absorbers (the 16-absorber kernel, whose
    per-warp pipeline takes 37 KB of shared memory), HR2_MAX_MU angle nodes and
    HR2_MAX_TNODES temperature nodes (5 cubic elements), on a ragged 300-point range."""
    K = 16
    spec = W.TableSpec(K, np.linspace(300.0, 3000.0, 10), np.linspace(-4.0, 2.0, 8), 5000.0, 1.0, 330, seed=91)
    tabs = W.make_tables(spec)
    setup = W.make_setup(spec, 5011.0, 5310.0, 255, range(K), 8, 5, 3, 300.0, 10)
    assert setup.n_tnodes == 16
    st_ = storage[:4]
    t = eng.add_tables(spec, st_, tabs)
    s = eng.add_setup(t, setup, level_cache=(storage == "fp16-level-gridded"))
    theta = W.draw_params(setup, 3, 17, W.Prior(b=(0.9, 0.99), log_x=(-9.0, -4.0)))
    bins, hi, st = _run(eng, [s], np.zeros(3, np.int32), theta)
    assert np.all(st == 0)
    om = oracle_model(tables_as_stored(tabs, st_), setup)
    tol = FLUX_RTOL if st_ == "fp16" else FP64_RTOL
    for i in range(3):
        _compare(om, theta[i], bins[i], hi[i], tol, setup.n_nu)


# ------------------------------------------------------------ linear-sigma interpolation option
@pytest.mark.parametrize("storage", ["fp16-level-gridded", "fp64"])
@pytest.mark.parametrize("case", TINY[1:], ids=[f"nu{c[0]}_L{c[1]}_K{c[2]}_mu{c[5]}" for c in TINY[1:]])
def test_linear_option_tiny_grids_match_oracle(eng, storage, case):
    n_nu, L, K, nT, nP, nmu, R, nb, off, (Ke, q) = case
    spec = W.TableSpec(K, np.linspace(300.0, 2500.0, nT), np.linspace(-4.0, 2.0, nP), 5000.0, 1.0,
                       n_nu + off + 3, seed=hash(case) % 1000 + 1)
    tabs = W.make_tables(spec)
    setup = W.make_setup(spec, 5000.0 + off, 5000.0 + off + n_nu - 1, L, range(K), nmu, Ke, q, R, nb)
    setup.interp = "linear"
    t = eng.add_tables(spec, storage[:4], tabs)
    s = eng.add_setup(t, setup, level_cache=(storage == "fp16-level-gridded"))
    theta = W.draw_params(setup, 4, 19, W.Prior(T1=(900.0, 2400.0), b=(0.85, 0.99)))
    bins, hi, st = _run(eng, [s], np.zeros(4, np.int32), theta, highres_ld=n_nu + 64)
    assert np.all(st == 0)
    om = oracle_model(tables_as_stored(tabs, storage[:4]), setup)
    tol = FLUX_RTOL if storage[:4] == "fp16" else FP64_RTOL
    for i in range(4):
        _compare(om, theta[i], bins[i], hi[i], tol, n_nu)


@pytest.mark.parametrize("storage", ["fp16", "fp64"])
def test_linear_option_on_the_batch_workload_with_lnl(eng, storage):
    """The 100-layer, 6-absorber setup with the linear option: spectra against
    the oracle run with the same option, and lnL near the data-generating
    sample.  Both options give different spectra (the option is not a no-op)."""
    wl = W.batch1024_l100_k6_nu8501()
    tabs = W.make_tables(wl.table)
    stored = tables_as_stored(tabs, storage)
    spec = dataclasses.replace(wl.setups[0], interp="linear")
    t = eng.add_tables(wl.table, storage, tabs)
    s = eng.add_setup(t, spec)
    om = oracle_model(stored, spec)
    truth = wl.truth(0)
    tb, ok = om.forward(truth)
    assert ok
    D, sig = W.mock_observation(tb, wl.seed + 5)
    eng.set_observation(s, D, sig)
    theta, _ = wl.params(8, seed_offset=31)
    near = np.repeat(truth[None, :], 3, axis=0)
    near[1:, 0] += np.array([1e-3, -1e-3])
    theta = np.concatenate([theta, near])
    sid = np.zeros(len(theta), np.int32)
    bins, hi, status = _run(eng, [s], sid, theta)
    assert np.all(status == 0)
    tol = FLUX_RTOL if storage == "fp16" else FP64_RTOL
    for i in range(len(theta)):
        _compare(om, theta[i], bins[i], hi[i], tol, spec.n_nu)
    om_log = oracle_model(stored, wl.setups[0])
    assert np.max(np.abs(om_log.forward(theta[0])[0] / bins[0] - 1.0)) > 1e-3
    lnl = eng.lnl([s], _dev(sid, torch.int32), _dev(bins.astype(np.float32), torch.float32)).cpu().numpy()
    for i in range(len(theta) - 3, len(theta)):
        ref = oracle.lnL(D, sig, om.forward(theta[i])[0])
        assert abs(lnl[i] - ref) < LNL_ATOL, (i, lnl[i], ref)


def test_linear_option_argument_errors(eng):
    spec, tabs = _absorber_spec(2, 5)
    t = eng.add_tables(spec, "fp16", tabs)
    setup = W.make_setup(spec, 5000.0, 5199.0, 8, range(2), 2, 1, 1, 0.0, 3)
    setup.interp = "linear"
    with pytest.raises(hr2.Hr2Error) as ei:                 # FP16 tables need the level-gridded operand
        eng.add_setup(t, setup, level_cache=False)
    assert ei.value.code == hr2.HR2_EINVAL
    lin = eng.add_setup(t, setup)
    log = eng.add_setup(t, dataclasses.replace(setup, interp="log10"))
    theta = W.draw_params(setup, 2, 3, W.Prior(b=(0.8, 0.95)))
    with pytest.raises(hr2.Hr2Error):                        # one option per batch
        _run(eng, [lin, log], np.array([0, 1], np.int32), theta)


# ------------------------------------------------------------ named workloads
_CACHE = {}


def _workload_on(eng, name, storage, n=None):
    key = (name, storage)
    if key not in _CACHE:
        wl = W.WORKLOADS[name]() if storage is None else W.WORKLOADS[name]()
        tabs = W.make_tables(wl.table)
        st = storage or wl.storage
        t = eng.add_tables(wl.table, st, tabs)
        setups = [eng.add_setup(t, s) for s in wl.setups]
        _CACHE[key] = (wl, tabs, tables_as_stored(tabs, st), setups, st, t)
    return _CACHE[key][:5]


def _tables_of(name, storage):
    return _CACHE[(name, storage)][5]


@pytest.mark.parametrize("storage", ["fp64", "fp16"])
def test_single_model_50_layers(eng, storage):
    wl, tabs, stored, setups, st = _workload_on(eng, "single_l50_k1_nu6001", storage)
    theta, sid = wl.params()
    bins, hi, status = _run(eng, setups, sid, theta)
    om = oracle_model(stored, wl.setups[0])
    tol = FLUX_RTOL if st == "fp16" else FP64_RTOL
    e = _compare(om, theta[0], bins[0], hi[0], tol, wl.setups[0].n_nu)
    print("single model", storage, "rel err (F+, bins):", e)


def _observation(eng, wl, stored, setups, g=0):
    om = oracle_model(stored, wl.setups[g])
    truth = wl.truth(g)
    tb, ok = om.forward(truth)
    assert ok
    D, sig = W.mock_observation(tb, wl.seed + g)
    eng.set_observation(setups[g], D, sig)
    return om, truth, D, sig


@pytest.mark.parametrize("storage", ["fp16", "fp64"])
def test_batch_100_layers_reduced_with_lnl(eng, storage):
    wl, tabs, stored, setups, st = _workload_on(eng, "batch1024_l100_k6_nu8501", storage)
    om, truth, D, sig = _observation(eng, wl, stored, setups)
    theta, sid = wl.params(12)
    # near-truth samples: the truth and small perturbations of it
    near = np.repeat(truth[None, :], 4, axis=0)
    near[1:, 0] += np.array([1e-3, -2e-3, 5e-4])
    near[1:, 3:10] *= 1.0 + np.array([1e-3, -1e-3, 2e-3])[:, None]
    theta = np.concatenate([theta, near])
    sid = np.zeros(len(theta), np.int32)
    bins, hi, status = _run(eng, setups, sid, theta)
    assert np.all(status == 0)
    tol = FLUX_RTOL if st == "fp16" else FP64_RTOL
    worst = 0.0
    ob_all = []
    for i in range(len(theta)):
        e = _compare(om, theta[i], bins[i], hi[i], tol, wl.setups[0].n_nu)
        worst = max(worst, *e)
        ob_all.append(om.forward(theta[i])[0])
    print(storage, "worst rel flux err", worst)
    # likelihood on the GPU's own bins (FP64 reduction) and end to end
    bins_t = _dev(bins.astype(np.float32), torch.float32)
    lnl = eng.lnl(setups, _dev(sid, torch.int32), bins_t).cpu().numpy()
    for i in range(len(theta)):
        ref_same = oracle.lnL(D, sig, bins[i])
        assert abs(lnl[i] - ref_same) <= 1e-9 * abs(ref_same) + 1e-9
    for i in range(len(theta) - 4, len(theta)):
        ref = oracle.lnL(D, sig, ob_all[i])
        d_sig = (bins[i] - ob_all[i]) / sig
        print("sample %d: dlnL %.3e  max|dDm|/sigma %.3e  max Dm/sigma %.1f  max rel bin err %.2e"
              % (i, lnl[i] - ref, np.max(np.abs(d_sig)), np.max(ob_all[i] / sig),
                 np.max(np.abs(bins[i] / ob_all[i] - 1))))
    for i in range(len(theta) - 4, len(theta)):
        ref = oracle.lnL(D, sig, ob_all[i])
        assert abs(lnl[i] - ref) < LNL_ATOL, (i, lnl[i], ref)
    # far from the data (the prior draws) lnL is large and |dlnL| may exceed LNL_ATOL, but it
    # must stay within what the flux tolerance allows: with |Dm_gpu - Dm| <= e_b per bin,
    # e_b = tol (|Dm_b| + 1e-6 max|Dm|) (the relative-error gate with its floor),
    # |dlnL| <= sum e_b |D_b - Dm_b| / s_b^2 + sum e_b^2 / (2 s_b^2)   (Eq. 19 expanded)
    for i in range(len(theta) - 4):
        ref = oracle.lnL(D, sig, ob_all[i])
        e = tol * (np.abs(ob_all[i]) + 1e-6 * np.max(np.abs(ob_all[i])))
        bound = np.sum(e * np.abs(D - ob_all[i]) / sig ** 2) + np.sum(e ** 2 / (2 * sig ** 2))
        print("sample %d: lnL %.4e  dlnL %.3e  bound %.3e" % (i, ref, lnl[i] - ref, bound))
        assert abs(lnl[i] - ref) <= bound + 1e-9 * abs(ref), (i, lnl[i] - ref, bound)
    # error inflation (Eqs. 22-23)
    eps = np.full(len(theta), np.log10(np.median(sig) ** 2))
    eps[0] = np.nan
    lnl_e = eng.lnl(setups, _dev(sid, torch.int32), bins_t, _dev(eps, torch.float64)).cpu().numpy()
    for i in range(len(theta)):
        ref = oracle.lnL(D, sig, bins[i], eps[i])
        assert abs(lnl_e[i] - ref) <= 1e-9 * abs(ref) + 1e-9


def test_batch_1024_full_size_sampled(eng):
    """The benchmark's workload and launch shape; 12 samples checked fully."""
    wl, tabs, stored, setups, st = _workload_on(eng, "batch1024_l100_k6_nu8501", "fp16")
    theta, sid = wl.params()
    assert len(theta) == 1024
    bins, hi, status = _run(eng, setups, sid, theta)
    om = oracle_model(stored, wl.setups[0])
    pick = np.random.default_rng(0).choice(1024, 12, replace=False)
    for i in pick:
        _compare(om, theta[i], bins[i], hi[i], FLUX_RTOL, wl.setups[0].n_nu)
    assert np.all(np.isfinite(bins[status == 0]))


def test_uneven_three_setups_sampled_and_alone_equals_mix(eng):
    wl, tabs, stored, setups, st = _workload_on(eng, "uneven2048_3setups", "fp16")
    theta, sid = wl.params()
    bins, hi, status = _run(eng, setups, sid, theta, highres_ld=max(s.n_nu for s in wl.setups))
    rng = np.random.default_rng(1)
    for g, s in enumerate(wl.setups):
        om = oracle_model(stored, s)
        idx = np.nonzero(sid == g)[0]
        for i in rng.choice(idx, 2, replace=False):
            _compare(om, theta[i], bins[i], hi[i], FLUX_RTOL, s.n_nu)
    # a sample's result does not depend on the rest of the batch
    sub = rng.choice(len(theta), 37, replace=False)
    b2, h2, _ = _run(eng, setups, sid[sub], theta[sub], highres_ld=hi.shape[1])
    assert np.array_equal(b2, bins[sub])
    assert np.array_equal(h2, hi[sub])


@pytest.mark.parametrize("sc", ["linear", "parabolic"])
def test_single_setup_launch_equals_the_mixed_launch(eng, sc):
    """A launch with one setup runs the sweep compiled with the setup index fixed (the
    angle-node constants at fixed parameter offsets); the same samples in a launch with
    several setups run the general sweep.  Same arithmetic: the same bits, for each setup
    of the uneven batch (6-10 absorbers, 81-121 levels; the first four with the parabolic
    source)."""
    wl, tabs, stored, setups, st = _workload_on(eng, "uneven2048_3setups", "fp16")
    theta, sid = wl.params(48, seed_offset=31)
    if sc == "parabolic":
        t = _tables_of("uneven2048_3setups", "fp16")
        setups = [eng.add_setup(t, dataclasses.replace(s, sc="parabolic")) for s in wl.setups[:4]]
        keep = sid < 4
        theta, sid = theta[keep], sid[keep]
    ld = max(s.n_nu for s in wl.setups)
    b_mix, h_mix, _ = _run(eng, setups, sid, theta, highres_ld=ld)
    for g in range(len(setups)):
        idx = np.nonzero(sid == g)[0]
        if len(idx) == 0:
            continue
        b1, h1, status = _run(eng, [setups[g]], np.zeros(len(idx), np.int32), theta[idx], highres_ld=ld)
        assert np.all(status == 0)
        nb = wl.setups[g].n_bins
        assert np.array_equal(b1[:, :nb], b_mix[idx][:, :nb]), g
        assert np.array_equal(h1, h_mix[idx]), g


def test_direct_fp16_path_on_uneven_setups(eng):
    """The bilinear-in-place FP16 path (no level-gridded operand) on mixed setups."""
    wl, tabs, stored, setups, st = _workload_on(eng, "uneven2048_3setups", "fp16")
    t = _tables_of("uneven2048_3setups", "fp16")
    direct = [eng.add_setup(t, s, level_cache=False) for s in wl.setups]
    theta, sid = wl.params(60, seed_offset=9)
    bins, hi, status = _run(eng, direct, sid, theta, highres_ld=max(s.n_nu for s in wl.setups))
    for g, s in enumerate(wl.setups):
        om = oracle_model(stored, s)
        for i in np.nonzero(sid == g)[0][:1]:
            _compare(om, theta[i], bins[i], hi[i], FLUX_RTOL, s.n_nu)
    with pytest.raises(hr2.Hr2Error):             # one batch takes setups of one kind
        _run(eng, [setups[0], direct[1]], np.zeros(2, np.int32), theta[:2])


def test_two_pass_direct_path_is_the_one_pass_result(eng):
    """Small batches on tables read in place run in two passes (every level's absorption
    coefficient first, then the sweep reading it back) with the one-pass arithmetic: the same
    spectra bit for bit, for mixed setups, batch sizes around the threshold and a sample with
    an invalid setup index; and the oracle agrees."""
    wl, tabs, stored, setups, st = _workload_on(eng, "uneven2048_3setups", "fp16")
    t = _tables_of("uneven2048_3setups", "fp16")
    direct = [eng.add_setup(t, s, level_cache=False) for s in wl.setups]
    theta, sid = wl.params(7, seed_offset=21)
    sid = sid.copy()
    sid[5] = -1
    ld = max(s.n_nu for s in wl.setups)
    old = hr2.hr2_get_launch_config(eng.ctx)
    try:
        eng.set_launch_config(2, 8, 1, 0, 0)
        one = _run(eng, direct, sid, theta, highres_ld=ld)
        for m in (1, 3, 7):
            eng.set_launch_config(2, 8, 1, 0, m)
            two = _run(eng, direct, sid[:m], theta[:m], highres_ld=ld)
            for x, y in zip(two, one):
                assert np.array_equal(x, y[:m], equal_nan=True)
    finally:
        eng.set_launch_config(*old)
    assert one[2][5] == hr2.HR2_SAMPLE_BAD_SETUP and np.all(np.isnan(one[0][5]))
    for i in (0, 6):
        g = int(sid[i])
        _compare(oracle_model(stored, wl.setups[g]), theta[i], one[0][i], one[1][i], FLUX_RTOL, wl.setups[g].n_nu)


def test_small_batches_use_every_warp(eng):
    """Batches smaller than a work item (1, 2, 3 samples) give the same results as inside a large batch."""
    wl, tabs, stored, setups, st = _workload_on(eng, "batch1024_l100_k6_nu8501", "fp16")
    theta, sid = wl.params(8, seed_offset=21)
    ref = _run(eng, setups, sid, theta)
    for m in (1, 2, 3):
        got = _run(eng, setups, sid[:m], theta[:m])
        assert np.array_equal(got[0], ref[0][:m]) and np.array_equal(got[1], ref[1][:m])


@pytest.mark.parametrize("K,n_mu", [(12, 8), (9, 6), (6, 4)])
def test_stage_variants_agree_bitwise(eng, K, n_mu):
    """The level-gridded kernels with more than 4 angle nodes and an absorber
    bound of 8 or more run with two shared-memory stages below 16 samples and
    one stage from 16 up; the two variants (and the one-stage kernels of the
    other shapes at any batch size) give bit-identical spectra, and both match
    the oracle."""
    spec, tabs = _absorber_spec(K, 90 + K)
    setup = W.make_setup(spec, 5000.0, 5299.0, 24, range(K), n_mu, 3, 2, 300.0, 6)
    t = eng.add_tables(spec, "fp16", tabs)
    s = eng.add_setup(t, setup)
    theta = W.draw_params(setup, 40, 61, W.Prior(b=(0.8, 0.97)))
    sid = np.zeros(40, np.int32)
    big = _run(eng, [s], sid, theta)
    for m in (1, 5, 15):
        small = _run(eng, [s], sid[:m], theta[:m])
        assert np.array_equal(small[0], big[0][:m]) and np.array_equal(small[1], big[1][:m])
    # the depth asked for explicitly (where both exist), with wider items
    old = hr2.hr2_get_launch_config(eng.ctx)
    try:
        for stages in (1, 2):
            eng.set_launch_config(2, 8, 2, stages)
            for m in (3, 40):
                got = _run(eng, [s], sid[:m], theta[:m])
                assert np.array_equal(got[0], big[0][:m]) and np.array_equal(got[1], big[1][:m])
    finally:
        eng.set_launch_config(*old)
    om = oracle_model(tables_as_stored(tabs, "fp16"), setup)
    for i in (0, 17, 39):
        _compare(om, theta[i], big[0][i], big[1][i], FLUX_RTOL, 300)


def test_launch_shapes_agree_bitwise(eng):
    """Every launch shape the autotuner may pick (samples and wavenumber tiles per work item,
    CTAs per SM) computes each sample and point the same way."""
    wl, tabs, stored, setups, st = _workload_on(eng, "uneven2048_3setups", "fp16")
    theta, sid = wl.params(96, seed_offset=3)
    ref = None
    old = hr2.hr2_get_launch_config(eng.ctx)
    try:
        for shape in ((1, 1, 1, 0), (4, 2, 1, 0), (8, 3, 2, 0), (16, 1, 4, 0), (2, 8, 3, 0), (2, 8, 16, 0)):
            eng.set_launch_config(*shape)
            out = _run(eng, setups, sid, theta, highres_ld=10001)
            if ref is None:
                ref = out
            else:
                assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])
    finally:
        eng.set_launch_config(*old)


def test_invalid_samples_flagged(eng):
    wl, tabs, stored, setups, st = _workload_on(eng, "batch1024_l100_k6_nu8501", "fp16")
    om, truth, D, sig = _observation(eng, wl, stored, setups)
    theta = np.repeat(truth[None], 5, axis=0)
    theta[1, 1] = -1.0                 # f <= 0
    theta[2, W.P_X0] = 0.1             # abundances sum above 1
    theta[3, W.P_T0 + 2] = -50.0       # negative temperature node
    sid = np.array([0, 0, 0, 0, 3], np.int32)   # last: setup index out of range
    bins, hi, status = _run(eng, setups, sid, theta)
    assert status[0] == 0
    assert status[1] & hr2.HR2_SAMPLE_BAD_SCALE
    assert status[2] & hr2.HR2_SAMPLE_BAD_ABUND
    assert status[3] & hr2.HR2_SAMPLE_BAD_T
    assert status[4] == hr2.HR2_SAMPLE_BAD_SETUP
    assert np.all(np.isnan(bins[1:]))
    lnl = eng.lnl(setups, _dev(sid, torch.int32), _dev(bins.astype(np.float32), torch.float32)).cpu().numpy()
    assert np.isfinite(lnl[0]) and np.all(lnl[1:] == -np.inf)


def test_evaluate_host_matches_device_calls(eng):
    wl, tabs, stored, setups, st = _workload_on(eng, "batch1024_l100_k6_nu8501", "fp16")
    _observation(eng, wl, stored, setups)
    theta, sid = wl.params(64, seed_offset=5)
    out_bins = np.zeros((64, 300), np.float32)
    lnl_h = eng.evaluate_host(setups, sid, theta, out_bins=out_bins)
    bins, hi, status = _run(eng, setups, sid, theta)
    lnl_d = eng.lnl(setups, _dev(sid, torch.int32), _dev(bins.astype(np.float32), torch.float32)).cpu().numpy()
    assert np.array_equal(out_bins.astype(np.float64), bins)
    assert np.array_equal(lnl_h, lnl_d)


def test_empty_batch_and_argument_errors(eng):
    wl, tabs, stored, setups, st = _workload_on(eng, "batch1024_l100_k6_nu8501", "fp16")
    e = torch.empty((0, 300), dtype=torch.float32, device="cuda")
    hr2.forward_model_batch(eng.ctx, setups, torch.empty(0, dtype=torch.int32, device="cuda"),
                            torch.empty((0, hr2.HR2_NPARAM), dtype=torch.float64, device="cuda"), e)
    theta, sid = wl.params(2)
    small = torch.empty((2, 10), dtype=torch.float32, device="cuda")
    with pytest.raises(hr2.Hr2Error) as ei:
        hr2.forward_model_batch(eng.ctx, setups, _dev(sid, torch.int32), _dev(theta, torch.float64), small)
    assert ei.value.code == hr2.HR2_EINVAL
    with pytest.raises(hr2.Hr2Error) as ei:
        bad = W.make_setup(wl.table, 4000.0, 12500.0, 100, range(6), 4, 3, 2, 300.0, 300)
        bad.nu_first = wl.table.n_nu - 10
        eng.add_setup(_tables_of("batch1024_l100_k6_nu8501", "fp16"), bad)
    assert ei.value.code == hr2.HR2_EINVAL
    with pytest.raises(hr2.Hr2Error) as ei:      # a bin with no point in it
        edges = np.array([4000.0, 4000.2, 4000.4, 5000.0])
        s = W.make_setup(wl.table, 4000.0, 5000.0, 10, [0], 2, 1, 1, 0.0, 3)
        s.bin_edges = edges
        eng.add_setup(_tables_of("batch1024_l100_k6_nu8501", "fp16"), s)
    assert ei.value.code == hr2.HR2_EINVAL


def test_memory_budget_admission():
    e = Engine(0, mem_budget_bytes=1 << 20)
    try:
        wl = W.batch1024_l100_k6_nu8501()
        with pytest.raises(hr2.Hr2Error) as ei:
            e.add_tables(wl.table, "fp16", W.make_tables(wl.table))
        assert ei.value.code == hr2.HR2_ENOMEM
        assert e.memory()[0] <= 1 << 20
    finally:
        e.close()


def test_level_gridded_operand_where_it_fits():
    """level_cache='auto' builds the level-gridded operand only where it fits the context's budget
    (and half the free device memory); otherwise the setup streams the operand (built per call
    into a ring that fits the budget) and reads the FP16 tables directly below 32 samples, with
    the same results as a setup created without the operand there.  The operand's size is
    levels x (T cells) x (absorbers + 2 CIA rows) x tiles of 128 points x 8 bytes."""
    spec, tabs = _absorber_spec(6, 77)
    setup = W.make_setup(spec, 5000.0, 5299.0, 24, range(6), 4, 3, 2, 300.0, 6)
    theta = W.draw_params(setup, 20, 71, W.Prior())
    sid = np.zeros(20, np.int32)
    n_tiles = (setup.nu_first + setup.n_nu - 1) // 128 - setup.nu_first // 128 + 1
    operand = (setup.n_layers + 1) * (len(spec.T_grid) - 1) * (6 + 2) * n_tiles * 128 * 8
    with Engine(0) as big:
        t = big.add_tables(spec, "fp16", tabs)
        s_auto = big.add_setup(t, setup, level_cache="auto")
        s_direct = big.add_setup(t, setup, level_cache=False)
        b, ob, lg = hr2.hr2_setup_memory(s_auto)
        assert lg and ob == operand and b > ob
        b2, ob2, lg2 = hr2.hr2_setup_memory(s_direct)
        assert not lg2 and ob2 == 0 and b2 == b - ob
        ref_direct = _run(big, [s_direct], sid, theta)
        theta64 = W.draw_params(setup, 64, 72, W.Prior())
        ref64 = _run(big, [s_direct], np.zeros(64, np.int32), theta64)
    with Engine(0) as probe:
        t = probe.add_tables(spec, "fp16", tabs)
        tables_bytes = probe.memory()[0]
    # a budget that holds the tables and the setup without the operand, not with it
    with Engine(0, mem_budget_bytes=tables_bytes + b2 + operand // 2) as small:
        t = small.add_tables(spec, "fp16", tabs)
        s = small.add_setup(t, setup, level_cache="auto")
        assert hr2.hr2_setup_memory(s)[2] is False
        assert hr2.hr2_setup_streamed(s)
        got = _run(small, [s], sid, theta)
        assert np.array_equal(got[0], ref_direct[0]) and np.array_equal(got[1], ref_direct[1])
        # 64 samples stream the operand through a ring that fits what the budget leaves
        got64 = _run(small, [s], np.zeros(64, np.int32), theta64)
        used, budget = small.memory()
        assert used <= budget
        for i in range(64):
            assert rel_flux_err(got64[1][i], ref64[1][i].astype(np.float64)) <= 2e-5
            assert rel_flux_err(got64[0][i], ref64[0][i].astype(np.float64)) <= 2e-5
        with pytest.raises(hr2.Hr2Error) as ei:
            small.add_setup(t, dataclasses.replace(setup, interp="linear"), level_cache="auto")
        assert ei.value.code == hr2.HR2_ENOMEM


@pytest.mark.slow
def test_large_tables_sampled(eng):
    """290001-point, 12-absorber FP16 tables (~2 GB), batch 256, 8 nodes, R=1000 -> 2000 bins."""
    wl = W.large_l100_k12_nu290001_b256()
    spec = wl.table
    h2h2, h2he = W.cia_tables(spec)
    t = hr2.create_opacity_tables(eng.ctx, spec.T_grid, spec.log10p_grid, spec.nu0, spec.dnu, spec.n_nu,
                                  spec.masses, None, h2h2, h2he, hr2.HR2_STORE_FP16_OFFSET)
    from tests.helpers import fp16_offset_dequantise
    stored = np.empty((spec.n_species, len(spec.T_grid), len(spec.log10p_grid), spec.n_nu))
    for s in range(spec.n_species):
        v = W.species_table(spec, s)
        hr2.hr2_tables_upload_species(eng.ctx, t, s, v)
        stored[s] = fp16_offset_dequantise(v)
        del v
    s0 = eng.add_setup(t, wl.setups[0])
    theta, sid = wl.params()
    bins, hi, status = _run(eng, [s0], sid, theta)
    tabs = dict(T_grid=spec.T_grid, log10p_grid=spec.log10p_grid, nu0=spec.nu0, dnu=spec.dnu,
                log10_sigma=stored, log10_cia_h2h2=fp16_offset_dequantise(h2h2),
                log10_cia_h2he=fp16_offset_dequantise(h2he), species_mass=spec.masses)
    om = oracle_model(tabs, wl.setups[0])
    rng = np.random.default_rng(2)
    idx = np.sort(rng.choice(spec.n_nu, 1500, replace=False))
    sel = np.sort(rng.choice(wl.setups[0].n_bins, 10, replace=False))
    for i in (0, 131):
        ref, ok = om.top_flux_at(theta[i], idx)
        assert ok
        assert rel_flux_err(hi[i][idx], ref) <= FLUX_RTOL
        refb, _ = om.bins_at(theta[i], sel)
        assert rel_flux_err(bins[i][sel], refb) <= FLUX_RTOL
    # the same batch on the streamed operand: no 62 GB operand, a ring of one group of tiles
    s1 = eng.add_setup(t, wl.setups[0], level_cache="stream")
    b1, h1, st1 = _run(eng, [s1], sid, theta)
    assert np.all(st1 == 0)
    for i in (0, 131):
        ref, _ = om.top_flux_at(theta[i], idx)
        assert rel_flux_err(h1[i][idx], ref) <= FLUX_RTOL
        refb, _ = om.bins_at(theta[i], sel)
        assert rel_flux_err(b1[i][sel], refb) <= FLUX_RTOL
