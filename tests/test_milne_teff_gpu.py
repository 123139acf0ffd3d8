"""Milne's temperature profile (Sect. 2.5) and the effective-temperature
post-processing (Sect. 2.6) through the C ABI, against the oracle.

The library's Hopf function comes from Chandrasekhar's H-function
representation, the oracle's from solving Milne's integral equation; the two
agree to ~1e-8 in q (both tables read by cubic interpolation), which moves
the flux by well under 1e-7, so the plain FP64 path keeps its usual 2e-7 gate
on Milne setups and the FP16 paths their 1e-4."""
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
    sd = torch.as_tensor(sid, dtype=torch.int32, device="cuda")
    eng.forward(setups, sd, torch.as_tensor(theta, device="cuda"), bins, hi, st)
    torch.cuda.synchronize()
    return bins, hi, st, sd


@pytest.mark.parametrize("storage", ["fp16-level-gridded", "fp16-direct", "fp64"])
def test_milne_profile_matches_oracle(eng, storage):
    spec = W.TableSpec(3, np.linspace(300.0, 3000.0, 8), np.linspace(-4.0, 2.0, 6), 5000.0, 1.0, 700, seed=61)
    tabs = W.make_tables(spec)
    setup = W.make_setup(spec, 5003.0, 5650.0, 40, [0, 1, 2], 4, 2, 1, 400.0, 20)
    setup.profile = "milne"
    st_ = storage[:4]
    t = eng.add_tables(spec, st_, tabs)
    s = eng.add_setup(t, setup, level_cache=(storage == "fp16-level-gridded"))
    theta = W.draw_params(setup, 6, 8, W.Prior(t_bar=(500.0, 1800.0), log_kappa=(-3.0, 0.5)))
    bins, hi, st, _ = _run(eng, [s], np.zeros(6, np.int32), theta, setup.n_nu)
    assert np.all(st.cpu().numpy() == 0)
    om = oracle_model(tables_as_stored(tabs, st_), setup)
    tol = FLUX_RTOL if st_ == "fp16" else FP64_RTOL
    b, h = bins.cpu().numpy().astype(np.float64), hi.cpu().numpy().astype(np.float64)
    for i in range(6):
        ob, otop, ok = om.forward(theta[i], want_top=True)
        assert ok
        assert rel_flux_err(h[i], otop) <= tol
        assert rel_flux_err(b[i], ob) <= tol


def test_mixed_profiles_in_one_batch(eng):
    spec = W.TableSpec(2, np.linspace(300.0, 3000.0, 6), np.linspace(-4.0, 2.0, 5), 5000.0, 1.0, 300, seed=62)
    tabs = W.make_tables(spec)
    fe = W.make_setup(spec, 5000.0, 5299.0, 24, [0, 1], 3, 2, 2, 300.0, 8)
    mi = W.make_setup(spec, 5010.0, 5280.0, 30, [0, 1], 3, 2, 2, 300.0, 8)
    mi.profile = "milne"
    t = eng.add_tables(spec, "fp16", tabs)
    setups = [eng.add_setup(t, fe), eng.add_setup(t, mi)]
    sid = np.array([0, 1, 1, 0, 1], np.int32)
    theta = np.concatenate([W.draw_params([fe, mi][g], 1, 40 + i, W.Prior(b=(0.8, 0.97))) for i, g in enumerate(sid)])
    bins, hi, st, _ = _run(eng, setups, sid, theta, 300)
    stored = tables_as_stored(tabs, "fp16")
    h = hi.cpu().numpy().astype(np.float64)
    for i, g in enumerate(sid):
        sp = [fe, mi][g]
        _, otop, ok = oracle_model(stored, sp).forward(theta[i], want_top=True)
        assert rel_flux_err(h[i, : sp.n_nu], otop) <= FLUX_RTOL


@pytest.mark.parametrize("profile", ["fe", "milne"])
def test_effective_temperature_matches_oracle(eng, profile):
    """T_eff over a 500-10000 cm^-1 (1-20 micron) setup."""
    spec = W.TableSpec(2, np.linspace(200.0, 3000.0, 8), np.linspace(-4.0, 2.0, 5), 500.0, 1.0, 9501, seed=63)
    tabs = W.make_tables(spec)
    setup = W.make_setup(spec, 500.0, 10000.0, 30, [0, 1], 2, 3, 2, 0.0, 10)
    setup.profile = profile
    t = eng.add_tables(spec, "fp16", tabs)
    s = eng.add_setup(t, setup)
    theta = W.draw_params(setup, 5, 9, W.Prior(b=(0.8, 0.97), t_bar=(500.0, 1500.0), log_kappa=(-3.0, 0.0)))
    bins, hi, st, sd = _run(eng, [s], np.zeros(5, np.int32), theta, setup.n_nu)
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    hr2.hr2_effective_temperature(eng.ctx, [s], sd, hi, out)
    teff = out.cpu().numpy()
    om = oracle_model(tables_as_stored(tabs, "fp16"), setup)
    for i in range(5):
        assert teff[i] == pytest.approx(om.effective_temperature(theta[i]), rel=1e-5)


def test_profile_argument_error(eng, monkeypatch):
    spec = W.TableSpec(1, np.linspace(300.0, 3000.0, 3), np.linspace(-4.0, 2.0, 3), 5000.0, 1.0, 64, seed=2)
    t = eng.add_tables(spec, "fp16", W.make_tables(spec))
    setup = W.make_setup(spec, 5000.0, 5063.0, 4, [0], 2, 1, 1, 0.0, 2)
    monkeypatch.setitem(hr2.PROFILE, "bogus", 7)          # a profile code the library does not know
    with pytest.raises(hr2.Hr2Error) as ei:
        hr2.hr2_setup_create(eng.ctx, t, setup.nu_first, setup.n_nu, 4, [0], 2, 1, 1, 0.0, setup.bin_edges,
                             profile="bogus")
    assert ei.value.code == hr2.HR2_EINVAL
