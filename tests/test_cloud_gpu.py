"""The gray cloud layer (parameters HR2_P_CLOUD..) through the C ABI against
the oracle, on the three paths, mixed with cloud-free setups."""
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


@pytest.mark.parametrize("storage", ["fp16-level-gridded", "fp16-direct", "fp64"])
def test_cloudy_setups_match_oracle(eng, storage):
    spec = W.TableSpec(3, np.linspace(300.0, 3000.0, 7), np.linspace(-4.0, 2.0, 6), 5000.0, 1.0, 400, seed=71)
    tabs = W.make_tables(spec)
    clear = W.make_setup(spec, 5000.0, 5399.0, 30, [0, 1, 2], 4, 2, 2, 300.0, 12)
    cloudy = W.make_setup(spec, 5007.0, 5390.0, 36, [0, 1, 2], 4, 2, 2, 300.0, 12)
    cloudy.cloud = True
    st_ = storage[:4]
    t = eng.add_tables(spec, st_, tabs)
    lc = storage == "fp16-level-gridded"
    setups = [eng.add_setup(t, clear, level_cache=lc), eng.add_setup(t, cloudy, level_cache=lc)]
    sid = np.array([1, 0, 1, 1, 0, 1, 1], np.int32)
    prior = W.Prior(b=(0.8, 0.97), log_tau_cloud=(-1.0, 1.5), log_p_cloud=(-2.5, 0.5))
    theta = np.concatenate([W.draw_params([clear, cloudy][g], 1, 300 + i, prior) for i, g in enumerate(sid)])
    b, h, st = _run(eng, setups, sid, theta, 400)
    assert np.all(st == 0)
    stored = tables_as_stored(tabs, st_)
    tol = FLUX_RTOL if st_ == "fp16" else FP64_RTOL
    for i, g in enumerate(sid):
        sp = [clear, cloudy][g]
        ob, otop, ok = oracle_model(stored, sp).forward(theta[i], want_top=True)
        assert ok
        assert rel_flux_err(h[i, : sp.n_nu], otop) <= tol
        assert rel_flux_err(b[i, : sp.n_bins], ob) <= tol
    # the cloud matters: the same parameters without it give another spectrum
    no = oracle_model(stored, clear)
    i = int(np.nonzero(sid == 1)[0][0])
    assert np.max(np.abs(no.forward(theta[i], want_top=True)[1][7:391] / h[i, :384] - 1)) > 1e-3


def test_invalid_cloud_is_flagged(eng):
    spec = W.TableSpec(1, np.linspace(300.0, 3000.0, 3), np.linspace(-4.0, 2.0, 3), 5000.0, 1.0, 128, seed=72)
    t = eng.add_tables(spec, "fp16", W.make_tables(spec))
    cloudy = W.make_setup(spec, 5000.0, 5127.0, 10, [0], 2, 1, 1, 0.0, 4)
    cloudy.cloud = True
    s = eng.add_setup(t, cloudy)
    theta = W.draw_params(cloudy, 3, 5, W.Prior(b=(0.8, 0.97)))
    theta[1, W.P_CLOUD + 2] = 0.3                     # f_c > 1: bottom above the top
    theta[2, W.P_CLOUD] = np.nan
    b, h, st = _run(eng, [s], np.zeros(3, np.int32), theta, 128)
    assert st[0] == 0
    assert st[1] == hr2.HR2_SAMPLE_BAD_CLOUD and st[2] == hr2.HR2_SAMPLE_BAD_CLOUD
    assert np.all(np.isnan(h[1:]))
