"""GPU tests of the runtime around the kernels: CUDA-graph replay, the launch
autotuner and the continuous-batching server (each result the same alone and
in the mix)."""
import numpy as np
import pytest

from paper_1910_01070_b300 import autotune, graphs, hr2, serving
from paper_1910_01070_b300 import workloads as W
from paper_1910_01070_b300.engine import Engine

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def uneven():
    from paper_1910_01070_b300 import build
    build.build()
    wl = W.uneven2048_3setups()
    eng = Engine(0)
    t = eng.add_tables(wl.table, "fp16", W.make_tables(wl.table))
    setups = [eng.add_setup(t, s) for s in wl.setups]
    for h, s in zip(setups, wl.setups):       # any positive data will do for equality tests
        eng.set_observation(h, np.full(s.n_bins, 3e-16), np.full(s.n_bins, 5e-17))
    yield wl, eng, setups
    eng.close()


def test_graph_replay_matches_direct_calls(uneven):
    wl, eng, setups = uneven
    nb = max(s.n_bins for s in wl.setups)
    nn = max(s.n_nu for s in wl.setups)
    cap = graphs.CapturedBatch(eng.ctx, setups, 256, nb, nn)
    for seed in (1, 2):
        theta, sid = wl.params(200, seed_offset=seed)
        lnl_g, bins_g = cap.run(torch.as_tensor(theta), torch.as_tensor(sid))
        lnl_g, bins_g = lnl_g.cpu().numpy().copy(), bins_g.cpu().numpy().copy()
        th, sd = torch.as_tensor(theta, device="cuda"), torch.as_tensor(sid, device="cuda")
        bins = torch.empty((200, nb), dtype=torch.float32, device="cuda")
        eng.forward(setups, sd, th, bins)
        lnl = eng.lnl(setups, sd, bins)
        torch.cuda.synchronize()
        for g, s in enumerate(wl.setups):
            rows = np.nonzero(sid == g)[0]
            assert np.array_equal(bins_g[rows, : s.n_bins], bins.cpu().numpy()[rows, : s.n_bins])
        assert np.array_equal(lnl_g, lnl.cpu().numpy())


def test_autotuner_picks_a_candidate_and_caches_it(uneven, tmp_path):
    wl, eng, setups = uneven
    theta, sid = wl.params(512, seed_offset=4)
    th, sd = torch.as_tensor(theta, device="cuda"), torch.as_tensor(sid, device="cuda")
    bins = torch.empty((512, max(s.n_bins for s in wl.setups)), dtype=torch.float32, device="cuda")
    info = [autotune.setup_info_from_spec(s) for s in wl.setups]
    cands = [(2, 4), (4, 4), (8, 2)]
    path = str(tmp_path / "tune.json")
    old = hr2.hr2_get_launch_config(eng.ctx)
    try:
        best, timings = autotune.tune(eng.ctx, setups, sd, th, bins, info, cands, reps=1, path=path)
        assert best in cands and set(timings) == set(cands) and all(v > 0 for v in timings.values())
        assert hr2.hr2_get_launch_config(eng.ctx) == best
        again, t2 = autotune.tune(eng.ctx, setups, sd, th, bins, info, cands, path=path)
        assert again == best and t2 == {}                         # served from the cache
    finally:
        hr2.hr2_set_launch_config(eng.ctx, *old)


def test_server_result_is_the_same_alone_and_in_the_mix(uneven):
    wl, eng, setups = uneven
    shapes = [(s.n_bins, s.n_nu, s.n_layers + 1) for s in wl.setups]
    srv = serving.Server(eng.ctx, setups, shapes, slots=2, max_batch=1024, mem_budget=1 << 30)
    rng = np.random.default_rng(3)
    reqs = []
    for rid in range(24):
        g = int(rng.integers(0, len(wl.setups)))
        n = int(rng.integers(32, 300))
        reqs.append(serving.Request(rid=rid, stream=rid % 16, setup=g,
                                    params=W.draw_params(wl.setups[g], n, 1000 + rid, wl.prior)))
    for r in reqs:
        r.t_arrival = srv.clock()
        srv.submit(r)
    srv.drain()
    assert len(srv.done) == 24 and srv.mem_in_use == 0
    assert srv.batches >= 2 and all(r.latency > 0 for r in srv.done)
    for r in reqs[:6]:
        alone = eng.evaluate_host(setups, np.full(r.n, r.setup, np.int32), r.params)
        assert np.array_equal(alone, r.lnl)


def test_open_loop_serving_reports_latency(uneven):
    wl, eng, setups = uneven
    shapes = [(s.n_bins, s.n_nu, s.n_layers + 1) for s in wl.setups]
    srv = serving.Server(eng.ctx, setups, shapes, slots=3, max_batch=2048, mem_budget=2 << 30)
    lo = np.zeros(hr2.HR2_NPARAM)
    hi = np.zeros(hr2.HR2_NPARAM)
    streams, templates = [], []
    for k in range(16):
        g = k % len(wl.setups)
        t = wl.truth(g)
        lo_k, hi_k = t.copy(), t.copy()
        lo_k[0], hi_k[0] = 4.0, 5.5
        lo_k[1], hi_k[1] = 0.5, 2.0
        nsp = len(wl.setups[g].species)
        lo_k[19:19 + nsp], hi_k[19:19 + nsp] = -8.0, -2.0
        streams.append(serving.RetrievalStream(k, g, lo_k, hi_k, rate=20.0, seed=k))
        templates.append(t)
    stats = serving.run_open_loop(srv, streams, templates, duration=1.5)
    assert stats["requests"] > 10 and stats["samples"] > 1000
    assert 0 < stats["p50_ms"] <= stats["p99_ms"]
    assert all(np.all(np.isfinite(r.lnl)) for r in srv.done)
