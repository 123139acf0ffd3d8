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
    cands = [(2, 4, 1, 0, 4), (4, 4, 2, 0, 4), (8, 2, 4, 0, 4)]
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


def _requests(wl, count, seed, lo_n=32, hi_n=300):
    rng = np.random.default_rng(seed)
    reqs = []
    for rid in range(count):
        g = int(rng.integers(0, len(wl.setups)))
        n = int(rng.integers(lo_n, hi_n))
        reqs.append(serving.Request(rid=rid, stream=rid % 16, setup=g,
                                    params=W.draw_params(wl.setups[g], n, 1000 * seed + rid, wl.prior)))
    return reqs


def _shapes(wl):
    return [(s.n_bins, s.n_nu, s.n_layers + 1) for s in wl.setups]


@pytest.mark.parametrize("graphs", [True, False])
def test_server_result_is_the_same_alone_and_in_the_mix(uneven, graphs):
    wl, eng, setups = uneven
    srv = serving.Server(eng.ctx, setups, _shapes(wl), slots=2, max_batch=1024, mem_budget=64 << 30,
                         queue_limit=1 << 20, graphs=graphs)
    reqs = _requests(wl, 24, 3)
    for r in reqs:
        r.t_arrival = srv.clock()
        assert srv.submit(r)
    srv.drain()
    assert len(srv.done) == 24 and srv.mem_in_use == 0
    assert srv.batches >= 2 and all(r.latency > 0 and r.status == serving.DONE for r in srv.done)
    for r in reqs[:6]:
        alone = eng.evaluate_host(setups, np.full(r.n, r.setup, np.int32), r.params)
        assert np.array_equal(alone, r.lnl)


def test_server_memory_is_the_context_s_and_its_own(uneven):
    """The budget counts what the context holds (tables, setups with their operands,
    workspaces) plus the server's buffers; a budget below that is refused."""
    wl, eng, setups = uneven
    used, _ = hr2.hr2_ctx_memory(eng.ctx)
    with pytest.raises(ValueError):
        serving.Server(eng.ctx, setups, _shapes(wl), slots=1, max_batch=256, mem_budget=used, graphs=False)
    srv = serving.Server(eng.ctx, setups, _shapes(wl), slots=1, max_batch=256, mem_budget=64 << 30,
                         queue_limit=1 << 20, graphs=False)
    assert srv.device_bytes >= hr2.hr2_ctx_memory(eng.ctx)[0]
    assert srv.pool_bytes >= 256 * srv.bytes_per_sample > 0
    # admission never lets the in-flight footprint exceed the reserved pool
    reqs = _requests(wl, 12, 5, 100, 250)
    for r in reqs:
        srv.submit(r)
    peak = 0
    while not srv.idle():
        srv.step()
        peak = max(peak, srv.mem_in_use)
        assert srv.mem_in_use <= srv.pool_bytes
    assert peak > 0 and srv.mem_in_use == 0 and len(srv.done) == 12


def test_server_faults_stay_with_their_request(uneven):
    """Host-side faults: one request's consumer raises, one request is cancelled before it is
    launched; every other request's lnL is bit-identical to evaluating it alone, and the
    server's memory accounting returns to zero."""
    wl, eng, setups = uneven
    srv = serving.Server(eng.ctx, setups, _shapes(wl), slots=2, max_batch=512, mem_budget=64 << 30,
                         queue_limit=1 << 20)
    reqs = _requests(wl, 16, 7)
    seen = []

    def consumer(req):
        seen.append(req.rid)
        if req.rid == 5:
            raise RuntimeError("consumer of request 5 failed")

    for r in reqs:
        r.callback = consumer
        r.t_arrival = srv.clock()
        srv.submit(r)
    assert srv.cancel(11)                   # still queued: withdrawn before any launch
    assert not srv.cancel(999)
    srv.drain()
    assert srv.mem_in_use == 0 and srv.idle()
    by_id = {r.rid: r for r in reqs}
    assert by_id[11].status == serving.CANCELLED and by_id[11].lnl is None and 11 not in seen
    assert by_id[5].status == serving.FAILED and isinstance(by_id[5].error, RuntimeError)
    assert np.all(np.isfinite(by_id[5].lnl))         # its result was delivered before the consumer failed
    for r in reqs:
        if r.rid == 11:
            continue
        alone = eng.evaluate_host(setups, np.full(r.n, r.setup, np.int32), r.params)
        assert np.array_equal(alone, r.lnl), r.rid
        if r.rid != 5:
            assert r.status == serving.DONE and r.error is None


def test_server_sheds_load_past_its_queue_bound(uneven):
    wl, eng, setups = uneven
    srv = serving.Server(eng.ctx, setups, _shapes(wl), slots=1, max_batch=256, mem_budget=64 << 30,
                         queue_limit=600, graphs=False)
    reqs = _requests(wl, 20, 9, 150, 250)
    accepted = [srv.submit(r) for r in reqs]      # all at once, before any step
    assert not all(accepted) and any(accepted)
    assert sum(r.n for r, ok in zip(reqs, accepted) if ok) <= 600
    assert len(srv.rejected) == accepted.count(False)
    assert all(r.status == serving.REJECTED and r.lnl is None for r in srv.rejected)
    srv.drain()
    assert len(srv.done) == accepted.count(True) and srv.mem_in_use == 0


def test_graph_pool_picks_the_smallest_bucket_and_matches_direct_calls(uneven):
    wl, eng, setups = uneven
    nb = max(s.n_bins for s in wl.setups)
    nn = max(s.n_nu for s in wl.setups)
    pool = graphs.GraphPool(eng.ctx, setups, nb, nn, min_n=64, max_n=256)
    assert pool.sizes == [64, 128, 256]
    assert pool.bucket_for(1).n == 64 and pool.bucket_for(64).n == 64 and pool.bucket_for(65).n == 128
    assert pool.bucket_for(256).n == 256
    with pytest.raises(ValueError):
        pool.bucket_for(257)
    for m, seed in ((40, 1), (200, 2)):
        theta, sid = wl.params(m, seed_offset=seed)
        lnl_g, _ = pool.run(torch.as_tensor(theta), torch.as_tensor(sid))
        lnl_g = lnl_g.cpu().numpy().copy()
        alone = eng.evaluate_host(setups, sid.astype(np.int32), theta)
        assert np.array_equal(lnl_g, alone)


def test_open_loop_serving_reports_latency(uneven):
    wl, eng, setups = uneven
    shapes = [(s.n_bins, s.n_nu, s.n_layers + 1) for s in wl.setups]
    srv = serving.Server(eng.ctx, setups, shapes, slots=2, max_batch=1024, mem_budget=64 << 30)
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
