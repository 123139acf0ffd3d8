"""Host-side logic that needs no GPU: serving admission and packing, the
autotuner's shape keys, cache and choice, and the benchmark's multi-rank
timing reduction over gloo (world size 2)."""
import collections
import os

import numpy as np
import pytest

from paper_1910_01070_b300 import autotune
from paper_1910_01070_b300 import serving
from paper_1910_01070_b300 import workloads as W


def _req(rid, n, setup=0):
    return serving.Request(rid=rid, stream=0, setup=setup, params=np.zeros((n, W.NPARAM)))


def test_admission_is_fifo_and_respects_budget():
    pending = collections.deque([_req(0, 100), _req(1, 300), _req(2, 50)])
    admitted = collections.deque()
    fp = lambda r: r.n * 10
    used = serving.admit(pending, admitted, 0, 4200, fp)
    assert [r.rid for r in admitted] == [0, 1] and used == 4000
    assert [r.rid for r in pending] == [2]            # 4000 + 500 > 4200: waits
    used = serving.admit(pending, admitted, used - 1000, 4200, fp)    # request 0 finished
    assert [r.rid for r in admitted] == [0, 1, 2] and used == 3500


def test_head_of_queue_is_never_overtaken():
    pending = collections.deque([_req(0, 400), _req(1, 10)])
    admitted = collections.deque()
    used = serving.admit(pending, admitted, 0, 1000, lambda r: r.n * 10)
    assert len(admitted) == 0 and used == 0          # the small one waits behind the big one


def test_packing_takes_whole_requests_in_order():
    admitted = collections.deque([_req(0, 300), _req(1, 500), _req(2, 400), _req(3, 100)])
    batch = serving.pack(admitted, 1000)
    assert [(r.rid, off) for r, off in batch] == [(0, 0), (1, 300)]
    assert [r.rid for r in admitted] == [2, 3]
    batch = serving.pack(admitted, 1000)
    assert [(r.rid, off) for r, off in batch] == [(2, 0), (3, 400)]


def test_queue_bound_counts_pending_and_admitted_samples():
    assert not serving.over_queue_limit(300, 300, 600)
    assert serving.over_queue_limit(301, 300, 600)
    assert serving.over_queue_limit(0, 601, 600)


def test_cancel_removes_only_the_named_request():
    pending = collections.deque([_req(0, 10), _req(1, 20)])
    admitted = collections.deque([_req(2, 30)])
    r = serving.cancel_from([pending, admitted], 2)
    assert r.rid == 2 and len(admitted) == 0 and [q.rid for q in pending] == [0, 1]
    assert serving.cancel_from([pending, admitted], 7) is None
    assert [q.rid for q in pending] == [0, 1]


def test_graph_buckets_cover_every_batch_size():
    sizes = serving.bucket_sizes(1024)
    assert sizes == [64, 128, 256, 512, 1024]
    assert serving.bucket_sizes(300) == [64, 128, 256, 300]
    assert serving.pick_bucket(sizes, 1) == 64 and serving.pick_bucket(sizes, 65) == 128
    assert serving.pick_bucket(sizes, 1024) == 1024
    with pytest.raises(ValueError):
        serving.pick_bucket(sizes, 1025)


def test_retrieval_stream_is_seeded_and_contracts():
    lo = np.zeros(W.NPARAM)
    hi = np.zeros(W.NPARAM)
    lo[0], hi[0] = 4.0, 5.5
    s1 = serving.RetrievalStream(0, 0, lo, hi, rate=10.0, seed=5)
    s2 = serving.RetrievalStream(0, 0, lo, hi, rate=10.0, seed=5)
    t = np.zeros(W.NPARAM)
    r1, r2 = s1.make_request(0, t), s2.make_request(0, t)
    assert np.array_equal(r1.params, r2.params) and 32 <= r1.n <= 512
    assert np.all((r1.params[:, 0] >= 4.0) & (r1.params[:, 0] <= 5.5))
    r1.lnl = -np.arange(r1.n, dtype=float)
    w0 = s1.width[0]
    s1.feedback(r1)
    assert s1.width[0] < w0 and np.array_equal(s1.center, r1.params[0])


def test_autotune_shape_key_and_cache(tmp_path):
    info = [{"K": 6, "L": 100, "n_mu": 4, "n_nu": 8501, "cached": 1}]
    k1 = autotune.shape_key(info, 1000)
    k2 = autotune.shape_key(info, 1024)
    assert k1 == k2 and k1.startswith("n1024|")
    assert autotune.shape_key(info, 1025) != k1
    path = str(tmp_path / "tune.json")
    autotune.save_cache({k1: [4, 4]}, path)
    assert autotune.load_cache(path) == {k1: [4, 4]}
    assert autotune.load_cache(str(tmp_path / "missing.json")) == {}
    assert autotune.pick_best({(8, 2, 1, 0, 4): 7.0, (4, 4, 1, 0, 4): 6.9, (2, 8, 2, 0, 4): 6.9}) == (2, 8, 2, 0, 4)
    assert autotune._as_shape([4, 4]) == (4, 4, 1, 0, autotune.DEFAULT_SHAPE[4])


def test_autotune_candidates_span_the_tile_shape():
    few = autotune.candidates_for([{"K": 6, "L": 100, "n_mu": 4, "n_nu": 8501, "cached": 1}])
    assert {c[2] for c in few} == {1, 2, 4} and {c[3] for c in few} == {0}
    assert len(few) == len(autotune.GRIDS) * 3 and len(set(few)) == len(few)
    both = autotune.candidates_for([{"K": 12, "L": 100, "n_mu": 8, "n_nu": 290001, "cached": 1}])
    assert {c[3] for c in both} == {0, 1, 2} and len(both) == 3 * len(few)
    assert {c[4] for c in few} == {autotune.DEFAULT_SHAPE[4]}
    direct = autotune.candidates_for([{"K": 12, "L": 100, "n_mu": 8, "n_nu": 290001, "cached": 0}], n=3)
    assert {c[4] for c in direct} == {0, 4} and len(direct) == 2 * len(few)


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    w, r, _ = bench.dist_setup(None)
    m = bench.max_over_ranks(w, float(10 + r))
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    out.put((r, w, m))


def test_bench_rank_reduction_over_gloo():
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert res == [(0, 2, 11.0), (1, 2, 11.0)]
