"""The allocation-free entry point against the ordinary one.

forward_model_batch_noalloc exists for callers that may not let a library
allocate device memory (an application whose device memory belongs to
another allocator, or a latency-critical loop that cannot accept the
synchronisation cudaMalloc may imply).  It must give what
forward_model_batch gives, bit for bit (the same kernels on the same inputs).
Two calls in a row with different batches check that the shared static
scratch, which keeps the previous call's contents, does not leak into the next
result; a second, larger call must leave every measure of device memory where
it was; and a bounded wait that runs out must come back through
hr2_noalloc_check.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1910_01070_b300 import hr2
from paper_1910_01070_b300 import workloads as W
from paper_1910_01070_b300.engine import Engine

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_matches_forward_model_batch_twice_in_a_row():
    """Both entry points run the same kernels on the same inputs, so the results
    agree bit for bit; the second, smaller call must not see the first call's
    leftovers in the shared array."""
    from paper_1910_01070_b300 import build
    build.build()
    wl = W.uneven2048_3setups()
    with Engine(0) as eng:
        t = eng.add_tables(wl.table, "fp16", W.make_tables(wl.table))
        setups = [eng.add_setup(t, s) for s in wl.setups]
        nb = max(s.n_bins for s in wl.setups)
        nn = max(s.n_nu for s in wl.setups)
        for n, seed in ((96, 11), (40, 12)):      # two calls in a row, different batches
            theta, sid = wl.params(n, seed_offset=seed)
            th = torch.as_tensor(theta, device="cuda")
            sd = torch.as_tensor(sid, device="cuda")
            ref_b = torch.empty((n, nb), dtype=torch.float32, device="cuda")
            ref_h = torch.empty((n, nn), dtype=torch.float32, device="cuda")
            eng.forward(setups, sd, th, ref_b, ref_h)
            out_b = torch.full((n, nb), -1.0, dtype=torch.float32, device="cuda")
            out_h = torch.full((n, nn), -1.0, dtype=torch.float32, device="cuda")
            st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            hr2.forward_model_batch_noalloc(eng.ctx, setups, sd, th, out_b, out_h, st)
            hr2.hr2_noalloc_check(eng.ctx)
            torch.cuda.synchronize()
            for g, s in enumerate(wl.setups):
                rows = np.nonzero(sid == g)[0]
                if len(rows) == 0:
                    continue
                rb, ob = ref_b.cpu().numpy()[rows, : s.n_bins], out_b.cpu().numpy()[rows, : s.n_bins]
                rh, oh = ref_h.cpu().numpy()[rows, : s.n_nu], out_h.cpu().numpy()[rows, : s.n_nu]
                assert np.array_equal(ob, rb)
                assert np.array_equal(oh, rh)
            assert np.all(st.cpu().numpy() == 0)


def test_noalloc_allocates_no_device_memory():
    """After a first round of calls (which looks up the array's address and
    loads the kernels), further calls, a larger batch after a smaller one,
    change neither the driver's free device memory nor what torch's caching
    allocator holds, nor the context's own accounting."""
    wl = W.batch1024_l100_k6_nu8501()
    with Engine(0) as eng:
        t = eng.add_tables(wl.table, "fp16", W.make_tables(wl.table))
        s = eng.add_setup(t, wl.setups[0])
        bufs = {}
        for n in (16, 200):
            bufs[n] = (torch.empty((n, 300), dtype=torch.float32, device="cuda"),
                       torch.empty((n, 8501), dtype=torch.float32, device="cuda"))
        params = {}
        for rnd in range(2):
            for n in (16, 200):
                theta, sid = wl.params(n, seed_offset=10 * rnd + n)
                params[rnd, n] = (torch.as_tensor(theta, device="cuda"), torch.as_tensor(sid, device="cuda"))
        torch.cuda.synchronize()

        def call(rnd, n):
            th, sd = params[rnd, n]
            ob, oh = bufs[n]
            hr2.forward_model_batch_noalloc(eng.ctx, [s], sd, th, ob, oh)
            hr2.hr2_noalloc_check(eng.ctx)

        call(0, 16)
        call(0, 200)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        reserved0 = torch.cuda.memory_reserved()
        used0 = eng.memory()[0]
        call(1, 16)
        call(1, 200)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_reserved() == reserved0
        assert eng.memory()[0] == used0
        assert np.all(np.isfinite(bufs[200][0].cpu().numpy()))


def test_noalloc_reports_an_expired_wait():
    """The error word of the allocation-free path lives in the static array;
    hr2_noalloc_check returns it (the bounded-wait test hook makes a stage's
    wait run out, nothing faults), and the next call is clean again."""
    wl = W.tiny(n_nu=300, n_layers=12, n_species=3, n_T=4, n_p=3, n_mu=3, resolving_power=200.0, n_bins=6)
    with Engine(0) as eng:
        t = eng.add_tables(wl.table, "fp16", W.make_tables(wl.table))
        s = eng.add_setup(t, wl.setups[0])
        theta, sid = wl.params(24, seed_offset=9)
        th, sd = torch.as_tensor(theta, device="cuda"), torch.as_tensor(sid, device="cuda")
        ref_b = torch.empty((24, 6), dtype=torch.float32, device="cuda")
        ref_h = torch.empty((24, 300), dtype=torch.float32, device="cuda")
        hr2.forward_model_batch_noalloc(eng.ctx, [s], sd, th, ref_b, ref_h)
        hr2.hr2_noalloc_check(eng.ctx)
        hr2.hr2_set_wait_limit(eng.ctx, 200000)
        hr2.hr2_set_wait_fault(eng.ctx, True)
        ob = torch.empty((24, 6), dtype=torch.float32, device="cuda")
        oh = torch.empty((24, 300), dtype=torch.float32, device="cuda")
        hr2.forward_model_batch_noalloc(eng.ctx, [s], sd, th, ob, oh)
        with pytest.raises(hr2.Hr2Error) as ei:
            hr2.hr2_noalloc_check(eng.ctx)
        assert ei.value.code == hr2.HR2_ETIMEDOUT
        hr2.hr2_set_wait_fault(eng.ctx, False)
        hr2.hr2_set_wait_limit(eng.ctx, 2000000000)
        hr2.forward_model_batch_noalloc(eng.ctx, [s], sd, th, ob, oh)
        hr2.hr2_noalloc_check(eng.ctx)
        assert np.array_equal(ob.cpu().numpy(), ref_b.cpu().numpy())
        assert np.array_equal(oh.cpu().numpy(), ref_h.cpu().numpy())


def test_noalloc_rejects_batches_beyond_its_scratch():
    wl = W.batch1024_l100_k6_nu8501()
    with Engine(0) as eng:
        t = eng.add_tables(wl.table, "fp16", W.make_tables(wl.table))
        s = eng.add_setup(t, wl.setups[0])
        n = 4096                                   # 4096 x 101 levels x 64 B > 8 MiB
        theta, sid = wl.params(n)
        out_b = torch.empty((n, 300), dtype=torch.float32, device="cuda")
        out_h = torch.empty((n, 8501), dtype=torch.float32, device="cuda")
        with pytest.raises(hr2.Hr2Error) as ei:
            hr2.forward_model_batch_noalloc(eng.ctx, [s], torch.as_tensor(sid, device="cuda"),
                                            torch.as_tensor(theta, device="cuda"), out_b, out_h)
        assert ei.value.code == hr2.HR2_EINVAL
        assert "scratch" in str(ei.value)
