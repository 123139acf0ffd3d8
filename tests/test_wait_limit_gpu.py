"""The forward kernel's bounded pipeline waits, made to run out on the GPU
without harming it.

Every wait of the level-gridded kernel's copy pipeline gives up after the
context's wait limit, sets the batch's error word, lets its own copies land
and stops its warp.  hr2_set_wait_fault arms each work item's first stage for
bytes that never arrive (a flag that nothing sets), so that this path runs
deterministically; nothing faults, traps or hangs.  The checks: the call
itself succeeds, the error comes back as HR2_ETIMEDOUT (hr2_stream_check,
hr2_evaluate_host), the kernel ends within a bounded time (its copies drained),
and the next normal batch on the same stream gives exactly what a fresh
context gives.
"""
import time

import numpy as np
import pytest

from paper_1910_01070_b300 import hr2
from paper_1910_01070_b300 import workloads as W
from paper_1910_01070_b300.engine import Engine

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHORT_LIMIT = 200000        # SM cycles (~0.1 ms): the injected stage wait gives up after this


def _tiny():
    wl = W.tiny(n_nu=300, n_layers=12, n_species=3, n_T=4, n_p=3, n_mu=3, resolving_power=200.0, n_bins=6)
    return wl, W.make_tables(wl.table)


def _run(eng, setups, theta, sid, stream):
    n = theta.shape[0]
    nb = hr2.hr2_setup_info(setups[0])[0]
    nn = hr2.hr2_setup_info(setups[0])[1]
    bins = torch.full((n, nb), -7.0, dtype=torch.float32, device="cuda")
    hi = torch.full((n, nn), -7.0, dtype=torch.float32, device="cuda")
    th = torch.as_tensor(theta, device="cuda")
    sd = torch.as_tensor(sid, device="cuda")
    hr2.forward_model_batch(eng.ctx, setups, sd, th, bins, hi, None, stream)
    return bins, hi


def test_wait_limit_default_and_argument_errors():
    with Engine(0) as eng:
        assert hr2.hr2_get_wait_limit(eng.ctx) == 2000000000
        hr2.hr2_set_wait_limit(eng.ctx, 12345)
        assert hr2.hr2_get_wait_limit(eng.ctx) == 12345
        with pytest.raises(hr2.Hr2Error) as ei:
            hr2.hr2_set_wait_limit(eng.ctx, -1)
        assert ei.value.code == hr2.HR2_EINVAL


def test_expired_wait_reports_timeout_and_the_next_batch_is_clean():
    from paper_1910_01070_b300 import build
    build.build()
    wl, tabs = _tiny()
    theta, sid = wl.params(37, seed_offset=3)
    stream = torch.cuda.Stream()
    # a fresh context's result, the reference
    with Engine(0) as fresh:
        t = fresh.add_tables(wl.table, "fp16", tabs)
        s = fresh.add_setup(t, wl.setups[0])
        with torch.cuda.stream(stream):
            ref_b, ref_h = _run(fresh, [s], theta, sid, stream)
        hr2.hr2_stream_check(fresh.ctx, stream)
        ref_b, ref_h = ref_b.cpu().numpy(), ref_h.cpu().numpy()
    assert np.all(np.isfinite(ref_b)) and np.all(np.isfinite(ref_h))

    with Engine(0) as eng:
        t = eng.add_tables(wl.table, "fp16", tabs)
        s = eng.add_setup(t, wl.setups[0])
        D = ref_b[0].astype(np.float64)
        eng.set_observation(s, D, np.full(D.shape, 0.1 * float(np.median(D))))
        hr2.hr2_set_wait_limit(eng.ctx, SHORT_LIMIT)
        hr2.hr2_set_wait_fault(eng.ctx, True)
        with torch.cuda.stream(stream):
            t0 = time.perf_counter()
            _run(eng, [s], theta, sid, stream)          # the launch itself succeeds
        with pytest.raises(hr2.Hr2Error) as ei:
            hr2.hr2_stream_check(eng.ctx, stream)
        waited = time.perf_counter() - t0
        assert ei.value.code == hr2.HR2_ETIMEDOUT
        # each warp gives up once (short limit) and drains for ~1e7 cycles:
        # far below a second even with the many persistent warps in turn
        assert waited < 5.0
        # the host-buffer entry point reports the same through its return code
        out = np.empty(37)
        with pytest.raises(hr2.Hr2Error) as ei:
            hr2.hr2_evaluate_host(eng.ctx, [s], sid.astype(np.int32), theta, out, None, None, stream)
        assert ei.value.code == hr2.HR2_ETIMEDOUT

        # hook off, default limit: the same stream and workspace give exactly
        # what the fresh context gave, and the error word is clear again
        hr2.hr2_set_wait_fault(eng.ctx, False)
        hr2.hr2_set_wait_limit(eng.ctx, 2000000000)
        with torch.cuda.stream(stream):
            b, h = _run(eng, [s], theta, sid, stream)
        hr2.hr2_stream_check(eng.ctx, stream)
        assert np.array_equal(b.cpu().numpy(), ref_b)
        assert np.array_equal(h.cpu().numpy(), ref_h)
        hr2.hr2_evaluate_host(eng.ctx, [s], sid.astype(np.int32), theta, out, None, None, stream)
        assert np.all(np.isfinite(out))


def test_a_short_limit_alone_changes_nothing_when_the_copies_arrive():
    """The limit bounds how long a wait may take; a batch whose copies arrive
    within it is unaffected (bit for bit)."""
    wl, tabs = _tiny()
    theta, sid = wl.params(64, seed_offset=5)
    with Engine(0) as eng:
        t = eng.add_tables(wl.table, "fp16", tabs)
        s = eng.add_setup(t, wl.setups[0])
        b0, h0 = _run(eng, [s], theta, sid, None)
        hr2.hr2_stream_check(eng.ctx, None)
        hr2.hr2_set_wait_limit(eng.ctx, 20000000)       # ~10 ms, far above a copy's latency
        b1, h1 = _run(eng, [s], theta, sid, None)
        hr2.hr2_stream_check(eng.ctx, None)
        assert np.array_equal(b0.cpu().numpy(), b1.cpu().numpy())
        assert np.array_equal(h0.cpu().numpy(), h1.cpu().numpy())
