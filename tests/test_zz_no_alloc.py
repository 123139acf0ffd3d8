"""The allocation-free entry point against the ordinary one.

forward_model_batch_noalloc exists for callers that may not let a library
allocate device memory (an application whose device memory belongs to
another allocator, or a latency-critical loop that cannot accept the
synchronisation cudaMalloc may imply).  It must give what
forward_model_batch gives.  Two calls in a row with different batches check
that the shared static scratch, which keeps the previous call's contents,
does not leak into the next result.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1910_01070_b300 import hr2
from paper_1910_01070_b300 import workloads as W
from paper_1910_01070_b300.engine import Engine
from tests.helpers import FLUX_RTOL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel(a, b):
    a = a.astype(np.float64)
    b = b.astype(np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-30)))


def test_noalloc_matches_forward_model_batch_twice_in_a_row():
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
            torch.cuda.synchronize()
            for g, s in enumerate(wl.setups):
                rows = np.nonzero(sid == g)[0]
                if len(rows) == 0:
                    continue
                rb, ob = ref_b.cpu().numpy()[rows, : s.n_bins], out_b.cpu().numpy()[rows, : s.n_bins]
                rh, oh = ref_h.cpu().numpy()[rows, : s.n_nu], out_h.cpu().numpy()[rows, : s.n_nu]
                assert _rel(ob, rb) <= FLUX_RTOL
                assert _rel(oh, rh) <= FLUX_RTOL
            assert np.all(st.cpu().numpy() == 0)


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
