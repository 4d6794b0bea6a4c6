"""sj_join_noalloc: the join for callers that cannot allocate device memory
(code running under someone else's CUDA graph capture, plug-ins whose host
owns every allocation).  It is called here through the C ABI with
caller-owned buffers and compared with sj_join_into, the allocating entry
point, pair for pair (integer results: exact), on two calls in a row.

This file is collected last on purpose, so that a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_1908_11740_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sorted(a):
    a = np.asarray(a, np.int32).reshape(-1, 2)
    return a[np.lexsort((a[:, 1], a[:, 0]))]


def test_noalloc_matches_join_into_twice():
    from paper_1908_11740_gb300 import build, sj

    build.build()
    lib = sj.load()
    ctx = sj.sj_create(0)
    try:
        stream = torch.cuda.current_stream()
        cases = [inputs.uniform_pair(20_000, 30_000, max_extent=6e-3, seed=21),
                 inputs.degenerate_pair(900, 700, seed=22)]
        for (R, S), K in zip(cases, (128, 16)):
            dR, dS = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
            g = sj.make_grid(K)
            n_ref = sj.sj_count(ctx, dR, dS, g)
            ref = torch.empty((n_ref + 1, 2), dtype=torch.int32, device="cuda")
            n = sj.sj_join_into(ctx, dR, dS, g, ref)
            torch.cuda.synchronize()
            want = _sorted(ref[:n].cpu().numpy())
            for call in range(2):
                out = torch.full((n_ref + 16, 2), -1, dtype=torch.int32, device="cuda")
                got_n = ctypes.c_int64(-1)
                st = lib.sj_join_noalloc(dR.data_ptr(), len(R), dS.data_ptr(), len(S), ctypes.byref(g),
                                         out.data_ptr(), out.shape[0], ctypes.byref(got_n),
                                         ctypes.c_void_p(stream.cuda_stream))
                torch.cuda.synchronize()
                assert st == sj.SJ_OK, f"call {call}: status {st}"
                assert got_n.value == n
                np.testing.assert_array_equal(_sorted(out[:n].cpu().numpy()), want)
                assert (out[n:] == -1).all()
        # a buffer that is too small reports the required count
        R, S = cases[0]
        dR, dS = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
        g = sj.make_grid(128)
        small = torch.empty((4, 2), dtype=torch.int32, device="cuda")
        got_n = ctypes.c_int64(-1)
        st = lib.sj_join_noalloc(dR.data_ptr(), len(R), dS.data_ptr(), len(S), ctypes.byref(g),
                                 small.data_ptr(), 4, ctypes.byref(got_n), ctypes.c_void_p(stream.cuda_stream))
        assert st == sj.SJ_EOVERFLOW and got_n.value == sj.sj_count(ctx, dR, dS, g)
        # sizes beyond the fixed scratch are refused before any work
        big = torch.zeros((70_000, 4), dtype=torch.float32, device="cuda")
        st = lib.sj_join_noalloc(big.data_ptr(), 70_000, dS.data_ptr(), len(S), ctypes.byref(g),
                                 small.data_ptr(), 4, ctypes.byref(got_n), ctypes.c_void_p(stream.cuda_stream))
        assert st == sj.SJ_EINVAL
    finally:
        sj.sj_destroy(ctx)
