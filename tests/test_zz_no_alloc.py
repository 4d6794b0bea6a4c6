"""sj_join_noalloc: the join for callers that cannot allocate device memory
(plug-ins whose host process owns every device allocation, callers on a
latency-critical path that cannot pay for cudaMalloc/cudaFree).  It is called
here through the C ABI with caller-owned buffers and compared, pair for pair
(integer results: exact), with sj_join_into, the allocating entry point, and
with the oracle, on two calls in a row.  The limits are exercised too: sizes
beyond them are refused before any work, and an input within the size limits
whose replicated entries exceed the fixed scratch is refused by the device
check with nothing written.

This file is collected last on purpose, so that a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1908_11740_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sorted(a):
    a = np.asarray(a, np.int32).reshape(-1, 2)
    return a[np.lexsort((a[:, 1], a[:, 0]))]


def _noalloc(lib, sj, dR, nR, dS, nS, g, out, cap, stream):
    got_n = ctypes.c_int64(-1)
    st = lib.sj_join_noalloc(dR.data_ptr(), nR, dS.data_ptr(), nS, ctypes.byref(g),
                             out.data_ptr() if out is not None else None, cap, ctypes.byref(got_n),
                             ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return st, got_n.value


def test_noalloc_matches_join_into_twice():
    from paper_1908_11740_gb300 import build, sj

    build.build()
    lib = sj.load()
    ctx = sj.sj_create(0)
    try:
        stream = torch.cuda.current_stream()
        cases = [inputs.uniform_pair(20_000, 30_000, max_extent=6e-3, seed=21),
                 inputs.degenerate_pair(900, 700, seed=22),
                 inputs.gis_pair(65_536, 65_536, seed=23, median_extent=5e-4)]
        for (R, S), K in zip(cases, (128, 16, 256)):
            want_oracle = oracle.pbsm(R, S, K)
            dR, dS = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
            g = sj.make_grid(K)
            n_ref = sj.sj_count(ctx, dR, dS, g)
            ref = torch.empty((n_ref + 1, 2), dtype=torch.int32, device="cuda")
            n = sj.sj_join_into(ctx, dR, dS, g, ref)
            torch.cuda.synchronize()
            want = _sorted(ref[:n].cpu().numpy())
            np.testing.assert_array_equal(want, want_oracle)
            for call in range(2):
                out = torch.full((n_ref + 16, 2), -1, dtype=torch.int32, device="cuda")
                st, got_n = _noalloc(lib, sj, dR, len(R), dS, len(S), g, out, out.shape[0], stream)
                assert st == sj.SJ_OK, f"call {call}: status {st}"
                assert got_n == n
                np.testing.assert_array_equal(_sorted(out[:n].cpu().numpy()), want)
                assert (out[n:] == -1).all()
        # a buffer that is too small reports the required count
        R, S = cases[0]
        dR, dS = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
        g = sj.make_grid(128)
        small = torch.full((4, 2), -1, dtype=torch.int32, device="cuda")
        st, got_n = _noalloc(lib, sj, dR, len(R), dS, len(S), g, small, 4, stream)
        assert st == sj.SJ_EOVERFLOW and got_n == sj.sj_count(ctx, dR, dS, g)
        assert (small == -1).all()
        # sizes beyond the fixed scratch are refused before any work
        big = torch.zeros((70_000, 4), dtype=torch.float32, device="cuda")
        st, _ = _noalloc(lib, sj, big, 70_000, dS, len(S), g, small, 4, stream)
        assert st == sj.SJ_EINVAL
        st, _ = _noalloc(lib, sj, dR, len(R), dS, len(S), sj.make_grid(300), small, 4, stream)
        assert st == sj.SJ_EINVAL           # 90,000 tiles > 65,536
    finally:
        sj.sj_destroy(ctx)


def test_noalloc_entry_cap_detected_on_device():
    """60,000 rectangles per side (within the size limit), each 3.5 tiles wide
    and high on a 256 x 256 grid: at least 16 replicated entries each, far
    beyond the 131,072 entries per side the scratch holds.  The device check
    refuses the join with SJ_EINVAL and the output buffer stays untouched."""
    from paper_1908_11740_gb300 import build, sj

    build.build()
    lib = sj.load()
    rng = np.random.default_rng(24)
    n, K = 60_000, 256
    w = 3.5 / K

    def rects():
        c = rng.uniform(w, 1.0 - w, (n, 2))
        return np.concatenate([c - w / 2, c + w / 2], axis=1).astype(np.float32)

    R, S = rects(), rects()
    assert len(oracle.cells(R, K)) == n
    c = oracle.cells(R, K)
    assert int(((c[:, 1] - c[:, 0] + 1) * (c[:, 3] - c[:, 2] + 1)).sum()) > 131_072
    dR, dS = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
    out = torch.full((1024, 2), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(2):
        st, got_n = _noalloc(lib, sj, dR, n, dS, n, sj.make_grid(K), out, out.shape[0], stream)
        assert st == sj.SJ_EINVAL
        assert got_n == 0
        assert (out == -1).all()
    # the scratch is still usable afterwards
    R2, S2 = inputs.uniform_pair(5_000, 6_000, max_extent=1e-2, seed=25)
    want = oracle.pbsm(R2, S2, 64)
    dR2, dS2 = torch.from_numpy(R2).cuda(), torch.from_numpy(S2).cuda()
    out = torch.full((len(want) + 8, 2), -1, dtype=torch.int32, device="cuda")
    st, got_n = _noalloc(lib, sj, dR2, len(R2), dS2, len(S2), sj.make_grid(64), out, out.shape[0], stream)
    assert st == sj.SJ_OK and got_n == len(want)
    np.testing.assert_array_equal(_sorted(out[:got_n].cpu().numpy()), want)
