"""Parity at the benchmark's full size and launch configuration: the
GIS-shaped join |R| = 10M, |S| = 20M on a 3000 x 3000 grid (and 1000 x 1000),
the complete sorted pair set against the single-threaded oracle, plus the
properties that hold at any size (no duplicates, count == sj_count, the
host-buffer entry point returns the same set)."""
import numpy as np
import pytest

import oracle
from paper_1908_11740_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def data():
    return inputs.gis_pair()          # 10M x 20M, seed 2


@pytest.fixture(scope="module")
def sj():
    from paper_1908_11740_gb300 import build, sj as binding

    build.build()
    return binding


def sorted_pairs(a):
    a = np.asarray(a, np.int32)
    return a[np.lexsort((a[:, 1], a[:, 0]))]


@pytest.mark.parametrize("K", [3000, 1000])
def test_gis_full_size_exact(sj, data, K):
    R, S = data
    want = oracle.pbsm(R, S, K)
    ctx = sj.sj_create(0)
    try:
        dR, dS = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
        g = sj.make_grid(K)
        got = sj.sj_join(ctx, dR, dS, g, sj.make_opts("two_pass")).cpu().numpy()
        assert len(np.unique(got.view(np.int64))) == len(got)          # no duplicates
        np.testing.assert_array_equal(sorted_pairs(got), want)
        assert sj.sj_count(ctx, dR, dS, g) == len(want)
        if K == 3000:
            host = sj.sj_join_host(ctx, R, S, g).numpy()
            np.testing.assert_array_equal(sorted_pairs(host), want)
            # sorted on the device: equal to the oracle without a host sort
            srt = sj.sj_join(ctx, dR, dS, g, sj.make_opts("two_pass", sort_output=True)).cpu().numpy()
            np.testing.assert_array_equal(srt, want)
    finally:
        sj.sj_destroy(ctx)
