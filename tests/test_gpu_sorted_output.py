"""sj_opts.sort_output: the pairs come back in ascending (r, s) order, sorted
on the device (stable LSD radix sort of the pairs), and must equal the
oracle's sorted pair set element by element without any host-side sort."""
import numpy as np
import pytest

import oracle
from paper_1908_11740_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sj():
    from paper_1908_11740_gb300 import build, sj as binding

    build.build()
    return binding


@pytest.fixture(scope="module")
def ctx(sj):
    c = sj.sj_create(0)
    yield c
    sj.sj_destroy(c)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.mark.parametrize("mode", ["two_pass", "one_pass_heur", "one_pass"])
@pytest.mark.parametrize("grid", [64, 700])
def test_sorted_join_modes(sj, ctx, mode, grid):
    R, S = inputs.gis_pair(200_000, 300_000, seed=41, median_extent=2e-4)
    want = oracle.pbsm(R, S, 100)
    assert len(want) > 10_000
    model = None
    if mode == "one_pass":
        from paper_1908_11740_gb300 import learn
        model, _ = learn.load(ctx, learn.DEFAULT_MODEL)
        sj.sj_set_model(ctx, model)
    try:
        got = sj.sj_join(ctx, dev(R), dev(S), sj.make_grid(grid), sj.make_opts(mode, sort_output=True))
        np.testing.assert_array_equal(got.cpu().numpy(), want)
    finally:
        if model is not None:
            sj.sj_set_model(ctx, None)
            model.free()


@pytest.mark.parametrize("n_r,n_s,ext", [(1, 1, 0.5), (2, 3, 0.6), (3000, 50, 0.05), (9000, 9000, 0.02)])
def test_sorted_small_and_ragged(sj, ctx, n_r, n_s, ext):
    # pair counts around the sort's tile of 8192 pairs and its warp slices
    R, S = inputs.uniform_pair(n_r, n_s, max_extent=ext, seed=n_r + n_s)
    want = oracle.pbsm(R, S, 16)
    got = sj.sj_join(ctx, dev(R), dev(S), sj.make_grid(16), sj.make_opts("two_pass", sort_output=True))
    np.testing.assert_array_equal(got.cpu().numpy().reshape(-1, 2), want)


def test_sorted_single_level_and_into(sj, ctx):
    # dense duplicates: tiles beyond shared memory (single-level path)
    R, S = inputs.zipf_pair(60_000, 60_000, seed=5, rho=0.3, lattice=64)
    want = oracle.pbsm(R, S, 50)
    g = sj.make_grid(50)
    o = sj.make_opts("two_pass", sort_output=True)
    got = sj.sj_join(ctx, dev(R), dev(S), g, o)
    assert sj.sj_last_stats(ctx)["path"] == 0
    np.testing.assert_array_equal(got.cpu().numpy(), want)
    buf = torch.empty((len(want), 2), dtype=torch.int32, device="cuda")
    n = sj.sj_join_into(ctx, dev(R), dev(S), g, buf, o)
    assert n == len(want)
    np.testing.assert_array_equal(buf.cpu().numpy(), want)


def test_sorted_distance_join(sj, ctx):
    P, Q = inputs.gis_points(100_000, 150_000, seed=43)
    want = oracle.dist_pbsm(P, Q, 1e-3, 200)
    got = sj.sj_distance_join(ctx, dev(P), dev(Q), 1e-3, sj.make_grid(500),
                              sj.make_opts("two_pass", sort_output=True))
    np.testing.assert_array_equal(got.cpu().numpy(), want)
