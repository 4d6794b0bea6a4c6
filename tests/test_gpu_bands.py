"""GPU parity of the block join's heavy-block paths against the oracle.

The two-level join stages a block whose tile entries exceed shared memory in
several bands of tiles; such a block first lists its entries per tile row in
a global pool (and reads its whole L1 range when the pool is exhausted).
The one-pass join collects a block's pairs in shared memory, then in a
global spill area per CTA, and re-sweeps a block whose pairs exceed both.
Every case below drives one of these paths and must return exactly the
oracle's pairs, in every join mode.
"""
import numpy as np
import pytest

import oracle

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


def sorted_pairs(t):
    a = t.cpu().numpy().astype(np.int32)
    return a[np.lexsort((a[:, 1], a[:, 0]))] if len(a) else a.reshape(0, 2)


def rects(g, n, lo, hi, wmax):
    c = g.uniform(lo, hi, (n, 2))
    w = g.uniform(0.0, wmax, (n, 2))
    return np.concatenate([c - w / 2, c + w / 2], axis=1).astype(np.float32)


MODES = ["two_pass", "one_pass_heur"]


def check_all_modes(sj, ctx, R, S, K, want=None):
    want = oracle.pbsm(R, S, K) if want is None else want
    for mode in MODES:
        got = sorted_pairs(sj.sj_join(ctx, dev(R), dev(S), sj.make_grid(K), sj.make_opts(mode, margin=0.0)))
        st = sj.sj_last_stats(ctx)
        np.testing.assert_array_equal(got, want, err_msg=mode)
        assert st["path"] == 1, "expected the two-level path"
    n = sj.sj_count(ctx, dev(R), dev(S), sj.make_grid(K))
    assert n == len(want)
    return want


def test_wide_rectangles_many_bands_and_pool_exhaustion(sj, ctx):
    # every rectangle covers about 3 x 3 tiles: blocks hold ~9x more tile
    # entries than L1 entries, so they need many bands and their row lists
    # outgrow the pool after a few blocks (the rest read their L1 range)
    g = np.random.default_rng(71)
    R = rects(g, 12_000, 0.0, 1.0, 0.06)
    S = rects(g, 12_000, 0.0, 1.0, 0.06)
    want = check_all_modes(sj, ctx, R, S, 64)
    assert len(want) > 100_000
    assert np.array_equal(want, oracle.brute(R, S))


@pytest.mark.parametrize("n_cluster", [1_000, 4_000])
def test_dense_cluster_pairs_spill_and_resweep(sj, ctx, n_cluster):
    # a cluster inside one block of 32 x 32 tiles on a 500 x 500 grid (block
    # 7 spans [0.448, 0.512) on both axes): ~1e4 pairs in one block (shared
    # buffer -> spill area) or ~1.6e5 (beyond the spill: the block is swept
    # again), plus a uniform background
    g = np.random.default_rng(72 + n_cluster)
    R = np.concatenate([rects(g, 20_000, 0.0, 1.0, 2e-3), rects(g, n_cluster, 0.452, 0.472, 2e-3)])
    S = np.concatenate([rects(g, 20_000, 0.0, 1.0, 2e-3), rects(g, n_cluster, 0.452, 0.472, 2e-3)])
    want = check_all_modes(sj, ctx, R, S, 500)
    inside = np.count_nonzero(R[want[:, 0], 0] > 0.45)
    assert inside > (5_000 if n_cluster == 1_000 else 50_000)


def test_dense_cluster_learned_sizing(sj, ctx):
    # the learned one-pass join (packaged model) on the same kind of cluster
    from paper_1908_11740_gb300 import learn

    g = np.random.default_rng(75)
    R = np.concatenate([rects(g, 30_000, 0.0, 1.0, 1e-3), rects(g, 2_000, 0.452, 0.472, 2e-3)])
    S = np.concatenate([rects(g, 30_000, 0.0, 1.0, 1e-3), rects(g, 2_000, 0.452, 0.472, 2e-3)])
    want = oracle.pbsm(R, S, 500)
    model, _ = learn.load(ctx)
    try:
        sj.sj_set_model(ctx, model)
        got = sorted_pairs(sj.sj_join(ctx, dev(R), dev(S), sj.make_grid(500), sj.make_opts("one_pass")))
        np.testing.assert_array_equal(got, want)
    finally:
        sj.sj_set_model(ctx, None)
        model.free()
