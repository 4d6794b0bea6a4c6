"""GPU parity: the CUDA join through the C ABI against the CPU oracle.

Pairs are compared as sorted int32 (r, s) arrays, element by element (the
bar is bit-exact: the method involves no rounding other than the cell
function, which both sides compute in float32).  Per-tile counts and the
tile that reports each pair are compared too, since both sides use the same
float32 cell function.
"""
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


def sorted_pairs(t):
    a = t.cpu().numpy().astype(np.int32)
    return a[np.lexsort((a[:, 1], a[:, 0]))] if len(a) else a.reshape(0, 2)


def gpu_join(sj, ctx, R, S, nx, ny=None, ext=(0.0, 0.0, 1.0, 1.0), mode="two_pass", sort_output=False):
    g = sj.make_grid(nx, ny, *ext)
    out = sj.sj_join(ctx, dev(R), dev(S), g, sj.make_opts(mode, sort_output))
    torch.cuda.synchronize()
    return out


def test_fig1_instance(sj, ctx):
    from test_oracle_pins import load_fig1

    R, S, pairs, _ = load_fig1()
    got = sorted_pairs(gpu_join(sj, ctx, R, S, 3))
    np.testing.assert_array_equal(got, pairs[:, :2])
    cr, cs, tp = sj.sj_tile_stats(ctx, dev(R), dev(S), sj.make_grid(3))
    want_tp = np.bincount(pairs[:, 2], minlength=9)
    np.testing.assert_array_equal(tp.cpu().numpy(), want_tp)


def test_uniform_plain_join_64(sj, ctx):
    R, S = inputs.uniform_pair()          # |R| = |S| = 10^4, extents U[0, 2e-3]
    want = oracle.brute(R, S)
    got = sorted_pairs(gpu_join(sj, ctx, R, S, 64))
    np.testing.assert_array_equal(got, want)
    assert sj.sj_count(ctx, dev(R), dev(S), sj.make_grid(64)) == len(want)


@pytest.mark.parametrize("grid", [(1, 1), (2, 2), (7, 7), (16, 16), (64, 64), (5, 1), (1, 9), (13, 4),
                                  (300, 300)])
def test_degenerate_inputs_any_grid(sj, ctx, grid):
    R, S = inputs.degenerate_pair(900, 800, seed=7)
    want = oracle.brute(R, S)
    got = sorted_pairs(gpu_join(sj, ctx, R, S, *grid))
    np.testing.assert_array_equal(got, want)


def test_grid_over_subwindow(sj, ctx):
    R, S = inputs.uniform_pair(3000, 3000, max_extent=0.02, seed=3)
    want = oracle.brute(R, S)
    got = sorted_pairs(gpu_join(sj, ctx, R, S, 9, 9, (0.2, 0.3, 0.7, 0.6)))
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("K", [16, 100, 500])
def test_tile_counts_and_reporting_tiles(sj, ctx, K):
    R, S = inputs.gis_pair(20000, 30000, seed=5, median_extent=2e-3)
    _, info = oracle.pbsm(R, S, K, per_tile=True)
    cr, cs, tp = sj.sj_tile_stats(ctx, dev(R), dev(S), sj.make_grid(K))
    np.testing.assert_array_equal(cr.cpu().numpy(), info["cnt_r"])
    np.testing.assert_array_equal(cs.cpu().numpy(), info["cnt_s"])
    np.testing.assert_array_equal(tp.cpu().numpy(), info["pairs"])


def test_partition_segments(sj, ctx):
    # Sec. 3.4 steps 2-4: per-tile counts, prefix sums, and each tile's
    # segment holding exactly the rectangles that overlap it, with the
    # first-column / first-row flags of the duplicate test.
    R, S = inputs.uniform_pair(5000, 4000, max_extent=0.05, seed=8)
    K = 24
    part = sj.sj_partition(ctx, dev(R), dev(S), sj.make_grid(K))
    try:
        v = part.view()
        T = K * K
        torch.cuda.synchronize()
        o = sj.device_view(v.off, (T + 1, 2), torch.int32).cpu().numpy().view(np.uint32)
        idr = sj.device_view(v.id_r, (v.e_r,), torch.int32).cpu().numpy().view(np.uint32)
        mr = sj.device_view(v.ent_r, (v.e_r, 4), torch.float32).cpu().numpy()
        np.testing.assert_array_equal(np.diff(o[:, 0].astype(np.int64)), oracle.tile_counts(R, K))
        np.testing.assert_array_equal(np.diff(o[:, 1].astype(np.int64)), oracle.tile_counts(S, K))
        assert v.e_r == o[T, 0] and v.e_s == o[T, 1]
        mask = (1 << 30) - 1
        cells = np.array([[oracle.cell(float(r[k]), 0.0, 1.0, K) for k in range(4)] for r in R])
        for t in range(T):
            cx, cy = t % K, t // K
            seg = idr[o[t, 0]:o[t + 1, 0]]
            ids = seg & mask
            want = np.nonzero((cells[:, 0] <= cx) & (cx <= cells[:, 2]) &
                              (cells[:, 1] <= cy) & (cy <= cells[:, 3]))[0]
            np.testing.assert_array_equal(np.sort(ids), want)
            np.testing.assert_array_equal((seg >> 30) & 1, (cells[ids, 0] == cx).astype(np.uint32))
            np.testing.assert_array_equal(seg >> 31, (cells[ids, 1] == cy).astype(np.uint32))
            np.testing.assert_array_equal(mr[o[t, 0]:o[t + 1, 0]], R[ids])
        got = sorted_pairs(sj.sj_part_join(ctx, part))
        np.testing.assert_array_equal(got, oracle.pbsm(R, S, K))
        got2 = sorted_pairs(sj.sj_part_join(ctx, part))      # reusable
        np.testing.assert_array_equal(got2, got)
    finally:
        part.free()


def test_large_tiles(sj, ctx):
    # a few tiles hold thousands of entries (more than one shared-memory
    # chunk): the segmented radix sort + global sweep path
    g = np.random.default_rng(12)
    n = 12000
    cx = np.where(g.random(n) < 0.7, 0.51 + 0.02 * g.random(n), g.random(n))
    cy = np.where(g.random(n) < 0.7, 0.52 + 0.02 * g.random(n), g.random(n))
    R = inputs.rects_from_centres(cx, cy, g.uniform(0, 4e-3, n), g.uniform(0, 4e-3, n))
    cx = np.where(g.random(n) < 0.7, 0.51 + 0.02 * g.random(n), g.random(n))
    cy = np.where(g.random(n) < 0.7, 0.52 + 0.02 * g.random(n), g.random(n))
    S = inputs.rects_from_centres(cx, cy, g.uniform(0, 4e-3, n), g.uniform(0, 4e-3, n))
    for K in (8, 40):
        want = oracle.pbsm(R, S, K)
        got = sorted_pairs(gpu_join(sj, ctx, R, S, K))
        np.testing.assert_array_equal(got, want)
        _, info = oracle.pbsm(R, S, K, per_tile=True)
        assert (info["cnt_r"] + info["cnt_s"] + 1 > 1024).any()
        _, _, tp = sj.sj_tile_stats(ctx, dev(R), dev(S), sj.make_grid(K))
        np.testing.assert_array_equal(tp.cpu().numpy(), info["pairs"])


@pytest.mark.parametrize("K", [50, 200, 1000])
def test_gis_layers_scaled(sj, ctx, K):
    # 1% of the GIS-shaped workload (100k x 200k), denser extents so the
    # result is sizeable
    R, S = inputs.gis_pair(100_000, 200_000, seed=2, median_extent=2e-4)
    want = oracle.pbsm(R, S, K)
    got = sorted_pairs(gpu_join(sj, ctx, R, S, K))
    np.testing.assert_array_equal(got, want)


def test_zipf_skew_scaled(sj, ctx):
    R, S = inputs.zipf_pair(150_000, 150_000, seed=3, rho=0.02, lattice=256,
                            r_max_extent=4e-4, s_max_extent=4e-3)
    for K in (64, 256):
        want = oracle.pbsm(R, S, K)
        got = sorted_pairs(gpu_join(sj, ctx, R, S, K))
        np.testing.assert_array_equal(got, want)


def test_empty_and_tiny_inputs(sj, ctx):
    R, S = inputs.uniform_pair(10, 10, max_extent=0.5, seed=4)
    E = np.zeros((0, 4), np.float32)
    for a, b in ((R, E), (E, S), (E, E), (R[:1], S[:1])):
        got = sorted_pairs(gpu_join(sj, ctx, a, b, 4))
        np.testing.assert_array_equal(got, oracle.brute(a, b))
        assert sj.sj_count(ctx, dev(a), dev(b), sj.make_grid(4)) == len(oracle.brute(a, b))


def test_invalid_inputs_rejected(sj, ctx):
    R, S = inputs.uniform_pair(100, 100, seed=4)
    g = sj.make_grid(8)
    for bad in (np.nan, np.inf):
        B = R.copy()
        B[5, 2] = bad
        with pytest.raises(sj.SJError) as e:
            sj.sj_join(ctx, dev(B), dev(S), g)
        assert e.value.status == sj.SJ_EINVAL
    B = R.copy()
    B[7, 0], B[7, 2] = 0.6, 0.5          # xl > xu
    with pytest.raises(sj.SJError) as e:
        sj.sj_join(ctx, dev(B), dev(S), g)
    assert e.value.status == sj.SJ_EINVAL
    for bad_grid in (sj.make_grid(0), sj.make_grid(4, 4, 0.5, 0.0, 0.5, 1.0), sj.make_grid(1 << 25, 1)):
        with pytest.raises(sj.SJError) as e:
            sj.sj_join(ctx, dev(R), dev(S), bad_grid)
        assert e.value.status == sj.SJ_EINVAL
    # misaligned start (one float into the buffer)
    buf = dev(np.concatenate([R.ravel(), np.zeros(4, np.float32)]))
    mis = buf[1:1 + 400].view(100, 4)
    with pytest.raises(sj.SJError):
        sj.sj_join(ctx, mis, dev(S), g)
    # the context stays usable after errors
    np.testing.assert_array_equal(sorted_pairs(sj.sj_join(ctx, dev(R), dev(S), g)), oracle.brute(R, S))


def test_join_into_overflow_reports_required(sj, ctx):
    R, S = inputs.uniform_pair(3000, 3000, max_extent=0.02, seed=6)
    want = oracle.brute(R, S)
    small = torch.empty((len(want) // 2, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(sj.SJError) as e:
        sj.sj_join_into(ctx, dev(R), dev(S), sj.make_grid(32), small)
    assert e.value.status == sj.SJ_EOVERFLOW and e.value.required == len(want)
    big = torch.empty((len(want) + 5, 2), dtype=torch.int32, device="cuda")
    n = sj.sj_join_into(ctx, dev(R), dev(S), sj.make_grid(32), big)
    torch.cuda.synchronize()
    assert n == len(want)
    np.testing.assert_array_equal(sorted_pairs(big[:n]), want)


def test_repeated_calls_and_growth(sj, ctx):
    # workspace grows from small to large problems and stays correct
    for n, ext, K in ((500, 0.01, 4), (60_000, 2e-3, 300), (2000, 0.05, 16)):
        R, S = inputs.uniform_pair(n, n, max_extent=ext, seed=n)
        np.testing.assert_array_equal(sorted_pairs(gpu_join(sj, ctx, R, S, K)), oracle.pbsm(R, S, K))
