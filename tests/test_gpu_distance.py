"""GPU parity of the eps-distance join on points (Sec. 1: squares of side eps,
intersection join, distance refinement) through the C ABI against the CPU
oracle.

The distance decision is taken in binary64 in the same fixed order on both
sides, so the pair sets must be identical (compared as sorted int32 arrays,
element by element).  The GPU's squares and the oracle's are built
independently (both only need to hold the exact square of side eps), so the
candidate counts may differ; the results may not."""
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


def srt(t):
    a = t.cpu().numpy().astype(np.int32) if isinstance(t, torch.Tensor) else np.asarray(t, np.int32)
    return a[np.lexsort((a[:, 1], a[:, 0]))] if len(a) else a.reshape(0, 2)


def gpu_dist(sj, ctx, P, Q, eps, nx, ny=None, mode="two_pass", ext=(0.0, 0.0, 1.0, 1.0)):
    out, nc = sj.sj_distance_join(ctx, dev(P), dev(Q), eps, sj.make_grid(nx, ny, *ext), sj.make_opts(mode),
                                  return_candidates=True)
    torch.cuda.synchronize()
    return out, nc


def _offsets(r):
    return [(a, b) for a in range(-r, r + 1) for b in range(-r, r + 1) if a * a + b * b <= r * r]


def _lattice_pairs(n, m, s, t, offs):
    out = [(i * n + j, (i + a - s) * m + (j + b - t)) for i in range(n) for j in range(n) for a, b in offs
           if 0 <= i + a - s < m and 0 <= j + b - t < m]
    return np.array(sorted(out), np.int32).reshape(-1, 2)


@pytest.mark.parametrize("r", [0, 1, 2, 5])
@pytest.mark.parametrize("grid", [1, 7, 64, 300])
def test_lattice_closed_form(sj, ctx, r, grid):
    h = 1.0 / 64
    P = inputs.lattice_points(40, h, 0.25, 0.25)
    Q = inputs.lattice_points(33, h, 0.25 + 3 * h, 0.25 - 2 * h)
    want = _lattice_pairs(40, 33, 3, -2, _offsets(r))
    got, nc = gpu_dist(sj, ctx, P, Q, np.float32(r * h), grid)
    np.testing.assert_array_equal(srt(got), want)
    assert nc >= len(want)


@pytest.mark.parametrize("r", [1, 3])
def test_lattice_just_below_radius(sj, ctx, r):
    h = 1.0 / 64
    P = inputs.lattice_points(30, h, 0.25, 0.25)
    eps = np.nextafter(np.float32(r * h), np.float32(0))
    want = _lattice_pairs(30, 30, 0, 0, [(a, b) for a, b in _offsets(r) if a * a + b * b < r * r])
    got, _ = gpu_dist(sj, ctx, P, P, eps, 16)
    np.testing.assert_array_equal(srt(got), want)


@pytest.mark.parametrize("seed,n_p,n_q,eps,grid", [
    (1, 3000, 5000, 0.01, 64), (2, 20000, 30000, 0.003, 200), (3, 50000, 40000, 0.001, 700),
    (4, 5000, 100, 0.05, 20), (5, 1, 20000, 0.2, 50)])
def test_uniform_points(sj, ctx, seed, n_p, n_q, eps, grid):
    rng = np.random.default_rng(seed)
    P = rng.random((n_p, 2)).astype(np.float32)
    Q = (rng.random((n_q, 2)) * 1.1 - 0.05).astype(np.float32)
    want = oracle.dist_pbsm(P, Q, eps, 50)
    got, nc = gpu_dist(sj, ctx, P, Q, eps, grid)
    np.testing.assert_array_equal(srt(got), want)
    assert nc >= len(want)


@pytest.mark.parametrize("mode", ["two_pass", "one_pass_heur"])
@pytest.mark.parametrize("eps,grid", [(5e-4, 500), (2e-3, 100), (1e-4, 2000)])
def test_clustered_points(sj, ctx, mode, eps, grid):
    P, Q = inputs.gis_points(200_000, 300_000, seed=21)
    want = oracle.dist_pbsm(P, Q, eps, 400)
    assert len(want) > 1000
    got, _ = gpu_dist(sj, ctx, P, Q, eps, grid, mode=mode)
    np.testing.assert_array_equal(srt(got), want)


def test_duplicates_and_dense_tiles(sj, ctx):
    # few distinct locations, thousands of copies each: tiles far above the
    # shared-memory capacity (the single-level path with its large-tile sort)
    rng = np.random.default_rng(8)
    base = rng.random((40, 2)).astype(np.float32)
    P = base[rng.integers(0, 40, 30_000)]
    Q = np.concatenate([base[rng.integers(0, 40, 20_000)], rng.random((5000, 2)).astype(np.float32)])
    for eps in (0.0, 1e-3, 0.02):
        want = oracle.dist_pbsm(P, Q, eps, 30)
        got, _ = gpu_dist(sj, ctx, P, Q, eps, 64)
        np.testing.assert_array_equal(srt(got), want)


def test_path_points_on_the_fly_and_materialised(sj, ctx):
    """The two-level path reads the points and forms the squares as it loads
    them; a tile beyond shared memory sends the join to the single-level
    path, which gets materialised squares.  Both give the oracle's set."""
    P, Q = inputs.gis_points(100_000, 150_000, seed=44)
    want = oracle.dist_pbsm(P, Q, 5e-4, 200)
    got, _ = gpu_dist(sj, ctx, P, Q, 5e-4, 400)
    assert sj.sj_last_stats(ctx)["path"] == 1
    np.testing.assert_array_equal(srt(got), want)
    # three points repeated thousands of times: their tiles hold more than
    # 3,072 entries (about 3,300 each)
    rng = np.random.default_rng(45)
    base = rng.random((3, 2)).astype(np.float32)
    Ph = np.concatenate([base[np.arange(6_000) % 3], P[:20_000]])
    Qh = np.concatenate([base[np.arange(4_000) % 3], Q[:20_000]])
    want = oracle.dist_pbsm(Ph, Qh, 2e-3, 50)
    for mode in ("two_pass", "one_pass_heur"):
        got, _ = gpu_dist(sj, ctx, Ph, Qh, 2e-3, 64, mode=mode)
        assert sj.sj_last_stats(ctx)["path"] == 0
        np.testing.assert_array_equal(srt(got), want)
    # the context's next rectangle join reads rectangles again
    R, S = inputs.gis_pair(30_000, 40_000, seed=46)
    got = sj.sj_join(ctx, dev(R), dev(S), sj.make_grid(100))
    np.testing.assert_array_equal(srt(got), oracle.pbsm(R, S, 100))


def test_tiny_and_negative_coordinates(sj, ctx):
    rng = np.random.default_rng(12)
    P = np.concatenate([rng.random((300, 2)) * 1e-30, -rng.random((300, 2)) * 1e-3,
                        rng.random((300, 2)) * 2e-3 - 1e-3]).astype(np.float32)
    Q = np.concatenate([rng.random((400, 2)) * 1e-30, rng.random((400, 2)) * 2e-3 - 1e-3]).astype(np.float32)
    for eps in (1e-31, 1e-4, 4e-4):
        want = oracle.dist_brute(P, Q, eps)
        got, _ = gpu_dist(sj, ctx, P, Q, eps, 32, ext=(-1e-3, -1e-3, 1e-3, 1e-3))
        np.testing.assert_array_equal(srt(got), want)


def test_empty_inputs(sj, ctx):
    P = np.zeros((0, 2), np.float32)
    Q = np.random.default_rng(1).random((100, 2)).astype(np.float32)
    for a, b in ((P, Q), (Q, P), (P, P)):
        got, nc = gpu_dist(sj, ctx, a, b, 0.1, 8)
        assert got.shape == (0, 2) and nc == 0
    got, nc = gpu_dist(sj, ctx, Q[:50], Q[50:], 0.0, 8)   # no coincident points
    assert got.shape == (0, 2)


def test_invalid_arguments(sj, ctx):
    P = dev(np.random.default_rng(2).random((64, 2)))
    g = sj.make_grid(8)
    for eps in (float("nan"), -1e-3, float("inf"), 1e30):
        with pytest.raises(sj.SJError) as ei:
            sj.sj_distance_join(ctx, P, P, eps, g)
        assert ei.value.status == sj.SJ_EINVAL
    bad = P.clone()
    bad[5, 1] = float("nan")
    with pytest.raises(sj.SJError) as ei:
        sj.sj_distance_join(ctx, bad, P, 0.1, g)
    assert ei.value.status == sj.SJ_EINVAL
    flat = torch.zeros(2 * 64 + 1, dtype=torch.float32, device="cuda")
    shifted = flat[1:].view(64, 2)                     # 4-byte aligned only
    with pytest.raises(sj.SJError) as ei:
        sj.sj_distance_join(ctx, shifted, P, 0.1, g)
    assert ei.value.status == sj.SJ_EINVAL
    # the context stays usable
    got = sj.sj_distance_join(ctx, P, P, 0.0, g)
    assert got.shape[0] == 64


def test_into_and_overflow(sj, ctx):
    rng = np.random.default_rng(4)
    P = rng.random((4000, 2)).astype(np.float32)
    Q = rng.random((6000, 2)).astype(np.float32)
    want = oracle.dist_pbsm(P, Q, 0.01, 20)
    g = sj.make_grid(40)
    short = torch.empty((len(want) - 1, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(sj.SJError) as ei:
        sj.sj_distance_join_into(ctx, dev(P), dev(Q), 0.01, g, short)
    assert ei.value.status == sj.SJ_EOVERFLOW and ei.value.required == len(want)
    buf = torch.full((len(want) + 10, 2), -7, dtype=torch.int32, device="cuda")
    n = sj.sj_distance_join_into(ctx, dev(P), dev(Q), 0.01, g, buf)
    assert n == len(want)
    np.testing.assert_array_equal(srt(buf[:n]), want)
    assert (buf[n:] == -7).all().item()


def test_repeated_calls_and_interleaving(sj, ctx):
    # the workspace is shared with the rectangle join: interleave both
    P, Q = inputs.gis_points(50_000, 80_000, seed=31)
    R, S = inputs.gis_pair(30_000, 40_000, seed=32)
    want_d = oracle.dist_pbsm(P, Q, 1e-3, 100)
    want_r = oracle.pbsm(R, S, 100)
    for _ in range(2):
        got, _ = gpu_dist(sj, ctx, P, Q, 1e-3, 300)
        np.testing.assert_array_equal(srt(got), want_d)
        got = sj.sj_join(ctx, dev(R), dev(S), sj.make_grid(300))
        np.testing.assert_array_equal(srt(got), want_r)


def test_full_size_gis_points(sj):
    """The benchmark workload: |P| = 10M, |Q| = 20M mixture points, eps =
    5e-5, grid 2000 x 2000, every pair against the oracle; learned one-pass
    and two-pass candidate joins give the same set."""
    P, Q = inputs.gis_points(seed=2)
    want = oracle.dist_pbsm(P, Q, 5e-5, 2000)
    c = sj.sj_create(0)
    try:
        dP, dQ = dev(P), dev(Q)
        g = sj.make_grid(2000)
        got, nc = sj.sj_distance_join(c, dP, dQ, 5e-5, g, sj.make_opts("two_pass"), return_candidates=True)
        assert nc >= len(want) > 1_000_000
        got = got.cpu().numpy()
        assert len(np.unique(got.view(np.int64))) == len(got)
        np.testing.assert_array_equal(srt(got), want)
        from paper_1908_11740_gb300 import learn
        model, _ = learn.load(c, learn.DEFAULT_MODEL)
        sj.sj_set_model(c, model)
        got1 = sj.sj_distance_join(c, dP, dQ, 5e-5, g, sj.make_opts("one_pass"))
        np.testing.assert_array_equal(srt(got1), want)
        first = sj.sj_last_stats(c)
        # the model learned rectangle joins and under-sizes these squares;
        # the context's capacity calibration removes the re-runs on later calls
        for _ in range(2):
            got1 = sj.sj_distance_join(c, dP, dQ, 5e-5, g, sj.make_opts("one_pass"))
            np.testing.assert_array_equal(srt(got1), want)
        st = sj.sj_last_stats(c)
        assert st["one_pass"] == 1 and st["capacity"] >= len(want), (first, st)
        assert st["refit_items"] == 0, (first, st)
        sj.sj_set_model(c, None)
        model.free()
    finally:
        sj.sj_destroy(c)
