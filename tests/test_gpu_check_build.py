"""The debug build with bounds checks (-DSJ_CHECK=1, build(check=True)).

Every data-dependent index of the kernels (offsets from atomics, scans,
counts and searches) is checked against its bound in that build; a failed
check records its site, skips the access and makes the call return
SJ_EINTERNAL naming the site.  It stands in for compute-sanitizer.  Here the
debug library is loaded beside the normal one and every path of the join
runs through it on small inputs: the two-level path in every mode and
variant, the single-level path with large tiles, stripes, a band of rows,
the distance join, batches, the partition reuse and the join without
allocation.  Each result must equal the oracle's and no check may fail.
Then the self-test: with SJ_CHECK_SELFTEST set, the two-pass write is given
one slot fewer than its pairs, so the check of the last write fails (the
write is skipped); the call must report it, and the same context must then
join correctly again."""
import ctypes
import os

import numpy as np
import pytest

import oracle
from paper_1908_11740_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sj():
    """The binding switched to the debug library for this module."""
    from paper_1908_11740_gb300 import build, sj as binding

    build.build()
    path = build.build(check=True)
    saved = binding._lib
    binding._lib = None
    binding.load(path)
    try:
        yield binding
    finally:
        binding._lib = saved


@pytest.fixture(scope="module")
def ctx(sj):
    c = sj.sj_create(0)
    yield c
    sj.sj_destroy(c)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def srt(t):
    a = np.asarray(t.cpu().numpy() if hasattr(t, "cpu") else t, np.int32).reshape(-1, 2)
    return a[np.lexsort((a[:, 1], a[:, 0]))]


@pytest.fixture(scope="module")
def gis():
    R, S = inputs.gis_pair(150_000, 250_000, seed=71, median_extent=2e-4)
    return R, S, oracle.pbsm(R, S, 300)


@pytest.mark.parametrize("variant", [{}, {"axis": "adaptive"}, {"dedup": "gbda"}])
@pytest.mark.parametrize("mode", ["two_pass", "one_pass_heur"])
def test_two_level_modes_and_variants(sj, ctx, gis, mode, variant):
    R, S, want = gis
    got = sj.sj_join(ctx, dev(R), dev(S), sj.make_grid(300), sj.make_opts(mode, **variant))
    np.testing.assert_array_equal(srt(got), want)
    assert sj.sj_last_stats(ctx)["path"] == 1


def test_learned_one_pass_and_sorted_output(sj, ctx, gis):
    from paper_1908_11740_gb300 import learn

    R, S, want = gis
    model, _ = learn.load(ctx)
    try:
        sj.sj_set_model(ctx, model)
        opts = sj.make_opts("one_pass", sort_output=True)
        got = sj.sj_join(ctx, dev(R), dev(S), sj.make_grid(300), opts).cpu().numpy()
        np.testing.assert_array_equal(got, want)   # already in (r, s) order
        # an under-sized plan: blocks re-run exactly
        p = np.zeros(learn.N_PARAMS, np.float32)
        zero = sj.Model(ctx, p)
        try:
            sj.sj_set_model(ctx, zero)
            got = sj.sj_join(ctx, dev(R), dev(S), sj.make_grid(300), sj.make_opts("one_pass", margin=0.0))
            np.testing.assert_array_equal(srt(got), want)
            assert sj.sj_last_stats(ctx)["refit_items"] > 0
        finally:
            sj.sj_set_model(ctx, None)
            zero.free()
    finally:
        sj.sj_set_model(ctx, None)
        model.free()


@pytest.mark.parametrize("mode", ["two_pass", "one_pass_heur"])
def test_single_level_large_tiles(sj, ctx, mode):
    # hot tiles of ~30k entries, beyond shared memory: the single-level path with its large-tile
    # sort and sweep (4.4e5 pairs)
    R, S = inputs.zipf_pair(150_000, 150_000, seed=131, lattice=256, r_max_extent=1e-4, s_max_extent=1e-3,
                            rho=0.02)
    want = oracle.pbsm(R, S, 200)
    got = sj.sj_join(ctx, dev(R), dev(S), sj.make_grid(200), sj.make_opts(mode))
    np.testing.assert_array_equal(srt(got), want)
    assert sj.sj_last_stats(ctx)["path"] == 0


@pytest.mark.parametrize("vertical", [True, False])
def test_stripes(sj, ctx, gis, vertical):
    R, S, _ = gis
    nx, ny = (400, 1) if vertical else (1, 400)
    want = oracle.pbsm(R, S, nx, ny)
    got = sj.sj_join(ctx, dev(R), dev(S), sj.make_grid(nx, ny))
    np.testing.assert_array_equal(srt(got), want)
    assert sj.sj_last_stats(ctx)["path"] == 2


def test_degenerate_inputs(sj, ctx):
    R, S = inputs.degenerate_pair(3000, 2500, seed=73)
    for K in (1, 7, 64):
        want = oracle.pbsm(R, S, K)
        np.testing.assert_array_equal(srt(sj.sj_join(ctx, dev(R), dev(S), sj.make_grid(K))), want)


def test_bands_of_rows(sj, ctx, gis):
    R, S, want = gis
    g = sj.make_grid(300)
    parts = [srt(sj.sj_join_rows(ctx, dev(R), dev(S), g, r0, r1, sj.make_opts("two_pass", sort_output=True)))
             for r0, r1 in ((0, 97), (97, 180), (180, 300))]
    got = np.concatenate(parts)
    np.testing.assert_array_equal(srt(got), want)


@pytest.mark.parametrize("mode", ["two_pass", "one_pass_heur"])
def test_distance_join(sj, ctx, mode):
    P, Q = inputs.gis_points(60_000, 90_000, seed=74)
    eps = 1e-3
    want = oracle.dist_pbsm(P, Q, eps, 200)
    got = sj.sj_distance_join(ctx, dev(P), dev(Q), eps, sj.make_grid(200), sj.make_opts(mode))
    np.testing.assert_array_equal(srt(got), want)


@pytest.mark.parametrize("mode", ["two_pass", "one_pass_heur"])
def test_batch(sj, ctx, mode):
    joins = [inputs.uniform_pair(3000 + 500 * j, 4000, max_extent=5e-3, seed=75 + j) for j in range(6)]
    joins.append(inputs.degenerate_pair(400, 300, seed=81))
    pairs, offs = sj.sj_join_batch(ctx, [dev(r) for r, _ in joins], [dev(s) for _, s in joins],
                                   opts=sj.make_opts(mode))
    got = pairs.cpu().numpy()
    for j, (r, s) in enumerate(joins):
        np.testing.assert_array_equal(srt(got[offs[j]:offs[j + 1]]), oracle.brute(r, s))


def test_partition_reuse(sj, ctx, gis):
    R, S, want = gis
    part = sj.sj_partition(ctx, dev(R), dev(S), sj.make_grid(300))
    try:
        for _ in range(2):
            np.testing.assert_array_equal(srt(sj.sj_part_join(ctx, part)), want)
    finally:
        part.free()


def test_join_without_allocation(sj, ctx):
    R, S = inputs.uniform_pair(20_000, 30_000, max_extent=6e-3, seed=82)
    want = oracle.pbsm(R, S, 128)
    dR, dS = dev(R), dev(S)
    out = torch.full((len(want) + 8, 2), -1, dtype=torch.int32, device="cuda")
    n = ctypes.c_int64(-1)
    st = sj.load().sj_join_noalloc(dR.data_ptr(), len(R), dS.data_ptr(), len(S), ctypes.byref(sj.make_grid(128)),
                                   out.data_ptr(), out.shape[0], ctypes.byref(n),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert st == sj.SJ_OK and n.value == len(want)
    np.testing.assert_array_equal(srt(out[:n.value]), want)


def test_failed_check_is_reported_and_the_context_recovers(sj, ctx, gis):
    R, S, want = gis
    g = sj.make_grid(300)
    os.environ["SJ_CHECK_SELFTEST"] = "1"
    try:
        with pytest.raises(sj.SJError) as ei:
            sj.sj_join(ctx, dev(R), dev(S), g, sj.make_opts("two_pass"))
    finally:
        del os.environ["SJ_CHECK_SELFTEST"]
    assert ei.value.status == sj.SJ_EINTERNAL
    assert "bounds check failed at blocked.cu:" in str(ei.value)
    np.testing.assert_array_equal(srt(sj.sj_join(ctx, dev(R), dev(S), g, sj.make_opts("two_pass"))), want)
