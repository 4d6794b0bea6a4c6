"""GPU parity of the stripe path (1D partitioning, Sec. 3.1): on an nx x 1
grid (vertical stripes, swept along y) or a 1 x ny grid (horizontal stripes,
swept along x), every stripe is sorted along the stripe in shared memory and
joined by the forward scan with the one-comparison duplicate test.  The pairs
equal the oracle's (PBSM on the same stripes, pinned by brute force) for
uniform, GIS-shaped, skew-light and degenerate inputs, a single stripe, wide
rectangles over many stripes, two-pass and one-pass modes (the stripe path is
exact two-pass) and sorted output; a stripe beyond shared memory sends the
join to the general path, still exact."""
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


def sorted_pairs(a):
    a = np.asarray(a.cpu().numpy() if hasattr(a, "cpu") else a, np.int32).reshape(-1, 2)
    return a[np.lexsort((a[:, 1], a[:, 0]))]


CASES = {
    "uniform": lambda: inputs.uniform_pair(60_000, 80_000, max_extent=4e-3, seed=121),
    "gis": lambda: inputs.gis_pair(200_000, 300_000, seed=122, median_extent=1e-4),
    "zipf": lambda: inputs.zipf_pair(60_000, 60_000, seed=123, lattice=128, r_max_extent=2e-3,
                                     s_max_extent=5e-3, rho=0.0),
    "degenerate": lambda: inputs.degenerate_pair(3000, 2500, seed=124),
    "wide": lambda: inputs.uniform_pair(20_000, 20_000, max_extent=0.2, seed=125),
}


@pytest.mark.parametrize("K", [1, 7, 200, 1500])
@pytest.mark.parametrize("vertical", [True, False])
@pytest.mark.parametrize("name", list(CASES))
def test_stripes_equal_oracle(sj, ctx, name, vertical, K):
    R, S = CASES[name]()
    nx, ny = (K, 1) if vertical else (1, K)
    want = oracle.pbsm(R, S, nx, ny)
    g = sj.make_grid(nx, ny)
    got = sj.sj_join(ctx, dev(R), dev(S), g)
    st = sj.sj_last_stats(ctx)
    np.testing.assert_array_equal(sorted_pairs(got), want)
    assert sj.sj_count(ctx, dev(R), dev(S), g) == len(want)
    if st["path"] == 2:
        assert st["blocks"] == K and st["block_side"] == 1


def test_stripe_path_taken_and_modes(sj, ctx):
    R, S = CASES["gis"]()
    g = sj.make_grid(1000, 1)
    want = oracle.pbsm(R, S, 1000, 1)
    for opts in (sj.make_opts("two_pass"), sj.make_opts("one_pass_heur"), sj.make_opts("two_pass", sort_output=True)):
        got = sj.sj_join(ctx, dev(R), dev(S), g, opts)
        assert sj.sj_last_stats(ctx)["path"] == 2
        if opts.sort_output:
            np.testing.assert_array_equal(got.cpu().numpy(), want)
        else:
            np.testing.assert_array_equal(sorted_pairs(got), want)
    buf = torch.full((len(want) + 4, 2), -1, dtype=torch.int32, device="cuda")
    assert sj.sj_join_into(ctx, dev(R), dev(S), g, buf) == len(want)
    np.testing.assert_array_equal(sorted_pairs(buf[:len(want)]), want)
    assert (buf[len(want):] == -1).all()


@pytest.mark.parametrize("K", [200, 400])
def test_stripes_of_several_thousand_entries(sj, ctx, K):
    """Stripes of 5,000-15,000 entries (beyond one tile of the block join,
    within the stripe kernel's shared memory) take the stripe path."""
    R, S = inputs.uniform_pair(1_000_000, 1_500_000, max_extent=2e-4, seed=127)
    for nx, ny in ((K, 1), (1, K)):
        want = oracle.pbsm(R, S, nx, ny)
        got = sj.sj_join(ctx, dev(R), dev(S), sj.make_grid(nx, ny))
        st = sj.sj_last_stats(ctx)
        assert st["path"] == 2, st
        assert 3072 < (st["l1_entries_r"] + st["l1_entries_s"]) / K < 16384
        np.testing.assert_array_equal(sorted_pairs(got), want)


def test_stripe_beyond_shared_memory_falls_back(sj, ctx):
    """40,000 rectangles in one stripe (more than 16,384 entries): the general
    path joins it, exactly."""
    R, S = inputs.uniform_pair(20_000, 20_000, max_extent=1e-3, seed=126)
    R[:, [0, 2]] = R[:, [0, 2]] * 0.001          # every R and S inside stripe 0 of 1000
    S[:, [0, 2]] = S[:, [0, 2]] * 0.001
    g = sj.make_grid(1000, 1)
    want = oracle.pbsm(R, S, 1000, 1)
    got = sj.sj_join(ctx, dev(R), dev(S), g)
    assert sj.sj_last_stats(ctx)["path"] != 2
    np.testing.assert_array_equal(sorted_pairs(got), want)
