"""GPU parity of grouping-based duplicate avoidance (SJ_DEDUP_GBDA): the
block join with class mini-joins instead of the test of Eq. 1 returns
exactly the oracle's pairs (the oracle's own GBDA route and its PBSM agree,
both pinned by brute force), in two-pass and one-pass modes, with sorted
output, on uniform, GIS-shaped, skew-light and degenerate inputs (blocks in
several bands included), and at full size on the 10M x 20M GIS-shaped join."""
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
    from paper_1908_11740_gb300 import learn

    c = sj.sj_create(0)
    model, _ = learn.load(c)
    yield c, model
    sj.sj_set_model(c, None)
    model.free()
    sj.sj_destroy(c)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def sorted_pairs(a):
    a = np.asarray(a.cpu().numpy() if hasattr(a, "cpu") else a, np.int32).reshape(-1, 2)
    return a[np.lexsort((a[:, 1], a[:, 0]))]


CASES = {
    "uniform": (lambda: inputs.uniform_pair(100_000, 150_000, max_extent=4e-3, seed=111), (256, 256)),
    "gis_heavy": (lambda: inputs.gis_pair(300_000, 500_000, seed=112, median_extent=1e-4), (120, 120)),
    "zipf": (lambda: inputs.zipf_pair(100_000, 100_000, seed=113, lattice=128, r_max_extent=2e-3,
                                      s_max_extent=5e-3, rho=0.0), (200, 150)),
    "degenerate": (lambda: inputs.degenerate_pair(3000, 2500, seed=114), (16, 16)),
}


@pytest.mark.parametrize("mode", ["two_pass", "one_pass_heur", "one_pass"])
@pytest.mark.parametrize("name", list(CASES))
def test_gbda_equals_oracle(sj, ctx, name, mode):
    make, (nx, ny) = CASES[name]
    R, S = make()
    c, model = ctx
    sj.sj_set_model(c, model if mode == "one_pass" else None)
    want = oracle.pbsm_gbda(R, S, nx, ny)
    np.testing.assert_array_equal(want, oracle.pbsm(R, S, nx, ny))
    g = sj.make_grid(nx, ny)
    got = sj.sj_join(c, dev(R), dev(S), g, sj.make_opts(mode, dedup="gbda"))
    st = sj.sj_last_stats(c)
    np.testing.assert_array_equal(sorted_pairs(got), want)
    if st["path"] == 1:
        assert st["dedup"] == 1
    srt = sj.sj_join(c, dev(R), dev(S), g, sj.make_opts(mode, dedup="gbda", sort_output=True))
    np.testing.assert_array_equal(srt.cpu().numpy(), want)
    assert sj.sj_count(c, dev(R), dev(S), g) == len(want)


def test_gbda_with_adaptive_axis_is_rejected(sj, ctx):
    c, _ = ctx
    R, S = inputs.uniform_pair(1000, 1000, seed=115)
    with pytest.raises(sj.SJError) as e:
        sj.sj_join(c, dev(R), dev(S), sj.make_grid(16), sj.make_opts("two_pass", axis="adaptive", dedup="gbda"))
    assert e.value.status == sj.SJ_EINVAL


def test_gbda_full_size(sj, ctx):
    c, model = ctx
    R, S = inputs.gis_pair()
    want = oracle.pbsm_gbda(R, S, 3000)
    g = sj.make_grid(3000)
    dR, dS = dev(R), dev(S)
    for mode in ("two_pass", "one_pass"):
        sj.sj_set_model(c, model if mode == "one_pass" else None)
        got = sj.sj_join(c, dR, dS, g, sj.make_opts(mode, dedup="gbda"))
        assert sj.sj_last_stats(c)["dedup"] == 1
        np.testing.assert_array_equal(sorted_pairs(got), want)
