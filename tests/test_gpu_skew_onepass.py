"""One pass on the single-level path (the extent / skew stress workload,
whose hottest tiles exceed shared memory): the small tiles are counted, the
output holds their exact pairs plus one slot per candidate of the large
tiles, and the large-tile sweep appends each candidate chunk's pairs with one
atomic.  The pairs equal the oracle's in every one-pass mode, through the
library buffer, a caller buffer that holds the bound, a caller buffer that
does not (the exact two-pass join runs), and with sorted output."""
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


@pytest.fixture(scope="module")
def data():
    # 22 tiles beyond shared memory (the largest 59,722 entries), 8.3M pairs
    R, S = inputs.zipf_pair(300_000, 300_000, seed=131, lattice=256, r_max_extent=1e-4, s_max_extent=5e-4,
                            rho=0.3)
    return R, S, oracle.pbsm(R, S, 200)


@pytest.mark.parametrize("mode", ["one_pass_heur", "one_pass"])
def test_single_level_one_pass(sj, ctx, data, mode):
    R, S, want = data
    c, model = ctx
    sj.sj_set_model(c, model if mode == "one_pass" else None)
    g = sj.make_grid(200)
    dR, dS = dev(R), dev(S)
    got = sj.sj_join(c, dR, dS, g, sj.make_opts(mode))
    st = sj.sj_last_stats(c)
    assert st["path"] == 0 and st["one_pass"] == 1
    assert st["capacity"] >= len(want)
    np.testing.assert_array_equal(sorted_pairs(got), want)
    srt = sj.sj_join(c, dR, dS, g, sj.make_opts(mode, sort_output=True))
    np.testing.assert_array_equal(srt.cpu().numpy(), want)
    # a caller buffer that holds the bound: one pass; one that does not: exact two-pass
    big = torch.full((st["capacity"] + 8, 2), -1, dtype=torch.int32, device="cuda")
    n = sj.sj_join_into(c, dR, dS, g, big, sj.make_opts(mode))
    assert n == len(want) and sj.sj_last_stats(c)["one_pass"] == 1
    np.testing.assert_array_equal(sorted_pairs(big[:n]), want)
    exact = torch.full((len(want) + 3, 2), -1, dtype=torch.int32, device="cuda")
    n = sj.sj_join_into(c, dR, dS, g, exact, sj.make_opts(mode))
    assert n == len(want) and sj.sj_last_stats(c)["one_pass"] == 0
    np.testing.assert_array_equal(sorted_pairs(exact[:n]), want)
    assert (exact[n:] == -1).all()
