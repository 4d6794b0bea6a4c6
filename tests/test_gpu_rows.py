"""GPU parity of the band split of one join (sj_join_rows, the per-GPU share
when the tile rows of one join are split over several GPUs).

One GPU runs the bands of a plan one after the other through the C ABI:

* every band returns exactly the oracle's pairs whose reference tile
  (Eq. 1) lies in its rows, and the union over the bands is the oracle's
  join, with no pair in two bands (plans of 1, 2, 3 and 5 bands, two-pass
  and one-pass, sorted output);
* a rank that stages only its band's rectangles (dist.band_members) gets the
  same pairs after mapping its local ids back;
* edge cases: an empty band, the band of all rows (= sj_join), a band
  outside the grid (SJ_EINVAL), a too small caller buffer (SJ_EOVERFLOW with
  the required count), an invalid rectangle outside the band (SJ_EINVAL, as
  for the whole join)."""
import numpy as np
import pytest

import oracle
from paper_1908_11740_gb300 import dist, inputs

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


def ref_rows(R, S, pairs, g):
    cr = oracle.cells(R, g.nx, g.ny, g.x0, g.y0, g.x1, g.y1)[:, 2]
    cs = oracle.cells(S, g.nx, g.ny, g.x0, g.y0, g.x1, g.y1)[:, 2]
    return np.maximum(cr[pairs[:, 0]], cs[pairs[:, 1]])


@pytest.fixture(scope="module")
def data():
    R, S = inputs.gis_pair(400_000, 700_000, seed=91, median_extent=2e-4)
    return R, S, oracle.pbsm(R, S, 400, 300)


@pytest.mark.parametrize("mode", ["two_pass", "one_pass_heur"])
@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_bands_union_is_the_join(sj, ctx, data, world, mode):
    R, S, want = data
    g = sj.make_grid(400, 300)
    rows = ref_rows(R, S, want, g)
    bands = dist.band_plan(dist.row_loads(R, S, g), world)
    dR, dS = dev(R), dev(S)
    parts = []
    for row0, row1 in bands:
        got = sorted_pairs(sj.sj_join_rows(ctx, dR, dS, g, row0, row1, sj.make_opts(mode)))
        np.testing.assert_array_equal(got, want[(rows >= row0) & (rows < row1)])
        parts.append(got)
    union = np.concatenate(parts)
    np.testing.assert_array_equal(sorted_pairs(union), want)
    assert len(union) == len(want)


def test_staged_band_rectangles(sj, ctx, data):
    R, S, want = data
    g = sj.make_grid(400, 300)
    rows = ref_rows(R, S, want, g)
    for row0, row1 in dist.band_plan(dist.row_loads(R, S, g), 3):
        ir, is_ = dist.band_members(R, S, g, row0, row1)
        assert len(ir) < len(R) and len(is_) < len(S)
        local = sj.sj_join_rows(ctx, dev(R[ir]), dev(S[is_]), g, row0, row1,
                                sj.make_opts("two_pass", sort_output=True)).cpu().numpy()
        got = np.stack([ir[local[:, 0]], is_[local[:, 1]]], 1)
        np.testing.assert_array_equal(sorted_pairs(got), want[(rows >= row0) & (rows < row1)])


def test_band_edge_cases(sj, ctx, data):
    R, S, want = data
    g = sj.make_grid(400, 300)
    dR, dS = dev(R), dev(S)
    assert sj.sj_join_rows(ctx, dR, dS, g, 120, 120).shape[0] == 0
    np.testing.assert_array_equal(sorted_pairs(sj.sj_join_rows(ctx, dR, dS, g, 0, 300)), want)
    srt = sj.sj_join_rows(ctx, dR, dS, g, 0, 300, sj.make_opts("two_pass", sort_output=True)).cpu().numpy()
    np.testing.assert_array_equal(srt, want)
    for bad in ((-1, 5), (10, 5), (0, 301)):
        with pytest.raises(sj.SJError) as e:
            sj.sj_join_rows(ctx, dR, dS, g, *bad)
        assert e.value.status == sj.SJ_EINVAL
    rows = ref_rows(R, S, want, g)
    n_band = int(((rows >= 100) & (rows < 200)).sum())
    small = torch.full((3, 2), -1, dtype=torch.int32, device="cuda")
    with pytest.raises(sj.SJError) as e:
        sj.sj_join_rows_into(ctx, dR, dS, g, 100, 200, small)
    assert e.value.status == sj.SJ_EOVERFLOW
    buf = torch.full((n_band + 5, 2), -1, dtype=torch.int32, device="cuda")
    assert sj.sj_join_rows_into(ctx, dR, dS, g, 100, 200, buf) == n_band
    assert (buf[n_band:] == -1).all()
    bad = R.copy()
    bad[7] = [0.5, 0.99, 0.4, 0.995]          # xl > xu, far from rows 0-9
    with pytest.raises(sj.SJError) as e:
        sj.sj_join_rows(ctx, dev(bad), dS, g, 0, 10)
    assert e.value.status == sj.SJ_EINVAL
