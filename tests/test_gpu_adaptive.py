"""GPU parity of the adaptive sweep axis (Sec. 3.3, SJ_SWEEP_ADAPTIVE).

* the axis of every tile (sj_tile_axes) equals the oracle's choice from the
  Eq. 2 histograms (oracle.tile_axes), element by element: both sides decide
  on integer counts from the same float32 cell-function values;
* joins with the adaptive axis (two-pass, one-pass with the Eq. 2 and the
  learned sizing) return exactly the oracle's pairs, on elongated,
  GIS-shaped and degenerate inputs, including blocks staged in several
  bands, and the count of tiles swept along y matches the oracle;
* at full size (10M x 20M elongated rectangles) the same holds.
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
    "aniso": (lambda: inputs.aniso_pair(200_000, 300_000, seed=71, median_extent=1e-4), (300, 300)),
    "aniso_coarse": (lambda: inputs.aniso_pair(200_000, 300_000, seed=72, median_extent=1e-4), (60, 90)),
    "gis_heavy": (lambda: inputs.gis_pair(300_000, 500_000, seed=73, median_extent=1e-4), (120, 120)),
    "degenerate": (lambda: inputs.degenerate_pair(3000, 2500, seed=74), (16, 16)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_tile_axes_equal_oracle(sj, ctx, name):
    make, (nx, ny) = CASES[name]
    R, S = make()
    c, _ = ctx
    g = sj.make_grid(nx, ny)
    got = sj.sj_tile_axes(c, dev(R), dev(S), g).cpu().numpy()
    want, ix, iy = oracle.tile_axes(R, S, nx, ny)
    np.testing.assert_array_equal(got, want)
    if name.startswith("aniso"):
        both = (ix > 0) | (iy > 0)
        assert 0.2 < want[both].mean() < 0.8      # both axes in use


@pytest.mark.parametrize("mode", ["two_pass", "one_pass_heur", "one_pass"])
@pytest.mark.parametrize("name", list(CASES))
def test_adaptive_join_equals_oracle(sj, ctx, name, mode):
    make, (nx, ny) = CASES[name]
    R, S = make()
    c, model = ctx
    sj.sj_set_model(c, model if mode == "one_pass" else None)
    want = oracle.pbsm(R, S, nx, ny)
    g = sj.make_grid(nx, ny)
    got = sj.sj_join(c, dev(R), dev(S), g, sj.make_opts(mode, axis="adaptive"))
    st = sj.sj_last_stats(c)
    np.testing.assert_array_equal(sorted_pairs(got), want)
    if st["path"] == 1:
        ax, _, _ = oracle.tile_axes(R, S, nx, ny)
        assert st["y_sweep_tiles"] == int(ax.sum())
    # sorted on the device, and through a caller buffer
    srt = sj.sj_join(c, dev(R), dev(S), g, sj.make_opts(mode, axis="adaptive", sort_output=True))
    np.testing.assert_array_equal(srt.cpu().numpy(), want)


def test_adaptive_full_size(sj, ctx):
    """10M x 20M elongated rectangles (ten times longer along one axis) at the
    grid of the tile-extent rule."""
    c, model = ctx
    R, S = inputs.aniso_pair()
    K = 1750
    want = oracle.pbsm(R, S, K)
    ax, _, _ = oracle.tile_axes(R, S, K)
    dR, dS = dev(R), dev(S)
    g = sj.make_grid(K)
    np.testing.assert_array_equal(sj.sj_tile_axes(c, dR, dS, g).cpu().numpy(), ax)
    for mode in ("two_pass", "one_pass"):
        sj.sj_set_model(c, model if mode == "one_pass" else None)
        got = sj.sj_join(c, dR, dS, g, sj.make_opts(mode, axis="adaptive"))
        st = sj.sj_last_stats(c)
        np.testing.assert_array_equal(sorted_pairs(got), want)
        assert st["path"] == 1 and st["y_sweep_tiles"] == int(ax.sum())
