"""Pins of the oracle's sweep-axis choice (``oracle.tile_axes``, Sec. 3.3).

Eq. 2 estimates the pairs of R_T x S_T whose x-projections intersect by the
pairs sharing one of k = 8 divisions of the tile's x-projection.  Facts that
do not come from the oracle itself:

* every x-intersecting pair of a tile shares a division, so I^x_T is at least
  the brute-force count of x-intersecting pairs of the tile (y alike);
* with every projection a single point at a division centre, sharing a
  division and intersecting coincide: I^x_T equals the brute-force count;
* rectangles ten times wider than high give tiles swept along y, ten times
  higher than wide along x; tiles missing a side are swept along x;
* planted mistakes in a copy of the oracle (an off-by-one division, the
  comparison reversed, a histogram from the wrong axis) fail these pins.
"""
import ctypes
import subprocess

import numpy as np
import pytest

import oracle
from paper_1908_11740_gb300 import inputs


def _tile_members(A, nx, ny):
    c = oracle.cells(A, nx, ny)
    out = {}
    for i, (cx0, cx1, cy0, cy1) in enumerate(c):
        for cy in range(cy0, cy1 + 1):
            for cx in range(cx0, cx1 + 1):
                out.setdefault(cy * nx + cx, []).append(i)
    return out


def _intersecting(R, S, ri, si, axis):
    lo, hi = (0, 2) if axis == 0 else (1, 3)
    a, b = R[ri], S[si]
    return int(((a[:, None, lo] <= b[None, :, hi]) & (b[None, :, lo] <= a[:, None, hi])).sum())


@pytest.mark.parametrize("K", [1, 4, 9])
def test_estimate_bounds_intersecting_projections(K):
    R, S = inputs.uniform_pair(400, 500, max_extent=0.15, seed=61)
    ax, ix, iy = oracle.tile_axes(R, S, K)
    mr, ms = _tile_members(R, K, K), _tile_members(S, K, K)
    checked = 0
    for t in range(K * K):
        ri, si = mr.get(t, []), ms.get(t, [])
        if not ri or not si:
            assert ax[t] == 0
            continue
        assert ix[t] >= _intersecting(R, S, ri, si, 0)
        assert iy[t] >= _intersecting(R, S, ri, si, 1)
        assert ax[t] == int(iy[t] < ix[t])
        checked += 1
    assert checked >= K * K // 2


def test_estimate_exact_for_division_centres():
    """One tile over [0, 1]^2: division i of x is [i/8, (i+1)/8)."""
    g = np.random.default_rng(62)
    for axis in (0, 1):
        def seg(n):
            c = (g.integers(0, 8, n) + 0.5) / 8.0
            lo = g.uniform(0.0, 0.8, n)
            hi = lo + g.uniform(0.0, 0.19, n)
            a = np.empty((n, 4))
            if axis == 0:
                a[:, 0] = a[:, 2] = c
                a[:, 1], a[:, 3] = lo, hi
            else:
                a[:, 1] = a[:, 3] = c
                a[:, 0], a[:, 2] = lo, hi
            return a.astype(np.float32)

        R, S = seg(70), seg(90)
        _, ix, iy = oracle.tile_axes(R, S, 1)
        exact = _intersecting(R, S, np.arange(70), np.arange(90), axis)
        assert (ix if axis == 0 else iy)[0] == exact
        # the other axis: projections of length < 1/8 over 0.8, bounded below
        assert (iy if axis == 0 else ix)[0] >= _intersecting(R, S, np.arange(70), np.arange(90), 1 - axis)


def test_elongated_rectangles_pick_the_short_axis():
    g = np.random.default_rng(63)

    def rects(n, wide):
        c = g.uniform(0.05, 0.95, (n, 2))
        long_, short = 0.04, 0.004
        w, h = (long_, short) if wide else (short, long_)
        return np.stack([c[:, 0] - w / 2, c[:, 1] - h / 2, c[:, 0] + w / 2, c[:, 1] + h / 2], 1).astype(np.float32)

    for wide, want in ((True, 1), (False, 0)):
        R, S = rects(3000, wide), rects(3000, wide)
        ax, ix, iy = oracle.tile_axes(R, S, 4)
        both = (ix > 0) | (iy > 0)
        assert both.sum() == 16
        assert (ax[both] == want).mean() >= 0.95


MUTANTS = [
    ("division off by one", "if (8.0f * tl < a + 1.0f && 8.0f * tu >= a) h[i]++;",
     "if (8.0f * tl <= a && 8.0f * tu >= a) h[i]++;"),
    ("comparison reversed", "axis[t] = (uint8_t)(cr[t] > 0 && cs[t] > 0 && sy < sx);",
     "axis[t] = (uint8_t)(cr[t] > 0 && cs[t] > 0 && sy > sx);"),
    ("y histogram from x", "tile_histogram(er + orr[t], cr[t], row, g.gy0, g.ginvy, 1, hry);",
     "tile_histogram(er + orr[t], cr[t], row, g.gy0, g.ginvy, 0, hry);"),
    ("product dropped", "sx += hrx[i] * hsx[i];", "sx += hrx[i];"),
]


@pytest.mark.parametrize("name,orig,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutants_caught(tmp_path, name, orig, new):
    src = open(oracle._SRC).read()
    assert src.count(orig) == 1, orig
    path = tmp_path / "m.c"
    path.write_text(src.replace(orig, new))
    so = tmp_path / "libm.so"
    subprocess.check_call(["gcc", *oracle.CFLAGS, "-o", str(so), str(path), "-lm"])
    lib = oracle._configure(ctypes.CDLL(str(so)))
    real = oracle._load()
    caught = False
    try:
        oracle._lib = lib          # route the oracle through the mutant
        for pin in (test_estimate_exact_for_division_centres, test_elongated_rectangles_pick_the_short_axis,
                    lambda: test_estimate_bounds_intersecting_projections(4)):
            try:
                pin()
            except AssertionError:
                caught = True
                break
    finally:
        oracle._lib = real
    assert caught, f"mutant '{name}' not caught"
