"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* the hand-built Fig. 1 instance (tests/golden), derived by hand;
* a closed-form count for two square lattices (touching counts, equal x_l);
* brute force (the definition of Sec. 1) == Algorithm 1 == PBSM at any grid;
* invariants: no duplicates, grid independence, swap(R,S) transposes,
  permuting the inputs permutes the ids;
* per-tile counts against counts derived from the rectangles' cells.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1908_11740_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_fig1():
    R, S, pairs, meta = [], [], [], {}
    with open(os.path.join(GOLDEN, "fig1_pbsm_example.txt")) as f:
        for line in f:
            line = line.split("#")[0].split()
            if not line:
                continue
            k, v = line[0], line[1:]
            if k == "R":
                R.append([int(x) for x in v])
            elif k == "S":
                S.append([int(x) for x in v])
            elif k == "pair":
                pairs.append([int(x) for x in v])
            else:
                meta[k] = [float(x) for x in v]
    u = meta["unit"][0]
    R = (np.array(R, np.float64) / u).astype(np.float32)
    S = (np.array(S, np.float64) / u).astype(np.float32)
    return R, S, np.array(pairs, np.int64), meta


def test_fig1_golden_pairs_and_reporting_tile():
    R, S, pairs, meta = load_fig1()
    nx, ny = int(meta["grid"][0]), int(meta["grid"][1])
    out, info = oracle.pbsm(R, S, nx, ny, per_tile=True)
    np.testing.assert_array_equal(out, pairs[:, :2])
    # each pair reported exactly by the tile that holds its reference point
    want_tile = np.zeros(nx * ny, np.int64)
    np.add.at(want_tile, pairs[:, 2], 1)
    np.testing.assert_array_equal(info["pairs"], want_tile)
    np.testing.assert_array_equal(info["cnt_r"], np.array(meta["cnt_r"], np.int64))
    np.testing.assert_array_equal(info["cnt_s"], np.array(meta["cnt_s"], np.int64))
    # (r1, s1): both rectangles sit in tiles 0 and 3, reported once, in tile 0
    r, s, t_a, t_b = (int(x) for x in meta["found_in"])

    def tiles(rect):
        cx0, cx1 = oracle.cell(rect[0], 0, 1, nx), oracle.cell(rect[2], 0, 1, nx)
        cy0, cy1 = oracle.cell(rect[1], 0, 1, ny), oracle.cell(rect[3], 0, 1, ny)
        return {cy * nx + cx for cy in range(cy0, cy1 + 1) for cx in range(cx0, cx1 + 1)}

    assert tiles(R[r]) == {t_a, t_b} and tiles(S[s]) == {t_a, t_b}
    np.testing.assert_array_equal(oracle.brute(R, S), pairs[:, :2])
    np.testing.assert_array_equal(oracle.sweep(R, S), pairs[:, :2])


def _lattice(n, pitch, side, dx, dy):
    i = np.arange(n)
    gx, gy = np.meshgrid(i, i, indexing="ij")
    xl = gx.ravel() * pitch + dx
    yl = gy.ravel() * pitch + dy
    out = np.stack([xl, yl, xl + side, yl + side], 1).astype(np.float32)
    assert np.all(out.astype(np.float64) == np.stack([xl, yl, xl + side, yl + side], 1))
    return out


def _count_1d(n, lo, hi):
    """#{(i,k) in [0,n)^2 : lo <= k - i <= hi} = sum_m max(n - |m|, 0)."""
    return sum(max(n - abs(m), 0) for m in range(lo, hi + 1))


@pytest.mark.parametrize("a_u,b_u,dx_u,dy_u", [(8, 4, 0, 0), (5, 7, 3, -2), (4, 4, 4, 0), (0, 12, 1, 5)])
def test_lattice_closed_form(a_u, b_u, dx_u, dy_u):
    # R: n x n squares of side a on pitch d; S: side b, shifted by (dx, dy).
    # Closed overlap on an axis:  (k - i) d in [-(dx + b), a - dx]  (touching
    # included), so the pair count factorises into two 1-D lattice sums.
    n, u = 40, 1.0 / 256
    d = 4
    R = _lattice(n, d * u, a_u * u, 0.25, 0.25)
    S = _lattice(n, d * u, b_u * u, 0.25 + dx_u * u, 0.25 + dy_u * u)
    lo_x, hi_x = -((dx_u + b_u) // d), (a_u - dx_u) // d
    lo_y, hi_y = -((dy_u + b_u) // d), (a_u - dy_u) // d
    want = _count_1d(n, lo_x, hi_x) * _count_1d(n, lo_y, hi_y)
    assert len(oracle.brute(R, S)) == want
    assert len(oracle.sweep(R, S)) == want
    for k in (1, 3, 16, 50):
        assert len(oracle.pbsm(R, S, k)) == want


def _random_case(seed, n_r, n_s, kind):
    if kind == "uniform":
        return inputs.uniform_pair(n_r, n_s, max_extent=0.05, seed=seed)
    if kind == "gis":
        return inputs.gis_pair(n_r, n_s, seed=seed, median_extent=5e-3)
    if kind == "zipf":
        return inputs.zipf_pair(n_r, n_s, seed=seed, lattice=32, r_max_extent=2e-2,
                                s_max_extent=5e-2, rho=0.5)
    return inputs.degenerate_pair(n_r, n_s, seed=seed)


@pytest.mark.parametrize("kind", ["uniform", "gis", "zipf", "degenerate"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_three_routes_agree(kind, seed):
    R, S = _random_case(seed, 700, 900, kind)
    want = oracle.brute(R, S)
    assert len(want) > 0
    np.testing.assert_array_equal(oracle.sweep(R, S), want)
    for nx, ny in ((1, 1), (2, 2), (7, 7), (64, 64), (5, 1), (1, 9), (13, 4)):
        np.testing.assert_array_equal(oracle.pbsm(R, S, nx, ny), want)
    # a grid over a sub-window: everything outside falls into border tiles
    np.testing.assert_array_equal(oracle.pbsm(R, S, 9, 9, 0.2, 0.3, 0.7, 0.6), want)


def test_invariants():
    R, S = inputs.degenerate_pair(800, 700, seed=5)
    base = oracle.pbsm(R, S, 16)
    # no duplicates
    assert len(np.unique(base, axis=0)) == len(base)
    # swapping R and S transposes the pair set
    sw = oracle.pbsm(S, R, 16)[:, ::-1]
    sw = sw[np.lexsort((sw[:, 1], sw[:, 0]))]
    np.testing.assert_array_equal(sw, base)
    # permuting the inputs only renames the ids
    g = np.random.default_rng(3)
    pr, ps = g.permutation(len(R)), g.permutation(len(S))
    got = oracle.pbsm(R[pr], S[ps], 16)
    mapped = np.stack([pr[got[:, 0]], ps[got[:, 1]]], 1)
    mapped = mapped[np.lexsort((mapped[:, 1], mapped[:, 0]))]
    np.testing.assert_array_equal(mapped, base)


def test_cell_function_partitions_the_line():
    # monotone, clamped, and tile c starts where floor(v * n) first reaches c
    n = 7
    vs = np.sort(np.concatenate([np.linspace(-0.5, 1.5, 3001), np.arange(n + 1) / n]).astype(np.float32))
    cells = [oracle.cell(float(v), 0.0, 1.0, n) for v in vs]
    assert all(a <= b for a, b in zip(cells, cells[1:]))
    assert min(cells) == 0 and max(cells) == n - 1
    assert oracle.cell(0.0, 0.0, 1.0, 4) == 0 and oracle.cell(0.25, 0.0, 1.0, 4) == 1
    assert oracle.cell(-0.0, 0.0, 1.0, 4) == 0 and oracle.cell(1.0, 0.0, 1.0, 4) == 3


def test_tile_counts_match_cells():
    R, _ = inputs.uniform_pair(500, 1, max_extent=0.3, seed=9)
    nx, ny = 6, 5
    want = np.zeros(nx * ny, np.int64)
    for xl, yl, xu, yu in R:
        for cy in range(oracle.cell(yl, 0, 1, ny), oracle.cell(yu, 0, 1, ny) + 1):
            for cx in range(oracle.cell(xl, 0, 1, nx), oracle.cell(xu, 0, 1, nx) + 1):
                want[cy * nx + cx] += 1
    np.testing.assert_array_equal(oracle.tile_counts(R, nx, ny), want)
    _, info = oracle.pbsm(R, R, nx, ny, per_tile=True)
    np.testing.assert_array_equal(info["cnt_r"], want)


def test_uniform_plain_join_expected_count():
    # |R| = |S| = 10^4, extents U[0, 2e-3]: E[P] ~ n^2 (E w_R + E w_S)^2 = 400
    # minus border effects; brute force fixes it exactly.
    R, S = inputs.uniform_pair()
    P = oracle.brute(R, S)
    assert 300 < len(P) < 500
    np.testing.assert_array_equal(oracle.pbsm(R, S, 64), P)
