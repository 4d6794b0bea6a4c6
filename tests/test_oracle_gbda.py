"""Pins of the oracle's grouping-based duplicate avoidance (``oracle.pbsm_gbda``).

GBDA replaces the duplicate test of Eq. 1 by evaluating only 9 of the 16
group-group joins of each tile (classes A-D by where a rectangle's
projections begin).  Facts that do not come from the oracle itself:

* the hand-built Fig. 1 instance (tests/golden) and the square-lattice closed
  form (touching corners and edges, equal x_l) give the same pairs;
* on random, GIS-like, skewed and degenerate inputs at grids from 1 x 1 to
  64 x 64 (and sub-window grids), the pairs equal brute force (the
  definition of Sec. 1), with no pair twice;
* planted mistakes -- evaluating a skipped join (B with B), dropping an
  evaluated one (B with C, A with D), a strict class boundary, class C
  taken for D -- fail these pins.
"""
import ctypes
import subprocess

import numpy as np
import pytest

import oracle
from test_oracle_pins import _count_1d, _lattice, _random_case, load_fig1


def test_fig1_and_lattice():
    R, S, pairs, meta = load_fig1()
    nx, ny = int(meta["grid"][0]), int(meta["grid"][1])
    np.testing.assert_array_equal(oracle.pbsm_gbda(R, S, nx, ny), pairs[:, :2])
    n, u, d = 40, 1.0 / 256, 4
    for a_u, b_u, dx_u, dy_u in [(8, 4, 0, 0), (5, 7, 3, -2), (4, 4, 4, 0)]:
        R = _lattice(n, d * u, a_u * u, 0.25, 0.25)
        S = _lattice(n, d * u, b_u * u, 0.25 + dx_u * u, 0.25 + dy_u * u)
        want = _count_1d(n, -((dx_u + b_u) // d), (a_u - dx_u) // d) * \
            _count_1d(n, -((dy_u + b_u) // d), (a_u - dy_u) // d)
        for k in (1, 3, 16, 50):
            got = oracle.pbsm_gbda(R, S, k)
            assert len(got) == want
            assert len(np.unique(got.astype(np.int64) @ np.array([1 << 32, 1]))) == want


@pytest.mark.parametrize("kind", ["uniform", "gis", "zipf", "degenerate"])
@pytest.mark.parametrize("K", [1, 2, 7, 64])
def test_equals_brute_force(kind, K):
    R, S = _random_case(100 + K, 700, 900, kind)
    want = oracle.brute(R, S)
    np.testing.assert_array_equal(oracle.pbsm_gbda(R, S, K), want)
    np.testing.assert_array_equal(oracle.pbsm_gbda(R, S, K, max(1, K // 2), 0.2, 0.1, 0.7, 0.8), want)


MUTANTS = [
    ("evaluates B with B", "    {CL_B, CL_C}, {CL_C, CL_B},\n};", "    {CL_B, CL_C}, {CL_C, CL_B}, {CL_B, CL_B},\n};"),
    ("drops B with C", "    {CL_B, CL_C}, {CL_C, CL_B},\n};", "    {CL_C, CL_B}, {CL_C, CL_B},\n};"),
    ("drops A with D", "{CL_A, CL_C}, {CL_A, CL_D},", "{CL_A, CL_C}, {CL_A, CL_C},"),
    ("strict class boundary", "int xin = cell_of(e->xl, g->gx0, g->ginvx, g->nx) >= col;",
     "int xin = cell_of(e->xl, g->gx0, g->ginvx, g->nx) > col;"),
    ("C taken for D", "    if (yin) return CL_C;", "    if (yin) return CL_D;"),
]


@pytest.mark.parametrize("name,orig,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutants_caught(tmp_path, name, orig, new):
    src = open(oracle._SRC).read()
    assert src.count(orig) == 1, orig
    path = tmp_path / "m.c"
    path.write_text(src.replace(orig, new))
    so = tmp_path / "libm.so"
    subprocess.check_call(["gcc", *oracle.CFLAGS, "-o", str(so), str(path), "-lm"])
    real = oracle._load()
    caught = False
    try:
        oracle._lib = oracle._configure(ctypes.CDLL(str(so)))
        try:
            test_fig1_and_lattice()
            for kind in ("uniform", "degenerate"):
                for K in (2, 7):
                    R, S = _random_case(100 + K, 700, 900, kind)
                    got = oracle.pbsm_gbda(R, S, K)
                    oracle._lib = real
                    want = oracle.brute(R, S)
                    oracle._lib = oracle._configure(ctypes.CDLL(str(so)))
                    np.testing.assert_array_equal(got, want)
        except AssertionError:
            caught = True
    finally:
        oracle._lib = real
    assert caught, f"mutant '{name}' not caught"
