"""Pins of the oracle's eps-distance join on points (Sec. 1: every point
becomes a square of side eps, the squares are joined, and each intersecting
pair is refined by its distance).

The oracle has two routes, the definition (``dist_brute``) and the paper's
route (``dist_pbsm``: squares, PBSM, distance test).  They are pinned here by
facts that do not come from the oracle itself:

* integer lattices, where every distance is exact in binary64, so the result
  is a closed form: the pair set is built from the integer offsets (a, b) with
  a^2 + b^2 <= r^2, whose numbers for the infinite lattice are the published
  Gauss circle counts 1, 5, 13, 29, 49, 81 for r = 0..5;
* eps = 0, which leaves exactly the coincident points;
* scipy's KD-tree (``cKDTree.query_ball_point``), a library routine for the
  same question, on random points;
* the squares contain the exact square of side eps (checked in exact rational
  arithmetic);
* mutants: plausible mistakes planted in a copy of the oracle are caught.
"""
import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1908_11740_gb300 import inputs

SRC = os.path.join(os.path.dirname(oracle.__file__), "sj_oracle.c")


def _offsets(r):
    """Integer offsets (a, b) with a^2 + b^2 <= r^2."""
    return [(a, b) for a in range(-r, r + 1) for b in range(-r, r + 1) if a * a + b * b <= r * r]


def _lattice_points(n, pitch, x0, y0):
    i = np.arange(n)
    gx, gy = np.meshgrid(i, i, indexing="ij")   # index = ix * n + iy
    pts = np.stack([x0 + gx.ravel() * pitch, y0 + gy.ravel() * pitch], 1)
    out = pts.astype(np.float32)
    assert np.all(out.astype(np.float64) == pts)   # exact in float32
    return out


def _lattice_pairs(n, m, s, t, offs):
    """Closed form: P = n x n lattice, Q = m x m lattice shifted by (s, t)
    pitches; Q point (k, l) sits at P-lattice coordinates (k + s, l + t).
    Pairs (P (i, j), Q (k, l)) with (k + s - i, l + t - j) in offs."""
    out = []
    for i in range(n):
        for j in range(n):
            for a, b in offs:
                k, l = i + a - s, j + b - t
                if 0 <= k < m and 0 <= l < m:
                    out.append((i * n + j, k * m + l))
    out = np.array(sorted(out), np.int32).reshape(-1, 2)
    return out


def test_gauss_circle_counts():
    # numbers of lattice points in the closed disc of radius r (r = 0..5)
    assert [len(_offsets(r)) for r in range(6)] == [1, 5, 13, 29, 49, 81]


@pytest.mark.parametrize("r", [0, 1, 2, 3, 5])
@pytest.mark.parametrize("n,m,s,t", [(20, 20, 0, 0), (18, 13, 3, -2)])
def test_lattice_closed_form(r, n, m, s, t):
    h = 1.0 / 64
    P = _lattice_points(n, h, 0.25, 0.25)
    Q = _lattice_points(m, h, 0.25 + s * h, 0.25 + t * h)
    eps = np.float32(r * h)
    want = _lattice_pairs(n, m, s, t, _offsets(r))
    np.testing.assert_array_equal(oracle.dist_brute(P, Q, eps), want)
    for k in (1, 7, 32):
        np.testing.assert_array_equal(oracle.dist_pbsm(P, Q, eps, k), want)


@pytest.mark.parametrize("r", [1, 2, 5])
def test_lattice_just_below_radius(r):
    # eps one float32 step below r * h: the ring at distance exactly r * h
    # drops out (the test is "<=", so at eps = r * h it is in)
    n, h = 16, 1.0 / 64
    P = _lattice_points(n, h, 0.25, 0.25)
    eps = np.nextafter(np.float32(r * h), np.float32(0))
    inner = [(a, b) for a, b in _offsets(r) if a * a + b * b < r * r]
    want = _lattice_pairs(n, n, 0, 0, inner)
    np.testing.assert_array_equal(oracle.dist_brute(P, P, eps), want)
    np.testing.assert_array_equal(oracle.dist_pbsm(P, P, eps, 9), want)


def test_eps_zero_keeps_coincident_points():
    rng = np.random.default_rng(5)
    base = rng.random((50, 2)).astype(np.float32)
    P = base[rng.integers(0, 50, 300)]
    Q = base[rng.integers(0, 50, 200)]
    want = np.array(sorted((i, j) for i in range(len(P)) for j in range(len(Q))
                           if P[i, 0] == Q[j, 0] and P[i, 1] == Q[j, 1]), np.int32).reshape(-1, 2)
    assert len(want) > 0
    np.testing.assert_array_equal(oracle.dist_brute(P, Q, 0.0), want)
    np.testing.assert_array_equal(oracle.dist_pbsm(P, Q, 0.0, 16), want)


def _kdtree_pairs(P, Q, eps):
    spatial = pytest.importorskip("scipy.spatial")
    tree = spatial.cKDTree(Q.astype(np.float64))
    hits = tree.query_ball_point(P.astype(np.float64), r=float(eps), p=2.0)
    out = [(i, j) for i, js in enumerate(hits) for j in js]
    return np.array(sorted(out), np.int32).reshape(-1, 2)


@pytest.mark.parametrize("seed,eps", [(1, 0.01), (2, 0.03), (3, 0.005)])
def test_kdtree_agrees(seed, eps):
    rng = np.random.default_rng(seed)
    P = rng.random((1500, 2)).astype(np.float32)
    Q = (rng.random((2500, 2)) * 1.1 - 0.05).astype(np.float32)
    want = _kdtree_pairs(P, Q, eps)
    assert len(want) > 50
    np.testing.assert_array_equal(oracle.dist_brute(P, Q, eps), want)
    np.testing.assert_array_equal(oracle.dist_pbsm(P, Q, eps, 20), want)


def test_routes_agree_clustered_and_swap():
    R, S = inputs.gis_pair(4000, 6000, seed=11)
    P = ((R[:, :2] + R[:, 2:]) * 0.5).astype(np.float32)
    Q = ((S[:, :2] + S[:, 2:]) * 0.5).astype(np.float32)
    eps = np.float32(4e-3)
    a = oracle.dist_brute(P, Q, eps)
    assert len(a) > 1000
    for k in (1, 5, 40, 250):
        np.testing.assert_array_equal(oracle.dist_pbsm(P, Q, eps, k), a)
    b = oracle.dist_brute(Q, P, eps)
    np.testing.assert_array_equal(b[np.lexsort((b[:, 0], b[:, 1]))][:, ::-1], a)


def test_squares_hold_the_exact_square():
    rng = np.random.default_rng(7)
    P = np.concatenate([rng.random((400, 2)), rng.random((100, 2)) * 1e-30,
                        -rng.random((100, 2)) * 3.0]).astype(np.float32)
    for eps in (0.0, 1e-38, 3e-7, 0.125, 0.3, 7.0):
        sq = oracle.dist_squares(P, eps)
        h = Fraction(float(np.float32(eps))) / 2 * (1 + Fraction(1, 2 ** 21))
        for (x, y), (xl, yl, xu, yu) in zip(P.tolist(), sq.tolist()):
            fx, fy = Fraction(x), Fraction(y)
            assert Fraction(xl) <= fx - h and Fraction(xu) >= fx + h
            assert Fraction(yl) <= fy - h and Fraction(yu) >= fy + h


def test_candidates_superset():
    rng = np.random.default_rng(9)
    P = rng.random((800, 2)).astype(np.float32)
    Q = rng.random((900, 2)).astype(np.float32)
    eps = 0.02
    res, ncand = oracle.dist_pbsm(P, Q, eps, 12, return_candidates=True)
    sq_pairs = oracle.brute(oracle.dist_squares(P, eps), oracle.dist_squares(Q, eps))
    assert ncand == len(sq_pairs) >= len(res)
    assert set(map(tuple, res.tolist())) <= set(map(tuple, sq_pairs.tolist()))


# ---- mutants -------------------------------------------------------------
MUTANTS = [
    ("distance test strict", "return d2 <= e2;", "return d2 < e2;"),
    ("distance drops dy", "double d2 = dx * dx + dy * dy;", "double d2 = dx * dx;"),
    ("distance sign", "double dy = (double)p.y - (double)q.y;", "double dy = (double)p.y + (double)q.y;"),
    ("square half of eps/2", "float h = (float)((double)eps * 0.5 *", "float h = (float)((double)eps * 0.25 *"),
    ("square corner sign", "out[i].xl = nextafterf(P[i].x - h, -INFINITY);",
     "out[i].xl = nextafterf(P[i].x + h, -INFINITY);"),
    ("refine transposed", "if (within_eps(P[c.r], Q[c.s], e2)) res_push(res, c.r, c.s);",
     "if (within_eps(P[c.r], Q[c.s], e2)) res_push(res, c.s, c.r);"),
    ("brute transposed", "if (within_eps(P[i], Q[j], e2)) res_push(res, (int32_t)i, (int32_t)j);",
     "if (within_eps(P[i], Q[j], e2)) res_push(res, (int32_t)j, (int32_t)i);"),
]


def _mutant(tmp_path, orig, new):
    src = open(SRC).read()
    assert src.count(orig) == 1, orig
    path = tmp_path / "m.c"
    path.write_text(src.replace(orig, new))
    so = tmp_path / "libm.so"
    subprocess.check_call(["gcc", *oracle.CFLAGS, "-o", str(so), str(path), "-lm"])
    lib = ctypes.CDLL(str(so))
    V, I64, I, F = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_float
    lib.orc_res_count.restype = I64
    lib.orc_res_count.argtypes = [V]
    lib.orc_res_copy.argtypes = [V, V]
    lib.orc_res_free.argtypes = [V]
    lib.orc_dist_brute.restype = V
    lib.orc_dist_brute.argtypes = [V, I64, V, I64, F]
    lib.orc_dist_pbsm.restype = V
    lib.orc_dist_pbsm.argtypes = [V, I64, V, I64, F, I, I, F, F, F, F, V]
    return lib


def _call(lib, route, P, Q, eps):
    P = np.ascontiguousarray(P, np.float32)
    Q = np.ascontiguousarray(Q, np.float32)
    if route == "brute":
        res = lib.orc_dist_brute(P.ctypes.data, len(P), Q.ctypes.data, len(Q), eps)
    else:
        res = lib.orc_dist_pbsm(P.ctypes.data, len(P), Q.ctypes.data, len(Q), eps, 7, 7, 0.0, 0.0, 1.0, 1.0, None)
    n = lib.orc_res_count(res)
    out = np.empty((n, 2), np.int32)
    if n:
        lib.orc_res_copy(res, out.ctypes.data)
    lib.orc_res_free(res)
    return out[np.lexsort((out[:, 1], out[:, 0]))]


def _pins_hold(lib):
    h = 1.0 / 64
    P = _lattice_points(12, h, 0.25, 0.25)
    Q = _lattice_points(9, h, 0.25 + 3 * h, 0.25 - 2 * h)
    want = _lattice_pairs(12, 9, 3, -2, _offsets(2))
    rng = np.random.default_rng(3)
    Pr = rng.random((500, 2)).astype(np.float32)
    Qr = rng.random((700, 2)).astype(np.float32)
    want_r = _kdtree_pairs(Pr, Qr, 0.03)
    for route in ("brute", "pbsm"):
        if not np.array_equal(_call(lib, route, P, Q, np.float32(2 * h)), want):
            return False
        if not np.array_equal(_call(lib, route, Pr, Qr, 0.03), want_r):
            return False
    return True


@pytest.mark.parametrize("name,orig,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, name, orig, new):
    assert not _pins_hold(_mutant(tmp_path, orig, new)), f"mutant '{name}' passes every pin"


def test_unmutated_oracle_passes_pins(tmp_path):
    assert _pins_hold(_mutant(tmp_path, "return d2 <= e2;", "return d2 <= e2;"))
