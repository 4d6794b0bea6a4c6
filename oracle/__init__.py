"""TEST INFRASTRUCTURE: the CPU oracle of the spatial-join filter step.

Plain, slow, obviously correct implementations of what the GPU path computes,
written from the paper ("Parallel In-Memory Evaluation of Spatial Joins"):

* ``brute``  -- the definition of Sec. 1, every pair tested (C);
* ``sweep``  -- Algorithm 1, forward-scan plane sweep over the whole space (C);
* ``pbsm``   -- uniform-grid PBSM with replication, per-tile sort by x_l,
  Algorithm 1 per tile and the reference-point test of Eq. 1 (C);
* ``pbsm_gbda`` -- PBSM with grouping-based duplicate avoidance: four
  classes per tile by where the projections begin, 9 of the 16 group-group
  joins, no duplicate test (C);
* ``pbsm_digest`` -- the same PBSM with the pairs folded into an
  order-independent digest (count, sum and xor of the SplitMix64 output
  function of each pair) instead of stored: the check of 1e9-pair joins;
* ``tile_counts`` / ``cell`` -- the partitioning counts of Sec. 3.4 step 2;
* ``tile_axes`` -- the sweep axis of every tile from the Eq. 2 histograms of
  Sec. 3.3 (k = 8 divisions per tile axis, all rectangles counted);
* ``features`` / ``mlp``    -- in :mod:`oracle.learned` (numpy, float64);
* ``dist_brute`` / ``dist_pbsm`` -- the eps-distance join on points of Sec. 1
  (the definition; squares of side eps joined by PBSM, then refined) (C).

``pbsm_parallel`` (``pbsm_parallel.c``) is not part of the oracle: it is the
paper's multi-core evaluation (Sec. 3.4) with OpenMP, a CPU timing baseline
whose pairs the tests check against the oracle.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sj_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libsj_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no OpenMP, no vector intrinsics), and
    the multi-core baseline if the compiler supports OpenMP."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    try:
        build_parallel(force)
    except (OSError, subprocess.CalledProcessError):
        pass   # no OpenMP: the baseline is reported as unavailable
    return _LIB


_PAR_SRC = os.path.join(_HERE, "pbsm_parallel.c")
_PAR_LIB = os.path.join(_BUILD, "libpbsm_parallel.so")
_par = None


def build_parallel(force: bool = False) -> str:
    """Compile the multi-core PBSM baseline (gcc -fopenmp)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_PAR_LIB) or os.path.getmtime(_PAR_LIB) < os.path.getmtime(_PAR_SRC):
        tmp = _PAR_LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, "-fopenmp", "-o", tmp, _PAR_SRC, "-lm"],
                              stderr=subprocess.DEVNULL)
        os.replace(tmp, _PAR_LIB)
    return _PAR_LIB


def _load_parallel():
    global _par
    with _lock:
        if _par is None:
            lib = ctypes.CDLL(build_parallel())
            P, I64, I, F = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_float
            lib.pp_pbsm.restype = I64
            lib.pp_pbsm.argtypes = [P, I64, P, I64, I, I, F, F, F, F, I, P]
            lib.pp_free.restype = None
            lib.pp_free.argtypes = [P]
            lib.pp_max_threads.restype = I
            lib.pp_max_threads.argtypes = []
            _par = lib
        return _par


def parallel_threads() -> int:
    """Threads the multi-core baseline uses by default."""
    return _load_parallel().pp_max_threads()


def pbsm_parallel(R, S, nx: int, ny: int | None = None, x0: float = 0.0, y0: float = 0.0,
                  x1: float = 1.0, y1: float = 1.0, threads: int = 0, pairs: bool = True):
    """The paper's multi-core PBSM (Sec. 3.4) on ``threads`` threads (0 = all):
    the sorted int32[P, 2] pairs, or only their number with ``pairs=False``."""
    lib = _load_parallel()
    ny = nx if ny is None else ny
    R, S = _rects(R), _rects(S)
    out = ctypes.c_void_p()
    n = lib.pp_pbsm(R.ctypes.data, len(R), S.ctypes.data, len(S), nx, ny, x0, y0, x1, y1, threads,
                    ctypes.byref(out) if pairs else None)
    if n < 0:
        raise MemoryError("multi-core baseline: allocation failed or bad arguments")
    if not pairs:
        return int(n)
    try:
        a = np.ctypeslib.as_array(ctypes.cast(out, ctypes.POINTER(ctypes.c_int32)), shape=(n * 2,)).copy() \
            if n else np.zeros(0, np.int32)
    finally:
        if out.value:
            lib.pp_free(out)
    a = a.reshape(-1, 2)
    return a[np.lexsort((a[:, 1], a[:, 0]))] if len(a) else a


def _configure(lib):
    """Set the argument and result types of every oracle function on a
    loaded copy of the library (also used for planted-mistake copies)."""
    P, I64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    F = ctypes.c_float
    lib.orc_brute.restype = P
    lib.orc_brute.argtypes = [P, I64, P, I64]
    lib.orc_sweep.restype = P
    lib.orc_sweep.argtypes = [P, I64, P, I64, P]
    lib.orc_pbsm_ex.restype = P
    lib.orc_pbsm_ex.argtypes = [P, I64, P, I64, I, I, F, F, F, F, P, P, P, P]
    lib.orc_pbsm_gbda.restype = P
    lib.orc_pbsm_gbda.argtypes = [P, I64, P, I64, I, I, F, F, F, F]
    lib.orc_pbsm_digest.restype = I
    lib.orc_pbsm_digest.argtypes = [P, I64, P, I64, I, I, F, F, F, F, P]
    lib.orc_res_count.restype = I64
    lib.orc_res_count.argtypes = [P]
    lib.orc_res_failed.restype = I
    lib.orc_res_failed.argtypes = [P]
    lib.orc_res_copy.restype = None
    lib.orc_res_copy.argtypes = [P, P]
    lib.orc_res_free.restype = None
    lib.orc_res_free.argtypes = [P]
    lib.orc_cell.restype = I
    lib.orc_cell.argtypes = [F, F, F, I]
    lib.orc_cells.restype = None
    lib.orc_cells.argtypes = [P, I64, I, I, F, F, F, F, P]
    lib.orc_tile_axes.restype = I
    lib.orc_tile_axes.argtypes = [P, I64, P, I64, I, I, F, F, F, F, P, P, P]
    lib.orc_tile_counts.restype = None
    lib.orc_tile_counts.argtypes = [P, I64, I, I, F, F, F, F, P]
    lib.orc_dist_brute.restype = P
    lib.orc_dist_brute.argtypes = [P, I64, P, I64, F]
    lib.orc_dist_squares.restype = None
    lib.orc_dist_squares.argtypes = [P, I64, F, P]
    lib.orc_dist_pbsm.restype = P
    lib.orc_dist_pbsm.argtypes = [P, I64, P, I64, F, I, I, F, F, F, F, P]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        _lib = _configure(ctypes.CDLL(build()))
        return _lib


def _rects(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 4:
        raise ValueError("rectangles must be float32[n, 4] (xl, yl, xu, yu)")
    return a


def _take(lib, res) -> np.ndarray:
    if not res:
        raise MemoryError("oracle: allocation failed or bad arguments")
    try:
        if lib.orc_res_failed(res):
            raise MemoryError("oracle: result buffer allocation failed")
        n = lib.orc_res_count(res)
        out = np.empty((n, 2), np.int32)
        if n:
            lib.orc_res_copy(res, out.ctypes.data)
        return out
    finally:
        lib.orc_res_free(res)


def brute(R, S) -> np.ndarray:
    """All intersecting pairs by testing every (r, s); int32[P, 2] sorted."""
    lib = _load()
    R, S = _rects(R), _rects(S)
    return _take(lib, lib.orc_brute(R.ctypes.data, len(R), S.ctypes.data, len(S)))


def sweep(R, S, return_candidates: bool = False):
    """Algorithm 1 over the whole space; int32[P, 2] sorted by (r, s)."""
    lib = _load()
    R, S = _rects(R), _rects(S)
    nc = ctypes.c_int64(0)
    out = _take(lib, lib.orc_sweep(R.ctypes.data, len(R), S.ctypes.data, len(S),
                                   ctypes.addressof(nc)))
    return (out, nc.value) if return_candidates else out


def pbsm(R, S, nx: int, ny: int | None = None, x0: float = 0.0, y0: float = 0.0,
         x1: float = 1.0, y1: float = 1.0, per_tile: bool = False):
    """Single-threaded PBSM on an nx x ny grid over [x0,x1] x [y0,y1].

    Returns the sorted int32[P, 2] pairs; with ``per_tile`` also a dict of
    int64[ny*nx] arrays ``cnt_r``, ``cnt_s`` (replicated entries per tile),
    ``pairs`` (pairs reported by the tile) and the candidate count ``cand``
    (pairs that x-intersect, examined by Algorithm 1's inner loops)."""
    lib = _load()
    ny = nx if ny is None else ny
    R, S = _rects(R), _rects(S)
    T = nx * ny
    cr = np.zeros(T, np.int64) if per_tile else None
    cs = np.zeros(T, np.int64) if per_tile else None
    tp = np.zeros(T, np.int64) if per_tile else None
    nc = ctypes.c_int64(0)
    ptr = lambda a: a.ctypes.data if a is not None else None  # noqa: E731
    out = _take(lib, lib.orc_pbsm_ex(R.ctypes.data, len(R), S.ctypes.data, len(S),
                                     nx, ny, x0, y0, x1, y1, ptr(cr), ptr(cs), ptr(tp),
                                     ctypes.addressof(nc)))
    if per_tile:
        return out, {"cnt_r": cr, "cnt_s": cs, "pairs": tp, "cand": nc.value}
    return out


def pbsm_gbda(R, S, nx: int, ny: int | None = None, x0: float = 0.0, y0: float = 0.0,
              x1: float = 1.0, y1: float = 1.0) -> np.ndarray:
    """PBSM with grouping-based duplicate avoidance (classes A-D per tile,
    the 9 group-group joins that can report a pair first, no duplicate
    test); int32[P, 2] sorted."""
    lib = _load()
    ny = nx if ny is None else ny
    R, S = _rects(R), _rects(S)
    return _take(lib, lib.orc_pbsm_gbda(R.ctypes.data, len(R), S.ctypes.data, len(S), nx, ny, x0, y0, x1, y1))


def pbsm_digest(R, S, nx: int, ny: int | None = None, x0: float = 0.0, y0: float = 0.0,
                x1: float = 1.0, y1: float = 1.0) -> tuple[int, int, int]:
    """PBSM as :func:`pbsm`, returning only the digest of its pair set:
    (pairs, sum mod 2^64, xor) of mix(r << 32 | s) over the pairs, with mix
    the output function of SplitMix64 (Steele, Lea and Flood, 2014).  The
    digest does not depend on the order of the pairs; no pair is stored."""
    lib = _load()
    ny = nx if ny is None else ny
    R, S = _rects(R), _rects(S)
    out = np.zeros(3, np.uint64)
    if lib.orc_pbsm_digest(R.ctypes.data, len(R), S.ctypes.data, len(S), nx, ny, x0, y0, x1, y1,
                           out.ctypes.data) != 0:
        raise MemoryError("oracle: allocation failed or bad arguments")
    return int(out[0]), int(out[1]), int(out[2])


def cell(v: float, g0: float, g1: float, n: int) -> int:
    """Tile index of coordinate v on an n-tile axis over [g0, g1]."""
    return _load().orc_cell(v, g0, g1, n)


def tile_axes(R, S, nx: int, ny: int | None = None, x0=0.0, y0=0.0, x1=1.0, y1=1.0):
    """Sweep axis of every tile (uint8[ny*nx], row-major, 1 = y) from Eq. 2
    with k = 8 divisions per tile axis, and the estimates I^x, I^y
    (int64[ny*nx] each): y where I^y < I^x and the tile holds both sides."""
    lib = _load()
    ny = nx if ny is None else ny
    R, S = _rects(R), _rects(S)
    ax = np.zeros(nx * ny, np.uint8)
    ix = np.zeros(nx * ny, np.int64)
    iy = np.zeros(nx * ny, np.int64)
    if lib.orc_tile_axes(R.ctypes.data, len(R), S.ctypes.data, len(S), nx, ny, x0, y0, x1, y1,
                         ax.ctypes.data, ix.ctypes.data, iy.ctypes.data) != 0:
        raise MemoryError("oracle: allocation failed or bad arguments")
    return ax, ix, iy


def tile_counts(A, nx: int, ny: int | None = None, x0=0.0, y0=0.0, x1=1.0, y1=1.0):
    """Replicated entries per tile, int64[ny*nx] (row-major, row = y cell)."""
    lib = _load()
    ny = nx if ny is None else ny
    A = _rects(A)
    out = np.zeros(nx * ny, np.int64)
    lib.orc_tile_counts(A.ctypes.data, len(A), nx, ny, x0, y0, x1, y1, out.ctypes.data)
    return out


def cells(A, nx: int, ny: int | None = None, x0=0.0, y0=0.0, x1=1.0, y1=1.0) -> np.ndarray:
    """int32[n, 4]: (cx0, cx1, cy0, cy1) of every rectangle."""
    lib = _load()
    ny = nx if ny is None else ny
    A = _rects(A)
    out = np.zeros((len(A), 4), np.int32)
    lib.orc_cells(A.ctypes.data, len(A), nx, ny, x0, y0, x1, y1, out.ctypes.data)
    return out


def _points(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 2:
        raise ValueError("points must be float32[n, 2] (x, y)")
    return a


def dist_brute(P, Q, eps: float) -> np.ndarray:
    """All (i, j) with |P[i] - Q[j]| <= eps, every pair tested (binary64
    distance in a fixed order); int32[n, 2] sorted."""
    lib = _load()
    P, Q = _points(P), _points(Q)
    return _take(lib, lib.orc_dist_brute(P.ctypes.data, len(P), Q.ctypes.data, len(Q), eps))


def dist_squares(P, eps: float) -> np.ndarray:
    """float32[n, 4]: the square of side eps around every point, widened and
    rounded outward so that it holds the exact square."""
    lib = _load()
    P = _points(P)
    out = np.zeros((len(P), 4), np.float32)
    lib.orc_dist_squares(P.ctypes.data, len(P), eps, out.ctypes.data)
    return out


def dist_pbsm(P, Q, eps: float, nx: int, ny: int | None = None, x0: float = 0.0, y0: float = 0.0,
              x1: float = 1.0, y1: float = 1.0, return_candidates: bool = False):
    """The paper's route for the eps-distance join: squares of side eps, PBSM
    on an nx x ny grid, distance test of every intersecting pair."""
    lib = _load()
    ny = nx if ny is None else ny
    P, Q = _points(P), _points(Q)
    nc = ctypes.c_int64(0)
    out = _take(lib, lib.orc_dist_pbsm(P.ctypes.data, len(P), Q.ctypes.data, len(Q), eps,
                                       nx, ny, x0, y0, x1, y1, ctypes.addressof(nc)))
    return (out, nc.value) if return_candidates else out
