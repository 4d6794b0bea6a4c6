"""Thin Python binding of the C ABI in ``include/sj.h`` (argument marshalling
only; every step of the join runs in the CUDA library ``libsj.so``).

The functions carry the C names (``sj_create``, ``sj_join``, ...).  Device
memory comes from PyTorch: rectangles are CUDA ``float32[n, 4]`` tensors and
every buffer the library allocates (workspace and results) is a PyTorch
tensor handed out through the context's allocator hook, so results come back
as ``int32[P, 2]`` CUDA tensors without a copy.

The library must have been built (``paper_1908_11740_gb300.build.build()``);
there is no fallback of any kind: loading fails loudly when it is missing.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import build as _build

SJ_OK, SJ_EINVAL, SJ_ENOMEM, SJ_EOVERFLOW, SJ_ETIMEOUT, SJ_ECUDA, SJ_EINTERNAL = range(7)
SJ_TWO_PASS, SJ_ONE_PASS, SJ_ONE_PASS_HEUR, SJ_AUTO = range(4)
SJ_SWEEP_ADAPTIVE = 1
SJ_DEDUP_GBDA = 2
MODES = {"two_pass": SJ_TWO_PASS, "one_pass": SJ_ONE_PASS, "one_pass_heur": SJ_ONE_PASS_HEUR,
         "auto": SJ_AUTO}


class SJError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[{status}] {msg}")
        self.status = status


class sj_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("x0", ctypes.c_float),
                ("y0", ctypes.c_float), ("x1", ctypes.c_float), ("y1", ctypes.c_float)]


class sj_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("sort_output", ctypes.c_int32),
                ("margin", ctypes.c_float), ("flags", ctypes.c_int32)]


class sj_part_view(ctypes.Structure):
    _fields_ = [("n_tiles", ctypes.c_int64), ("e_r", ctypes.c_int64), ("e_s", ctypes.c_int64),
                ("off", ctypes.c_void_p), ("ent_r", ctypes.c_void_p), ("id_r", ctypes.c_void_p),
                ("ent_s", ctypes.c_void_p), ("id_s", ctypes.c_void_p)]


class sj_timing(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("n", ctypes.c_int64 * 13), ("ms", ctypes.c_double * 13)]


class sj_stats(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("block_side", ctypes.c_int32), ("blocks", ctypes.c_int64),
                ("work_items", ctypes.c_int64), ("l1_entries_r", ctypes.c_int64),
                ("l1_entries_s", ctypes.c_int64), ("entries_r", ctypes.c_int64),
                ("entries_s", ctypes.c_int64), ("npairs", ctypes.c_int64), ("one_pass", ctypes.c_int32),
                ("dedup", ctypes.c_int32), ("capacity", ctypes.c_int64), ("refit_items", ctypes.c_int64),
                ("y_sweep_tiles", ctypes.c_int64)]


SJ_MLP_FEATURES = 32
SJ_MLP_PARAMS = 6337


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None

# (name, restype, argtypes) of every exported symbol declared in include/sj.h
P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
SIGNATURES = [
    ("sj_create", I32, [ctypes.POINTER(P), I32, P]),
    ("sj_destroy", I32, [P]),
    ("sj_set_allocator", I32, [P, ALLOC_FN, FREE_FN, P]),
    ("sj_free", None, [P, P]),
    ("sj_last_error", ctypes.c_char_p, [P]),
    ("sj_strerror", ctypes.c_char_p, [I32]),
    ("sj_partition", I32, [P, P, I64, P, I64, ctypes.POINTER(sj_grid), ctypes.POINTER(P)]),
    ("sj_part_view_get", I32, [P, ctypes.POINTER(sj_part_view)]),
    ("sj_part_join", I32, [P, P, ctypes.POINTER(sj_opts), ctypes.POINTER(P), ctypes.POINTER(I64)]),
    ("sj_part_free", None, [P]),
    ("sj_count", I32, [P, P, I64, P, I64, ctypes.POINTER(sj_grid), ctypes.POINTER(I64)]),
    ("sj_join", I32, [P, P, I64, P, I64, ctypes.POINTER(sj_grid), ctypes.POINTER(sj_opts),
                      ctypes.POINTER(P), ctypes.POINTER(I64)]),
    ("sj_join_into", I32, [P, P, I64, P, I64, ctypes.POINTER(sj_grid), ctypes.POINTER(sj_opts),
                           P, I64, ctypes.POINTER(I64)]),
    ("sj_tile_stats", I32, [P, P, I64, P, I64, ctypes.POINTER(sj_grid), P, P, P]),
    ("sj_join_rows", I32, [P, P, I64, P, I64, ctypes.POINTER(sj_grid), I32, I32, ctypes.POINTER(sj_opts),
                           ctypes.POINTER(P), ctypes.POINTER(I64)]),
    ("sj_join_rows_into", I32, [P, P, I64, P, I64, ctypes.POINTER(sj_grid), I32, I32, ctypes.POINTER(sj_opts),
                                P, I64, ctypes.POINTER(I64)]),
    ("sj_join_host", I32, [P, P, I64, P, I64, ctypes.POINTER(sj_grid), ctypes.POINTER(sj_opts),
                           P, I64, ctypes.POINTER(I64)]),
    ("sj_timing_enable", I32, [P, I32]),
    ("sj_timing_read", I32, [P, ctypes.POINTER(sj_timing)]),
    ("sj_timing_phase_name", ctypes.c_char_p, [I32]),
    ("sj_last_stats", I32, [P, ctypes.POINTER(sj_stats)]),
    ("sj_mlp_create", I32, [P, ctypes.POINTER(P)]),
    ("sj_mlp_free", None, [P]),
    ("sj_mlp_set_params", I32, [P, P, P]),
    ("sj_mlp_get_params", I32, [P, P, P, P]),
    ("sj_mlp_forward", I32, [P, P, P, I64, P]),
    ("sj_mlp_grad", I32, [P, P, P, P, I64, P, P]),
    ("sj_mlp_train_step", I32, [P, P, P, P, I64, ctypes.c_float, P]),
    ("sj_set_schedule", I32, [P, I32]),
    ("sj_tile_axes", I32, [P, P, I64, P, I64, ctypes.POINTER(sj_grid), P]),
    ("sj_block_features", I32, [P, P, I64, P, I64, ctypes.POINTER(sj_grid), P, P, P, I64, ctypes.POINTER(I64)]),
    ("sj_set_model", I32, [P, P]),
    ("sj_extent_stats", I32, [P, P, I64, P, I64, P]),
    ("sj_set_tuning", I32, [P, I32]),
    ("sj_join_batch", I32, [P, I32, P, P, P, P, P, ctypes.POINTER(sj_opts), P, I64, P]),
    ("sj_join_noalloc", I32, [P, I64, P, I64, ctypes.POINTER(sj_grid), P, I64, ctypes.POINTER(I64), P]),
    ("sj_join_host_many", I32, [P, I32, P, P, P, P, P, ctypes.POINTER(sj_opts), P, P, P]),
    ("sj_distance_join", I32, [P, P, I64, P, I64, ctypes.c_float, ctypes.POINTER(sj_grid),
                               ctypes.POINTER(sj_opts), ctypes.POINTER(P), ctypes.POINTER(I64),
                               ctypes.POINTER(I64)]),
    ("sj_distance_join_into", I32, [P, P, I64, P, I64, ctypes.c_float, ctypes.POINTER(sj_grid),
                                    ctypes.POINTER(sj_opts), P, I64, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
]


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libsj.so (built beforehand); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run paper_1908_11740_gb300.build.build())")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def make_grid(nx: int, ny: int | None = None, x0=0.0, y0=0.0, x1=1.0, y1=1.0) -> sj_grid:
    return sj_grid(int(nx), int(nx if ny is None else ny), x0, y0, x1, y1)


def make_opts(mode="two_pass", sort_output=False, margin=0.25, axis="x", dedup="refpoint") -> sj_opts:
    """axis: "x" (Algorithm 1 along x in every tile) or "adaptive" (per tile,
    the axis with the smaller Eq. 2 estimate, SJ_SWEEP_ADAPTIVE); dedup:
    "refpoint" (the test of Eq. 1) or "gbda" (class mini-joins,
    SJ_DEDUP_GBDA)."""
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    if axis not in ("x", "adaptive"):
        raise ValueError("axis must be 'x' or 'adaptive'")
    if dedup not in ("refpoint", "gbda"):
        raise ValueError("dedup must be 'refpoint' or 'gbda'")
    flags = (SJ_SWEEP_ADAPTIVE if axis == "adaptive" else 0) | (SJ_DEDUP_GBDA if dedup == "gbda" else 0)
    return sj_opts(m, int(bool(sort_output)), float(margin), flags)


class _TorchAllocator:
    """Device buffers for the library, as PyTorch tensors kept alive here
    until the library frees them (or the caller takes a result)."""

    def __init__(self, device: torch.device):
        self.device = device
        self.live: dict[int, torch.Tensor] = {}
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, _user):
        t = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, ptr, _user):
        self.live.pop(int(ptr or 0), None)

    def take(self, ptr: int) -> torch.Tensor:
        return self.live.pop(int(ptr))


@dataclass
class Context:
    handle: int
    device: torch.device
    allocator: _TorchAllocator


def _check(ctx_handle, status):
    if status != SJ_OK:
        lib = load()
        msg = lib.sj_last_error(ctx_handle).decode() if ctx_handle else ""
        raise SJError(status, msg or lib.sj_strerror(status).decode())


def _rects(t: torch.Tensor, device) -> tuple[int, int]:
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or t.dim() != 2 or t.shape[1] != 4:
        raise TypeError("rectangles must be a float32 tensor of shape [n, 4]")
    if t.device != device:
        raise ValueError(f"rectangles on {t.device}, context on {device}")
    if not t.is_contiguous():
        raise ValueError("rectangles must be contiguous")
    return (t.data_ptr() if t.shape[0] else 0), int(t.shape[0])


def sj_create(device: int = 0, stream: torch.cuda.Stream | None = None) -> Context:
    lib = load()
    dev = torch.device("cuda", device)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    h = ctypes.c_void_p()
    st = lib.sj_create(ctypes.byref(h), device, ctypes.c_void_p(s.cuda_stream))
    if st != SJ_OK:
        raise SJError(st, lib.sj_strerror(st).decode())
    al = _TorchAllocator(dev)
    _check(h.value, lib.sj_set_allocator(h, al.alloc_cb, al.free_cb, None))
    return Context(h.value, dev, al)


def sj_destroy(ctx: Context) -> None:
    if ctx.handle:
        _check(ctx.handle, load().sj_destroy(ctx.handle))
        ctx.handle = 0
        ctx.allocator.live.clear()


def sj_join(ctx: Context, R: torch.Tensor, S: torch.Tensor, grid: sj_grid,
            opts: sj_opts | None = None) -> torch.Tensor:
    """All intersecting pairs as an int32[P, 2] CUDA tensor (r, s)."""
    lib = load()
    pr, nr = _rects(R, ctx.device)
    ps, ns = _rects(S, ctx.device)
    out = ctypes.c_void_p()
    n = ctypes.c_int64()
    st = lib.sj_join(ctx.handle, pr, nr, ps, ns, ctypes.byref(grid),
                     ctypes.byref(opts) if opts is not None else None, ctypes.byref(out), ctypes.byref(n))
    _check(ctx.handle, st)
    if n.value == 0:
        return torch.empty((0, 2), dtype=torch.int32, device=ctx.device)
    buf = ctx.allocator.take(out.value)
    return buf[: 8 * n.value].view(torch.int32).view(n.value, 2)


def sj_join_rows(ctx: Context, R: torch.Tensor, S: torch.Tensor, grid: sj_grid, row0: int, row1: int,
                 opts: sj_opts | None = None) -> torch.Tensor:
    """The pairs whose reference tile (Eq. 1) lies in tile rows [row0, row1):
    one band's share of the join, int32[P, 2] CUDA tensor (ids into R, S)."""
    lib = load()
    pr, nr = _rects(R, ctx.device)
    ps, ns = _rects(S, ctx.device)
    out = ctypes.c_void_p()
    n = ctypes.c_int64()
    st = lib.sj_join_rows(ctx.handle, pr, nr, ps, ns, ctypes.byref(grid), int(row0), int(row1),
                          ctypes.byref(opts) if opts is not None else None, ctypes.byref(out), ctypes.byref(n))
    _check(ctx.handle, st)
    if n.value == 0:
        return torch.empty((0, 2), dtype=torch.int32, device=ctx.device)
    buf = ctx.allocator.take(out.value)
    return buf[: 8 * n.value].view(torch.int32).view(n.value, 2)


def sj_join_rows_into(ctx: Context, R, S, grid: sj_grid, row0: int, row1: int, out: torch.Tensor,
                      opts: sj_opts | None = None) -> int:
    """sj_join_rows into a caller buffer (int32[cap, 2] CUDA tensor); returns
    the pair count, raises SJError(SJ_EOVERFLOW) when cap is too small."""
    lib = load()
    pr, nr = _rects(R, ctx.device)
    ps, ns = _rects(S, ctx.device)
    n = ctypes.c_int64()
    st = lib.sj_join_rows_into(ctx.handle, pr, nr, ps, ns, ctypes.byref(grid), int(row0), int(row1),
                               ctypes.byref(opts) if opts is not None else None,
                               out.data_ptr() if out.shape[0] else None, int(out.shape[0]), ctypes.byref(n))
    _check(ctx.handle, st)
    return n.value


def sj_join_into(ctx: Context, R, S, grid: sj_grid, out: torch.Tensor,
                 opts: sj_opts | None = None) -> int:
    """Write the pairs into ``out`` (int32[cap, 2]); returns their number.
    Raises SJError(SJ_EOVERFLOW) with the required count when out is short."""
    lib = load()
    pr, nr = _rects(R, ctx.device)
    ps, ns = _rects(S, ctx.device)
    if out.dtype != torch.int32 or out.dim() != 2 or out.shape[1] != 2 or not out.is_contiguous():
        raise TypeError("out must be a contiguous int32 tensor of shape [cap, 2]")
    n = ctypes.c_int64()
    st = lib.sj_join_into(ctx.handle, pr, nr, ps, ns, ctypes.byref(grid),
                          ctypes.byref(opts) if opts is not None else None,
                          out.data_ptr() if out.numel() else None, int(out.shape[0]), ctypes.byref(n))
    if st == SJ_EOVERFLOW:
        err = SJError(st, load().sj_last_error(ctx.handle).decode())
        err.required = n.value
        raise err
    _check(ctx.handle, st)
    return n.value


def _points(t: torch.Tensor, device) -> tuple[int, int]:
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or t.dim() != 2 or t.shape[1] != 2:
        raise TypeError("points must be a float32 tensor of shape [n, 2]")
    if t.device != device:
        raise ValueError(f"points on {t.device}, context on {device}")
    if not t.is_contiguous():
        raise ValueError("points must be contiguous")
    return (t.data_ptr() if t.shape[0] else 0), int(t.shape[0])


def sj_distance_join(ctx: Context, P: torch.Tensor, Q: torch.Tensor, eps: float, grid: sj_grid,
                     opts: sj_opts | None = None, return_candidates: bool = False):
    """All (i, j) with |P[i] - Q[j]| <= eps as an int32[n, 2] CUDA tensor;
    with ``return_candidates`` also the number of intersecting squares."""
    lib = load()
    pp, npn = _points(P, ctx.device)
    pq, nq = _points(Q, ctx.device)
    out = ctypes.c_void_p()
    n = ctypes.c_int64()
    nc = ctypes.c_int64()
    st = lib.sj_distance_join(ctx.handle, pp, npn, pq, nq, float(eps), ctypes.byref(grid),
                              ctypes.byref(opts) if opts is not None else None, ctypes.byref(out),
                              ctypes.byref(n), ctypes.byref(nc))
    _check(ctx.handle, st)
    if n.value == 0:
        res = torch.empty((0, 2), dtype=torch.int32, device=ctx.device)
    else:
        res = ctx.allocator.take(out.value)[: 8 * n.value].view(torch.int32).view(n.value, 2)
    return (res, nc.value) if return_candidates else res


def sj_distance_join_into(ctx: Context, P, Q, eps: float, grid: sj_grid, out: torch.Tensor,
                          opts: sj_opts | None = None) -> int:
    """Write the pairs within distance eps into ``out`` (int32[cap, 2]);
    returns their number.  SJError(SJ_EOVERFLOW) with ``required`` when short."""
    lib = load()
    pp, npn = _points(P, ctx.device)
    pq, nq = _points(Q, ctx.device)
    if out.dtype != torch.int32 or out.dim() != 2 or out.shape[1] != 2 or not out.is_contiguous():
        raise TypeError("out must be a contiguous int32 tensor of shape [cap, 2]")
    n = ctypes.c_int64()
    st = lib.sj_distance_join_into(ctx.handle, pp, npn, pq, nq, float(eps), ctypes.byref(grid),
                                   ctypes.byref(opts) if opts is not None else None,
                                   out.data_ptr() if out.numel() else None, int(out.shape[0]),
                                   ctypes.byref(n), None)
    if st == SJ_EOVERFLOW:
        err = SJError(st, load().sj_last_error(ctx.handle).decode())
        err.required = n.value
        raise err
    _check(ctx.handle, st)
    return n.value


def sj_count(ctx: Context, R, S, grid: sj_grid) -> int:
    lib = load()
    pr, nr = _rects(R, ctx.device)
    ps, ns = _rects(S, ctx.device)
    n = ctypes.c_int64()
    _check(ctx.handle, lib.sj_count(ctx.handle, pr, nr, ps, ns, ctypes.byref(grid), ctypes.byref(n)))
    return n.value


def sj_tile_stats(ctx: Context, R, S, grid: sj_grid):
    """(cnt_r, cnt_s, pairs_per_tile), each int32[ny*nx] (row-major)."""
    lib = load()
    pr, nr = _rects(R, ctx.device)
    ps, ns = _rects(S, ctx.device)
    T = grid.nx * grid.ny
    cr = torch.empty(T, dtype=torch.int32, device=ctx.device)
    cs = torch.empty(T, dtype=torch.int32, device=ctx.device)
    tp = torch.empty(T, dtype=torch.int32, device=ctx.device)
    _check(ctx.handle, lib.sj_tile_stats(ctx.handle, pr, nr, ps, ns, ctypes.byref(grid),
                                         cr.data_ptr(), cs.data_ptr(), tp.data_ptr()))
    return cr, cs, tp


def sj_tile_axes(ctx: Context, R, S, grid: sj_grid) -> torch.Tensor:
    """uint8[ny * nx] device tensor: the sweep axis SJ_SWEEP_ADAPTIVE gives
    every tile (1 = y), from the Eq. 2 histograms of Sec. 3.3."""
    pr, nr = _rects(R, ctx.device)
    ps, ns = _rects(S, ctx.device)
    out = torch.empty(int(grid.nx) * int(grid.ny), dtype=torch.uint8, device=ctx.device)
    _check(ctx.handle, load().sj_tile_axes(ctx.handle, pr, nr, ps, ns, ctypes.byref(grid), out.data_ptr()))
    return out


def sj_join_host_many(ctx: Context, Rs, Ss, grids, outs, opts: sj_opts | None = None) -> list[int]:
    """Join the host arrays (Rs[i], Ss[i]) on grids[i] one after the other,
    each join's input copy overlapping the previous join; the pairs of join i
    go to outs[i] (CPU int32[cap_i, 2] tensors, ideally pinned).  Returns the
    pair counts.  SJError(SJ_EOVERFLOW) carries ``required`` (all counts)."""
    lib = load()
    n = len(Rs)
    if not (len(Ss) == len(grids) == len(outs) == n):
        raise ValueError("Rs, Ss, grids and outs must have the same length")
    keep = []

    def host(a, cols, dtype):
        if not isinstance(a, torch.Tensor) or a.device.type != "cpu" or a.dtype != dtype or a.dim() != 2 \
                or a.shape[1] != cols or not a.is_contiguous():
            raise TypeError(f"host arrays must be contiguous CPU {dtype} tensors [n, {cols}]")
        keep.append(a)
        return a.data_ptr() if a.shape[0] else None, a.shape[0]

    P = ctypes.c_void_p
    pr, nr, ps, ns, po, cp = (P * n)(), (ctypes.c_int64 * n)(), (P * n)(), (ctypes.c_int64 * n)(), (P * n)(), \
        (ctypes.c_int64 * n)()
    for i in range(n):
        pr[i], nr[i] = host(Rs[i], 4, torch.float32)
        ps[i], ns[i] = host(Ss[i], 4, torch.float32)
        po[i], cp[i] = host(outs[i], 2, torch.int32)
    g = (sj_grid * n)(*grids)
    counts = (ctypes.c_int64 * n)()
    st = lib.sj_join_host_many(ctx.handle, n, pr, nr, ps, ns, g, ctypes.byref(opts) if opts is not None else None,
                               po, cp, counts)
    if st == SJ_EOVERFLOW:
        err = SJError(st, lib.sj_last_error(ctx.handle).decode())
        err.required = list(counts)
        raise err
    _check(ctx.handle, st)
    return list(counts)


def sj_join_host(ctx: Context, R, S, grid: sj_grid, out=None, opts: sj_opts | None = None):
    """Join HOST arrays (numpy float32[n,4] or CPU tensors, ideally pinned):
    the library copies them to the device, joins, and copies the pairs back
    into ``out`` (a CPU int32[cap, 2] tensor / array).  Returns the pairs."""
    lib = load()

    def host(a):
        if isinstance(a, torch.Tensor):
            if a.device.type != "cpu" or a.dtype != torch.float32 or a.dim() != 2 or a.shape[1] != 4:
                raise TypeError("host rectangles must be a CPU float32 tensor [n, 4]")
            a = a.contiguous()
            return a, a.data_ptr(), a.shape[0]
        import numpy as np
        a = np.ascontiguousarray(a, np.float32)
        return a, a.ctypes.data, a.shape[0]

    r, pr, nr = host(R)
    s_, ps, ns = host(S)
    if out is None:
        out = torch.empty((0, 2), dtype=torch.int32)
    n = ctypes.c_int64()
    o_ptr = out.data_ptr() if isinstance(out, torch.Tensor) else out.ctypes.data
    st = lib.sj_join_host(ctx.handle, pr if nr else None, nr, ps if ns else None, ns, ctypes.byref(grid),
                          ctypes.byref(opts) if opts is not None else None,
                          o_ptr if len(out) else None, len(out), ctypes.byref(n))
    if st == SJ_EOVERFLOW:
        out = torch.empty((n.value, 2), dtype=torch.int32, pin_memory=torch.cuda.is_available())
        st = lib.sj_join_host(ctx.handle, pr if nr else None, nr, ps if ns else None, ns, ctypes.byref(grid),
                              ctypes.byref(opts) if opts is not None else None,
                              out.data_ptr() if len(out) else None, len(out), ctypes.byref(n))
    _check(ctx.handle, st)
    return out[: n.value]


def sj_last_stats(ctx: Context) -> dict:
    st = sj_stats()
    _check(ctx.handle, load().sj_last_stats(ctx.handle, ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in sj_stats._fields_}


def sj_timing_enable(ctx: Context, on: bool = True) -> None:
    _check(ctx.handle, load().sj_timing_enable(ctx.handle, int(bool(on))))


def sj_timing_read(ctx: Context) -> dict:
    """{'launches': L, phase: (occurrences, ms), ...} since the last read."""
    lib = load()
    t = sj_timing()
    _check(ctx.handle, lib.sj_timing_read(ctx.handle, ctypes.byref(t)))
    out = {"launches": int(t.launches)}
    for i in range(13):
        name = lib.sj_timing_phase_name(i).decode()
        if name:
            out[name] = (int(t.n[i]), float(t.ms[i]))
    return out


class Partition:
    def __init__(self, ctx: Context, handle: int, keep):
        self.ctx, self.handle, self._keep = ctx, handle, keep

    def view(self) -> sj_part_view:
        v = sj_part_view()
        _check(self.ctx.handle, load().sj_part_view_get(self.handle, ctypes.byref(v)))
        return v

    def free(self):
        if self.handle:
            load().sj_part_free(self.handle)
            self.handle = 0


def sj_partition(ctx: Context, R, S, grid: sj_grid) -> Partition:
    lib = load()
    pr, nr = _rects(R, ctx.device)
    ps, ns = _rects(S, ctx.device)
    h = ctypes.c_void_p()
    _check(ctx.handle, lib.sj_partition(ctx.handle, pr, nr, ps, ns, ctypes.byref(grid), ctypes.byref(h)))
    return Partition(ctx, h.value, None)


def sj_part_join(ctx: Context, part: Partition, opts: sj_opts | None = None) -> torch.Tensor:
    lib = load()
    out = ctypes.c_void_p()
    n = ctypes.c_int64()
    _check(ctx.handle, lib.sj_part_join(ctx.handle, part.handle,
                                        ctypes.byref(opts) if opts is not None else None,
                                        ctypes.byref(out), ctypes.byref(n)))
    if n.value == 0:
        return torch.empty((0, 2), dtype=torch.int32, device=ctx.device)
    buf = ctx.allocator.take(out.value)
    return buf[: 8 * n.value].view(torch.int32).view(n.value, 2)


class _CudaArray:
    """Exposes a raw device pointer through __cuda_array_interface__."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def device_view(ptr: int, shape, dtype: torch.dtype) -> torch.Tensor:
    """Zero-copy read-only tensor over library-owned device memory (for
    inspection, e.g. of a partition's per-tile arrays)."""
    typestr = {torch.int32: "<i4", torch.float32: "<f4", torch.int64: "<i8", torch.uint8: "|u1"}[dtype]
    n = 1
    for s in shape:
        n *= int(s)
    if n == 0:
        return torch.empty(tuple(shape), dtype=dtype, device="cuda")
    return torch.as_tensor(_CudaArray(ptr, shape, typestr), device="cuda")


# ---- learned per-block result-count predictor --------------------------------
class Model:
    """An sj_mlp on a context (32 -> 64 -> 64 -> 1, bf16 weights)."""

    def __init__(self, ctx: Context, params=None):
        lib = load()
        h = ctypes.c_void_p()
        _check(ctx.handle, lib.sj_mlp_create(ctx.handle, ctypes.byref(h)))
        self.ctx, self.handle = ctx, h.value
        self.loss_buf = torch.zeros(1, dtype=torch.float32, device=ctx.device)
        if params is not None:
            self.set_params(params)

    def set_params(self, params):
        import numpy as np
        p = np.ascontiguousarray(params, np.float32)
        if p.shape != (SJ_MLP_PARAMS,):
            raise ValueError(f"expected {SJ_MLP_PARAMS} parameters")
        _check(self.ctx.handle, load().sj_mlp_set_params(self.ctx.handle, self.handle, p.ctypes.data))

    def get_params(self, inference: bool = False):
        import numpy as np
        master = np.empty(SJ_MLP_PARAMS, np.float32)
        inf = np.empty(SJ_MLP_PARAMS, np.float32) if inference else None
        _check(self.ctx.handle, load().sj_mlp_get_params(self.ctx.handle, self.handle, master.ctypes.data,
                                                         inf.ctypes.data if inf is not None else None))
        return (master, inf) if inference else master

    def forward(self, X: torch.Tensor) -> torch.Tensor:
        X = X.contiguous()
        y = torch.empty(X.shape[0], dtype=torch.float32, device=self.ctx.device)
        _check(self.ctx.handle, load().sj_mlp_forward(self.ctx.handle, self.handle, X.data_ptr(), X.shape[0],
                                                      y.data_ptr()))
        return y

    def grad(self, X: torch.Tensor, Y: torch.Tensor):
        g = torch.empty(SJ_MLP_PARAMS, dtype=torch.float32, device=self.ctx.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.ctx.device)
        X, Y = X.contiguous(), Y.contiguous()
        _check(self.ctx.handle, load().sj_mlp_grad(self.ctx.handle, self.handle, X.data_ptr(), Y.data_ptr(),
                                                   X.shape[0], g.data_ptr(), loss.data_ptr()))
        return g, loss

    def train_step(self, X: torch.Tensor, Y: torch.Tensor, lr: float) -> torch.Tensor:
        """One Adam step; returns the batch loss as a device scalar (no sync)."""
        _check(self.ctx.handle, load().sj_mlp_train_step(self.ctx.handle, self.handle, X.data_ptr(),
                                                         Y.data_ptr(), X.shape[0], float(lr),
                                                         self.loss_buf.data_ptr()))
        return self.loss_buf

    def free(self):
        if self.handle:
            load().sj_mlp_free(self.handle)
            self.handle = 0


def sj_set_model(ctx: Context, model: "Model | None") -> None:
    _check(ctx.handle, load().sj_set_model(ctx.handle, model.handle if model is not None else None))


def sj_block_features(ctx: Context, R, S, grid: sj_grid, with_blocks: bool = False):
    """(features float32[n, 32], labels float32[n][, block ids int32[n]]) of
    the blocks of a join: labels = log1p(exact pairs each block reports)."""
    lib = load()
    pr, nr = _rects(R, ctx.device)
    ps, ns = _rects(S, ctx.device)
    n = ctypes.c_int64()
    st = lib.sj_block_features(ctx.handle, pr, nr, ps, ns, ctypes.byref(grid), None, None, None, 0,
                               ctypes.byref(n))
    if st not in (SJ_OK, SJ_EOVERFLOW):
        _check(ctx.handle, st)
    m = max(n.value, 1)
    X = torch.empty((m, SJ_MLP_FEATURES), dtype=torch.float32, device=ctx.device)
    Y = torch.empty(m, dtype=torch.float32, device=ctx.device)
    B = torch.empty(m, dtype=torch.int32, device=ctx.device)
    _check(ctx.handle, lib.sj_block_features(ctx.handle, pr, nr, ps, ns, ctypes.byref(grid), X.data_ptr(),
                                             Y.data_ptr(), B.data_ptr(), m, ctypes.byref(n)))
    k = n.value
    return (X[:k], Y[:k], B[:k]) if with_blocks else (X[:k], Y[:k])


def sj_join_batch(ctx: Context, Rs, Ss, grids=None, out: torch.Tensor | None = None,
                  opts: sj_opts | None = None):
    """Join every (Rs[j], Ss[j]) in one batched pass.  Returns (pairs
    int32[P, 2] device tensor, offsets int64[nj + 1]); the pairs of join j
    are pairs[offsets[j]:offsets[j+1]] (ids local to the join).  grids:
    list of sj_grid, or None for the rule-of-thumb grid of every join;
    opts.mode: two-pass (default) or one-pass sizing of the whole batch."""
    import numpy as np
    lib = load()
    nj = len(Rs)
    if len(Ss) != nj or nj == 0:
        raise ValueError("Rs and Ss must be non-empty lists of the same length")
    pr = (ctypes.c_void_p * nj)()
    ps = (ctypes.c_void_p * nj)()
    nr = (ctypes.c_int64 * nj)()
    ns = (ctypes.c_int64 * nj)()
    for j in range(nj):
        pr[j], nr[j] = _rects(Rs[j], ctx.device)
        ps[j], ns[j] = _rects(Ss[j], ctx.device)
    g = None
    if grids is not None:
        g = (sj_grid * nj)(*grids)
    offs = np.zeros(nj + 1, np.int64)
    buf = out if out is not None else torch.empty((0, 2), dtype=torch.int32, device=ctx.device)
    po = ctypes.byref(opts) if opts is not None else None
    st = lib.sj_join_batch(ctx.handle, nj, pr, nr, ps, ns, g, po, buf.data_ptr() if buf.numel() else None,
                           buf.shape[0], offs.ctypes.data)
    if st == SJ_EOVERFLOW and out is None:
        buf = torch.empty((int(offs[-1]), 2), dtype=torch.int32, device=ctx.device)
        st = lib.sj_join_batch(ctx.handle, nj, pr, nr, ps, ns, g, po, buf.data_ptr(), buf.shape[0],
                               offs.ctypes.data)
    _check(ctx.handle, st)
    return buf[: int(offs[-1])], offs


def sj_extent_stats(ctx: Context, R, S):
    """(sum w_R, sum h_R, sum w_S, sum h_S) of device rectangles."""
    import numpy as np
    pr, nr = _rects(R, ctx.device)
    ps, ns = _rects(S, ctx.device)
    out = np.zeros(4, np.float64)
    _check(ctx.handle, load().sj_extent_stats(ctx.handle, pr, nr, ps, ns, out.ctypes.data))
    return out


def sj_set_schedule(ctx: Context, heaviest_first: bool) -> None:
    """One-pass join: blocks heaviest predicted cost first (default) or in
    block order."""
    _check(ctx.handle, load().sj_set_schedule(ctx.handle, int(bool(heaviest_first))))


def sj_set_tuning(ctx: Context, block_target: int) -> None:
    _check(ctx.handle, load().sj_set_tuning(ctx.handle, int(block_target)))
