"""One process per GPU: rank setup, sharding of independent joins, and the
reduction of per-rank timings.

The filter step shards without a data-path exchange: tiles, and therefore
whole joins, are independent units (every pair is reported by exactly one
tile).  With N ranks,

* a batch of joins is split into N disjoint shards of about equal input
  size (each rank joins its shard with one batched call), and
* a single large workload is run as one independent instance per rank
  (weak scaling: rank r joins the instance drawn with seed base + r), or
* one join is split into contiguous bands of tile rows, one per rank,
  balanced by the entries per row (strong scaling).  Every pair is reported
  by the tile holding its reference point (Eq. 1), so disjoint bands give
  disjoint pair sets whose union is the join.  The exchange step is the
  staging of each band's rectangles -- those overlapping its rows -- into
  its GPU's own memory; no pair moves between ranks.

The only collectives are the barrier around the timed region and the
reduction of the results: the slowest rank's time (the job ends when the
last rank ends) and the sum of the pairs found.

    from paper_1908_11740_gb300 import dist
    env = dist.setup()                         # reads RANK / WORLD_SIZE / LOCAL_RANK
    mine = dist.shard(sizes, env.rank, env.world)
    bands = dist.band_plan(dist.row_loads(R, S, grid), env.world)
    idx_r, idx_s = dist.band_members(R, S, grid, *bands[env.rank])
    ms_job, pairs_job = dist.reduce_result(ms, pairs, env)
"""
from __future__ import annotations

import os
from dataclasses import dataclass

import numpy as np


@dataclass
class Env:
    rank: int
    world: int
    local_rank: int
    backend: str | None   # None: a single process, no process group


def setup(backend: str = "nccl") -> Env:
    """Read the launcher's environment; start the process group when there
    is more than one rank (MASTER_ADDR / MASTER_PORT come from the launcher)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    if world <= 1:
        return Env(0, 1, local, None)
    import torch.distributed as td

    if backend == "nccl":
        import torch

        torch.cuda.set_device(local)
    if not td.is_initialized():
        td.init_process_group(backend)
    return Env(rank, world, local, backend)


def teardown(env: Env) -> None:
    if env.backend is not None:
        import torch.distributed as td

        if td.is_initialized():
            td.destroy_process_group()


def shard(sizes, rank: int, world: int) -> list[int]:
    """Indices of the units rank `rank` takes: units in decreasing size, each
    given to the rank with the least total so far (ties: lowest rank).  The
    shards are disjoint, cover every unit, and every rank computes the same
    assignment from the same sizes."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    order = sorted(range(len(sizes)), key=lambda j: (-sizes[j], j))
    load = [0] * world
    owner = [0] * len(sizes)
    for j in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[j] = r
        load[r] += sizes[j]
    return [j for j in range(len(sizes)) if owner[j] == rank]


def cell_rows(A, ny: int, y0: float, y1: float):
    """First and last tile row of every rectangle: the cell function
    clamp(floor((y - y0) * gy), 0, ny - 1) with gy = ny / (y1 - y0), each
    operation rounded to float32 (numpy float32 arithmetic)."""
    A = np.asarray(A, np.float32)
    g0 = np.float32(y0)
    gy = np.float32(ny) / (np.float32(y1) - g0)

    def cell(v):
        t = (v - g0) * gy
        return np.clip(np.floor(t), 0, ny - 1).astype(np.int64)

    return cell(A[:, 1]), cell(A[:, 3])


def row_loads(R, S, grid) -> np.ndarray:
    """Replicated entries per tile row of the grid (both sides): a rectangle
    adds its column span to every row it overlaps."""
    nx, ny = int(grid.nx), int(grid.ny)
    load = np.zeros(ny + 1, np.int64)
    for A in (R, S):
        A = np.asarray(A, np.float32)
        if not len(A):
            continue
        r0, r1 = cell_rows(A, ny, grid.y0, grid.y1)
        gx = np.float32(nx) / (np.float32(grid.x1) - np.float32(grid.x0))
        c0 = np.clip(np.floor((A[:, 0] - np.float32(grid.x0)) * gx), 0, nx - 1).astype(np.int64)
        c1 = np.clip(np.floor((A[:, 2] - np.float32(grid.x0)) * gx), 0, nx - 1).astype(np.int64)
        w = c1 - c0 + 1
        np.add.at(load, r0, w)
        np.add.at(load, r1 + 1, -w)
    return np.cumsum(load)[:ny]


def band_plan(loads, world: int) -> list[tuple[int, int]]:
    """Split the rows into `world` contiguous bands [row0, row1) that cover
    every row once, cutting where the running load first reaches k / world of
    the total (k = 1 .. world - 1).  Bands may be empty when rows are fewer
    than ranks or one row carries most of the load."""
    loads = np.asarray(loads, np.int64)
    ny = len(loads)
    if world < 1:
        raise ValueError("world must be >= 1")
    pre = np.concatenate([[0], np.cumsum(loads)])
    total = int(pre[-1])
    cuts = [0]
    for k in range(1, world):
        target = total * k / world
        c = int(np.searchsorted(pre, target, side="left"))
        cuts.append(min(max(c, cuts[-1]), ny))
    cuts.append(ny)
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


def band_members(R, S, grid, row0: int, row1: int, margin: int = 1):
    """Indices of the rectangles of R and of S that a band's rank stages on
    its GPU: those overlapping rows [row0 - margin, row1 + margin).  Only the
    rectangles overlapping [row0, row1) are needed; the margin keeps the
    selection complete even if a host rounding differed from the device's
    cell function, and extra rectangles cannot change the band's pairs (the
    library keeps only pairs whose reference tile lies in the band)."""
    out = []
    for A in (R, S):
        if not len(A):
            out.append(np.zeros(0, np.int64))
            continue
        r0, r1 = cell_rows(A, int(grid.ny), grid.y0, grid.y1)
        out.append(np.flatnonzero((r0 < row1 + margin) & (r1 >= row0 - margin)))
    return out[0], out[1]


def instance_seed(base: int, env: Env) -> int:
    """Seed of this rank's independent instance (weak scaling)."""
    return base + env.rank


def barrier(env: Env) -> None:
    if env.backend is not None:
        import torch.distributed as td

        td.barrier()


def reduce_result(ms: float, pairs: int, env: Env) -> tuple[float, int]:
    """(max over ranks of ms, sum over ranks of pairs)."""
    if env.backend is None:
        return float(ms), int(pairs)
    import torch
    import torch.distributed as td

    dev = torch.device("cuda", torch.cuda.current_device()) if env.backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    p = torch.tensor([int(pairs)], dtype=torch.int64, device=dev)
    td.all_reduce(p, op=td.ReduceOp.SUM)
    return float(t.item()), int(p.item())
