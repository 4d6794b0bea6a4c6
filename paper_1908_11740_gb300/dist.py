"""One process per GPU: rank setup, sharding of independent joins, and the
reduction of per-rank timings.

The filter step shards without a data-path exchange: tiles, and therefore
whole joins, are independent units (every pair is reported by exactly one
tile).  With N ranks,

* a batch of joins is split into N disjoint shards of about equal input
  size (each rank joins its shard with one batched call), and
* a single large workload is run as one independent instance per rank
  (weak scaling: rank r joins the instance drawn with seed base + r).

The only collectives are the barrier around the timed region and the
reduction of the results: the slowest rank's time (the job ends when the
last rank ends) and the sum of the pairs found.

    from paper_1908_11740_gb300 import dist
    env = dist.setup()                         # reads RANK / WORLD_SIZE / LOCAL_RANK
    mine = dist.shard(sizes, env.rank, env.world)
    ms_job, pairs_job = dist.reduce_result(ms, pairs, env)
"""
from __future__ import annotations

import os
from dataclasses import dataclass


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
