"""The multi-rank host logic on CPU: two `gloo` ranks (world_size 2,
127.0.0.1) go through setup, the sharding of a batch of joins, the barrier
and the reduction of results, as bench.py does with one rank per GPU.

* the shards of the ranks are disjoint, cover every join and are balanced by
  input size (largest first to the least-loaded rank);
* every rank draws a different independent instance (weak scaling);
* the job time is the slowest rank's, the job's pairs are the sum over
  ranks;
* each rank joins its shard with the CPU oracle; the union of the ranks'
  pairs equals the oracle on the whole batch, so sharding loses and
  duplicates nothing."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

from paper_1908_11740_gb300 import dist, inputs  # noqa: E402


def test_shard_partition_and_balance():
    sizes = [5, 1, 9, 3, 3, 7, 2, 8]
    shards = [dist.shard(sizes, r, 3) for r in range(3)]
    flat = sorted(j for s in shards for j in s)
    assert flat == list(range(len(sizes)))
    loads = [sum(sizes[j] for j in s) for s in shards]
    assert max(loads) - min(loads) <= max(sizes)
    assert dist.shard(sizes, 0, 1) == list(range(len(sizes)))
    with pytest.raises(ValueError):
        dist.shard(sizes, 3, 3)


def test_single_process_env(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    env = dist.setup("gloo")
    assert (env.rank, env.world, env.backend) == (0, 1, None)
    assert dist.reduce_result(2.5, 7, env) == (2.5, 7)
    assert dist.instance_seed(2, env) == 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    import oracle

    env = dist.setup("gloo")
    joins = inputs.batch_pairs(n_joins=9, seed0=4000, n_min=200, n_max=3000, median_extent=3e-3)
    mine = dist.shard([len(r) + len(s) for r, s in joins], env.rank, env.world)
    pairs = {j: oracle.pbsm(joins[j][0], joins[j][1], 16) for j in mine}
    dist.barrier(env)
    local_ms = 10.0 + 5.0 * env.rank
    ms, total = dist.reduce_result(local_ms, sum(len(p) for p in pairs.values()), env)
    q.put((env.rank, mine, {j: p.tolist() for j, p in pairs.items()}, ms, total,
           dist.instance_seed(2, env)))
    dist.teardown(env)


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    shards = [r[1] for r in res]
    assert sorted(shards[0] + shards[1]) == list(range(9)) and not set(shards[0]) & set(shards[1])
    assert res[0][5] != res[1][5]                       # independent instances per rank
    assert res[0][3] == res[1][3] == 15.0               # slowest rank's time
    import oracle

    joins = inputs.batch_pairs(n_joins=9, seed0=4000, n_min=200, n_max=3000, median_extent=3e-3)
    got = {}
    for r in res:
        got.update(r[2])
    want_total = 0
    for j, (R, S) in enumerate(joins):
        want = oracle.brute(R, S)
        want_total += len(want)
        np.testing.assert_array_equal(np.asarray(got[j], np.int32).reshape(-1, 2), want)
    assert res[0][4] == res[1][4] == want_total          # pairs summed over ranks
