"""Band split of one join over several ranks (the multi-GPU partitioning of
one join), host logic on CPU.

* band_plan covers every tile row exactly once with contiguous bands and
  balances them by entries per row (no band above the even share by more
  than one row's load);
* the host cell rows used for planning equal the oracle's cell function;
* two `gloo` ranks each take a band, stage the rectangles that overlap it,
  join them with the CPU oracle on the full grid and keep the pairs whose
  reference tile (Eq. 1) lies in their band; the union over ranks is the
  oracle's join of the whole input and no pair appears in two bands."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from paper_1908_11740_gb300 import dist, inputs  # noqa: E402


class Grid:
    def __init__(self, nx, ny, x0=0.0, y0=0.0, x1=1.0, y1=1.0):
        self.nx, self.ny, self.x0, self.y0, self.x1, self.y1 = nx, ny, x0, y0, x1, y1


def test_cell_rows_match_oracle_cells():
    R, _ = inputs.gis_pair(20_000, 10, seed=81, median_extent=3e-3)
    R[:50] *= 1.3          # some coordinates outside the grid
    g = Grid(37, 53, 0.1, -0.05, 0.9, 1.05)
    r0, r1 = dist.cell_rows(R, g.ny, g.y0, g.y1)
    c = oracle.cells(R, g.nx, g.ny, g.x0, g.y0, g.x1, g.y1)
    np.testing.assert_array_equal(r0, c[:, 2])
    np.testing.assert_array_equal(r1, c[:, 3])
    loads = dist.row_loads(R, R[:0], g)
    per_tile = oracle.tile_counts(R, g.nx, g.ny, g.x0, g.y0, g.x1, g.y1).reshape(g.ny, g.nx)
    np.testing.assert_array_equal(loads, per_tile.sum(1))


@pytest.mark.parametrize("world", [1, 2, 3, 5, 8])
def test_band_plan_covers_and_balances(world):
    g = np.random.default_rng(world)
    loads = g.integers(0, 1000, 200) * (g.random(200) < 0.7)
    bands = dist.band_plan(loads, world)
    assert len(bands) == world and bands[0][0] == 0 and bands[-1][1] == 200
    for (a0, a1), (b0, b1) in zip(bands, bands[1:]):
        assert a1 == b0 and a0 <= a1
    share = loads.sum() / world
    for a0, a1 in bands:
        assert loads[a0:a1].sum() <= share + loads.max()
    # degenerate inputs: more ranks than rows, and no load at all
    assert dist.band_plan([5, 0, 7], 5)[-1][1] == 3
    assert [b for b in dist.band_plan(np.zeros(4, np.int64), 2)] == [(0, 0), (0, 4)]


def _band_pairs(R, S, g, row0, row1):
    """What one rank computes: its band's rectangles, the oracle's join on the
    full grid, the pairs whose reference row lies in the band, input ids."""
    ir, is_ = dist.band_members(R, S, g, row0, row1)
    sub = oracle.pbsm(R[ir], S[is_], g.nx, g.ny, g.x0, g.y0, g.x1, g.y1)
    cr = oracle.cells(R[ir], g.nx, g.ny, g.x0, g.y0, g.x1, g.y1)[:, 2]
    cs = oracle.cells(S[is_], g.nx, g.ny, g.x0, g.y0, g.x1, g.y1)[:, 2]
    ref = np.maximum(cr[sub[:, 0]], cs[sub[:, 1]])
    keep = sub[(ref >= row0) & (ref < row1)]
    return np.stack([ir[keep[:, 0]], is_[keep[:, 1]]], 1).astype(np.int32)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    import torch.distributed as td

    env = dist.setup("gloo")
    R, S = inputs.gis_pair(30_000, 40_000, seed=82, median_extent=2e-3)
    g = Grid(48, 48)
    bands = dist.band_plan(dist.row_loads(R, S, g), env.world)
    row0, row1 = bands[env.rank]
    mine = _band_pairs(R, S, g, row0, row1)
    gathered = [None] * env.world
    td.all_gather_object(gathered, (env.rank, bands, mine.tolist()))
    dist.barrier(env)
    ms, total = dist.reduce_result(1.0 + env.rank, len(mine), env)
    q.put((env.rank, gathered, ms, total))
    dist.teardown(env)


def test_two_gloo_ranks_bands_union_is_the_join():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    gathered = res[0][1]
    assert gathered == res[1][1]
    bands = gathered[0][1]
    assert bands[0][0] == 0 and bands[-1][1] == 48 and bands[0][1] == bands[1][0]
    parts = [np.asarray(p, np.int32).reshape(-1, 2) for _, _, p in sorted(gathered)]
    assert len(parts[0]) and len(parts[1])
    union = np.concatenate(parts)
    keys = union[:, 0].astype(np.int64) << 32 | union[:, 1].astype(np.int64)
    assert len(np.unique(keys)) == len(keys)             # no pair in two bands
    R, S = inputs.gis_pair(30_000, 40_000, seed=82, median_extent=2e-3)
    want = oracle.pbsm(R, S, 48)
    np.testing.assert_array_equal(union[np.lexsort((union[:, 1], union[:, 0]))], want)
    assert res[0][2] == res[1][2] == 2.0                 # slowest rank's time
    assert res[0][3] == res[1][3] == len(want)           # pairs summed over ranks
