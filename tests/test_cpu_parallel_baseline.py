"""The multi-core CPU baseline (the paper's parallel PBSM, Sec. 3.4, with
OpenMP) must return exactly the oracle's pairs, whatever the number of
threads and the grid; it is only a timing baseline, so it is checked here
against the oracle and never used as one."""
import numpy as np
import pytest

import oracle
from paper_1908_11740_gb300 import inputs


@pytest.fixture(scope="module")
def par():
    try:
        oracle.build_parallel()
    except Exception as e:  # pragma: no cover
        pytest.skip(f"no OpenMP: {e}")
    return oracle.pbsm_parallel


CASES = {
    "uniform": lambda: inputs.uniform_pair(20_000, 30_000, max_extent=5e-3, seed=61),
    "gis": lambda: inputs.gis_pair(100_000, 150_000, seed=62, median_extent=1e-4),
    "zipf": lambda: inputs.zipf_pair(30_000, 30_000, seed=63, rho=0.3, lattice=64),
    "degenerate": lambda: inputs.degenerate_pair(seed=64),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("grid", [(1, 1), (7, 3), (64, 64), (300, 300)])
@pytest.mark.parametrize("threads", [1, 2, 5])
def test_equals_oracle(par, case, grid, threads):
    R, S = CASES[case]()
    want = oracle.pbsm(R, S, 32)
    got = par(R, S, grid[0], grid[1], threads=threads)
    np.testing.assert_array_equal(got, want)
    assert par(R, S, grid[0], grid[1], threads=threads, pairs=False) == len(want)


def test_sub_window_and_empty(par):
    R, S = inputs.uniform_pair(5_000, 6_000, max_extent=0.02, seed=65)
    want = oracle.brute(R, S)
    # the grid covers only part of the space: outside rectangles go to the border tiles
    np.testing.assert_array_equal(par(R, S, 9, 4, 0.2, 0.3, 0.6, 0.5, threads=3), want)
    empty = np.zeros((0, 4), np.float32)
    assert par(empty, S, 8).shape == (0, 2)
    assert par(R, empty, 8, threads=4).shape == (0, 2)
