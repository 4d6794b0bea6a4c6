"""Pins of the oracle's digest route (``oracle.pbsm_digest``), the check used
for result sets too large to hold (the 1e9-pair skew joins).

* the mixer is the output function of SplitMix64 (Steele, Lea and Flood,
  2014): the first outputs of the generator seeded with 0 are published;
* a one-pair join has the digest of that pair alone (C mixer against them);
* on inputs small enough for brute force, the digest of PBSM equals the
  digest (computed with numpy in ``tests/pair_digest.py``) of the pairs of
  the definition, at several grids, on uniform, skewed and degenerate inputs;
* the digest ignores order but sees a changed, dropped or repeated pair.
"""
import numpy as np
import pytest

import oracle
from paper_1908_11740_gb300 import inputs
from pair_digest import combine, digest, mix


def test_mixer_is_splitmix64():
    gamma = 0x9E3779B97F4A7C15
    k = np.array([0, gamma, (2 * gamma) % (1 << 64)], np.uint64)
    got = [int(v) for v in mix(k)]
    # the first three outputs of SplitMix64 seeded with 0
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_single_pair_digest():
    R = np.array([[0.1, 0.1, 0.2, 0.2]], np.float32)
    S = np.array([[0.15, 0.15, 0.3, 0.3], [0.5, 0.5, 0.6, 0.6]], np.float32)
    assert oracle.pbsm_digest(R, S, 4) == (1, 0xE220A8397B1DCDAF, 0xE220A8397B1DCDAF)
    # (0, 1): key 1 << 0 = 1
    S2 = S[::-1].copy()
    h = int(mix(np.array([1], np.uint64))[0])
    assert oracle.pbsm_digest(R, S2, 4) == (1, h, h)
    # no pair
    assert oracle.pbsm_digest(R, S[1:], 4) == (0, 0, 0)


@pytest.mark.parametrize("K", [1, 3, 16, 64])
@pytest.mark.parametrize("kind", ["uniform", "zipf", "degenerate"])
def test_digest_equals_brute_force(kind, K):
    if kind == "uniform":
        R, S = inputs.uniform_pair(1500, 1800, max_extent=2e-2, seed=41)
    elif kind == "zipf":
        R, S = inputs.zipf_pair(1500, 1500, seed=42, rho=0.3)
    else:
        R, S = inputs.degenerate_pair(600, 500, seed=43)
    want = oracle.brute(R, S)
    assert len(want) > 50
    assert oracle.pbsm_digest(R, S, K) == digest(want)
    # and on a sub-window grid (coordinates outside fall into border tiles)
    assert oracle.pbsm_digest(R, S, K, K, 0.25, 0.25, 0.75, 0.75) == digest(want)


def test_digest_sees_changes_not_order():
    R, S = inputs.uniform_pair(2000, 2000, max_extent=2e-2, seed=44)
    p = oracle.brute(R, S)
    d = digest(p)
    rng = np.random.default_rng(0)
    assert digest(p[rng.permutation(len(p))]) == d
    assert combine([digest(p[:100]), digest(p[100:])]) == d
    q = p.copy()
    q[7, 1] += 1
    assert digest(q) != d
    assert digest(p[1:]) != d
    assert digest(np.concatenate([p, p[:1]])) != d
    # a transposed pair list (r and s swapped) differs as well
    assert digest(p[:, ::-1]) != d


def test_chunked_threaded_digest_equals_whole():
    """digest_device (chunks copied to the host and digested by several
    threads, as the full-size GPU tests use it) combines to the digest of the
    whole set, for chunk sizes that do and do not divide the length."""
    torch = pytest.importorskip("torch")
    from pair_digest import digest_device

    rng = np.random.default_rng(5)
    a = rng.integers(0, 1 << 30, (100_003, 2)).astype(np.int32)
    whole = digest(a)
    t = torch.from_numpy(a)
    for chunk in (1 << 10, 4_096, 100_003, 1 << 20):
        assert digest_device(t, chunk=chunk, threads=4) == whole
