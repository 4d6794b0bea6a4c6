"""Parity at full size for the extent / skew stress workload: |R| = |S| = 20M,
Zipf(1.2) centres on a 1024^2 lattice, R extents U[0, 1e-4], S extents
U[0, 1e-3], with S sharing R's hot spots with probability rho.  The three
rho values give about 7.2e7, 3e8 and 1e9 result pairs (the result-count
sweep of this workload; rho = 0 is its low end).

The whole pair set is compared with the oracle's: the single-threaded oracle
PBSM streams its pairs into an order-independent digest (exact count, sum
and xor of a 64-bit mix of every pair, ``oracle.pbsm_digest``), and the GPU
pairs are folded into the same digest on the host, chunk by chunk
(``tests/pair_digest.py``, written independently with numpy).  Beside it: no
pair occurs twice, the count equals sj_count, and the device-sorted output is
exactly the same set in (r, s) order.  The one-pass join of the same input
(small tiles counted, large tiles appended in one examination of their
candidates) gives the same digest."""
import numpy as np
import pytest

import oracle
from paper_1908_11740_gb300 import inputs
from pair_digest import digest_device

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 20_000_000
RHOS = [0.0, 5.2e-5, 2.1e-4]


@pytest.fixture(scope="module")
def sj():
    from paper_1908_11740_gb300 import build, sj as binding

    build.build()
    return binding


@pytest.fixture(scope="module")
def ctx(sj):
    c = sj.sj_create(0)
    yield c
    sj.sj_destroy(c)


@pytest.mark.parametrize("rho", RHOS)
def test_skew_full_size(sj, ctx, rho):
    R, S = inputs.zipf_pair(N, N, seed=3, rho=rho)
    dR, dS = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
    g = sj.make_grid(2000)
    pairs = sj.sj_join(ctx, dR, dS, g, sj.make_opts("two_pass"))
    P = pairs.shape[0]
    assert P > 5e7
    assert P == sj.sj_count(ctx, dR, dS, g)
    got = digest_device(pairs)
    want = oracle.pbsm_digest(R, S, 2000)
    print(f"\nrho {rho}: {P} pairs, digest {got[1]:#x} {got[2]:#x}")
    assert got == want
    # no pair twice
    key = pairs[:, 0].to(torch.int64) * (1 << 32) + pairs[:, 1].to(torch.int64)
    del pairs
    key, _ = torch.sort(key)
    assert int((key[1:] == key[:-1]).sum().item()) == 0
    # the device-sorted output (sort_output) is exactly this set in (r, s) order
    srt = sj.sj_join(ctx, dR, dS, g, sj.make_opts("two_pass", sort_output=True))
    skey = srt[:, 0].to(torch.int64) * (1 << 32) + srt[:, 1].to(torch.int64)
    assert torch.equal(skey, key)
    del srt, skey, key
    one = sj.sj_join(ctx, dR, dS, g, sj.make_opts("one_pass_heur"))
    assert sj.sj_last_stats(ctx)["one_pass"] == 1
    assert digest_device(one) == want
