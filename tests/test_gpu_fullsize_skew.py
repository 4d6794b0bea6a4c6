"""Parity at full size for the extent / skew stress workload: |R| = |S| = 20M,
Zipf(1.2) centres on a 1024^2 lattice, R extents U[0, 1e-4], S extents
U[0, 1e-3], with S sharing R's hot spots with probability rho.  The three
rho values give about 7.2e7, 3e8 and 1e9 result pairs (the result-count
sweep of this workload; rho = 0 is its low end).

The full pair set is too large for the single-threaded oracle in a test, so
the GPU result is checked on what the oracle can compute exactly at this
size, plus properties that hold at any size:

* the pair count equals sj_count, and no pair occurs twice;
* for a sample of R ids and a sample of S ids (random, plus ids in the
  hottest lattice cell), the GPU partners equal the brute-force partners
  over the whole other collection (the definition of Sec. 1);
* in a window around the hottest cell of R, the pairs whose reference point
  (Eq. 1) lies in the window equal those of the oracle PBSM run on the
  rectangles that overlap the window.
"""
import numpy as np
import pytest

import oracle
from paper_1908_11740_gb300 import inputs

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


def hottest_cell(A, lattice=1024):
    cx = np.clip(((A[:, 0] + A[:, 2]) * 0.5 * lattice).astype(np.int64), 0, lattice - 1)
    cy = np.clip(((A[:, 1] + A[:, 3]) * 0.5 * lattice).astype(np.int64), 0, lattice - 1)
    c = int(np.argmax(np.bincount(cy * lattice + cx, minlength=lattice * lattice)))
    return c % lattice, c // lattice


def partners_gpu(pairs, col, ids):
    """Sorted (r, s) rows of the GPU result whose column `col` is in ids."""
    sel = pairs[torch.isin(pairs[:, col], torch.as_tensor(ids, device=pairs.device))]
    a = sel.cpu().numpy()
    return a[np.lexsort((a[:, 1], a[:, 0]))]


@pytest.mark.parametrize("rho", RHOS)
def test_skew_full_size(sj, ctx, rho):
    R, S = inputs.zipf_pair(N, N, seed=3, rho=rho)
    dR, dS = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
    g = sj.make_grid(2000)
    pairs = sj.sj_join(ctx, dR, dS, g, sj.make_opts("two_pass"))
    P = pairs.shape[0]
    assert P == sj.sj_count(ctx, dR, dS, g)
    assert P > 5e7
    # no pair twice
    key = pairs[:, 0].to(torch.int64) * (1 << 32) + pairs[:, 1].to(torch.int64)
    key, _ = torch.sort(key)
    assert int((key[1:] == key[:-1]).sum().item()) == 0
    # the device-sorted output (sort_output) is exactly this set in (r, s) order
    srt = sj.sj_join(ctx, dR, dS, g, sj.make_opts("two_pass", sort_output=True))
    skey = srt[:, 0].to(torch.int64) * (1 << 32) + srt[:, 1].to(torch.int64)
    assert torch.equal(skey, key)
    del key, srt, skey

    rng = np.random.default_rng(17)
    hx, hy = hottest_cell(R)
    lat = 1024.0

    def in_cell(A):
        c = (A[:, 0] + A[:, 2]) * 0.5, (A[:, 1] + A[:, 3]) * 0.5
        return np.flatnonzero((np.floor(c[0] * lat) == hx) & (np.floor(c[1] * lat) == hy))

    # sampled R ids against all of S, sampled S ids against all of R
    r_ids = np.unique(np.concatenate([rng.choice(N, 150, replace=False),
                                      rng.choice(in_cell(R), 50, replace=False)])).astype(np.int32)
    s_ids = np.unique(np.concatenate([rng.choice(N, 150, replace=False),
                                      rng.choice(in_cell(S), min(50, len(in_cell(S))), replace=False)])).astype(np.int32)
    want_r = oracle.brute(R[r_ids], S)
    want_r[:, 0] = r_ids[want_r[:, 0]]
    np.testing.assert_array_equal(partners_gpu(pairs, 0, r_ids), want_r[np.lexsort((want_r[:, 1], want_r[:, 0]))])
    want_s = oracle.brute(R, S[s_ids])
    want_s[:, 1] = s_ids[want_s[:, 1]]
    np.testing.assert_array_equal(partners_gpu(pairs, 1, s_ids), want_s[np.lexsort((want_s[:, 1], want_s[:, 0]))])

    # every pair with its reference point in a window at the hot cell: the
    # 3 x 3 cells around it when S does not share the hot spot, else the
    # central 1/8 x 1/8 of the cell (where S shares it, the whole cell holds
    # most of the 1e8-1e9 pairs)
    if rho == 0.0:
        w0x, w0y, w1x, w1y = (hx - 1) / lat, (hy - 1) / lat, (hx + 2) / lat, (hy + 2) / lat
    else:
        w0x, w0y = (hx + 7 / 16) / lat, (hy + 7 / 16) / lat
        w1x, w1y = (hx + 9 / 16) / lat, (hy + 9 / 16) / lat

    def overlapping(A):
        return np.flatnonzero((A[:, 0] <= w1x) & (A[:, 2] >= w0x) & (A[:, 1] <= w1y) & (A[:, 3] >= w0y))

    ri, si = overlapping(R), overlapping(S)
    sub = oracle.pbsm(R[ri], S[si], 64, 64, np.float32(w0x), np.float32(w0y), np.float32(w1x), np.float32(w1y))
    sub = np.stack([ri[sub[:, 0]], si[sub[:, 1]]], axis=1).astype(np.int64)

    def ref_in_window(pr):
        rx = np.maximum(R[pr[:, 0], 0], S[pr[:, 1], 0])
        ry = np.maximum(R[pr[:, 0], 1], S[pr[:, 1], 1])
        return pr[(rx >= np.float32(w0x)) & (rx < np.float32(w1x)) & (ry >= np.float32(w0y)) & (ry < np.float32(w1y))]

    want_w = ref_in_window(sub)
    ri_t = torch.as_tensor(ri, device="cuda")
    cand = pairs[torch.isin(pairs[:, 0], ri_t)].cpu().numpy().astype(np.int64)
    got_w = ref_in_window(cand)
    want_w = want_w[np.lexsort((want_w[:, 1], want_w[:, 0]))]
    got_w = got_w[np.lexsort((got_w[:, 1], got_w[:, 0]))]
    assert len(want_w) > 1000
    np.testing.assert_array_equal(got_w, want_w)
