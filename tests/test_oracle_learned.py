"""Pins of the learned-part oracle (oracle/learned.py), CPU only.

* gradients of the float64 network against central finite differences;
* closed forms: zero weights (output = b3, dL/db3 = 2 mean(b3 - y), all
  other gradients zero) and the all-positive regime where the ReLU network
  is the linear map W3 W2 W1 x + ...;
* block features against hand-counted buckets on a tiny instance, and the
  block labels against the pairs of a brute-force join;
* the Eq. 2 estimate against brute-force counts of x- (y-) intersecting
  pairs: equal where every projection is a bucket centre, above otherwise.
"""
import numpy as np

import oracle
import oracle.learned as L
from paper_1908_11740_gb300 import inputs


def _params(seed, scale=0.3):
    g = np.random.default_rng(seed)
    return g.normal(0.0, scale, L.PARAMS)


def test_gradient_matches_finite_differences():
    g = np.random.default_rng(1)
    X = g.normal(0, 1, (7, L.FEAT))
    Y = g.normal(0, 1, 7)
    p = _params(2)
    loss, grad = L.mlp_loss_grad(p, X, Y)
    idx = np.concatenate([g.choice(L.PARAMS, 60, replace=False), [L.OFF_B3, L.OFF_W3, L.OFF_B1, L.OFF_B2]])
    h = 1e-6
    for i in idx:
        e = np.zeros(L.PARAMS)
        e[i] = h
        num = (L.mlp_loss_grad(p + e, X, Y)[0] - L.mlp_loss_grad(p - e, X, Y)[0]) / (2 * h)
        assert abs(num - grad[i]) <= 1e-6 * max(1.0, abs(num)), (i, num, grad[i])
    assert np.isclose(loss, np.mean((L.mlp_forward(p, X) - Y) ** 2))


def test_zero_weights_closed_form():
    p = np.zeros(L.PARAMS)
    p[L.OFF_B3] = 0.7
    X = np.random.default_rng(3).normal(0, 1, (5, L.FEAT))
    Y = np.arange(5.0)
    loss, grad = L.mlp_loss_grad(p, X, Y)
    assert np.allclose(L.mlp_forward(p, X), 0.7)
    assert np.isclose(loss, np.mean((0.7 - Y) ** 2))
    assert np.isclose(grad[L.OFF_B3], 2 * np.mean(0.7 - Y))
    # dL/dW3 is h2 = 0; every other gradient is zero because the ReLUs are closed
    assert np.allclose(np.delete(grad, L.OFF_B3), 0.0)


def test_linear_regime_closed_form():
    g = np.random.default_rng(4)
    W1 = g.uniform(0.1, 1, (L.H1, L.FEAT))
    W2 = g.uniform(0.1, 1, (L.H2, L.H1))
    W3 = g.uniform(-1, 1, L.H2)
    b1, b2, b3 = g.uniform(0, 1, L.H1), g.uniform(0, 1, L.H2), 0.3
    p = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3, [b3]])
    X = g.uniform(0, 1, (6, L.FEAT))           # all pre-activations positive
    want = ((X @ W1.T + b1) @ W2.T + b2) @ W3 + b3
    assert np.allclose(L.mlp_forward(p, X), want)
    # in that regime dL/dW1 = sum_n d_out_n (W3 W2)^T x_n^T
    Y = np.zeros(6)
    _, grad = L.mlp_loss_grad(p, X, Y)
    d_out = 2 * want / 6
    gW1 = np.outer(W3 @ W2, d_out @ X)
    assert np.allclose(grad[L.OFF_W1:L.OFF_B1].reshape(L.H1, L.FEAT), gW1)


def test_block_features_hand_counted():
    # 8 x 8 grid, blocks of 4 x 4 tiles (2 x 2 blocks); unit 1/64, exact.
    u = 1.0 / 64
    R = np.array([[1, 1, 2, 2], [9, 1, 30, 5], [40, 40, 41, 41]], np.float64) * u
    S = np.array([[0, 0, 20, 3], [33, 33, 60, 60], [5, 5, 6, 6], [10, 1, 12, 2]], np.float64) * u
    R, S = R.astype(np.float32), S.astype(np.float32)
    f = L.block_features(R, S, 8, 8, 4, phi=1)
    # Blocks are 4 tiles wide, so tile column c covers buckets 2c and 2c + 1.
    # block 0 (tiles 0-3 x 0-3): R0 (col 0, row 0), R1 (cols 1-3, row 0);
    # S0 (cols 0-2, row 0), S2 (col 0, row 0), S3 (col 1, row 0).
    hx_r = np.array([1, 1, 1, 1, 1, 1, 1, 1.0])           # R0: 0-1, R1: 2-7
    hy_r = np.array([2, 2, 0, 0, 0, 0, 0, 0.0])           # both in row 0: buckets 0-1
    hx_s = np.array([2, 2, 2, 2, 1, 1, 0, 0.0])           # S0: 0-5, S2: 0-1, S3: 2-3
    hy_s = np.array([3, 3, 0, 0, 0, 0, 0, 0.0])
    want = np.log1p(np.concatenate([hx_r, hy_r, hx_s, hy_s]))
    np.testing.assert_allclose(f[0], want)
    # block 3 (tiles 4-7 x 4-7): R2 (col 5, row 5 -> local 1), S1 (cols/rows 4-7 -> local 0-3)
    assert set(f) == {0, 3}
    r = np.array([0, 0, 1, 1, 0, 0, 0, 0.0])
    sfull = np.ones(8)
    want3 = np.log1p(np.concatenate([r, r, sfull, sfull]))
    np.testing.assert_allclose(f[3], want3)
    # sampling: with phi = 2 only rectangles 0, 2 of each side feed the
    # histograms, scaled by (exact entries / sampled entries)
    f2 = L.block_features(R, S, 8, 8, 4, phi=2)
    # block 0, R side: sampled R0 only (R1 has index 1), 2 exact entries
    np.testing.assert_allclose(f2[0][0:8], np.log1p(np.array([1, 1, 0, 0, 0, 0, 0, 0.0]) * 2 / 1))
    # block 0, S side: sampled S0 and S2 (indices 0 and 2), 3 exact entries
    np.testing.assert_allclose(f2[0][16:24], np.log1p(np.array([2, 2, 1, 1, 1, 1, 0, 0.0]) * 3 / 2))


def test_block_labels_sum_to_the_join():
    R, S = inputs.uniform_pair(2000, 2500, max_extent=0.03, seed=7)
    lab = L.block_labels(R, S, 40, 40, 8)
    assert sum(lab.values()) == len(oracle.brute(R, S))


def _x_overlaps(R, S, axis):
    lo, hi = (0, 2) if axis == 0 else (1, 3)
    return int(((R[:, None, lo] <= S[None, :, hi]) & (S[None, :, lo] <= R[:, None, hi])).sum())


def test_eq2_estimate_counts_bucket_sharing_pairs():
    """Eq. 2 (Sec. 3.3): I_x = sum_i |R_i^x| |S_i^x| counts the (r, s) pairs
    sharing an x bucket, an upper bound on the pairs whose x-projections
    intersect.  On one block of 8 x 8 tiles (bucket i = tile column i) with
    every rectangle of zero width at a bucket centre, two x-projections
    intersect exactly when they share the bucket, so I_x equals the
    brute-force count of x-intersecting pairs; zero-height rectangles pin I_y
    alike; for general rectangles inside the block I_x and I_y bound the
    brute-force counts from above."""
    g = np.random.default_rng(7)
    n_r, n_s = 40, 55

    def segments(n, axis):
        c = (g.integers(0, 8, n) + 0.5) / 8.0
        lo = g.uniform(0.0, 0.9, n)
        hi = np.minimum(lo + g.uniform(0.0, 0.3, n), 0.999)
        a = np.empty((n, 4))
        if axis == 0:   # zero width at bucket centres, random y extent
            a[:, 0] = a[:, 2] = c
            a[:, 1], a[:, 3] = lo, hi
        else:
            a[:, 1] = a[:, 3] = c
            a[:, 0], a[:, 2] = lo, hi
        return a.astype(np.float32)

    for axis in (0, 1):
        R, S = segments(n_r, axis), segments(n_s, axis)
        f = L.block_features(R, S, 8, 8, 8, phi=1)
        assert list(f) == [0]
        ix, iy = L.eq2_estimate(f[0][None, :])
        est = (ix if axis == 0 else iy)[0]
        assert np.isclose(est, _x_overlaps(R, S, axis), rtol=1e-12)
        other = (iy if axis == 0 else ix)[0]
        assert other >= _x_overlaps(R, S, 1 - axis) - 1e-9

    R, S = inputs.uniform_pair(60, 70, max_extent=0.3, seed=8)
    R, S = np.clip(R, 0.0, 0.999).astype(np.float32), np.clip(S, 0.0, 0.999).astype(np.float32)
    f = L.block_features(R, S, 8, 8, 8, phi=1)
    ix, iy = L.eq2_estimate(f[0][None, :])
    assert ix[0] >= _x_overlaps(R, S, 0) - 1e-9 and iy[0] >= _x_overlaps(R, S, 1) - 1e-9
    assert ix[0] > 0 and iy[0] > 0
