"""TEST INFRASTRUCTURE: float64 oracle of the learned result-count predictor.

* ``block_features`` -- the per-block Eq. 2 histograms (Sec. 3.3) with k = 8
  buckets over a block of G x G tiles, from a sample of one rectangle of
  every ``phi`` of each side (the sampling of Sec. 3.3), scaled to the
  block's exact entry count; features = log1p.  Local tile column c of a
  block G tiles wide spans [8c/G, 8(c+1)/G) in bucket units, so columns
  l0..l1 overlap buckets floor(8 l0 / G) .. floor((8 (l1 + 1) - 1) / G).
* ``block_labels`` -- the exact number of pairs each block reports, from the
  per-tile counts of the PBSM oracle (a block reports the pairs of its tiles).
* ``mlp_forward`` / ``mlp_loss_grad`` -- the 32 -> 64 -> 64 -> 1 ReLU network
  and the gradient of its mean squared error, written out layer by layer in
  float64 (backpropagation = the chain rule applied to each layer).
* ``eq2_estimate`` -- the non-learned estimate from the same histograms.

Only tests and the benchmark's CPU leg may use this module.
"""
from __future__ import annotations

import numpy as np

import oracle

FEAT, H1, H2, BINS = 32, 64, 64, 8
OFF_W1 = 0
OFF_B1 = OFF_W1 + H1 * FEAT
OFF_W2 = OFF_B1 + H1
OFF_B2 = OFF_W2 + H2 * H1
OFF_W3 = OFF_B2 + H2
OFF_B3 = OFF_W3 + H2
PARAMS = OFF_B3 + 1


def _blocks_of(c, G):
    return c[:, 0] // G, c[:, 1] // G, c[:, 2] // G, c[:, 3] // G


def block_counts(A, nx, ny, G):
    """Entries per block (a rectangle counts once in every block it
    overlaps); int64[BY*BX]."""
    bx_n, by_n = -(-nx // G), -(-ny // G)
    c = oracle.cells(A, nx, ny)
    bx0, bx1, by0, by1 = _blocks_of(c, G)
    out = np.zeros(bx_n * by_n, np.int64)
    for i in range(len(A)):
        for by in range(by0[i], by1[i] + 1):
            out[by * bx_n + bx0[i]: by * bx_n + bx1[i] + 1] += 1
    return out


def block_features(R, S, nx, ny, G, phi=16):
    """dict block id -> float64[32] features, for blocks holding both sides."""
    bx_n, by_n = -(-nx // G), -(-ny // G)
    nb = bx_n * by_n
    counts = [block_counts(R, nx, ny, G), block_counts(S, nx, ny, G)]
    raw = np.zeros((nb, 2, 2, BINS), np.int64)     # block, side, axis, bucket
    samp = np.zeros((nb, 2), np.int64)
    for side, A in enumerate((R, S)):
        c = oracle.cells(A, nx, ny)
        for i in range(0, len(A), phi):             # rectangles 0, phi, 2 phi, ...
            cx0, cx1, cy0, cy1 = (int(v) for v in c[i])
            for by in range(cy0 // G, cy1 // G + 1):
                for bx in range(cx0 // G, cx1 // G + 1):
                    b = by * bx_n + bx
                    lx0, lx1 = max(cx0 - bx * G, 0), min(cx1 - bx * G, G - 1)
                    ly0, ly1 = max(cy0 - by * G, 0), min(cy1 - by * G, G - 1)
                    # column c covers [8c/G, 8(c+1)/G) in bucket units
                    raw[b, side, 0, lx0 * BINS // G: ((lx1 + 1) * BINS - 1) // G + 1] += 1
                    raw[b, side, 1, ly0 * BINS // G: ((ly1 + 1) * BINS - 1) // G + 1] += 1
                    samp[b, side] += 1
    out = {}
    for b in range(nb):
        if counts[0][b] == 0 or counts[1][b] == 0:
            continue
        f = np.zeros(FEAT)
        for side in range(2):
            n = float(counts[side][b])
            for axis in range(2):
                if samp[b, side]:
                    h = raw[b, side, axis] * n / samp[b, side]
                else:
                    h = np.full(BINS, n / 8.0)
                f[side * 16 + axis * 8: side * 16 + axis * 8 + 8] = np.log1p(h)
        out[b] = f
    return out


def block_labels(R, S, nx, ny, G):
    """dict block id -> exact pairs reported by the block's tiles."""
    bx_n = -(-nx // G)
    _, info = oracle.pbsm(R, S, nx, ny, per_tile=True)
    tp = info["pairs"]
    t = np.arange(nx * ny)
    blk = (t // nx // G) * bx_n + (t % nx) // G
    per = np.bincount(blk, weights=tp, minlength=bx_n * (-(-ny // G))).astype(np.int64)
    return {b: int(per[b]) for b in range(len(per))}


def unpack(params):
    p = np.asarray(params, np.float64)
    W1 = p[OFF_W1:OFF_B1].reshape(H1, FEAT)
    b1 = p[OFF_B1:OFF_W2]
    W2 = p[OFF_W2:OFF_B2].reshape(H2, H1)
    b2 = p[OFF_B2:OFF_W3]
    W3 = p[OFF_W3:OFF_B3]
    b3 = p[OFF_B3]
    return W1, b1, W2, b2, W3, b3


def mlp_forward(params, X):
    """float64 outputs of the network for rows X[n, 32]."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    X = np.asarray(X, np.float64)
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ W3 + b3


def mlp_loss_grad(params, X, Y):
    """(loss, grad[PARAMS]) of mean((f(X) - Y)^2), float64."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    n = len(X)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    out = h2 @ W3 + b3
    err = out - Y
    loss = float(np.mean(err * err))
    d_out = 2.0 * err / n                         # d loss / d out
    g_W3 = h2.T @ d_out
    g_b3 = d_out.sum()
    d_z2 = np.outer(d_out, W3) * (z2 > 0)         # d loss / d z2
    g_W2 = d_z2.T @ h1
    g_b2 = d_z2.sum(0)
    d_z1 = (d_z2 @ W2) * (z1 > 0)                 # d loss / d z1
    g_W1 = d_z1.T @ X
    g_b1 = d_z1.sum(0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_W3, [g_b3]])
    return loss, g


def eq2_estimate(feat):
    """(I_x, I_y) of every row of block features: I_x = sum_i H_R^x[i] H_S^x[i]
    (Eq. 2), the pairs that share an x bucket (an upper bound on the pairs
    whose x-projections intersect), and I_y alike.  The sizing estimate of a
    block is I_x I_y / (n_R n_S) (x and y taken as independent); the cheaper
    sweep axis of a block is the one with the smaller estimate (Sec. 3.3)."""
    h = np.expm1(np.asarray(feat, np.float64))
    ix = (h[:, 0:8] * h[:, 16:24]).sum(1)
    iy = (h[:, 8:16] * h[:, 24:32]).sum(1)
    return ix, iy
