"""Training of the per-block result-count predictor of the one-pass join.

Samples are the blocks of joins the method itself runs: for each training
join, ``sj_block_features`` returns every block's 32 features and the exact
number of pairs the block reports (the label, as log1p).  The network is
trained on the GPU by the library's own kernels (``sj_mlp_train_step``:
forward, backward of the mean squared error, Adam).

    python -m paper_1908_11740_gb300.learn --out paper_1908_11740_gb300/models/block_pairs_mlp.npz

Training joins: the GIS-shaped layers (seeds 20-27, full size, grids 2000,
3000 and 4000), batched joins of uneven size (seeds 4100+, grid from the
tile-extent rule) and the extent / skew stress workload (20M x 20M, seeds
20-22, rho 0, 5.2e-5 and 2.1e-4, grid 2000).  The features carry no block
size, so the training joins use the grid family the model is applied to.
The skew joins' hottest tiles exceed shared memory, so they run on the
single-level path; their blocks' labels come from its per-tile pair counts
(sj_block_features does this by itself).  After training, the output bias
is shifted so that the summed predicted pairs of the GIS-shaped and batched
training blocks equal their summed exact pairs (regressing log counts
under-estimates sums); the skew blocks, whose sums run to 1e9 pairs, are
left out of that calibration.  Evaluation: a fresh seed (29) of the
GIS-shaped layers at full size.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_MODEL = os.path.join(HERE, "models", "block_pairs_mlp.npz")
FEATURE_VERSION = "eq2-histograms-k8-phi16-overlap-buckets-v1"
N_PARAMS = 6337
F, H1, H2 = 32, 64, 64


def init_params(seed: int, y_mean: float) -> np.ndarray:
    """He-normal weights, zero biases, output bias = mean label."""
    g = np.random.default_rng(seed)
    w1 = g.normal(0.0, np.sqrt(2.0 / F), (H1, F))
    w2 = g.normal(0.0, np.sqrt(2.0 / H1), (H2, H1))
    w3 = g.normal(0.0, np.sqrt(1.0 / H2), H2)
    p = np.concatenate([w1.ravel(), np.zeros(H1), w2.ravel(), np.zeros(H2), w3, [y_mean]])
    assert p.size == N_PARAMS
    return p.astype(np.float32)


def grid_rule(R, S) -> int:
    """Tile extent about 10x the average rectangle extent (Sec. 4.3)."""
    ext = np.concatenate([R[:, 2] - R[:, 0], R[:, 3] - R[:, 1], S[:, 2] - S[:, 0], S[:, 3] - S[:, 1]])
    m = float(np.mean(ext)) if ext.size else 1e-3
    return int(min(8000, max(16, round(1.0 / (10.0 * max(m, 1e-7))))))


SKEW_RHOS = (0.0, 5.2e-5, 2.1e-4)


def training_joins(scale: float = 1.0, n_batch: int = 16, grids=(2000, 3000, 4000), skew: bool = True):
    """(name, R, S, grid, calibrate) of every training join."""
    for seed in range(20, 28):
        R, S = inputs.gis_pair(int(10_000_000 * scale), int(20_000_000 * scale), seed=seed)
        for K in grids:
            yield f"gis seed {seed} K {K}", R, S, K, True
    for j, (R, S) in enumerate(inputs.batch_pairs(n_joins=n_batch, seed0=4100)):
        if len(R) < 2000 or len(S) < 2000:
            continue
        yield f"batch join {j}", R, S, grid_rule(R, S), True
    if skew:
        for seed, rho in zip(range(20, 23), SKEW_RHOS):
            n = int(20_000_000 * scale)
            R, S = inputs.zipf_pair(n, n, seed=seed, rho=rho)
            yield f"skew seed {seed} rho {rho}", R, S, 2000, False


def collect(ctx, joins, verbose=True):
    import torch

    from . import sj

    Xs, Ys, Cs = [], [], []
    for name, R, S, K, cal in joins:
        dR, dS = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
        try:
            X, Y = sj.sj_block_features(ctx, dR, dS, sj.make_grid(K))
        except sj.SJError as e:
            if verbose:
                print(f"skip {name}: {e}")
            continue
        Xs.append(X.clone())
        Ys.append(Y.clone())
        Cs.append(torch.full((X.shape[0],), bool(cal), dtype=torch.bool, device=X.device))
        if verbose:
            print(f"{name}: {X.shape[0]} blocks")
    return torch.cat(Xs), torch.cat(Ys), torch.cat(Cs)


def train(ctx, X, Y, epochs=60, batch=4096, lr=2e-3, seed=0, verbose=True):
    import torch

    from . import sj

    model = sj.Model(ctx, init_params(seed, float(Y.mean().item())))
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = X.shape[0]
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(X.device)
        Xp, Yp = X[perm].contiguous(), Y[perm].contiguous()
        lr_ep = lr * (0.5 * (1 + np.cos(np.pi * ep / epochs)))      # cosine decay
        tot = torch.zeros(1, device=X.device)
        nb = 0
        for i in range(0, n, batch):
            xb, yb = Xp[i:i + batch], Yp[i:i + batch]
            if xb.shape[0] < 2:
                continue
            tot += model.train_step(xb, yb, max(lr_ep, 1e-5))
            nb += 1
        hist.append(float((tot / max(nb, 1)).item()))
        if verbose and (ep % 10 == 0 or ep == epochs - 1):
            print(f"epoch {ep}: mse {hist[-1]:.4f}")
    return model, hist


def calibrate(model, X, Y):
    """Shift the output bias so that sum(expm1(pred)) == sum(expm1(Y)) on
    (X, Y); returns the shift (natural log)."""
    import torch

    pred = model.forward(X).double()
    want = torch.expm1(Y.double()).sum() + Y.shape[0]
    have = torch.exp(pred).sum()
    delta = float(torch.log(want / have).item())
    p = model.get_params()
    p[N_PARAMS - 1] += delta
    model.set_params(p)
    return delta


def save(model, path, header: dict):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    p = model.get_params()
    np.savez(path, params=p, header=json.dumps(header))


def load(ctx, path=DEFAULT_MODEL):
    from . import sj

    d = np.load(path, allow_pickle=False)
    header = json.loads(str(d["header"]))
    if header.get("features") != FEATURE_VERSION:
        raise ValueError(f"model features {header.get('features')} != {FEATURE_VERSION}")
    return sj.Model(ctx, d["params"]), header


def sizing_report(ctx, model, R, S, K, margin=0.25):
    """Capacity / exact pairs of the one-pass join with the model and with
    the Eq. 2 estimate, and their re-run block counts."""
    import torch

    from . import sj

    dR, dS = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
    g = sj.make_grid(K)
    out = {}
    for name, mode in (("learned", "one_pass"), ("eq2", "one_pass_heur")):
        if mode == "one_pass":
            sj.sj_set_model(ctx, model)
        P = sj.sj_join(ctx, dR, dS, g, sj.make_opts(mode, margin=margin)).shape[0]
        st = sj.sj_last_stats(ctx)
        out[name] = {"pairs": P, "capacity": st["capacity"], "ratio": st["capacity"] / max(P, 1),
                     "refit_blocks": st["refit_items"], "blocks": st["work_items"]}
    sj.sj_set_model(ctx, None)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_MODEL)
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--eval-seed", type=int, default=29)
    ap.add_argument("--no-skew", action="store_true", help="leave the skew stress joins out of training")
    a = ap.parse_args(argv)

    import torch

    from . import build, sj

    build.build()
    ctx = sj.sj_create(0)
    t0 = time.time()
    X, Y, C = collect(ctx, training_joins(a.scale, skew=not a.no_skew))
    t1 = time.time()
    model, hist = train(ctx, X, Y, epochs=a.epochs)
    delta = calibrate(model, X[C].contiguous(), Y[C].contiguous())
    torch.cuda.synchronize()
    t2 = time.time()
    R, S = inputs.gis_pair(seed=a.eval_seed)
    Xe, Ye = sj.sj_block_features(ctx, torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda(), sj.make_grid(3000))
    pe = model.forward(Xe)
    mae = float((pe - Ye).abs().mean().item())
    rep = sizing_report(ctx, model, R, S, 3000)
    header = {"features": FEATURE_VERSION, "arch": "32-64-64-1 relu, bf16 weights, fp32 accumulate",
              "train_samples": int(X.shape[0]), "train_mse": hist[-1], "epochs": a.epochs,
              "train_joins": ("gis seeds 20-27 at scale %g, grids 2000/3000/4000; batch joins seeds 4100-4115" % a.scale)
              + ("" if a.no_skew else "; skew 20M x 20M seeds 20-22, rho %s, grid 2000" % (SKEW_RHOS,)),
              "train_skew_samples": int((~C).sum().item()),
              "calibrated_on": "gis and batch blocks",
              "bias_calibration": delta,
              "eval": {"workload": "gis 10M x 20M seed %d grid 3000" % a.eval_seed, "block_mae_log1p": mae,
                       "sizing": rep},
              "seconds": {"collect": t1 - t0, "train": t2 - t1}}
    save(model, a.out, header)
    print(json.dumps(header, indent=1))
    model.free()
    sj.sj_destroy(ctx)


if __name__ == "__main__":
    main()
