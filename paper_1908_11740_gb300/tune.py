"""Autotuner of the join's grid and block size.

Starting point: the rule of Sec. 4.3 -- tiles about ten times the average
rectangle extent (K = 1 / (10 * mean extent) on the unit square).  The
tuner then times joins on the GPU for grids K * f and block sizes b around
that point and keeps the fastest (f, b) per (device, input-size bucket,
extent bucket) in a JSON cache; later joins of the same bucket use it
without measuring.

    from paper_1908_11740_gb300 import tune
    grid, block = tune.tuned(ctx, R, S)            # cached or measured
    grids = tune.tuned_batch(ctx, Rs, Ss)          # one grid per join of a batch
"""
from __future__ import annotations

import json
import math
import os
import time

FACTORS = (0.5, 0.71, 1.0, 1.41, 2.0)
BLOCK_TARGETS = (768, 1536, 3072)
DEFAULT_CACHE = os.environ.get("SJ_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache",
                                                              "sj_tune.json"))


def rule_k(mean_extent: float, kmax: int = 8192) -> int:
    """Tiles about ten times the average extent (Sec. 4.3)."""
    if not mean_extent > 0:
        return kmax
    return int(min(kmax, max(1, round(1.0 / (10.0 * mean_extent)))))


def bucket(n_total: int, mean_extent: float) -> str:
    """Cache key part: powers of two of the input size and of the extent."""
    nb = int(math.floor(math.log2(max(n_total, 1))))
    eb = int(math.floor(math.log2(max(mean_extent, 1e-12))))
    return f"n2^{nb}/e2^{eb}"


def mean_extent(ctx, R, S) -> float:
    from . import sj

    s = sj.sj_extent_stats(ctx, R, S)
    n = 2 * (R.shape[0] + S.shape[0])
    return float(s.sum() / n) if n else 0.0


class Cache:
    def __init__(self, path: str = DEFAULT_CACHE):
        self.path = path
        self.data = {}
        if path and os.path.exists(path):
            try:
                with open(path) as f:
                    self.data = json.load(f)
            except (OSError, ValueError):
                self.data = {}

    def get(self, device: str, key: str):
        return self.data.get(device, {}).get(key)

    def put(self, device: str, key: str, value: dict):
        self.data.setdefault(device, {})[key] = value
        if self.path:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.data, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def _time_join(ctx, R, S, grid, reps=3):
    import torch

    from . import sj

    opts = sj.make_opts("two_pass")
    sj.sj_join(ctx, R, S, grid, opts)          # warm-up (workspace, caches)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        sj.sj_join(ctx, R, S, grid, opts)
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / reps


def measure(ctx, R, S, factors=FACTORS, blocks=BLOCK_TARGETS, reps=3):
    """Time every (factor, block target); returns (best dict, all results)."""
    from . import sj

    m = mean_extent(ctx, R, S)
    k0 = rule_k(m)
    results = []
    for f in factors:
        k = max(1, int(round(k0 * f)))
        for b in blocks:
            sj.sj_set_tuning(ctx, b)
            t = _time_join(ctx, R, S, sj.make_grid(k), reps)
            results.append({"factor": f, "k": k, "block_target": b, "seconds": t})
    sj.sj_set_tuning(ctx, 1536)
    best = min(results, key=lambda r: r["seconds"])
    return {"factor": best["factor"], "block_target": best["block_target"], "rule_k": k0,
            "mean_extent": m}, results


def tuned(ctx, R, S, cache: Cache | None = None, device_name: str | None = None, measure_if_missing=True):
    """(grid, block_target) for joining R and S: cached per bucket, else the
    rule of thumb, measured and cached when measure_if_missing."""
    import torch

    from . import sj

    cache = cache if cache is not None else Cache()
    dev = device_name or torch.cuda.get_device_name(ctx.device)
    m = mean_extent(ctx, R, S)
    key = bucket(R.shape[0] + S.shape[0], m)
    hit = cache.get(dev, key)
    if hit is None and measure_if_missing:
        hit, _ = measure(ctx, R, S)
        cache.put(dev, key, hit)
    f = hit["factor"] if hit else 1.0
    b = hit["block_target"] if hit else 1536
    return sj.make_grid(max(1, int(round(rule_k(m) * f)))), b


def tuned_batch(ctx, Rs, Ss, cache: Cache | None = None, device_name: str | None = None,
                measure_if_missing=True, factors=FACTORS, reps=2):
    """The grid of every join of a batch: the rule of Sec. 4.3 scaled by the
    factor cached for the join's (size, extent) bucket.  A bucket without an
    entry is measured once, on its largest join, over the grid factors (the
    block target of a batch is one for all joins and is not tuned here)."""
    import torch

    from . import sj

    cache = cache if cache is not None else Cache()
    dev = device_name or torch.cuda.get_device_name(ctx.device)
    means = [mean_extent(ctx, R, S) for R, S in zip(Rs, Ss)]
    keys = [bucket(R.shape[0] + S.shape[0], m) for R, S, m in zip(Rs, Ss, means)]
    factor = {}
    for key in sorted(set(keys)):
        hit = cache.get(dev, key)
        if hit is None and measure_if_missing:
            j = max((i for i, k in enumerate(keys) if k == key), key=lambda i: Rs[i].shape[0] + Ss[i].shape[0])
            hit, _ = measure(ctx, Rs[j], Ss[j], factors=factors, blocks=(1536,), reps=reps)
            cache.put(dev, key, hit)
        factor[key] = hit["factor"] if hit else 1.0
    return [sj.make_grid(max(1, int(round(rule_k(m) * factor[k])))) for m, k in zip(means, keys)]
