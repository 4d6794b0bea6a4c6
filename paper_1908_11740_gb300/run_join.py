"""Command-line driver: run joins of a synthetic workload through the C ABI.

    python -m paper_1908_11740_gb300.run_join --workload gis --scale 0.25 --grid 3000 --reps 3

Useful to time or profile one configuration (for example under ncu, whose
kernel filter then selects the launches to capture).  Prints the pair count
and the per-phase device times of the last repetition.
"""
from __future__ import annotations

import argparse
import json

from . import inputs


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="gis", choices=["gis", "uniform", "zipf"])
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the default sizes")
    ap.add_argument("--grid", type=int, default=3000)
    ap.add_argument("--stripes", default=None, choices=["vertical", "horizontal"],
                    help="1D grid of --grid stripes instead of a --grid x --grid grid")
    ap.add_argument("--axis", default="x", choices=["x", "adaptive"])
    ap.add_argument("--dedup", default="refpoint", choices=["refpoint", "gbda"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--mode", default="two_pass")
    ap.add_argument("--rho", type=float, default=0.0)
    ap.add_argument("--model", default=None,
                    help="trained predictor (.npz) for --mode one_pass/auto; default: the packaged one")
    a = ap.parse_args(argv)

    import torch

    from . import build, sj

    build.build()
    if a.workload == "gis":
        R, S = inputs.gis_pair(int(10_000_000 * a.scale), int(20_000_000 * a.scale), seed=2)
    elif a.workload == "zipf":
        R, S = inputs.zipf_pair(int(20_000_000 * a.scale), int(20_000_000 * a.scale), seed=3, rho=a.rho)
    else:
        R, S = inputs.uniform_pair(int(10_000_000 * a.scale), int(10_000_000 * a.scale), seed=1)
    dR, dS = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
    ctx = sj.sj_create(0)
    model = None
    try:
        if a.mode in ("one_pass", "auto"):
            from . import learn
            model, _ = learn.load(ctx, a.model or learn.DEFAULT_MODEL)
            sj.sj_set_model(ctx, model)
        if a.stripes == "vertical":
            g = sj.make_grid(a.grid, 1)
        elif a.stripes == "horizontal":
            g = sj.make_grid(1, a.grid)
        else:
            g = sj.make_grid(a.grid)
        opts = sj.make_opts(a.mode, axis=a.axis, dedup=a.dedup)
        n = 0
        for i in range(a.reps):
            if i == a.reps - 1:
                sj.sj_timing_enable(ctx, True)
            n = sj.sj_join(ctx, dR, dS, g, opts).shape[0]
        t = sj.sj_timing_read(ctx)
        torch.cuda.synchronize()
        print(json.dumps({"pairs": n, "stats": sj.sj_last_stats(ctx),
                          "phases_ms": {k: v[1] for k, v in t.items() if k != "launches" and v[0]}}))
    finally:
        if model is not None:
            sj.sj_set_model(ctx, None)
            model.free()
        sj.sj_destroy(ctx)


if __name__ == "__main__":
    main()
