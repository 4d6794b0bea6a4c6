"""Benchmark of the spatial-join filter step on one GB300 (or N, one process
per GPU, each joining its own independent workload: weak scaling).

Workload: the GIS-shaped plain join, |R| = 10M, |S| = 20M float32 MBRs
(64-component Gaussian mixture + 20% uniform background, log-normal extents
with median 2e-5), on a uniform grid (default 3000 x 3000, the rule of thumb
"tile extent about 10x the average rectangle extent").  A step is one full
join: partition (count, scan, scatter), per-tile sort, sweep, duplicate test
and output, device-resident inputs -> device pair buffer with its count on
the host.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1908_11740_gb300 import dist as sjdist  # noqa: E402
from paper_1908_11740_gb300 import inputs  # noqa: E402

METRIC = "join time and result pairs/s on 1 GB300; learned one-pass vs plain two-pass"
UNIT = "pairs/s"
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", type=int, default=3000)
    ap.add_argument("--mode", default="one_pass",
                    help="one_pass (learned sizing, the headline), two_pass or one_pass_heur")
    ap.add_argument("--model", default=None, help="trained predictor (.npz); default: the packaged one")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the other join modes")
    ap.add_argument("--n-r", type=int, default=10_000_000)
    ap.add_argument("--n-s", type=int, default=20_000_000)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--cpu-frac", type=float, default=0.125,
                    help="CPU sample: rectangles whose centre has y < frac")
    ap.add_argument("--workload", default="gis", choices=["gis", "batch", "skew", "distance", "aniso", "bands", "gbda", "stripes", "link"],
                    help="gis: the 10M x 20M GIS-shaped join (default); batch: 256 joins of uneven size; "
                         "skew: the 20M x 20M Zipf extent / skew stress; aniso: 10M x 20M elongated "
                         "rectangles, sweep along x against the adaptive axis of Sec. 3.3; bands: the gis join "
                         "split into one band of tile rows per rank (the default for gis with N > 1); gbda: "
                         "the gis join with Eq. 1 against GBDA duplicate avoidance; stripes: the gis join on "
                         "1D grids (stripe kernel) against the 2D grid; link: the host link's copy bandwidth "
                         "and a copy running beside a join")
    ap.add_argument("--aniso-grids", default="1750,600",
                    help="aniso: grids to time (1750: the tile-extent rule; 600: coarse tiles)")
    ap.add_argument("--rho", type=float, default=2.1e-4,
                    help="skew: probability that S shares R's hot spots (2.1e-4: about 1e9 pairs)")
    ap.add_argument("--skew-mode", default="one_pass_heur", choices=["one_pass_heur", "two_pass"],
                    help="skew: one pass (small tiles counted, large tiles appended) or the exact two-pass join")
    ap.add_argument("--skew-grid", type=int, default=500,
                    help="skew: tiles per axis (500: fastest of 500-3000 on this workload)")
    ap.add_argument("--split", default="bands", choices=["bands", "instances"],
                    help="gis with N > 1 ranks: bands = one join split into N bands of tile rows balanced by "
                         "entries (strong scaling, each rank stages its band's rectangles); instances = an "
                         "independent join per rank (weak scaling)")
    ap.add_argument("--joins", type=int, default=256)
    ap.add_argument("--batch-grids", default="rule", choices=["rule", "tuned"],
                    help="batch: grids by the rule of Sec. 4.3 or by the measured tuner (tune.tuned_batch)")
    ap.add_argument("--eps", type=float, default=5e-5, help="distance of the eps-distance join")
    ap.add_argument("--dist-grid", type=int, default=2000, help="grid of the eps-distance join")
    return ap.parse_args()


def workload_name(a):
    return (f"GIS-shaped plain join |R|={a.n_r:,} |S|={a.n_s:,} fp32 MBRs, 64-comp Gaussian mixture "
            f"+20% uniform, log-normal extents median 2e-5 sigma 1; grid {a.grid}x{a.grid}")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def load_traffic():
    """ncu DRAM bytes per launch of the dominant kernel, from the committed
    profile summary (None when absent or stale)."""
    p = os.path.join(ROOT, "profiles", "traffic_gis_10Mx20M.txt")
    out = {}
    if os.path.exists(p):
        for line in open(p):
            line = line.split("#")[0].strip()
            if ":" in line:
                k, v = line.split(":", 1)
                try:
                    out[k.strip()] = float(v)
                except ValueError:
                    pass
    return out


class ClockSampler:
    """nvidia-smi SM clock / throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.seek(0)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_sample(R, S, frac):
    """Sub-join of the rectangles whose centre lies in the strip y < frac
    (every tile row of that strip, same tile size as the GPU grid)."""
    r = R[(R[:, 1] + R[:, 3]) * 0.5 < frac]
    s = S[(S[:, 1] + S[:, 3]) * 0.5 < frac]
    return r, s


def run_cpu_oracle(R, S, args, reps=1):
    import oracle

    r, s = cpu_sample(R, S, args.cpu_frac)
    ny = max(1, int(round(args.grid * args.cpu_frac)))
    times, npairs = [], 0
    for _ in range(reps):
        t0 = time.perf_counter()
        p = oracle.pbsm(r, s, args.grid, ny, 0.0, 0.0, 1.0, args.cpu_frac)
        times.append(time.perf_counter() - t0)
        npairs = len(p)
    t = statistics.median(times)
    return {"value": npairs / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"single-threaded oracle PBSM on the strip y<{args.cpu_frac} of the same workload "
                       f"({len(r):,} x {len(s):,} rectangles, {npairs:,} pairs, grid {args.grid}x{ny}), "
                       f"{t:.2f} s per run")}, t


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def run_cpu_parallel(R, S, args, reps=3):
    """The paper's multi-core PBSM (Sec. 3.4, OpenMP) on every host core,
    on the same strip as the oracle's sample: context for the GPU numbers,
    beside the single-core oracle.  Never fails the benchmark."""
    try:
        import oracle

        r, s = cpu_sample(R, S, args.cpu_frac)
        ny = max(1, int(round(args.grid * args.cpu_frac)))
        threads = oracle.parallel_threads()
        oracle.pbsm_parallel(r, s, args.grid, ny, 0.0, 0.0, 1.0, args.cpu_frac, pairs=False)   # warm
        times, npairs = [], 0
        for _ in range(reps):
            t0 = time.perf_counter()
            npairs = oracle.pbsm_parallel(r, s, args.grid, ny, 0.0, 0.0, 1.0, args.cpu_frac, pairs=False)
            times.append(time.perf_counter() - t0)
        t = statistics.median(times)
        return {"value": npairs / t, "unit": UNIT, "cores": threads, "kind": "paper Sec. 3.4 multi-core PBSM (OpenMP)",
                "cpu_model": cpu_model(),
                "sample": f"the oracle's strip ({len(r):,} x {len(s):,} rectangles, {npairs:,} pairs), "
                          f"{t * 1e3:.1f} ms per run on {threads} threads"}
    except Exception as e:  # noqa: BLE001 - a baseline must never break the benchmark
        return {"unavailable": f"{type(e).__name__}: {e}"[:200]}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    R, S = inputs.gis_pair(args.n_r, args.n_s, seed=args.seed)
    for _ in range(args.warmup):
        pass  # the oracle has no warm state; warm-up runs would only burn CPU time
    vals = []
    cb = None
    for _ in range(args.steps):
        cb, t = run_cpu_oracle(R, S, args)
        vals.append(t)
    t = statistics.median(vals)
    value = cb["value"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(args), "grid": args.grid, "sample": cb["sample"]},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# Algorithmic bytes per launch of each single-kernel phase: every input
# rectangle read once (16 B), every stored entry written / read once as the
# 20 B (MBR + id) it carries, every pair written once (8 B).  E is the
# number of entries the kernel's partition level stores in device memory.
def alg_bytes(phase, n_in, E, P):
    return {"count": 16 * n_in, "scatter": 16 * n_in + 20 * E, "sweep_count": 20 * E,
            "sweep_write": 20 * E + 8 * P}.get(phase)


KERNELS = {
    1: {"count": "k_bcount", "scatter": "k_bscatter_shared", "sweep_count": "k_bjoin<COUNT>",
        "sweep_write": "k_bjoin<WRITE>", "sweep_reserve": "k_bjoin<RESERVE>"},
    0: {"count": "k_count", "scatter": "k_scatter", "sweep_count": "k_sweep_chunks<COUNT>",
        "sweep_write": "k_sweep_chunks<WRITE>", "sweep_reserve": "k_sweep_chunks<RESERVE>"},
}


def ours(args):
    import torch

    from paper_1908_11740_gb300 import build, sj

    env = sjdist.setup("nccl")
    world, rank, local = env.world, env.rank, env.local_rank
    torch.cuda.set_device(local)
    build.build()
    # each rank joins its own independent workload (weak scaling)
    R, S = inputs.gis_pair(args.n_r, args.n_s, seed=sjdist.instance_seed(args.seed, env))
    hR = torch.from_numpy(R).pin_memory()
    hS = torch.from_numpy(S).pin_memory()
    dR, dS = hR.cuda(), hS.cuda()
    ctx = sj.sj_create(local)
    grid = sj.make_grid(args.grid)
    model = model_header = None
    if args.mode in ("one_pass", "auto"):
        from paper_1908_11740_gb300 import learn
        model, model_header = learn.load(ctx, args.model or learn.DEFAULT_MODEL)
        sj.sj_set_model(ctx, model)
    opts = sj.make_opts(args.mode)
    stream = torch.cuda.current_stream()

    def timed(o, steps):
        """ms per join over `steps` joins (CUDA events on the stream), phases."""
        for _ in range(max(3, args.warmup)):
            sj.sj_join(ctx, dR, dS, grid, o)
        torch.cuda.synchronize()
        sjdist.barrier(env)
        torch.cuda.synchronize()
        sj.sj_timing_enable(ctx, True)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        npairs = 0
        for _ in range(steps):
            out = sj.sj_join(ctx, dR, dS, grid, o)
            npairs = out.shape[0]
            del out
        ev1.record(stream)
        torch.cuda.synchronize()
        sjdist.barrier(env)
        tm = sj.sj_timing_read(ctx)
        sj.sj_timing_enable(ctx, False)
        return ev0.elapsed_time(ev1) / steps, tm, npairs

    P = sj.sj_join(ctx, dR, dS, grid, sj.make_opts("two_pass")).shape[0]
    last2 = sj.sj_last_stats(ctx)
    path = last2["path"]
    E1 = last2["l1_entries_r"] + last2["l1_entries_s"] if path == 1 else None
    cr, cs, _ = sj.sj_tile_stats(ctx, dR, dS, grid)
    E = int(cr.sum().item()) + int(cs.sum().item())
    del cr, cs
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms, timing, P_main = timed(opts, args.steps)
    clk = clocks.stop()
    assert P_main == P, (P_main, P)
    last = sj.sj_last_stats(ctx)
    compare = {}
    if not args.no_compare:
        for name in ("two_pass", "one_pass_heur"):
            if name == args.mode:
                continue
            cms, ctm, cP = timed(sj.make_opts(name), max(3, args.steps // 2))
            cl = sj.sj_last_stats(ctx)
            compare[name] = {"ms_per_step": cms, "value": cP / (cms / 1e3), "pairs": cP,
                             "capacity": cl["capacity"] if cl["one_pass"] else None,
                             "refit_blocks": cl["refit_items"] if cl["one_pass"] else None}
        if args.mode == "one_pass":
            # the plan's heaviest-first block order against plain block order
            sj.sj_set_schedule(ctx, False)
            cms, ctm, cP = timed(opts, max(3, args.steps // 2))
            sj.sj_set_schedule(ctx, True)
            compare["one_pass_block_order"] = {"ms_per_step": cms, "value": cP / (cms / 1e3), "pairs": cP,
                                               "block_join_ms": round(ctm["sweep_write"][1] / max(3, args.steps // 2), 4)}
    ms, p_all = sjdist.reduce_result(ms, P, env)
    value = p_all / (ms / 1e3)

    # end to end from pinned host buffers: every step copies its inputs to the
    # device, joins and copies its pairs back.  sj_join_host_many runs a
    # sequence of such joins with each input copy overlapping the previous
    # join; sj_join_host (one call per join, copy then join) is timed too.
    hout = torch.empty((P + 1024, 2), dtype=torch.int32).pin_memory()
    e2e_steps = max(3, min(args.steps, 20))
    many = lambda k: sj.sj_join_host_many(ctx, [hR] * k, [hS] * k, [grid] * k, [hout] * k, opts)  # noqa: E731
    many(2)
    sjdist.barrier(env)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    counts = many(e2e_steps)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    e2e_ms, _ = sjdist.reduce_result(e2e_ms, P, env)
    assert counts == [P] * e2e_steps
    for _ in range(2):
        sj.sj_join_host(ctx, hR, hS, grid, hout, opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        res = sj.sj_join_host(ctx, hR, hS, grid, hout, opts)
    torch.cuda.synchronize()
    serial_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    serial_ms, _ = sjdist.reduce_result(serial_ms, P, env)
    assert res.shape[0] == P

    phases = {k: v for k, v in timing.items() if k != "launches" and v[0] > 0}
    n_in = args.n_r + args.n_s
    kern = dict(KERNELS[path])
    if args.mode.startswith("one_pass"):
        kern["sweep_write"] = kern["sweep_reserve"]
    cand = {k: v for k, v in phases.items() if k in kern and k != "sweep_reserve"}
    dom = max(cand, key=lambda k: cand[k][1])
    dom_ms = cand[dom][1] / cand[dom][0]
    ab = alg_bytes(dom, n_in, E1 if path == 1 else E, P)
    peak, peak_kind = load_peaks()
    achieved = ab / (dom_ms / 1e3) / 1e9
    traffic = load_traffic().get(kern[dom])
    b_join = 16 * n_in + 40 * E + 8 * P

    cpu = cpu_par = None
    if rank == 0 and not args.no_cpu:
        cpu, _ = run_cpu_oracle(R, S, args)
        cpu_par = run_cpu_parallel(R, S, args)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(args), "grid": args.grid, "mode": args.mode,
                       "model": (model_header or {}).get("features") if model_header else None,
                       "one_pass_capacity": last["capacity"] if last["one_pass"] else None,
                       "one_pass_refit_blocks": last["refit_items"] if last["one_pass"] else None,
                       "pairs": P, "entries": E, "l1_entries": E1,
                       "path": "two-level (blocks of %d x %d tiles)" % (last["block_side"], last["block_side"])
                       if path == 1 else "single-level",
                       "l2": "inputs 480 MB > 129 MB L2 (no flush needed)",
                       "per_rank": "independent join per GPU, seed 2 + rank"},
            "roofline": {"bound": "hbm", "kernel": kern[dom], "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                         else "fallback 6.8 TB/s", "traffic": traffic,
                         "alg_bytes_per_launch": ab, "launch_ms": dom_ms},
            "join_roofline": {"alg_bytes": b_join, "achieved_gbs": b_join / (ms / 1e3) / 1e9,
                              "frac": b_join / (ms / 1e3) / 1e9 / peak},
            "phases_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in phases.items()},
            "compare": compare,
            "cpu_baseline": cpu,
            "cpu_parallel_baseline": cpu_par,
            "e2e": {"value": p_all / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": 16 * n_in, "d2h_bytes_per_step": 8 * P,
                    "api": f"sj_join_host_many ({e2e_steps} joins from pinned host buffers, each input copy "
                           f"overlapping the previous join)",
                    "serial": {"value": p_all / (serial_ms / 1e3), "ms_per_step": serial_ms,
                               "api": "sj_join_host, one call per join (copy, join, copy back)"}},
            "clocks": clk,
            "gpu_launches": timing["launches"],
        }
        print(json.dumps(line), flush=True)
    sj.sj_set_model(ctx, None)
    if model is not None:
        model.free()
    sj.sj_destroy(ctx)
    sjdist.teardown(env)


def batch_arm(args):
    """256 independent joins (sizes log-uniform in [1e3, 2e6] per side), grids
    by the rule of thumb per join (or the measured tuner, --batch-grids
    tuned).  With N ranks the joins are split into N disjoint shards of about
    equal input size (no data-path collective); each rank joins its shard in
    one batched call.  Total work is fixed as N grows (strong scaling);
    value = all pairs / the slowest rank's time.  Beside it: the phases of the
    same batch launched without graphs (a second context), the algorithmic
    bytes over the HBM peak, and the oracle on a bounded sample of the joins."""
    import torch

    from paper_1908_11740_gb300 import build, sj

    env = sjdist.setup("nccl")
    torch.cuda.set_device(env.local_rank)
    build.build()
    joins = inputs.batch_pairs(n_joins=args.joins)
    mine = sjdist.shard([len(r) + len(s) for r, s in joins], env.rank, env.world)
    Rs = [torch.from_numpy(joins[j][0]).cuda() for j in mine]
    Ss = [torch.from_numpy(joins[j][1]).cuda() for j in mine]
    n_in = sum(len(r) + len(s) for r, s in joins)
    ctx = sj.sj_create(env.local_rank)
    grids = None
    if args.batch_grids == "tuned":
        from paper_1908_11740_gb300 import tune

        grids = tune.tuned_batch(ctx, Rs, Ss, cache=tune.Cache(os.path.join(tempfile.gettempdir(), "sj_tune.json")))
    pairs, offs = sj.sj_join_batch(ctx, Rs, Ss, grids)
    st = sj.sj_last_stats(ctx)
    E1 = st["l1_entries_r"] + st["l1_entries_s"]
    out = torch.empty((int(offs[-1]) + 1, 2), dtype=torch.int32, device="cuda")
    for _ in range(max(3, args.warmup)):
        sj.sj_join_batch(ctx, Rs, Ss, grids, out=out)
    torch.cuda.synchronize()
    clocks = ClockSampler(env.local_rank)
    clocks.start()
    time.sleep(0.3)
    sjdist.barrier(env)
    torch.cuda.synchronize()
    sj.sj_timing_enable(ctx, True)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        sj.sj_join_batch(ctx, Rs, Ss, grids, out=out)
    ev1.record(stream)
    torch.cuda.synchronize()
    sjdist.barrier(env)
    tm = sj.sj_timing_read(ctx)
    clk = clocks.stop()
    ms, P = sjdist.reduce_result(ev0.elapsed_time(ev1) / args.steps, int(offs[-1]), env)
    # one-pass sizing of the whole batch: the learned model and the Eq. 2 estimate
    from paper_1908_11740_gb300 import learn

    model, _ = learn.load(ctx, args.model or learn.DEFAULT_MODEL)
    sj.sj_set_model(ctx, model)
    one = {}
    for name in ("one_pass", "one_pass_heur"):
        o = sj.make_opts(name)
        for _ in range(max(3, args.warmup)):
            sj.sj_join_batch(ctx, Rs, Ss, grids, out=out, opts=o)
        torch.cuda.synchronize()
        sjdist.barrier(env)
        sj.sj_timing_enable(ctx, True)
        ev0.record(stream)
        for _ in range(args.steps):
            sj.sj_join_batch(ctx, Rs, Ss, grids, out=out, opts=o)
        ev1.record(stream)
        torch.cuda.synchronize()
        sjdist.barrier(env)
        tmo = sj.sj_timing_read(ctx)
        sj.sj_timing_enable(ctx, False)
        lo = sj.sj_last_stats(ctx)
        one[name] = {"ms_per_step": ev0.elapsed_time(ev1) / args.steps, "capacity": lo["capacity"],
                     "refit_blocks": lo["refit_items"], "launches": tmo["launches"],
                     "phases_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in tmo.items()
                                            if k != "launches" and v[0]}}
    sj.sj_set_model(ctx, None)
    model.free()
    ms_one, _ = sjdist.reduce_result(one["one_pass"]["ms_per_step"], 0, env)
    # the same batch without graphs: direct launches, phases timed
    os.environ["SJ_BATCH_GRAPHS"] = "0"
    ctx_direct = sj.sj_create(env.local_rank)
    del os.environ["SJ_BATCH_GRAPHS"]
    for _ in range(2):
        sj.sj_join_batch(ctx_direct, Rs, Ss, grids, out=out)
    torch.cuda.synchronize()
    sj.sj_timing_enable(ctx_direct, True)
    ev0.record(stream)
    for _ in range(args.steps):
        sj.sj_join_batch(ctx_direct, Rs, Ss, grids, out=out)
    ev1.record(stream)
    torch.cuda.synchronize()
    tmd = sj.sj_timing_read(ctx_direct)
    ms_direct = ev0.elapsed_time(ev1) / args.steps
    sj.sj_destroy(ctx_direct)
    cpu = None
    if env.rank == 0 and not args.no_cpu:
        import oracle

        t, npairs, nrect, k = 0.0, 0, 0, 0
        for R, S in joins:   # bounded sample: the first joins, about 4M rectangles
            K = int(grids[k].nx) if grids is not None and k < len(grids) else None
            from paper_1908_11740_gb300 import learn

            K = K or learn.grid_rule(R, S)
            t0 = time.perf_counter()
            npairs += len(oracle.pbsm(R, S, K))
            t += time.perf_counter() - t0
            nrect += len(R) + len(S)
            k += 1
            if nrect >= 4_000_000 or t > 20:
                break
        cpu = {"value": npairs / t, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"single-threaded oracle PBSM on the first {k} joins of the batch ({nrect:,} rectangles, "
                         f"{npairs:,} pairs, rule-of-thumb grids), {t:.2f} s"}
    if env.rank == 0:
        peak, _ = load_peaks()
        b_alg = 16 * n_in + 40 * E1 + 8 * P
        line = {"metric": METRIC + " (batched joins)", "value": P / (ms_one / 1e3), "unit": UNIT,
                "n_gpus": env.world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_one,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": f"{args.joins} independent joins, per-side sizes log-uniform in [1e3, 2e6], "
                                       f"uniform / mixture centres, log-normal extents median 1e-4",
                           "rectangles": n_in, "pairs": P, "l1_entries": E1,
                           "grids": "measured tuner per join" if grids is not None else "rule of thumb per join",
                           "mode": "batched learned one-pass (packaged model), direct launches",
                           "one_pass_capacity": one["one_pass"]["capacity"],
                           "one_pass_refit_blocks": one["one_pass"]["refit_blocks"],
                           "sharding": "joins split over ranks by input size, no data-path collective"},
                "join_roofline": {"alg_bytes": b_alg, "alg_bytes_formula": "16 (n_R + n_S) + 40 E1 + 8 P (E1 = L1 "
                                  "entries, a lower bound of the per-tile entries)",
                                  "achieved_gbs": b_alg / (ms_one / 1e3) / 1e9,
                                  "frac": b_alg / (ms_one / 1e3) / 1e9 / peak},
                "gpu_launches": one["one_pass"]["launches"], "clocks": clk,
                "input_gbs": 16 * n_in / (ms_one / 1e3) / 1e9,
                "compare": {"two_pass": {"ms_per_step": ms, "value": P / (ms / 1e3),
                                         "mode": "batched two-pass, CUDA graphs replayed",
                                         "launches": tm["launches"]},
                            "one_pass_heur": one["one_pass_heur"],
                            "one_pass_phases_ms_per_step": one["one_pass"]["phases_ms_per_step"]},
                "direct_launches": {"ms_per_step": ms_direct,
                                    "phases_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in tmd.items()
                                                           if k != "launches" and v[0]}},
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    sj.sj_destroy(ctx)
    sjdist.teardown(env)


def skew_arm(args):
    """Extent / skew stress: |R| = |S| = 20M, Zipf(1.2) centres on a 1024^2
    lattice, R extents U[0, 1e-4], S extents U[0, 1e-3], S sharing R's hot
    spots with probability rho; grid --skew-grid (500 x 500).  Hot lattice cells hold
    millions of entries, so the join runs on the single-level path (global
    segmented radix sort of the large tiles).  By default the one-pass join
    (the small tiles counted, the large tiles' pairs appended after them in
    one examination of their candidates, into an output sized by the small
    tiles' pairs plus one slot per large-tile candidate); the exact two-pass
    join is timed alongside.  The output is 8 bytes per pair (7.7 GB at
    rho = 2.1e-4)."""
    import torch

    from paper_1908_11740_gb300 import build, sj

    env = sjdist.setup("nccl")
    torch.cuda.set_device(env.local_rank)
    build.build()
    R, S = inputs.zipf_pair(20_000_000, 20_000_000, seed=sjdist.instance_seed(3, env), rho=args.rho)
    dR, dS = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
    ctx = sj.sj_create(env.local_rank)
    g = sj.make_grid(args.skew_grid)
    # one pass (small tiles counted, large tiles appended) is the default; the
    # exact two-pass join is timed alongside
    o = sj.make_opts(args.skew_mode)
    for _ in range(max(3, args.warmup)):
        sj.sj_join(ctx, dR, dS, g, o)
    torch.cuda.synchronize()
    clocks = ClockSampler(env.local_rank)
    clocks.start()
    time.sleep(0.3)
    sjdist.barrier(env)
    sj.sj_timing_enable(ctx, True)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(1, min(args.steps, 10))
    ev0.record(stream)
    for _ in range(steps):
        out = sj.sj_join(ctx, dR, dS, g, o)
        P = out.shape[0]
        del out
    ev1.record(stream)
    torch.cuda.synchronize()
    sjdist.barrier(env)
    tm = sj.sj_timing_read(ctx)
    sj.sj_timing_enable(ctx, False)
    clk = clocks.stop()
    st = sj.sj_last_stats(ctx)
    ms, P_all = sjdist.reduce_result(ev0.elapsed_time(ev1) / steps, P, env)
    other = "two_pass" if args.skew_mode != "two_pass" else "one_pass_heur"
    o2 = sj.make_opts(other)
    sj.sj_join(ctx, dR, dS, g, o2)
    torch.cuda.synchronize()
    sj.sj_timing_enable(ctx, True)
    ev0.record(stream)
    for _ in range(steps):
        out = sj.sj_join(ctx, dR, dS, g, o2)
        del out
    ev1.record(stream)
    torch.cuda.synchronize()
    tm2 = sj.sj_timing_read(ctx)
    ms2 = ev0.elapsed_time(ev1) / steps
    if env.rank == 0:
        n_in = 40_000_000
        E = st["entries_r"] + st["entries_s"]
        line = {"metric": METRIC + " (extent / skew stress)", "value": P_all / (ms / 1e3), "unit": UNIT,
                "n_gpus": env.world, "steps": steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": f"Zipf(1.2) skew |R|=|S|=20M, rho={args.rho}, grid {args.skew_grid}x{args.skew_grid}",
                           "pairs": P, "entries": E, "mode": args.skew_mode,
                           "one_pass_capacity": st["capacity"] if st["one_pass"] else None,
                           "path": "single-level" if st["path"] == 0 else "two-level"},
                "compare": {other: {"ms_per_step": ms2, "value": P / (ms2 / 1e3),
                                    "phases_ms_per_step": {k: round(v[1] / steps, 4) for k, v in tm2.items()
                                                           if k != "launches" and v[0]}}},
                "join_roofline": {"alg_bytes": 16 * n_in + 40 * E + 8 * P,
                                  "achieved_gbs": (16 * n_in + 40 * E + 8 * P) / (ms / 1e3) / 1e9},
                "gpu_launches": tm["launches"], "clocks": clk,
                "phases_ms_per_step": {k: round(v[1] / steps, 4) for k, v in tm.items()
                                       if k != "launches" and v[0]}}
        print(json.dumps(line), flush=True)
    sj.sj_destroy(ctx)
    sjdist.teardown(env)


def distance_arm(args):
    """eps-distance join on points (Sec. 1): |P| = 10M, |Q| = 20M points with
    the GIS-shaped mixture distribution, eps = 5e-5, grid 2000 x 2000 (tiles
    about ten times eps).  Squares of side eps, the candidate join (the
    learned one-pass join by default, two-pass timed alongside), binary64
    distance test and ordered compaction, inputs resident.  The oracle (squares,
    PBSM, distance test) is timed on a strip of the same workload."""
    import torch

    from paper_1908_11740_gb300 import build, learn, sj

    env = sjdist.setup("nccl")
    torch.cuda.set_device(env.local_rank)
    build.build()
    P, Q = inputs.gis_points(args.n_r, args.n_s, seed=sjdist.instance_seed(args.seed, env))
    dP, dQ = torch.from_numpy(P).cuda(), torch.from_numpy(Q).cuda()
    ctx = sj.sj_create(env.local_rank)
    model, _ = learn.load(ctx, args.model or learn.DEFAULT_MODEL)
    sj.sj_set_model(ctx, model)
    g = sj.make_grid(args.dist_grid)
    stream = torch.cuda.current_stream()

    def timed(mode, steps):
        o = sj.make_opts(mode)
        for _ in range(max(3, args.warmup)):
            sj.sj_distance_join(ctx, dP, dQ, args.eps, g, o)
        torch.cuda.synchronize()
        sjdist.barrier(env)
        sj.sj_timing_enable(ctx, True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            out, nc = sj.sj_distance_join(ctx, dP, dQ, args.eps, g, o, return_candidates=True)
            npairs = out.shape[0]
            del out
        ev1.record(stream)
        torch.cuda.synchronize()
        sjdist.barrier(env)
        tm = sj.sj_timing_read(ctx)
        sj.sj_timing_enable(ctx, False)
        return ev0.elapsed_time(ev1) / steps, tm, npairs, nc

    clocks = ClockSampler(env.local_rank)
    clocks.start()
    time.sleep(0.3)
    steps = max(1, min(args.steps, 20))
    ms, tm, npairs, ncand = timed(args.mode, steps)
    clk = clocks.stop()
    st = sj.sj_last_stats(ctx)
    cms, _, cP, _ = timed("two_pass", max(3, steps // 2))
    assert cP == npairs
    ms, P_all = sjdist.reduce_result(ms, npairs, env)
    cpu = None
    if env.rank == 0 and not args.no_cpu:
        import oracle

        frac = 0.125
        p = P[P[:, 1] < frac]
        q = Q[Q[:, 1] < frac]
        ny = max(1, int(round(args.dist_grid * frac)))
        t0 = time.perf_counter()
        res = oracle.dist_pbsm(p, q, args.eps, args.dist_grid, ny, 0.0, 0.0, 1.0, frac)
        t = time.perf_counter() - t0
        cpu = {"value": len(res) / t, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"single-threaded oracle (squares, PBSM, distance test) on the strip y<{frac}: "
                         f"{len(p):,} x {len(q):,} points, {len(res):,} pairs, {t:.2f} s"}
    if env.rank == 0:
        n_in = args.n_r + args.n_s
        E = st["l1_entries_r"] + st["l1_entries_s"] if st["path"] == 1 else st["entries_r"] + st["entries_s"]
        b_alg = 8 * n_in + 40 * E + 8 * npairs
        peak, _ = load_peaks()
        line = {"metric": METRIC + " (eps-distance join on points)", "value": P_all / (ms / 1e3), "unit": UNIT,
                "n_gpus": env.world, "steps": steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic",
                "config": {"workload": f"eps-distance join, |P|={args.n_r:,} |Q|={args.n_s:,} mixture points, "
                                       f"eps={args.eps}, grid {args.dist_grid}x{args.dist_grid}",
                           "pairs": npairs, "candidates": ncand, "mode": args.mode,
                           "one_pass_capacity": st["capacity"] if st["one_pass"] else None,
                           "one_pass_refit_blocks": st["refit_items"] if st["one_pass"] else None,
                           "stored_entries": E,
                           "path": "two-level" if st["path"] == 1 else "single-level"},
                "join_roofline": {"alg_bytes": b_alg, "achieved_gbs": b_alg / (ms / 1e3) / 1e9,
                                  "frac": b_alg / (ms / 1e3) / 1e9 / peak},
                "compare": {"two_pass": {"ms_per_step": cms, "value": cP / (cms / 1e3)}},
                "cpu_baseline": cpu, "gpu_launches": tm["launches"], "clocks": clk,
                "phases_ms_per_step": {k: round(v[1] / steps, 4) for k, v in tm.items()
                                       if k != "launches" and v[0]}}
        print(json.dumps(line), flush=True)
    sj.sj_set_model(ctx, None)
    model.free()
    sj.sj_destroy(ctx)
    sjdist.teardown(env)


def bands_arm(args):
    """One GIS-shaped join (10M x 20M, seed 2, grid 3000) split over the N
    ranks by contiguous bands of tile rows balanced by entries per row
    (dist.band_plan).  Each rank stages only the rectangles that overlap its
    band (dist.band_members) on its GPU and joins its band (sj_join_rows,
    learned one-pass): the pairs whose reference tile lies in the band.  The
    union over ranks is the join; no pair moves between ranks.  Strong
    scaling: value = all pairs / the slowest rank's time.  e2e: every step
    copies the band's rectangles from pinned host memory, joins and copies
    the pairs back."""
    import torch

    from paper_1908_11740_gb300 import build, learn, sj

    env = sjdist.setup("nccl")
    torch.cuda.set_device(env.local_rank)
    build.build()
    R, S = inputs.gis_pair(args.n_r, args.n_s, seed=args.seed)
    ctx = sj.sj_create(env.local_rank)
    grid = sj.make_grid(args.grid)
    bands = sjdist.band_plan(sjdist.row_loads(R, S, grid), env.world)
    row0, row1 = bands[env.rank]
    ir, is_ = sjdist.band_members(R, S, grid, row0, row1)
    hR = torch.from_numpy(np.ascontiguousarray(R[ir])).pin_memory()
    hS = torch.from_numpy(np.ascontiguousarray(S[is_])).pin_memory()
    dR, dS = hR.cuda(), hS.cuda()
    model, _ = learn.load(ctx, args.model or learn.DEFAULT_MODEL)
    sj.sj_set_model(ctx, model)
    opts = sj.make_opts(args.mode)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        P = sj.sj_join_rows(ctx, dR, dS, grid, row0, row1, opts).shape[0]
    torch.cuda.synchronize()
    clocks = ClockSampler(env.local_rank)
    clocks.start()
    time.sleep(0.3)
    sjdist.barrier(env)
    torch.cuda.synchronize()
    sj.sj_timing_enable(ctx, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        out = sj.sj_join_rows(ctx, dR, dS, grid, row0, row1, opts)
        del out
    ev1.record(stream)
    torch.cuda.synchronize()
    sjdist.barrier(env)
    tm = sj.sj_timing_read(ctx)
    clk = clocks.stop()
    ms, P_all = sjdist.reduce_result(ev0.elapsed_time(ev1) / args.steps, P, env)
    # end to end: the band's rectangles host -> device, join, pairs -> host
    e2e_steps = max(3, min(args.steps, 20))
    sjdist.barrier(env)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        dR.copy_(hR, non_blocking=True)
        dS.copy_(hS, non_blocking=True)
        host = sj.sj_join_rows(ctx, dR, dS, grid, row0, row1, opts).cpu()
    torch.cuda.synchronize()
    e2e_ms, _ = sjdist.reduce_result((time.perf_counter() - t0) * 1e3 / e2e_steps, P, env)
    assert host.shape[0] == P
    if env.rank == 0:
        line = {"metric": METRIC, "value": P_all / (ms / 1e3), "unit": UNIT, "n_gpus": env.world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": workload_name(args), "grid": args.grid, "mode": args.mode,
                           "split": f"{env.world} bands of tile rows balanced by entries: {bands}",
                           "pairs": P_all, "l2": "inputs 480 MB > 129 MB L2 (no flush needed)"},
                "e2e": {"value": P_all / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
                        "h2d_bytes_per_step": 16 * (len(ir) + len(is_)), "d2h_bytes_per_step": 8 * P,
                        "api": "rank 0's band: copy of its rectangles, sj_join_rows, copy of its pairs"},
                "gpu_launches": tm["launches"], "clocks": clk,
                "phases_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in tm.items()
                                       if k != "launches" and v[0]}}
        print(json.dumps(line), flush=True)
    sj.sj_set_model(ctx, None)
    model.free()
    sj.sj_destroy(ctx)
    sjdist.teardown(env)


def _variant_table(args, env, ctx, dR, dS, grids, variants):
    """ms per join of every (grid, mode, variant) with inputs resident, CUDA
    events on the stream; returns ({name: result}, steps)."""
    import torch

    from paper_1908_11740_gb300 import sj

    stream = torch.cuda.current_stream()
    steps = max(3, min(args.steps, 20))
    results = {}
    for K in grids:
        g = sj.make_grid(K)
        for mode in ("two_pass", "one_pass"):
            for vname, kw in variants:
                o = sj.make_opts(mode, **kw)
                for _ in range(max(3, args.warmup)):
                    sj.sj_join(ctx, dR, dS, g, o)
                torch.cuda.synchronize()
                sjdist.barrier(env)
                sj.sj_timing_enable(ctx, True)
                ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                for _ in range(steps):
                    out = sj.sj_join(ctx, dR, dS, g, o)
                    P = out.shape[0]
                    del out
                ev1.record(stream)
                torch.cuda.synchronize()
                sjdist.barrier(env)
                tm = sj.sj_timing_read(ctx)
                sj.sj_timing_enable(ctx, False)
                st = sj.sj_last_stats(ctx)
                ph = {k: round(v[1] / steps, 4) for k, v in tm.items() if k != "launches" and v[0]}
                results[f"K{K} {mode} {vname}"] = {
                    "launches": tm["launches"],
                    "ms_per_step": round(ev0.elapsed_time(ev1) / steps, 4), "pairs": P,
                    "block_join_ms": ph.get("sweep_write"), "count_pass_ms": ph.get("sweep_count"),
                    "y_sweep_tiles": st["y_sweep_tiles"], "gbda": st["dedup"],
                    "path": "two-level" if st["path"] == 1 else "single-level"}
    return results, steps


def aniso_arm(args):
    """Adaptive sweep axis (Sec. 3.3): |R| = 10M, |S| = 20M rectangles ten
    times longer along one axis than the other (half the mixture components
    wide, half tall), at the grid of the tile-extent rule and at a coarse
    grid.  Every tile swept along x against every tile swept along the axis
    with the smaller Eq. 2 estimate (k = 8 divisions per tile axis), in the
    two-pass and the learned one-pass join; inputs resident."""
    import torch

    from paper_1908_11740_gb300 import build, learn, sj

    env = sjdist.setup("nccl")
    torch.cuda.set_device(env.local_rank)
    build.build()
    R, S = inputs.aniso_pair(args.n_r, args.n_s, seed=sjdist.instance_seed(5, env))
    dR, dS = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
    ctx = sj.sj_create(env.local_rank)
    model, _ = learn.load(ctx, args.model or learn.DEFAULT_MODEL)
    sj.sj_set_model(ctx, model)
    clocks = ClockSampler(env.local_rank)
    clocks.start()
    time.sleep(0.3)
    grids = [int(k) for k in args.aniso_grids.split(",")]
    results, steps = _variant_table(args, env, ctx, dR, dS, grids,
                                    [("x", {"axis": "x"}), ("adaptive", {"axis": "adaptive"})])
    clk = clocks.stop()
    head = results[f"K{grids[0]} one_pass adaptive"]
    ms, P_all = sjdist.reduce_result(head["ms_per_step"], head["pairs"], env)
    if env.rank == 0:
        line = {"metric": METRIC + " (adaptive sweep axis, elongated rectangles)", "value": P_all / (ms / 1e3),
                "unit": UNIT, "n_gpus": env.world, "steps": steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": f"elongated rectangles |R|={args.n_r:,} |S|={args.n_s:,}, aspect 10, "
                                       f"GIS-shaped mixture centres, grid {grids[0]}x{grids[0]}, learned one-pass, "
                                       f"adaptive axis", "pairs": head["pairs"]},
                "compare": results, "gpu_launches": head["launches"], "clocks": clk}
        print(json.dumps(line), flush=True)
    sj.sj_set_model(ctx, None)
    model.free()
    sj.sj_destroy(ctx)
    sjdist.teardown(env)


def stripes_arm(args):
    """1D partitioning (Sec. 3.1): the GIS-shaped 10M x 20M join on vertical
    stripes (K x 1, swept along y) and horizontal stripes (1 x K, swept
    along x) through the stripe kernel, against the 2D grid (3000 x 3000) and
    against the same stripes on the general path (a second context created
    with SJ_STRIPES=0); exact two-pass, inputs resident."""
    import torch

    from paper_1908_11740_gb300 import build, sj

    env = sjdist.setup("nccl")
    torch.cuda.set_device(env.local_rank)
    build.build()
    R, S = inputs.gis_pair(args.n_r, args.n_s, seed=sjdist.instance_seed(args.seed, env))
    dR, dS = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
    ctx = sj.sj_create(env.local_rank)
    os.environ["SJ_STRIPES"] = "0"
    ctx_general = sj.sj_create(env.local_rank)
    del os.environ["SJ_STRIPES"]
    stream = torch.cuda.current_stream()
    steps = max(3, min(args.steps, 20))

    def timed(c, g):
        o = sj.make_opts("two_pass")
        for _ in range(max(3, args.warmup)):
            sj.sj_join(c, dR, dS, g, o)
        torch.cuda.synchronize()
        sjdist.barrier(env)
        sj.sj_timing_enable(c, True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            out = sj.sj_join(c, dR, dS, g, o)
            P = out.shape[0]
            del out
        ev1.record(stream)
        torch.cuda.synchronize()
        sjdist.barrier(env)
        tm = sj.sj_timing_read(c)
        sj.sj_timing_enable(c, False)
        st = sj.sj_last_stats(c)
        return {"ms_per_step": round(ev0.elapsed_time(ev1) / steps, 4), "pairs": P, "launches": tm["launches"],
                "path": {0: "single-level", 1: "two-level", 2: "stripes"}[st["path"]],
                "stored_entries": st["l1_entries_r"] + st["l1_entries_s"] if st["path"] else
                st["entries_r"] + st["entries_s"],
                "phases_ms": {k: round(v[1] / steps, 4) for k, v in tm.items() if k != "launches" and v[0]}}

    clocks = ClockSampler(env.local_rank)
    clocks.start()
    time.sleep(0.3)
    res = {}
    for name, c, (nx, ny) in (("vertical 3000 x 1, stripe kernel", ctx, (3000, 1)),
                              ("vertical 7000 x 1, stripe kernel", ctx, (7000, 1)),
                              ("horizontal 1 x 3000, stripe kernel", ctx, (1, 3000)),
                              ("2D 3000 x 3000", ctx, (3000, 3000)),
                              ("vertical 3000 x 1, general path", ctx_general, (3000, 1)),
                              ("horizontal 1 x 3000, general path", ctx_general, (1, 3000))):
        res[name] = timed(c, sj.make_grid(nx, ny))
    clk = clocks.stop()
    head = res["vertical 7000 x 1, stripe kernel"]
    ms, P_all = sjdist.reduce_result(head["ms_per_step"], head["pairs"], env)
    if env.rank == 0:
        line = {"metric": METRIC + " (1D stripes)", "value": P_all / (ms / 1e3), "unit": UNIT,
                "n_gpus": env.world, "steps": steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": f"GIS-shaped plain join |R|={args.n_r:,} |S|={args.n_s:,}, 7000 vertical "
                                       f"stripes swept along y, two-pass", "pairs": head["pairs"]},
                "compare": res, "gpu_launches": head["launches"], "clocks": clk}
        print(json.dumps(line), flush=True)
    sj.sj_destroy(ctx_general)
    sj.sj_destroy(ctx)
    sjdist.teardown(env)


def link_arm(args):
    """The host link behind the end-to-end numbers: the copy of the GIS-shaped
    join's inputs (480 MB) host -> device from page-locked memory, the copy of
    its pairs back, each alone; then the input copy on a second stream while
    the learned one-pass join runs on the first, against each alone.  CUDA
    events; the copies are single cudaMemcpyAsync calls (torch copy_)."""
    import torch

    from paper_1908_11740_gb300 import build, learn, sj

    env = sjdist.setup("nccl")
    torch.cuda.set_device(env.local_rank)
    build.build()
    R, S = inputs.gis_pair(args.n_r, args.n_s, seed=args.seed)
    hin = torch.from_numpy(np.concatenate([R, S])).pin_memory()
    din = hin.cuda()
    dR, dS = din[:len(R)], din[len(R):]
    ctx = sj.sj_create(env.local_rank)
    model, _ = learn.load(ctx, args.model or learn.DEFAULT_MODEL)
    sj.sj_set_model(ctx, model)
    g = sj.make_grid(args.grid)
    o = sj.make_opts("one_pass")
    pairs = sj.sj_join(ctx, dR, dS, g, o)
    hout = torch.empty(pairs.shape, dtype=pairs.dtype).pin_memory()
    dcopy = torch.empty_like(din)
    main, side = torch.cuda.current_stream(), torch.cuda.Stream()
    steps = max(3, min(args.steps, 20))

    def timed(fn, stream):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    def h2d():
        with torch.cuda.stream(side):
            dcopy.copy_(hin, non_blocking=True)

    def d2h():
        with torch.cuda.stream(side):
            hout.copy_(pairs, non_blocking=True)

    def join():
        out = sj.sj_join(ctx, dR, dS, g, o)
        del out

    h2d_ms, d2h_ms, join_ms = timed(h2d, side), timed(d2h, side), timed(join, main)
    # both at once: the copy on the side stream, the join on the main stream
    for _ in range(2):
        h2d(); join()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev = []
    for _ in range(steps):
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        j0, j1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(side)
        h2d()
        c1.record(side)
        j0.record(main)
        join()
        j1.record(main)
        torch.cuda.synchronize()
        ev.append((c0.elapsed_time(c1), j0.elapsed_time(j1)))
    both_ms = (time.perf_counter() - t0) * 1e3 / steps
    if env.rank == 0:
        nb = hin.numel() * 4
        line = {"metric": "host link: copy bandwidth and copy / join overlap", "value": nb / (h2d_ms / 1e3) / 1e9,
                "unit": "GB/s (host -> device, page-locked)", "n_gpus": env.world, "steps": steps,
                "warmup": 2, "ms_per_step": h2d_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"{nb / 1e6:.0f} MB of inputs of the GIS-shaped join, "
                                       f"{pairs.shape[0]:,} pairs back"},
                "h2d": {"ms": h2d_ms, "gbs": nb / (h2d_ms / 1e3) / 1e9},
                "d2h": {"ms": d2h_ms, "gbs": hout.numel() * 4 / (d2h_ms / 1e3) / 1e9},
                "join_alone_ms": join_ms,
                "together": {"copy_ms": float(np.median([c for c, _ in ev])),
                             "join_ms": float(np.median([j for _, j in ev])),
                             "wall_ms_per_step": both_ms}}
        print(json.dumps(line), flush=True)
    sj.sj_set_model(ctx, None)
    model.free()
    sj.sj_destroy(ctx)
    sjdist.teardown(env)


def gbda_arm(args):
    """Duplicate avoidance: the GIS-shaped 10M x 20M join with the
    reference-point test of Eq. 1 against GBDA (class mini-joins, no test per
    pair), two-pass and learned one-pass, at the rule-of-thumb grid and at a
    coarse grid; inputs resident."""
    import torch

    from paper_1908_11740_gb300 import build, learn, sj

    env = sjdist.setup("nccl")
    torch.cuda.set_device(env.local_rank)
    build.build()
    R, S = inputs.gis_pair(args.n_r, args.n_s, seed=sjdist.instance_seed(args.seed, env))
    dR, dS = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
    ctx = sj.sj_create(env.local_rank)
    model, _ = learn.load(ctx, args.model or learn.DEFAULT_MODEL)
    sj.sj_set_model(ctx, model)
    clocks = ClockSampler(env.local_rank)
    clocks.start()
    time.sleep(0.3)
    grids = [args.grid, 1000]
    results, steps = _variant_table(args, env, ctx, dR, dS, grids,
                                    [("refpoint", {"dedup": "refpoint"}), ("gbda", {"dedup": "gbda"})])
    clk = clocks.stop()
    head = results[f"K{grids[0]} one_pass gbda"]
    ms, P_all = sjdist.reduce_result(head["ms_per_step"], head["pairs"], env)
    if env.rank == 0:
        line = {"metric": METRIC + " (GBDA duplicate avoidance)", "value": P_all / (ms / 1e3),
                "unit": UNIT, "n_gpus": env.world, "steps": steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": workload_name(args) + ", learned one-pass, GBDA", "pairs": head["pairs"]},
                "compare": results, "gpu_launches": head["launches"], "clocks": clk}
        print(json.dumps(line), flush=True)
    sj.sj_set_model(ctx, None)
    model.free()
    sj.sj_destroy(ctx)
    sjdist.teardown(env)


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "batch":
        batch_arm(args)
    elif args.workload == "skew":
        skew_arm(args)
    elif args.workload == "distance":
        distance_arm(args)
    elif args.workload == "aniso":
        aniso_arm(args)
    elif args.workload == "gbda":
        gbda_arm(args)
    elif args.workload == "stripes":
        stripes_arm(args)
    elif args.workload == "link":
        link_arm(args)
    elif args.workload == "bands" or (int(os.environ.get("WORLD_SIZE", "1")) > 1 and args.split == "bands"):
        bands_arm(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
