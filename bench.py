"""Benchmark of the lensing remap on the Nside 4096, spin-2, K=32 workload.

One step lenses one batch of 2^24 consecutive RING targets (a twelfth of the
sky) of an Nside 4096 Q/U map resident in HBM; successive steps walk around
the sky.  ``value`` is the mixed-precision path's throughput (points/s, whole
job over all ranks); the FP64 path is timed on the same batches for the
mixed-vs-FP64 ratio.  Inputs are larger than L2 (3.2 GB map, 268 MB of
deflections per step), so no L2 flush is needed.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) the sky is split into contiguous RING ranges, one per
rank, and every rank lenses batches of its own range of the replicated map
(weak scaling, no collective on the data path); timings are bracketed by
barriers and the maximum over ranks is reported by rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402

METRIC = "lensed pts/s at Nside 4096 spin-2 K=32, mixed vs FP64 @2e-4 rel err; p50/p99 ms"
# DRAM bytes (read + write) per target of the mixed spin-2 K=32 kernel a plan call launches
# (batch_kernel<1,2,32>), from the ncu capture of `bench.py --profile-case mixed` (13.866 MB for
# 2^18 targets; profiles/batch_kernel_c3_full_sets.md), scaled to a launch by its target count
MIXED_DRAM_BYTES_PER_POINT = 13.865984e6 / (1 << 18)
# warp instructions per target of the same kernel in the same capture (6.717 G for 2^18 targets):
# with the measured point rate, the issue rate against 4 sub-partitions x 152 SMs x 2.07 GHz
MIXED_WARP_INSTR_PER_POINT = 6.716570991e9 / (1 << 18)
ISSUE_PEAK_PER_S = 4 * 152 * 2.07e9
BATCH = 1 << 24
W = wl.C3


def _hbm_peak_gbs() -> float:
    """Measured copy bandwidth of the GB300s (MEASURED_PEAKS.json, hbm_gbs) when the
    file is present, else the profiling recipe's fallback of 6.8 TB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


HBM_PEAK_GBS = _hbm_peak_gbs()
# where the nvidia-smi clock samples of the timed regions are written
OUT_DIR = os.environ.get("FLINTS_BENCH_OUT", "/tmp")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", choices=["c3", "c3aug", "c4", "c5", "ss", "pipeline", "spin1", "paper"],
                    default="c3",
                    help="c3: Nside 4096 spin 2 (default); c3aug: the same with the augmented (xi+, xi-) "
                         "estimator; c4: 64-map batched persistent launch; c5: serving; ss: supersampling "
                         "Nside 2048 -> 4096; pipeline: synthesis of T, Q/U and the deflection + lensing; "
                         "spin1: a deflection field (spin 1) lensed at Nside 4096; paper: the 9/36-pixel stencil "
                         "with tabulated inverses (lensing at 4096, supersampling 2048 -> 4096)")
    ap.add_argument("--duration", type=float, default=45.0, help="c5: seconds of Poisson arrivals")
    ap.add_argument("--serving-seconds", type=float, default=15.0,
                    help="c3: seconds of the Poisson serving leg appended to the run (0: none)")
    ap.add_argument("--profile-case", choices=["mixed", "fp64", "paper1", "paper2", "paper1m", "paper2m", "paper2q", "paper2qm"], default=None,
                    help="small case for ncu: two launches on 2^18 targets of the resident c3 map (mixed, "
                         "fp64), or on 2^20 targets of the tabulated-inverse route at level 1 or 2 (m: mixed; q: "
                         "spin-2 Q/U)")
    return ap.parse_args()


def run_profile_case_paper(y: int, precision: str = "fp64", spin: int = 0):
    """Two launches of the tabulated-inverse apply kernel (Nside 4096 lensing, level y;
    spin 0 T or spin 2 Q/U) on 2^20 targets of a ring band (the second one is the one
    to capture)."""
    import torch

    import paper_1003_4984_gb300 as fl

    fl.load_library()
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev)
    g.manual_seed(8)
    n = 1 << 20
    nside = 4096
    m = torch.randn((12 * nside * nside, 2) if spin else (12 * nside * nside,), dtype=torch.float64, device=dev,
                    generator=g)
    defl = torch.randn((n, 2), dtype=torch.float64, device=dev, generator=g) * wl.DEFLECTION_RMS
    if spin:
        cl_ee, cl_bb = W.cl()
        plan = fl.PaperPlan(nside, cl_ee, y, precision, spin=2, cl_bb=cl_bb)
    else:
        plan = fl.PaperPlan(nside, wl.cl_tt(4096, 2500.0), y, precision)
    for _ in range(2):
        out, var = plan.lens(m, defl, first=100_000_000, count=n)
    torch.cuda.synchronize()
    info = plan.info()
    assert info["window"] == 0 and info["failed_slots"] == 0, info
    print(json.dumps({"profile_case": f"paper_y{y}_{precision}_spin{spin}", "points": n, "K": info["K"]}))


def run_profile_case(precision: str):
    """Two launches of the c3 lens kernel on 2^18 targets (the second one is the one to capture)."""
    import torch

    import paper_1003_4984_gb300 as fl

    if precision.startswith("paper"):
        return run_profile_case_paper(int(precision[5]), "mixed" if precision.endswith("m") else "fp64",
                                      2 if "q" in precision else 0)
    fl.load_library()
    cl, bb = W.cl()
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    n = 1 << 18
    qu = torch.randn((W.npix, 2), dtype=torch.float64, device=dev, generator=g)
    defl = torch.randn((n, 2), dtype=torch.float64, device=dev, generator=g) * (wl.DEFLECTION_RMS / math.sqrt(2))
    out = torch.empty((n, 2), dtype=torch.float64, device=dev)
    var = torch.empty(n, dtype=torch.float64, device=dev)
    plan = fl.Plan(W.nside, cl, bb, spin=2, K=W.K, precision=precision)
    for _ in range(2):
        plan.lens(qu, defl, out, var, first=100_000_000, count=n)
    torch.cuda.synchronize()
    st = plan.stats()
    assert st["failed"] == 0, st
    print(json.dumps({"profile_case": precision, "points": n, "stats": st}))


def config(n_gpus):
    return {"workload": "c3: spin-2 Q/U, Nside 4096 (201,326,592 px), lmax 4096, C_l^EE = 0.05 x C_l^TT shape "
                        "(damping l = 2500), B = 0, K = 32",
            "batch_points": BATCH, "npix": W.npix, "nside": W.nside, "lmax": W.lmax, "K": W.K, "spin": 2,
            "l2": "inputs larger than L2 (3.2 GB resident map, 268 MB deflections per step)",
            "parallelism": f"{n_gpus} rank(s): one sky split into contiguous RING ranges balanced by count, one "
                           f"per rank, source map replicated, no data-path collective (weak: 2^24 targets per "
                           f"rank per step)"}


# ------------------------------------------------------------ CPU oracle leg
def _oracle_worker(args):
    first, count, seed, aug = args
    sys.path.insert(0, ROOT)
    from oracle import kriging as kr
    from oracle import xi

    cl, bb = W.cl()
    t_max, n = xi.grid_rule(np.abs(cl) + np.abs(bb), W.K, W.nside)
    if (t_max, n) not in _TABLE_CACHE:
        _TABLE_CACHE[(t_max, n)] = xi.spin2_tables(cl, bb, t_max, n)
    tp, tm, x0 = _TABLE_CACHE[(t_max, n)]
    pix = np.arange(first, first + count)
    defl = wl.random_deflection(count, seed + first)
    qu = wl.HashedMap(W.npix, 6, 2)
    t0 = time.time()
    kr.lens(W.nside, W.K, 2, qu, defl, pix, tp, x0, f_minus=tm if aug else None)
    return count, time.time() - t0


_TABLE_CACHE: dict = {}


def _paper_oracle_worker(args):
    first, count, y = args
    sys.path.insert(0, ROOT)
    from oracle import faces as fc
    from oracle import xi

    nside, lmax = 4096, 4096
    cl = wl.cl_tt(lmax, 2500.0)
    t_max, n = fc.paper_grid_rule(cl, nside, y)
    if ("paper", t_max, n) not in _TABLE_CACHE:
        _TABLE_CACHE[("paper", t_max, n)] = xi.spin0_table(cl, t_max, n)
    tab, x0 = _TABLE_CACHE[("paper", t_max, n)]
    pix = np.arange(first, first + count)
    defl = wl.random_deflection(count, 77 + first)
    t0 = time.time()
    fc.paper_lens(nside, y, wl.HashedMap(12 * nside * nside, 9, 1), defl, pix, tab, x0, classes=True)
    return count, time.time() - t0


def cpu_oracle_paper(seconds: float, y: int = 1):
    """Time the oracle's class route of the tabulated-inverse lensing (Nside 4096 T,
    level y) on a bounded sample, on all host cores (spawned processes)."""
    import multiprocessing as mp

    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    per = 512
    npix = 12 * 4096 * 4096
    # chunk starts spread over the whole sky in a seeded random order, so that the
    # calibration chunks sample caps and belt alike
    spread = [int(v) for v in np.random.default_rng(5).integers(0, npix - per, 100_000)]
    with ctx.Pool(cores) as pool:
        # calibrate on one chunk per core taken across the sky (caps hold more classes)
        pool.map(_paper_oracle_worker, [(spread[0], 16, y)] * cores)  # warm each process
        t = time.time()
        res = pool.map(_paper_oracle_worker, [(s_, per, y) for s_ in spread[:cores]])
        rate = cores * per / max(time.time() - t, 1e-9)
        chunks = max(cores, int(seconds * rate / per))
        t = time.time()
        res += pool.map(_paper_oracle_worker, [(s_, per, y) for s_ in spread[cores:cores + chunks]])
        wall = time.time() - t
        res = res[cores:]
    pts = sum(r[0] for r in res)
    return {"value": pts / wall, "unit": "pts/s", "cores": cores, "kind": "oracle",
            "sample": f"{pts} targets of Nside 4096 T lensing, level {y}, in {chunks} chunks of {per} consecutive "
                      f"RING pixels (hashed-normal map values, per-pixel deflections; the oracle's class route), "
                      f"{wall:.1f} s wall on {cores} spawned processes"}


def cpu_oracle(seconds: float, aug: bool = False):
    """Time the oracle (as it stands) on a bounded sample of the workload on all host cores."""
    import multiprocessing as mp

    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    per = 256
    # calibrate on one chunk, then size the sample to about `seconds` of wall time
    with ctx.Pool(cores, initializer=None if aug else _oracle_init) as pool:
        n0, t0 = pool.map(_oracle_worker, [(50_000_000, per, 11, aug)])[0]
        rate1 = n0 / max(t0, 1e-9)
        chunks = max(cores, int(seconds * rate1 * cores / per))
        starts = [(50_000_000 + 7919 * per * k) % (W.npix - per) for k in range(chunks)]
        t = time.time()
        res = pool.map(_oracle_worker, [(s, per, 11, aug) for s in starts])
        wall = time.time() - t
    pts = sum(r[0] for r in res)
    return {"value": pts / wall, "unit": "pts/s", "cores": cores, "kind": "oracle",
            "sample": f"{pts} targets of the c3 workload{' (augmented estimator)' if aug else ''} in {chunks} chunks of {per} consecutive RING pixels "
                      f"(hashed-normal Q/U values, per-pixel deflections), {wall:.1f} s wall on {cores} spawned "
                      f"processes"}


# ------------------------------------------------------------------ clocks
class Clocks:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self, gpu_index: int):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9 or not p[0].isdigit() or int(p[0]) != gpu_index:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons)}


# ---------------------------------------------------------------- our arm
def measured_peaks():
    """FP32 and FP64 multiply-add throughput measured on this GPU before the timed region
    (flints_measure_fma_peak), next to the peaks derived from unit counts and clocks."""
    import paper_1003_4984_gb300 as fl
    from paper_1003_4984_gb300 import flops

    return {"fp32_tflops": max(fl.measure_fma_peak("mixed") for _ in range(3)),
            "fp64_tflops": max(fl.measure_fma_peak("fp64") for _ in range(3)),
            "fp32_derived_tflops": flops.FP32_PEAK_TFLOPS, "fp64_nominal_tflops": flops.FP64_PEAK_TFLOPS,
            "how": "flints_measure_fma_peak: independent FMA chains on every SM, best of 3, CUDA events"}


def roofline_entry(rate, flops_per_point, peak_tflops, kernel, peak_note, **extra):
    """ALU roofline of a lens kernel: the method's algorithmic flops per point times the
    measured point rate, against a measured pipe peak."""
    achieved = rate * flops_per_point / 1e12
    out = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
           "frac": achieved / peak_tflops, "flops_per_point": flops_per_point, "kernel": kernel,
           "peak_note": peak_note}
    out.update(extra)
    return out


def run_ours(args):
    import torch

    import paper_1003_4984_gb300 as fl
    from paper_1003_4984_gb300 import flops

    from paper_1003_4984_gb300 import ranks

    world, rank, local = ranks.rank_env()
    if world > 1:
        torch.cuda.set_device(local)
    dist = ranks.init("nccl")
    # the CPU baseline runs first, before any GPU work (spawned pool)
    aug = args.workload == "c3aug"
    flags = fl.FLINTS_SPIN2_AUGMENTED if aug else 0
    cpu = cpu_oracle(args.cpu_seconds, aug) if (rank == 0 and world == 1) else None

    dev = torch.device("cuda", local)
    fl.load_library()
    peaks = measured_peaks()
    cl, bb = W.cl()
    stream = torch.cuda.current_stream(dev)
    # one sky, the same on every rank (replicated source map); the targets are split into
    # contiguous RING ranges, one per rank, and each rank keeps the deflections of its range
    bounds = ranks.shard_bounds(W.npix, world)[rank]
    g = torch.Generator(device=dev)
    g.manual_seed(ranks.seed(1234))
    qu = torch.randn((W.npix, 2), dtype=torch.float64, device=dev, generator=g)
    defl_sky = torch.randn((W.npix, 2), dtype=torch.float64, device=dev, generator=g) * (
        wl.DEFLECTION_RMS / math.sqrt(2))
    defl = defl_sky[bounds[0]:bounds[1]].clone()
    del defl_sky
    out = torch.empty((BATCH, 2), dtype=torch.float64, device=dev)
    var = torch.empty(BATCH, dtype=torch.float64, device=dev)
    plans = {p: fl.Plan(W.nside, cl, bb, spin=2, K=W.K, precision=p, flags=flags) for p in ("mixed", "fp64")}

    def window(i):
        first, count = ranks.step_window(bounds, i, BATCH)
        return first, count, defl[first - bounds[0]:first - bounds[0] + count]

    def step(plan, i):
        first, count, d = window(i)
        plan.lens(qu, d, out[:count], var[:count], first=first, count=count)
        return count

    def timed(plan, steps, warmup):
        for i in range(warmup):
            step(plan, i)
        torch.cuda.synchronize(dev)
        ranks.barrier(dist)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record(stream)
        pts = 0
        for i in range(steps):
            pts += step(plan, warmup + i)
            ev[i + 1].record(stream)
        torch.cuda.synchronize(dev)
        per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
        total = ranks.max_over_ranks(ev[0].elapsed_time(ev[steps]), dist, dev)
        return total, per, pts

    plans["mixed"].reset_stats()
    with Clocks(os.path.join(OUT_DIR, f"bench_clocks_r{rank}.csv")) as clk:
        total_ms, per, pts = timed(plans["mixed"], args.steps, args.warmup)
    clocks = clk.summary(local)
    st = plans["mixed"].stats()
    fp_total, fp_per, fp_pts = timed(plans["fp64"], max(1, args.fp64_steps), 1)

    # the same mixed steps (same target windows) through the batched path: one persistent
    # launch per step from a captured CUDA graph (job-table upload, queue reset, class
    # kernels); each step re-stages its job on the host once the previous replay is done
    batched = None
    if not aug:
        batch = fl.Batch(1)
        bcfg = fl.LaunchCfg(8, 0, 16)

        def stage(i):
            b_first, b_count, b_defl = window(i)
            batch.stage([(plans["mixed"], b_first, b_count, qu, b_defl, out[:b_count], var[:b_count], None)],
                        bcfg.tile_points)
            return b_count

        side = torch.cuda.Stream(dev)
        stage(0)
        batch.launch(bcfg, stream=side)
        torch.cuda.synchronize(dev)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            batch.launch(bcfg, stream=side)
        for i in range(args.warmup):
            stage(i)
            graph.replay()
            torch.cuda.synchronize(dev)
        ranks.barrier(dist)
        cur = torch.cuda.current_stream(dev)
        b_ms, b_pts = 0.0, 0
        for i in range(args.steps):
            b_pts += stage(args.warmup + i)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(cur)
            graph.replay()
            e1.record(cur)
            torch.cuda.synchronize(dev)
            b_ms += e0.elapsed_time(e1)
        b_total = ranks.max_over_ranks(b_ms, dist, dev)
        batched = {"value": ranks.job_rate(b_pts, b_total / 1e3, world), "unit": "pts/s",
                   "ms_per_step": b_total / args.steps, "steps": args.steps,
                   "launch": "CUDA graph replay of flints_batch_launch (job-table upload, queue reset, "
                             "persistent class kernels) on the same target windows as the timed steps"}
        del graph
        batch.close()

    # end to end through the public API with pinned host buffers: every step uploads its
    # deflections and a twelfth of the map (the whole-sky upload amortised over the 12
    # steps of a sky) and downloads value and variance.  Copies overlap the kernels of
    # neighbouring steps: uploads run on one stream into double buffers (the map share
    # into a staging buffer, copied into the resident map on the compute stream right
    # before the step's kernel, so no kernel reads map pixels while they are written),
    # downloads on another; events order each buffer's reuse.
    nb = 12
    slice_len = (W.npix + nb - 1) // nb
    h_map = torch.empty((W.npix, 2), dtype=torch.float64, pin_memory=True)
    h_defl = torch.empty((BATCH, 2), dtype=torch.float64, pin_memory=True)
    h_out = [torch.empty((BATCH, 2), dtype=torch.float64, pin_memory=True) for _ in range(2)]
    h_var = [torch.empty(BATCH, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    h_defl.copy_(defl[:BATCH])
    h_map.copy_(qu)
    d_defl = [torch.empty((BATCH, 2), dtype=torch.float64, device=dev) for _ in range(2)]
    d_stage = [torch.empty((slice_len, 2), dtype=torch.float64, device=dev) for _ in range(2)]
    d_out = [out, torch.empty_like(out)]
    d_var = [var, torch.empty_like(var)]
    up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    kernel_done = [torch.cuda.Event(), torch.cuda.Event()]
    drained = [torch.cuda.Event(), torch.cuda.Event()]
    in_ready = [torch.cuda.Event(), torch.cuda.Event()]
    for b in range(2):  # recorded once so that the first waits are satisfied
        kernel_done[b].record(stream)
        drained[b].record(stream)

    def e2e_step(i):
        b = i & 1
        s0 = (i % nb) * slice_len
        s1 = min(W.npix, s0 + slice_len)
        first, count, _ = window(i)
        with torch.cuda.stream(up):
            up.wait_event(kernel_done[b])  # step i - 2 no longer reads these buffers
            d_stage[b][:s1 - s0].copy_(h_map[s0:s1], non_blocking=True)
            d_defl[b][:count].copy_(h_defl[:count], non_blocking=True)
            in_ready[b].record(up)
        stream.wait_event(in_ready[b])
        stream.wait_event(drained[b])  # step i - 2's outputs are downloaded
        qu[s0:s1].copy_(d_stage[b][:s1 - s0], non_blocking=True)  # this step's share of the map
        plans["mixed"].lens(qu, d_defl[b][:count], d_out[b][:count], d_var[b][:count], first=first, count=count,
                            stream=stream)
        kernel_done[b].record(stream)
        with torch.cuda.stream(down):
            down.wait_event(kernel_done[b])
            h_out[b][:count].copy_(d_out[b][:count], non_blocking=True)
            h_var[b][:count].copy_(d_var[b][:count], non_blocking=True)
            drained[b].record(down)
        return count

    e2e_step(0)
    e2e_step(1)
    torch.cuda.synchronize(dev)
    ranks.barrier(dist)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    up.wait_event(e0)  # no copy of the timed steps starts before e0
    e2e_pts = 0
    for i in range(args.steps):
        e2e_pts += e2e_step(2 + i)
    stream.wait_event(drained[0])
    stream.wait_event(drained[1])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = ranks.max_over_ranks(e0.elapsed_time(e1), dist, dev)
    h2d = slice_len * 16 + BATCH * 16
    d2h = BATCH * 16 + BATCH * 8

    serving = None
    if world == 1 and args.serving_seconds > 0 and not aug:
        serving = serving_leg(dev, args.serving_seconds)

    if rank != 0:
        dist.destroy_process_group()
        return
    n_gpus = world
    ms_step = total_ms / args.steps
    value = ranks.job_rate(pts, total_ms / 1e3, n_gpus)
    fp_value = ranks.job_rate(fp_pts, fp_total / 1e3, n_gpus)
    rate = BATCH / (statistics.mean(per) / 1e3)  # one launch per step: the kernel's own rate
    rate64 = BATCH / (statistics.mean(fp_per) / 1e3)
    f_method = flops.augmented_flops(W.K, False) if aug else flops.fp64_flops(W.K, 2)
    f_issue = flops.augmented_flops(W.K, True) if aug else flops.mixed_fp32_flops(W.K, 2)
    roof = roofline_entry(
        rate, f_method, peaks["fp32_tflops"],
        ("lens_kernel<32,3,mixed>" if aug else "batch_kernel<1,2,32> (the class kernel a spin-2 K=32 mixed plan "
         "call launches)") + " (double-float on the FP32 pipe)",
        "measured FP32 multiply-add throughput in this run (flints_measure_fma_peak); derived peak "
        "152 SMs x 128 lanes x 2 x 2.07 GHz = %.1f TFLOP/s" % flops.FP32_PEAK_TFLOPS,
        traffic=None if aug else MIXED_DRAM_BYTES_PER_POINT * BATCH,
        traffic_note="dram bytes read + written per launch, from the ncu capture of 2^18 targets scaled to "
                     "the launch (outputs of that case stayed in L2; at 2^24 targets 24 B/point more are "
                     "written back)",
        flops_convention="the method's own arithmetic per point (FP64 operation count, flops.fp64_flops): "
                         "the double-float path executes the same steps, each as several FP32 instructions",
        issue_flops_per_point=f_issue,
        issue_note="FP32 flops per point of the plain double-float cost model (instruction cost, not "
                   "algorithmic work; an upper estimate: the anchored accumulation executes fewer, and "
                   "issue_rate holds the measured instruction count)",
        issue_frac=rate * f_issue / 1e12 / peaks["fp32_tflops"],
        issue_rate=None if aug else {
            "warp_instr_per_point": MIXED_WARP_INSTR_PER_POINT,
            "achieved_per_s": rate * MIXED_WARP_INSTR_PER_POINT, "peak_per_s": ISSUE_PEAK_PER_S,
            "frac": rate * MIXED_WARP_INSTR_PER_POINT / ISSUE_PEAK_PER_S,
            "note": "instructions per target from the ncu capture of 2^18 targets; the issue slot is the "
                    "binding resource of the double-float emulation"},
        hbm={"bytes_per_point": 56, "achieved_gbs": rate * 56 / 1e9, "peak_gbs": HBM_PEAK_GBS,
             "frac": rate * 56 / 1e9 / HBM_PEAK_GBS})
    roof64 = roofline_entry(rate64, f_method, peaks["fp64_tflops"],
                            "lens_kernel<32,3,fp64>" if aug else "batch_kernel<0,2,32> (FP64)",
                            "measured FP64 multiply-add throughput in this run (flints_measure_fma_peak); "
                            "nominal 1.25 TFLOP/s")
    line = {
        "metric": METRIC + (" (augmented xi+/xi- estimator)" if aug else ""), "value": value, "unit": "pts/s",
        "n_gpus": n_gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 in/out; double-float (2 x f32: an FP64 emulation on the FP32 pipe) assembly, factor and solves; f64 geometry",
        "data": "synthetic: white-noise Q/U map (the work does not depend on the values) and per-pixel Gaussian "
                "deflections of 2.5 arcmin rms",
        "config": config(n_gpus),
        "step_p50_ms": float(np.percentile(per, 50)), "step_p99_ms": float(np.percentile(per, 99)),
        "serving": serving,
        "fp64": {"value": fp_value, "unit": "pts/s", "ms_per_step": statistics.mean(fp_per),
                 "steps": len(fp_per)},
        "mixed_over_fp64": value / fp_value,
        "batched": batched,
        "batched_over_fp64": None if batched is None else batched["value"] / fp_value,
        "mixed_stats": st,
        "e2e": {"value": ranks.job_rate(e2e_pts, e2e_ms / 1e3, n_gpus), "unit": "pts/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": args.steps},
        "roofline": roof,
        "roofline_fp64": roof64,
        "peaks_measured": peaks,
        "cpu_baseline": cpu,
        "clocks": clocks,
        # per timed step one plan call: store_one_job (its one-job table) + batch_kernel<1,2,32>
        "gpu_launches": 2 * args.steps,
    }
    print(json.dumps(line))


# ---------------------------------------------------------- c4 batched arm
C4_JOB = 1 << 20  # targets per map per step (whole map when smaller)


def run_c4(args):
    """64 maps of uneven Nside, K and spin (mixed precision) in one persistent,
    graph-captured launch per step; the launch shape comes from the autotuner."""
    import torch

    import paper_1003_4984_gb300 as fl
    from paper_1003_4984_gb300 import autotune

    fl.load_library()
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev)
    g.manual_seed(99)
    jobs, plans = [], []
    for w in wl.batched_maps(64):
        cl = wl.cl_tt(w.lmax, w.l_damp) if w.spin == 0 else wl.cl_ee(w.lmax, w.l_damp)
        plan = fl.Plan(w.nside, cl, spin=w.spin, K=w.K, precision="mixed")
        n = min(C4_JOB, w.npix)
        m = torch.randn((w.npix,) if w.spin == 0 else (w.npix, 2), dtype=torch.float64, device=dev, generator=g)
        d = torch.randn((n, 2), dtype=torch.float64, device=dev, generator=g) * (wl.DEFLECTION_RMS / math.sqrt(2))
        o = torch.empty((n,) if w.spin == 0 else (n, 2), dtype=torch.float64, device=dev)
        v = torch.empty(n, dtype=torch.float64, device=dev)
        first = (w.npix - n) // 2
        jobs.append((plan, first, n, m, d, o, v, None))
        plans.append(plan)
    points = sum(j[2] for j in jobs)
    batch = fl.Batch(len(jobs))
    cfg = autotune.tune_batch(batch, jobs, cands=[fl.LaunchCfg(w, 0, t) for w in (2, 4, 8) for t in (8, 16)])
    batch.stage(jobs, cfg.tile_points)
    stream = torch.cuda.Stream(dev)
    batch.launch(cfg, stream=stream)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        batch.launch(cfg, stream=stream)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    cur = torch.cuda.current_stream(dev)
    ev[0].record(cur)
    for i in range(args.steps):
        graph.replay()
        ev[i + 1].record(cur)
    torch.cuda.synchronize(dev)
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total = ev[0].elapsed_time(ev[-1])
    # the same jobs as one launch per job (no batching) for comparison
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    for (plan, first, n, m, d, o, v, _) in jobs:
        plan.lens(m, d, o, v, first=first, count=n)
    e1.record(cur)
    torch.cuda.synchronize(dev)
    seq_ms = e0.elapsed_time(e1)
    st = {"failed": sum(p.stats()["failed"] for p in plans), "fallback": sum(p.stats()["fallback"] for p in plans)}
    classes = {}
    for w in wl.batched_maps(64):
        classes[f"K{w.K}/spin{w.spin}"] = classes.get(f"K{w.K}/spin{w.spin}", 0) + 1
    print(json.dumps({
        "metric": "lensed pts/s, 64-map batched persistent launch (c4)", "value": points * args.steps / (total / 1e3),
        "unit": "pts/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 in/out; double-float factor", "data": "synthetic white-noise maps, Gaussian deflections 2.5' rms",
        "config": {"workload": "c4: 64 maps, Nside in {256,512,1024,2048}, K in {16,24,32,48}, spin in {0,2}, "
                               "lmax = min(2 Nside, 4096), mixed precision; up to 2^20 targets per map per step",
                   "points_per_step": points, "classes": classes, "launch": list(cfg.key()),
                   "graph": "one CUDA graph replay per step (job upload, queue reset, one persistent kernel per (precision, spin, K) class; empty classes exit at once)"},
        "p50_ms": float(np.percentile(per, 50)), "p99_ms": float(np.percentile(per, 99)),
        "per_job_launches": {"ms": seq_ms, "value": points / (seq_ms / 1e3)},
        "stats": st, "gpu_launches": 16 * args.steps}))


# ------------------------------------------------------------ c5 serving arm
def serving_leg(dev, duration: float, seed: int = 5):
    """Poisson stream of lensing requests (point counts log-uniform in [1e4, 1e8],
    spin 0/2, K 16/32, Nside 512..4096) served with continuous batching under a
    150 GB HBM budget (resident maps and plans included) at about 80 % of the
    capacity measured by a calibration burst; latency = completion - arrival."""
    import torch

    import paper_1003_4984_gb300 as fl
    from paper_1003_4984_gb300.serving import LensServer, Request, latency_stats

    fl.load_library()
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    server = LensServer(hbm_budget=150e9, batch_points=1 << 22, chunk_points=1 << 21, max_jobs=64,
                        device=dev.index or 0)
    for nside in (512, 1024, 2048, 4096):
        for spin in (0, 2):
            lmax = min(2 * nside, 4096)
            ld = 0.61 * lmax if lmax < 4096 else 2500.0
            cl = wl.cl_tt(lmax, ld) if spin == 0 else wl.cl_ee(lmax, ld)
            npix = 12 * nside * nside
            m = torch.randn((npix,) if spin == 0 else (npix, 2), dtype=torch.float64, device=dev, generator=g)
            server.register_map(nside, spin, m, cl)

    def defl_maker(count, sd):
        def make():
            gg = torch.Generator(device=dev)
            gg.manual_seed(sd)
            return torch.randn((count, 2), dtype=torch.float64, device=dev, generator=gg) * (
                wl.DEFLECTION_RMS / math.sqrt(2))
        return make

    # capacity: a calibration run of 24 requests arriving at once
    cal = wl.job_stream(24, 1e9, seed=499, max_points=4e6)
    creqs = [Request(i, (j.nside, j.spin), j.K, j.first, j.count, defl_maker(j.count, 10_000 + i)) for i, j in
             enumerate(cal)]
    t = time.perf_counter()
    server.run(creqs)
    torch.cuda.synchronize(dev)
    capacity = sum(r.count for r in creqs) / (time.perf_counter() - t)
    server.finished.clear()
    launches0 = server.launches
    mean_points = (1e8 - 1e4) / math.log(1e8 / 1e4)
    rate = 0.8 * capacity / mean_points
    n_jobs = max(10, int(rate * duration))
    stream = wl.job_stream(n_jobs, rate, seed=500)
    reqs = [Request(i, (j.nside, j.spin), j.K, j.first, j.count, defl_maker(j.count, i), arrival=j.arrival_s)
            for i, j in enumerate(stream)]
    done = server.run(reqs)
    torch.cuda.synchronize(dev)
    st = latency_stats(done)
    failed = sum(p.stats()["failed"] for p in server.plans.values())
    server.close()
    return {"p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"], "max_ms": st["max_ms"],
            "pts_per_s": st["points_per_s"], "requests": st["requests"], "points": st["points"],
            "span_s": st["span_s"], "arrival_rate_hz": rate, "capacity_pts_per_s": capacity,
            "launches": server.launches - launches0, "failed": failed,
            "load": "Poisson arrivals at 80 % of the measured capacity, point counts log-uniform in [1e4, 1e8] "
                    "(capped at Npix), spin 0/2, K 16/32, Nside 512..4096, mixed precision, 150 GB HBM budget "
                    "including the resident maps and xi tables, deflections generated on the device at "
                    "admission; latency = completion - arrival"}


def run_c5(args):
    """The serving load alone, for ``--duration`` seconds of arrivals."""
    import torch

    dev = torch.device("cuda", 0)
    sv = serving_leg(dev, args.duration)
    print(json.dumps({
        "metric": "serving latency p50/p99 (ms) and lensed pts/s under Poisson load (c5)",
        "value": sv["pts_per_s"], "unit": "pts/s", "n_gpus": 1, "higher_is_better": True,
        "p50_ms": sv["p50_ms"], "p99_ms": sv["p99_ms"], "serving": sv,
        "config": {"workload": "c5: " + sv["load"], "batch_points": 1 << 22, "chunk_points": 1 << 21},
        "data": "synthetic white-noise maps; deflections generated on the device at admission",
        "gpu_launches": 16 * sv["launches"]}))


# ----------------------------------------------------------- reference arm
REF_STEP = 1 << 16  # targets per step of the reference arm (the oracle on the host cores)
REF_CHUNK = 256


def _oracle_init():
    """Pool initializer: build the oracle's correlation tables once per process."""
    sys.path.insert(0, ROOT)
    from oracle import xi

    cl, bb = W.cl()
    t_max, n = xi.grid_rule(np.abs(cl) + np.abs(bb), W.K, W.nside)
    if (t_max, n) not in _TABLE_CACHE:
        _TABLE_CACHE[(t_max, n)] = xi.spin2_tables(cl, bb, t_max, n)


def run_reference(args):
    """The reference arm: the FP64 oracle (as it stands) on all host cores, on the same
    workload, metric and unit as our arm.  One step is a bounded sample of REF_STEP
    targets -- REF_STEP / REF_CHUNK chunks of consecutive RING targets spread over the
    sky, a different set each step -- timed by wall clock around the whole step; the
    warm-up steps run the same way untimed.  Under torchrun only rank 0 runs."""
    import multiprocessing as mp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    steps, warm = max(1, args.steps), max(0, args.warmup)
    nchunk = REF_STEP // REF_CHUNK
    rng = np.random.default_rng(2718)

    def chunks():
        starts = rng.integers(0, W.npix - REF_CHUNK, nchunk)
        return [(int(s_), REF_CHUNK, 11, False) for s_ in starts]

    ctx = mp.get_context("spawn")
    per = []
    with ctx.Pool(cores, initializer=_oracle_init) as pool:
        for _ in range(warm):
            pool.map(_oracle_worker, chunks())
        for _ in range(steps):
            work = chunks()
            t = time.perf_counter()
            res = pool.map(_oracle_worker, work)
            per.append(time.perf_counter() - t)
            assert sum(r[0] for r in res) == REF_STEP
    total = sum(per)
    value = steps * REF_STEP / total
    sample = (f"{steps} steps of {REF_STEP} targets of the c3 workload, each {nchunk} chunks of {REF_CHUNK} "
              f"consecutive RING pixels at seeded random places on the sky (hashed-normal Q/U values, per-pixel "
              f"deflections), {total:.1f} s wall on {cores} spawned processes; the GPU arm's step is {BATCH} "
              f"targets")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pts/s", "n_gpus": world,
            "steps": steps, "warmup": warm, "ms_per_step": 1e3 * total / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (see cpu_baseline.sample)",
            "config": dict(config(world), step_points=REF_STEP),
            "step_p50_ms": float(np.percentile(per, 50)) * 1e3, "step_p99_ms": float(np.percentile(per, 99)) * 1e3,
            "cpu_baseline": {"value": value, "unit": "pts/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "pts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------- supersampling arm
def run_ss(args):
    """Supersampling (Sec. 2.6, Table 1 row Nside 2048 -> 4096, lmax 4096): an Nside
    2048 map predicted at the pixel centres of the Nside 4096 grid, K = 32, spin 0,
    2^24 targets per step.  Also reports the predicted precision sqrt(<sigma^2>)/sigma_map,
    Table 1's precision column (its stencils have 9 and 36 neighbours)."""
    import torch

    import paper_1003_4984_gb300 as fl
    from paper_1003_4984_gb300 import flops

    fl.load_library()
    Wc = wl.C2
    nout = 2 * Wc.nside
    npix_out = 12 * nout * nout
    cl, _ = Wc.cl()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    g = torch.Generator(device=dev)
    g.manual_seed(4242)
    m = torch.randn(Wc.npix, dtype=torch.float64, device=dev, generator=g)
    out = torch.empty(BATCH, dtype=torch.float64, device=dev)
    var = torch.empty(BATCH, dtype=torch.float64, device=dev)
    nb = npix_out // BATCH
    res = {}
    for precision, steps in (("mixed", args.steps), ("fp64", max(1, args.fp64_steps))):
        plan = fl.Plan(Wc.nside, cl, spin=0, K=Wc.K, precision=precision)
        for i in range(args.warmup):
            plan.supersample(m, nout, out, var, first=(i % nb) * BATCH, count=BATCH)
        torch.cuda.synchronize(dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record(stream)
        for i in range(steps):
            plan.supersample(m, nout, out, var, first=((args.warmup + i) % nb) * BATCH, count=BATCH)
            ev[i + 1].record(stream)
        torch.cuda.synchronize(dev)
        per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
        res[precision] = (BATCH * steps / (ev[0].elapsed_time(ev[steps]) / 1e3), per, plan.info().xi0, plan.stats())
        plan.close()
    value, per, xi0, st = res["mixed"]
    precision_pred = math.sqrt(float(var.mean()) / xi0)  # last batch, FP64 plan
    peaks = measured_peaks()
    roof = roofline_entry(BATCH / (statistics.mean(per) / 1e3), flops.fp64_flops(Wc.K, 0), peaks["fp32_tflops"],
                          "batch_kernel<1,0,32>", "measured FP32 multiply-add throughput in this run",
                          traffic=None, issue_flops_per_point=flops.mixed_fp32_flops(Wc.K, 0))
    print(json.dumps({
        "metric": "supersampled pts/s, Nside 2048 -> 4096, lmax 4096, K=32, spin 0", "value": value,
        "unit": "pts/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(per), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 in/out; double-float factor", "data": "synthetic white-noise Nside 2048 map",
        "config": {"workload": "supersampling: Nside 2048 (lmax 4096, damping l = 2500) -> Nside 4096 pixel "
                               "centres, K = 32", "batch_points": BATCH,
                   "l2": "inputs larger than L2 (403 MB map, 2^24 targets per step)"},
        "fp64": {"value": res["fp64"][0], "ms_per_step": statistics.mean(res["fp64"][1])},
        "mixed_over_fp64": value / res["fp64"][0],
        "predicted_precision": precision_pred,
        "paper_table1": "Nside 2048 -> 4096, l 4096: 3e-3 (9 neighbours), 3e-4 (36 neighbours); serial "
                        "Xeon E5410 3.3 / 19 min per map",
        "roofline": roof, "peaks_measured": peaks,
        "mixed_stats": st, "gpu_launches": 2 * args.steps}))


# -------------------------------------------------------------- spin-1 arm
def run_spin1(args):
    """A spin-1 field -- a deflection d = grad phi, C^E_l = l(l+1) C^phiphi_l -- remapped
    at Nside 4096 (lmax 4096, K = 32), 2^24 targets per step, mixed and FP64."""
    import torch

    import paper_1003_4984_gb300 as fl
    from paper_1003_4984_gb300 import flops

    fl.load_library()
    nside, lmax, K = W.nside, W.lmax, W.K
    npix = 12 * nside * nside
    ell = np.arange(lmax + 1)
    cle = wl.cl_phiphi(lmax) * ell * (ell + 1.0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    g = torch.Generator(device=dev)
    g.manual_seed(77)
    m = torch.randn((npix, 2), dtype=torch.float64, device=dev, generator=g) * wl.DEFLECTION_RMS
    nb = npix // BATCH
    defl = torch.randn((nb * BATCH, 2), dtype=torch.float64, device=dev, generator=g) * (wl.DEFLECTION_RMS / math.sqrt(2))
    out = torch.empty((BATCH, 2), dtype=torch.float64, device=dev)
    var = torch.empty(BATCH, dtype=torch.float64, device=dev)
    res = {}
    for precision, steps in (("mixed", args.steps), ("fp64", max(1, args.fp64_steps))):
        plan = fl.Plan(nside, cle, spin=1, K=K, precision=precision)

        def step(i):
            b = i % nb
            plan.lens(m, defl[b * BATCH:(b + 1) * BATCH], out, var, first=b * BATCH, count=BATCH)

        for i in range(args.warmup):
            step(i)
        torch.cuda.synchronize(dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record(stream)
        for i in range(steps):
            step(args.warmup + i)
            ev[i + 1].record(stream)
        torch.cuda.synchronize(dev)
        per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
        res[precision] = (BATCH * steps / (ev[0].elapsed_time(ev[steps]) / 1e3), per, plan.stats())
        plan.close()
    value, per, st = res["mixed"]
    peaks = measured_peaks()
    roof = roofline_entry(BATCH / (statistics.mean(per) / 1e3), flops.fp64_flops(K, 1), peaks["fp32_tflops"],
                          "lens_kernel<32,1,mixed>", "measured FP32 multiply-add throughput in this run",
                          traffic=None, issue_flops_per_point=flops.mixed_fp32_flops(K, 1))
    print(json.dumps({
        "metric": "lensed pts/s of a spin-1 deflection field at Nside 4096, K=32", "value": value, "unit": "pts/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(per),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 in/out; double-float factor", "data": "synthetic white-noise spin-1 map, Gaussian deflections",
        "config": {"workload": "spin 1: Nside 4096, lmax 4096, C^E = l(l+1) C^phiphi (2.5 arcmin rms), K = 32",
                   "batch_points": BATCH},
        "fp64": {"value": res["fp64"][0], "ms_per_step": statistics.mean(res["fp64"][1])},
        "mixed_over_fp64": value / res["fp64"][0],
        "roofline": roof, "peaks_measured": peaks,
        "mixed_stats": st, "gpu_launches": args.steps}))


# ----------------------------------------------------------- pipeline arm
def run_pipeline(args):
    """Table 2's total on the GPU: from Gaussian a_lm of T, E and phi (Nside 4096,
    lmax 4096), synthesise the unlensed T and Q/U maps and the deflection
    grad(phi) (spin-1 synthesis), then lens T and Q/U over the whole sky
    (mixed path, K = 32, batches of 2^24 targets).  One step = one lensed T+P map."""
    import torch

    import paper_1003_4984_gb300 as fl

    fl.load_library()
    nside, lmax, K = W.nside, W.lmax, W.K
    npix = 12 * nside * nside
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ell = torch.arange(lmax + 1, dtype=torch.float64, device=dev)
    cl_t = torch.from_numpy(wl.cl_tt(lmax, 2500.0)).to(dev)
    cl_e, _ = W.cl()
    cl_e = torch.from_numpy(cl_e).to(dev)
    cl_p = torch.from_numpy(wl.cl_phiphi(lmax)).to(dev)
    g = torch.Generator(device=dev)
    g.manual_seed(2024)

    def alm(cl):  # Gaussian a_lm with <|a_lm|^2> = C_l (m = 0 real)
        a = torch.randn((lmax + 1, lmax + 1, 2), dtype=torch.float64, device=dev, generator=g)
        a *= torch.sqrt(cl / 2.0)[:, None, None]
        a[:, 0, 0] *= math.sqrt(2.0)
        a[:, 0, 1] = 0.0
        a = torch.view_as_complex(a)
        return torch.tril(a).contiguous()

    a_t, a_e = alm(cl_t), alm(cl_e)
    a_d = (alm(cl_p) * torch.sqrt(ell * (ell + 1.0))[:, None]).contiguous()  # E of the spin-1 deflection
    t0 = time.time()
    syn = {0: fl.Synth(nside, lmax, 0), 1: fl.Synth(nside, lmax, 1), 2: fl.Synth(nside, lmax, 2)}
    torch.cuda.synchronize(dev)
    synth_plan_s = time.time() - t0
    t0 = time.time()
    plan_t = fl.Plan(nside, wl.cl_tt(lmax, 2500.0), spin=0, K=K, precision="mixed", flags=fl.FLINTS_NO_VARIANCE)
    cl_ee, bb = W.cl()
    plan_p = fl.Plan(nside, cl_ee, bb, spin=2, K=K, precision="mixed", flags=fl.FLINTS_NO_VARIANCE)
    lens_plan_s = time.time() - t0
    tmap = torch.empty(npix, dtype=torch.float64, device=dev)
    qu = torch.empty((npix, 2), dtype=torch.float64, device=dev)
    defl = torch.empty((npix, 2), dtype=torch.float64, device=dev)
    out_t = torch.empty(npix, dtype=torch.float64, device=dev)
    out_p = torch.empty((npix, 2), dtype=torch.float64, device=dev)
    ev = {}

    def step():
        for k in ("s_t", "s_p", "s_d", "l_t", "l_p", "end"):
            ev.setdefault(k, torch.cuda.Event(enable_timing=True))
        ev["s_t"].record(stream)
        syn[0].run(a_t, None, tmap)
        ev["s_p"].record(stream)
        syn[2].run(a_e, None, qu)
        ev["s_d"].record(stream)
        syn[1].run(a_d, None, defl)
        ev["l_t"].record(stream)
        for b0 in range(0, npix, BATCH):
            n = min(BATCH, npix - b0)
            plan_t.lens(tmap, defl[b0:b0 + n], out_t[b0:b0 + n], first=b0, count=n)
        ev["l_p"].record(stream)
        for b0 in range(0, npix, BATCH):
            n = min(BATCH, npix - b0)
            plan_p.lens(qu, defl[b0:b0 + n], out_p[b0:b0 + n], first=b0, count=n)
        ev["end"].record(stream)

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    steps = max(1, args.steps)
    parts = {"synth_T": [], "synth_QU": [], "synth_deflection": [], "lens_T": [], "lens_QU": [], "total": []}
    with Clocks(os.path.join(OUT_DIR, "bench_clocks_pipeline.csv")) as clk:
        for _ in range(steps):
            step()
            torch.cuda.synchronize(dev)
            parts["synth_T"].append(ev["s_t"].elapsed_time(ev["s_p"]))
            parts["synth_QU"].append(ev["s_p"].elapsed_time(ev["s_d"]))
            parts["synth_deflection"].append(ev["s_d"].elapsed_time(ev["l_t"]))
            parts["lens_T"].append(ev["l_t"].elapsed_time(ev["l_p"]))
            parts["lens_QU"].append(ev["l_p"].elapsed_time(ev["end"]))
            parts["total"].append(ev["s_t"].elapsed_time(ev["end"]))
    ms = {k: statistics.mean(v) for k, v in parts.items()}
    st_t, st_p = plan_t.stats(), plan_p.stats()
    print(json.dumps({
        "metric": "seconds per lensed T+Q/U map at Nside 4096 (synthesis of T, Q/U, deflection + lensing)",
        "value": ms["total"] / 1e3, "unit": "s", "n_gpus": 1, "steps": steps, "warmup": max(1, args.warmup),
        "ms_per_step": ms["total"], "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 synthesis; lensing double-float factor, f64 geometry",
        "data": "synthetic Gaussian a_lm of the c3 spectra (T damping l = 2500, E = 0.05 T shape, B = 0, "
                "C^phiphi ~ l^-4 at 2.5 arcmin rms)",
        "config": {"workload": "pipeline: Nside 4096 (201,326,592 px), lmax 4096, K = 32, T and Q/U, mixed",
                   "batch_points": BATCH},
        "breakdown_ms": ms, "synth_plans_s": synth_plan_s, "lens_plans_s": lens_plan_s,
        "lens_stats": {"T": st_t, "QU": st_p},
        "paper_table2": "FLINTS Nside 4096, 9 neighbours: interpolation 22 min, total 51 min (+16 min init), "
                        "serial Xeon E5410",
        "clocks": clk.summary(0), "gpu_launches": 30 * steps}))
    for s_ in syn.values():
        s_.close()


# ------------------------------------------------- tabulated-inverse arm
def run_paper(args):
    """The paper's own route (Secs. 2.3-2.5): the pixel-centred stencil of 9 (y = 1)
    and 36 (y = 2) pixels with L^-1 (the factor of S^-1) tabulated per symmetry
    class of central pixels, two triangular matrix-vector products per target,
    in FP64 and in double-float (mixed).  Lensing of an Nside 4096, lmax 4096
    temperature map (Table 2's configuration) and supersampling Nside 2048 ->
    4096 (Table 1's), 2^24 targets per step.  The plan time (stencils and L^-1
    tabulation) is Table 2's "init" column."""
    import torch

    import paper_1003_4984_gb300 as fl
    from paper_1003_4984_gb300 import flops

    # the CPU baseline runs first, before any GPU work (spawned pool)
    cpu = cpu_oracle_paper(args.cpu_seconds, 1)
    fl.load_library()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    g = torch.Generator(device=dev)
    g.manual_seed(777)
    lmax = 4096
    cl = wl.cl_tt(lmax, 2500.0)
    steps, warm = max(1, args.steps), max(3, args.warmup)
    out = torch.empty(BATCH, dtype=torch.float64, device=dev)
    var = torch.empty(BATCH, dtype=torch.float64, device=dev)
    res = {}
    clk_path = os.path.join(OUT_DIR, "bench_clocks_paper.csv")
    cl_ee, cl_bb = W.cl()
    with Clocks(clk_path) as clk:
        for task, nside, nout, spin in (("lens", 4096, None, 0), ("supersample", 2048, 4096, 0),
                                        ("lens_qu", 4096, None, 2), ("lens_qu_aug", 4096, None, 2)):
            npix = 12 * nside * nside
            m = torch.randn((npix, 2) if spin == 2 else (npix,), dtype=torch.float64, device=dev, generator=g)
            ntgt = 12 * (nout or nside) ** 2
            nb = ntgt // BATCH
            defl = None
            if task.startswith("lens"):
                defl = torch.randn((BATCH, 2), dtype=torch.float64, device=dev, generator=g) * wl.DEFLECTION_RMS
            out = torch.empty((BATCH, 2) if spin == 2 else (BATCH,), dtype=torch.float64, device=dev)
            for y in (1, 2):
                for precision in (("fp64",) if task.endswith("aug") else ("fp64", "mixed")):
                    torch.cuda.synchronize(dev)
                    t0 = time.perf_counter()
                    if spin == 2:
                        plan = fl.PaperPlan(nside, cl_ee, y, precision, spin=2, cl_bb=cl_bb,
                                            augmented=task.endswith("aug"))
                    else:
                        plan = fl.PaperPlan(nside, cl, y, precision)
                    torch.cuda.synchronize(dev)
                    plan_s = time.perf_counter() - t0
                    info = plan.info()

                    def step(i):
                        first = (i % nb) * BATCH
                        if task.startswith("lens"):
                            plan.lens(m, defl, first=first, count=BATCH, out=out, var=var)
                        else:
                            plan.supersample(m, nout, first=first, count=BATCH, out=out, var=var)

                    for i in range(warm):
                        step(i)
                    torch.cuda.synchronize(dev)
                    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
                    ev[0].record(stream)
                    for i in range(steps):
                        step(warm + i)
                        ev[i + 1].record(stream)
                    torch.cuda.synchronize(dev)
                    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
                    K = info["K"]
                    sec = statistics.mean(per) / 1e3
                    arm = {
                        "value": BATCH * steps / (ev[0].elapsed_time(ev[steps]) / 1e3), "unit": "pts/s",
                        "ms_per_step": statistics.mean(per), "K": K, "plan_s": plan_s, "slots": info["slots"],
                        "table_bytes": info["table_bytes"], "device_bytes": info["device_bytes"],
                        "window": info["window"],
                        "nugget_slots": info["nugget_slots"], "failed_slots": info["failed_slots"],
                        "predicted_precision": math.sqrt(float(var.mean()) / info["xi0"])}
                    # the method's flops per target (whatever precision executes them), and for
                    # double-float arms the FP32 instruction cost of the emulation beside them
                    f_method = flops.paper_augmented_fp64_flops(K) if task.endswith("aug") else flops.paper_fp64_flops(K, spin)
                    arm["method_tflops"] = f_method * BATCH / sec / 1e12
                    if precision == "mixed":
                        arm["issue_fp32_tflops"] = flops.paper_mixed_fp32_flops(K, spin) * BATCH / sec / 1e12
                    res[f"{task}_y{y}_{precision}"] = arm
                    plan.close()
                    torch.cuda.empty_cache()
            del m, defl
            torch.cuda.empty_cache()
    head = res["lens_y1_mixed"]
    ratios = {f"{t}_y{y}": res[f"{t}_y{y}_mixed"]["value"] / res[f"{t}_y{y}_fp64"]["value"]
              for t in ("lens", "supersample", "lens_qu") for y in (1, 2)}
    peaks = measured_peaks()
    roof = roofline_entry(head["value"], flops.paper_fp64_flops(9), peaks["fp32_tflops"], "paper::apply_kernel_df<9>",
                          "measured FP32 multiply-add throughput in this run", traffic=None,
                          issue_flops_per_point=flops.paper_mixed_fp32_flops(9))
    roof64 = roofline_entry(res["lens_y1_fp64"]["value"], flops.paper_fp64_flops(9), peaks["fp64_tflops"],
                            "paper::apply_kernel<9>", "measured FP64 multiply-add throughput in this run")
    print(json.dumps({
        "metric": "lensed pts/s, Nside 4096 T, lmax 4096, paper stencil (9 px) with tabulated inverses, mixed vs FP64",
        "value": head["value"], "unit": "pts/s", "n_gpus": 1, "steps": steps, "warmup": warm,
        "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 in/out; double-float chords, lookups and triangular products",
        "data": "synthetic white-noise maps, Gaussian deflections of 2.5 arcmin rms",
        "config": {"workload": "tabulated inverse: lensing Nside 4096 T (y = 1, 2; FP64 and mixed), "
                               "supersampling Nside 2048 -> 4096 (y = 1, 2; FP64 and mixed), lensing Nside 4096 "
                               "Q/U (spin 2, c3 spectra, y = 1, 2; FP64 and mixed; augmented xi+/xi- FP64), lmax 4096",
                   "batch_points": BATCH, "l2": "inputs larger than L2 (1.6 GB map, 268 MB of deflections)"},
        "fp64": {"value": res["lens_y1_fp64"]["value"], "ms_per_step": res["lens_y1_fp64"]["ms_per_step"]},
        "mixed_over_fp64": ratios, "arms": res,
        "paper_tables": "Table 2 (Nside 4096, 9 neighbours): init 16 min, interpolation 22 min per map; "
                        "Table 1 (2048 -> 4096): 3.3 min (9) / 19 min (36), precision 3e-3 / 3e-4; serial "
                        "Xeon E5410",
        "roofline": roof, "roofline_fp64": roof64, "peaks_measured": peaks,
        "cpu_baseline": cpu, "clocks": clk.summary(0), "gpu_launches": steps}))


if __name__ == "__main__":
    a = parse()
    if a.workload == "c4" and a.impl == "ours" and not a.profile_case:
        run_c4(a)
    elif a.workload == "c5" and a.impl == "ours" and not a.profile_case:
        run_c5(a)
    elif a.workload == "ss" and a.impl == "ours" and not a.profile_case:
        run_ss(a)
    elif a.workload == "pipeline" and a.impl == "ours" and not a.profile_case:
        run_pipeline(a)
    elif a.workload == "spin1" and a.impl == "ours" and not a.profile_case:
        run_spin1(a)
    elif a.workload == "paper" and a.impl == "ours" and not a.profile_case:
        run_paper(a)
    elif a.profile_case:
        run_profile_case(a.profile_case)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)  # c3, or c3aug
