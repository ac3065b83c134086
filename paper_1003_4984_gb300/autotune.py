"""Launch-shape autotuner for the lens kernels.

The results of a launch do not depend on its shape, only its speed does.  The
tuner times candidate shapes (warps per block, blocks per SM, targets per warp
tile) with CUDA events on a sample of the caller's own workload, keeps the
fastest, and caches it in a JSON file keyed by the GPU and the workload class,
so later plans of the same class reuse the choice without timing.
"""
from __future__ import annotations

import itertools
import json
import os
import threading

from .api import Batch, LaunchCfg, Plan

DEFAULT_CACHE = os.environ.get("FLINTS_AUTOTUNE_CACHE",
                               os.path.join(os.path.expanduser("~"), ".cache", "flints_autotune.json"))
_lock = threading.Lock()


def candidates(max_warps: int = 8):
    out = []
    for w, b, t in itertools.product((2, 4, 8), (0, 1, 2), (8, 16)):
        if w <= max_warps:
            out.append(LaunchCfg(w, b, t))
    return out


def _device_key():
    import torch

    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|{p.multi_processor_count}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(path, data):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time(fn, reps: int) -> float:
    import torch

    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def plan_key(plan: Plan) -> str:
    return f"plan|{_device_key()}|nside={plan.nside}|K={plan.K}|spin={plan.spin}|{plan.precision}"


def tune_plan(plan: Plan, map_, defl, first: int, count: int, cache: str = DEFAULT_CACHE, reps: int = 2,
              cands=None, force: bool = False) -> LaunchCfg:
    """Choose and set the fastest launch shape for ``plan`` on the given sample range."""
    import torch

    key = plan_key(plan)
    with _lock:
        data = _load(cache)
    if key in data and not force:
        cfg = LaunchCfg(*data[key]["cfg"])
        plan.set_launch(cfg)
        return cfg
    out = torch.empty((count,) if plan.spin == 0 else (count, 2), dtype=torch.float64, device=map_.device)
    var = torch.empty(count, dtype=torch.float64, device=map_.device)
    best, best_ms, table = None, float("inf"), []
    for cfg in cands or candidates():
        plan.set_launch(cfg)
        ms = _time(lambda: plan.lens(map_, defl, out, var, first=first, count=count), reps)
        table.append((cfg.key(), ms))
        if ms < best_ms:
            best, best_ms = cfg, ms
    plan.set_launch(best)
    with _lock:
        data = _load(cache)
        data[key] = {"cfg": list(best.key()), "ms": best_ms, "points": count, "tried": table}
        _save(cache, data)
    return best


def batch_key(jobs) -> str:
    classes = sorted({(p.K, p.spin, p.precision) for p, *_ in jobs})
    return f"batch|{_device_key()}|" + ",".join(f"K{k}s{s}{pr}" for k, s, pr in classes)


def tune_batch(batch: Batch, jobs, cache: str = DEFAULT_CACHE, reps: int = 1, cands=None,
               force: bool = False) -> LaunchCfg:
    """Choose the fastest launch shape for a staged batch of jobs (by full launches)."""
    key = batch_key(jobs)
    with _lock:
        data = _load(cache)
    if key in data and not force:
        return LaunchCfg(*data[key]["cfg"])
    best, best_ms, table = None, float("inf"), []
    for cfg in cands or candidates():
        batch.stage(jobs, cfg.tile_points)
        ms = _time(lambda: batch.launch(cfg), reps)
        table.append((cfg.key(), ms))
        if ms < best_ms:
            best, best_ms = cfg, ms
    batch.stage(jobs, best.tile_points)
    with _lock:
        data = _load(cache)
        data[key] = {"cfg": list(best.key()), "ms": best_ms, "tried": table}
        _save(cache, data)
    return best
