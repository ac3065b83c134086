"""Host-side layout of a multi-GPU run: one process per GPU (torchrun
environment), one sky split across the ranks.  Every target pixel is
independent (the per-pixel locality that makes the method suitable for
distributed memory, abstract and Sec. 5), so the targets of one map are cut
into contiguous RING ranges balanced by count, one per rank; each rank holds
the whole source map (replicated: a stencil may reach pixels of a neighbouring
range) and lenses its own range with no collective on the data path; outputs
stay sharded or are gathered to rank 0 afterwards.  Timings are bracketed by
barriers and joined by a MAX reduction, and the whole-job rate counts the
points of all ranks.

Backend-agnostic: the CUDA benchmark uses NCCL, the tests gloo on CPU.
"""
from __future__ import annotations

import os


def rank_env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the torchrun environment (1, 0, 0 when absent)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str):
    """torch.distributed initialised for world size > 1, else None."""
    world, _, _ = rank_env()
    if world <= 1:
        return None
    import torch.distributed as dist

    if not dist.is_initialized():
        dist.init_process_group(backend)
    return dist


def shard_bounds(n: int, world: int) -> list[tuple[int, int]]:
    """Contiguous [start, stop) target ranges of a sky of n targets, one per rank,
    balanced by count (sizes differ by at most one); they tile [0, n) once."""
    base, extra = divmod(int(n), int(world))
    out, start = [], 0
    for r in range(world):
        stop = start + base + (1 if r < extra else 0)
        out.append((start, stop))
        start = stop
    return out


def step_window(bounds: tuple[int, int], step: int, batch: int) -> tuple[int, int]:
    """(first, count) of benchmark step ``step`` on a rank whose range is ``bounds``:
    ``batch`` consecutive targets of the range, successive steps walking through it
    (a range shorter than the batch is lensed whole)."""
    start, stop = bounds
    length = stop - start
    if length <= batch:
        return start, length
    span = length - batch + 1
    return start + (step * batch) % span, batch


def lens_shard(lens_range, bounds: tuple[int, int], batch: int):
    """Lens a rank's whole range in calls of at most ``batch`` consecutive targets.

    ``lens_range(first, count)`` lenses targets [first, first+count) and returns
    (value, variance) tensors; the results are concatenated in RING order.  An
    empty range (a sky with fewer targets than ranks) makes one call with
    count 0, so the rank still holds typed empty tensors for the gather."""
    import torch

    start, stop = bounds
    if stop <= start:
        return lens_range(start, 0)
    vals, vars_ = [], []
    for first in range(start, stop, batch):
        v, s2 = lens_range(first, min(batch, stop - first))
        vals.append(v)
        vars_.append(s2)
    return torch.cat(vals), torch.cat(vars_)


def gather_shards(local, bounds: list[tuple[int, int]], dist, rank: int, dst: int = 0):
    """Whole-sky tensor on rank ``dst`` from every rank's range (None on the others;
    ``local`` itself when there is no process group).  Shards are padded to the
    longest one for the collective and trimmed afterwards."""
    if dist is None:
        return local
    import torch

    longest = max(b - a for a, b in bounds)
    pad = torch.zeros((longest,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[:local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in bounds] if rank == dst else None
    dist.gather(pad, parts, dst=dst)
    if rank != dst:
        return None
    return torch.cat([p[:b - a] for p, (a, b) in zip(parts, bounds)])


def seed(base: int) -> int:
    """Seed of the synthetic map and deflections: one sky, the same on every rank."""
    return base


def barrier(dist) -> None:
    if dist is not None:
        dist.barrier()


def max_over_ranks(x: float, dist, device=None) -> float:
    """The largest value of x over all ranks (x itself on one rank)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(points_per_rank: int, seconds_max: float, world: int) -> float:
    """Whole-job throughput: the points all ranks processed over the slowest rank's time."""
    return world * points_per_rank / seconds_max
