"""Host-side layout of a multi-GPU run: one process per GPU (torchrun
environment), independent problems per rank (every target pixel is
independent, so ranks lens their own maps and batches: weak scaling, no
collective on the data path); timings are bracketed by barriers and joined by
a MAX reduction, and the whole-job rate counts the points of all ranks.

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


def batch_index(rank: int, i: int, n_batches: int) -> int:
    """Target batch of step i on a rank: ranks start 5 batches apart around the sky."""
    return (rank * 5 + i) % n_batches


def seed(rank: int, base: int) -> int:
    """Per-rank seed of the synthetic map and deflections (independent problems)."""
    return base + rank


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
