"""Rank bookkeeping for running the volume term on several GPUs of one node.

Elements are independent (the volume term is block-diagonal per element), so
the path shards with no data-path exchange: each rank owns a contiguous block
of elements and computes it alone.  The only collective is a MAX of the
per-rank step time (one scalar), taken after the timed region.
"""
from __future__ import annotations

import os


def rank_world():
    """(rank, world_size, local_rank) from the torchrun environment (1 rank if unset)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n_total: int, rank: int, world: int):
    """Contiguous element range [e0, e1) of `rank` when n_total elements are
    split over `world` ranks (sizes differ by at most one)."""
    if world < 1 or not (0 <= rank < world) or n_total < 0:
        raise ValueError("bad shard arguments")
    q, r = divmod(n_total, world)
    e0 = rank * q + min(rank, r)
    return e0, e0 + q + (1 if rank < r else 0)


def weak_block_seed(rank: int, base: int = 2) -> int:
    """Seed of rank's own element block under weak scaling (each rank a full
    block of the workload, distinct data)."""
    return base + 10 * rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """MAX of a per-rank scalar (e.g. the timed region's duration)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(units_per_rank: float, world: int, t_max: float) -> float:
    """Whole-job throughput: the units all ranks processed / the slowest rank's time."""
    return units_per_rank * world / t_max
