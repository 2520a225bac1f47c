"""Replica (data-parallel, no exchange) helpers for multi-GPU runs.

Angles are independent, so N GPUs run N replicas of the same kernels on
their own shards: no collective touches the data.  The only inter-rank
operations are a barrier around the timed region and the max of the
per-rank times (the job finishes when the slowest rank does).  Works with
any torch.distributed backend (nccl on GPUs, gloo on CPU).
"""
from __future__ import annotations

import os


def rank_env():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_seed(base_seed: int, rank: int) -> int:
    """Seed of rank `rank`'s shard: every rank draws its own angles."""
    return base_seed + rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Max of a per-rank scalar over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job rate: all ranks' units divided by the slowest rank's time."""
    return units_per_rank * world / seconds
