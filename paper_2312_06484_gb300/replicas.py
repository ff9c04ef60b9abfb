"""Bookkeeping of a run on several GPUs.

The filter does not exchange data between GPUs here: a run on N GPUs is N replicas, one
process per GPU, each running its own independent chains (its own chain indices, hence its
own random streams).  The job's time is the slowest rank's, and its throughput counts the
work of every rank.
"""
from __future__ import annotations


def world():
    """(world_size, rank, local_rank) from the launcher's environment (1, 0, 0 without one)."""
    import os
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def chain_base(rank: int, chains_per_rank: int = 1) -> int:
    """First chain index of a rank: ranks own disjoint, contiguous chain ranges."""
    if rank < 0 or chains_per_rank < 1:
        raise ValueError("rank >= 0 and chains_per_rank >= 1")
    return rank * chains_per_rank


def max_over_ranks(value: float, device="cpu") -> float:
    """The largest value over all ranks (the value itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, seconds_slowest: float, world_size: int) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    if seconds_slowest <= 0:
        raise ValueError("time must be positive")
    return units_per_rank * world_size / seconds_slowest
