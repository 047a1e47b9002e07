"""Host logic of the multi-GPU benchmark path (one process per GPU).

Queries are independent, so ranks shard them with no data-path collective:
each rank solves its own batch (weak scaling) or its contiguous share of a
global batch.  The only collective is a MAX of the per-rank step time, so
the whole job is timed by its slowest rank.
"""
from __future__ import annotations

import os


def env():
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [start, stop) share of n queries for ``rank``."""
    base, extra = divmod(int(n), int(world))
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def rank_seed(seed: int, rank: int) -> int:
    """Seed of a rank's own batch (weak scaling)."""
    return int(seed) + int(rank)


def max_over_ranks(value: float, group=None, device=None) -> float:
    """MAX all-reduce of a float (identity without an initialised group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def job_throughput(queries_per_rank: int, world: int, step_ms: float) -> float:
    """Whole-job queries/s: all ranks' queries over the slowest rank's time."""
    return queries_per_rank * world / (step_ms * 1e-3)
