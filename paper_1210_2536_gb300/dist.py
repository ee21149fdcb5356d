"""Multi-process plumbing for replicated runs (one process per GPU).

SpMV on one matrix needs no exchange when every rank holds its own replica
(the data-parallel reading: independent problems per rank), so the only
collective is the timing reduction: the job's time is the slowest rank's, and
its throughput is all ranks' work over that time (weak scaling).
"""
from __future__ import annotations

import os


def world() -> tuple[int, int, int]:
    """(rank, local_rank, world_size) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of `value` over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_throughput(work_per_rank: float, seconds_max: float, world_size: int) -> float:
    """Whole-job throughput: every rank did `work_per_rank`; the job took the
    slowest rank's time."""
    return world_size * work_per_rank / seconds_max
