"""Spreading independent channels over ranks (one GPU per rank).

The X-step is trivially parallel over frequency channels (Section 2: the
channels are processed independently; Section 7 likewise), so a multi-GPU run
needs no collective on the data path: each rank correlates its own channels.
These helpers cover the bookkeeping: which channels a rank owns, the
max-over-ranks time of a timed region, and the job-wide throughput.
"""
from __future__ import annotations

from typing import Tuple


def channel_range(n_channels: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous [lo, hi) of the channels owned by ``rank`` of ``world``; the
    first ``n_channels % world`` ranks get one channel more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    base, extra = divmod(n_channels, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def max_over_ranks(value: float, group=None, device=None) -> float:
    """Maximum of ``value`` over the ranks of ``group`` (identity without an
    initialised process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def job_throughput(units_per_rank, seconds_max: float) -> float:
    """Work units of all ranks divided by the slowest rank's time."""
    total = float(sum(units_per_rank)) if hasattr(units_per_rank, "__iter__") else float(units_per_rank)
    return total / seconds_max
