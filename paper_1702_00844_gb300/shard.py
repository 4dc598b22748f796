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


def sum_over_ranks(value: float, group=None, device=None) -> float:
    """Sum of ``value`` over the ranks of ``group`` (identity without an
    initialised process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())


def corner_turn(x_local, S: int, C: int, T: int, I: int, dtype: str, group=None, reorder_fn=None):
    """The FX corner turn of Section 7 over the ranks of ``group``: before the
    exchange every rank holds all channels of its own stations, afterwards
    every rank holds its own channels of all stations.

    x_local: this rank's stations ``station_range(S, world, rank)`` in the
    station-major layout "sct", shape ``layout_shape(S/world, C, T, I, dtype,
    "sct")``. Returns this rank's channels ``channel_range(C, world, rank)``
    of all S stations in the correlator's layout "cst". S must be a multiple
    of the world size.

    One ``all_to_all_single`` per integration; the local permutations around
    it (into channel-major order before, and source rank <-> channel after)
    run through ``reorder_fn`` (default: the library's ``corr_reorder``, for
    device tensors)."""
    import torch
    import torch.distributed as dist
    from .corr import reorder as lib_reorder
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    if S % world:
        raise ValueError("corner_turn: the station count must be a multiple of the world size")
    if reorder_fn is None:
        if not x_local.is_cuda:
            raise ValueError("corner_turn: device tensors expected (or pass reorder_fn)")
        reorder_fn = lib_reorder
    Sr = S // world
    # 1. [I][Sr][C][T] -> [I][C][Sr][T]: each destination's channels contiguous
    x_cst = reorder_fn(x_local, Sr, C, T, I, dtype, "sct", "cst")
    if world == 1:
        return x_cst
    lo, hi = channel_range(C, world, rank)
    Cr = hi - lo
    sample_shape = tuple(x_cst.shape[4:])   # pols (x re/im)
    per_ch = Sr * T * x_cst[0, 0, 0, 0].numel() * x_cst.element_size()  # bytes per channel
    send_splits = [(channel_range(C, world, q)[1] - channel_range(C, world, q)[0]) * per_ch
                   for q in range(world)]
    outs = []
    for i in range(I):
        # exchanged as bytes, whatever the sample type
        send = x_cst[i].reshape(-1).view(torch.uint8)
        recv = torch.empty(world * Cr * per_ch, dtype=torch.uint8, device=x_cst.device)
        dist.all_to_all_single(recv, send, output_split_sizes=[Cr * per_ch] * world,
                               input_split_sizes=send_splits, group=group)
        # 2. recv = [source rank q][Cr][Sr][T] -> [Cr][q][Sr][T] = [Cr][S][T]: the
        # same permutation as "sct" -> "cst" with q as the station axis and
        # (station of q, time) as the time axis
        shaped = recv.view(x_cst.dtype).view((1, world, Cr, Sr * T) + sample_shape)
        outs.append(reorder_fn(shaped, world, Cr, Sr * T, 1, dtype, "sct", "cst")
                    .view((1, Cr, S, T) + sample_shape))
    return torch.cat(outs, 0) if I > 1 else outs[0]


def job_throughput(units_per_rank, seconds_max: float) -> float:
    """Work units of all ranks divided by the slowest rank's time."""
    total = float(sum(units_per_rank)) if hasattr(units_per_rank, "__iter__") else float(units_per_rank)
    return total / seconds_max
