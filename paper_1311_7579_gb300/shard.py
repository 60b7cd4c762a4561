"""Multi-GPU partitioning of the reweighting work (host logic only).

The path shards naturally: (event, point) pairs are independent.
  * By parameter points: each rank holds every sample and computes a contiguous
    slice of the point table; no exchange is needed to compute, and the slices
    are only gathered to assemble the full table of histograms.
  * By events: each rank holds a contiguous slice of a sample's events and
    computes partial histograms; the one exchange step is their sum, done here
    by gathering every rank's partials and adding them in rank order, so the
    result is identical on all ranks and does not depend on a collective's
    internal reduction order.
Collectives use torch.distributed (gloo on CPU, NCCL on GPUs).
"""
from __future__ import annotations


def split_range(n: int, world_size: int, rank: int, quantum: int = 1):
    """Contiguous [begin, begin + count) slice of n items for `rank`, slices
    balanced to within one quantum (slice starts are multiples of `quantum`)."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("bad world_size / rank")
    units = -(-n // quantum)
    base, extra = divmod(units, world_size)
    u0 = rank * base + min(rank, extra)
    u1 = u0 + base + (1 if rank < extra else 0)
    begin = min(n, u0 * quantum)
    end = min(n, u1 * quantum)
    return begin, end - begin


def shard_points(n_points: int, world_size: int, rank: int):
    return split_range(n_points, world_size, rank)


def shard_events(n_events: int, world_size: int, rank: int):
    """Event slices start on multiples of 64 events (the kernels' item granularity)."""
    return split_range(n_events, world_size, rank, quantum=64)


def gather_point_histograms(local, n_points: int, group=None):
    """local: tensor [n_samples, count_r, nbins] for this rank's point slice.
    Returns the full [n_samples, n_points, nbins] tensor on every rank."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size(group)
    counts = [shard_points(n_points, ws, r)[1] for r in range(ws)]
    width = max(counts)
    pad = torch.zeros(local.shape[0], width, local.shape[2], dtype=local.dtype, device=local.device)
    pad[:, :local.shape[1]] = local
    parts = [torch.empty_like(pad) for _ in range(ws)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([parts[r][:, :counts[r]] for r in range(ws)], dim=1)


def sum_event_histograms(local, group=None):
    """Sum of every rank's partial histograms, added in rank order (deterministic
    and identical on all ranks)."""
    import torch.distributed as dist
    import torch
    ws = dist.get_world_size(group)
    parts = [torch.empty_like(local) for _ in range(ws)]
    dist.all_gather(parts, local.contiguous(), group=group)
    total = parts[0].clone()
    for r in range(1, ws):
        total += parts[r]
    return total
