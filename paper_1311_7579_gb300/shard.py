"""Multi-GPU partitioning of the reweighting work: one process per GPU, the
histograms computed by the CUDA library on each rank.

The path shards naturally: (event, point) pairs are independent (Sec. 2.1: one
event per thread, every event's weight on its own).
  * By parameter points: each rank holds every sample and computes a contiguous
    slice of the point table (osc_histogram); no exchange is needed to compute,
    and the slices are only gathered to assemble the full table.
  * By events: each rank holds a contiguous slice of a sample's events.  The one
    exchange step is the sum of partial histograms.  Each rank computes its bins
    as exact integer digit columns (osc_histogram_digits) under the whole
    sample's fixed-point scale (osc_sample_set_bounds), the columns are summed
    with an integer all-reduce, and the total is converted once
    (osc_histogram_from_digits).  Integer addition is exact and associative, so
    the result is bit for bit that of one osc_histogram call over all events,
    on every rank, whatever the reduction order.
Collectives use torch.distributed (gloo on CPU tensors; NCCL works the same on
CUDA tensors).  This module marshals and exchanges; every bin is computed and
converted by the library's kernels.
"""
from __future__ import annotations

import numpy as np


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


def slice_sample(sample: dict, begin: int, count: int) -> dict:
    """The events [begin, begin + count) of a sample dict (path scalars kept)."""
    out = {k: (v[begin:begin + count] if isinstance(v, np.ndarray) else v) for k, v in sample.items()}
    out["n"] = count
    return out


def global_bounds(local_sample: dict, group=None):
    """(largest |w_mc|, largest E_true) over every rank's slice of a sample: the
    bounds osc_sample_set_bounds takes (an all-reduce of two maxima)."""
    import torch
    import torch.distributed as dist
    w = float(np.max(np.abs(local_sample["w_mc"]))) if local_sample["n"] else 0.0
    e = float(np.max(local_sample["e_true"])) if local_sample["n"] else 0.0
    t = torch.tensor([w, e], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t[0]), float(t[1])


def sum_digits(digits, group=None):
    """Word-wise sum over ranks of uint64 digit columns (numpy), with integer
    wrap-around: the digits of the exact total.  Returns a new uint64 array."""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(digits).view(np.int64).copy())
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.numpy().view(np.uint64)


def event_sharded_histogram(api, ctx, sample_ids, point_begin, n_points, prec, lo, hi, nbins, group=None):
    """Histograms of samples whose events are split over the ranks (each rank
    passes the ids of its own slices, loaded and bounded with
    osc_sample_set_bounds): bitwise the single-call result, on every rank."""
    digits = api.osc_histogram_digits(ctx, sample_ids, point_begin, n_points, prec, lo, hi, nbins)
    total = sum_digits(digits, group)
    return api.osc_histogram_from_digits(ctx, sample_ids, point_begin, n_points, nbins, total)


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


def point_sharded_histogram(api, ctx, sample_ids, n_points, prec, lo, hi, nbins, group=None):
    """Histograms of the whole point table, each rank computing its slice of the
    points with osc_histogram; the slices are gathered on every rank."""
    import torch
    import torch.distributed as dist
    ws, rank = dist.get_world_size(group), dist.get_rank(group)
    b, c = shard_points(n_points, ws, rank)
    n_s = len(sample_ids)
    if c > 0:
        local = api.osc_histogram(ctx, sample_ids, b, c, prec, lo, hi, nbins)
    else:
        local = np.zeros((n_s, 0, int(nbins)))
    return gather_point_histograms(torch.from_numpy(np.ascontiguousarray(local)), n_points, group).numpy()
