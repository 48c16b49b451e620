"""Data-parallel layout of the hologram path over ranks (one process per GPU).

Targets (and OSPR subframes) are independent: no step of an iteration
exchanges data between targets, so ranks split the targets and run with no
collective on the data path.  What crosses ranks is the bookkeeping around
it: the step time (max over ranks, since the job is as slow as its slowest
rank) and, for a caller that wants every result in one place, a final gather
of per-target outputs (MSE curves, holograms) in rank order.

Works with any torch.distributed backend: NCCL for CUDA tensors on GPU
ranks, gloo for CPU tensors (the multi-rank tests run on CPU).
"""
from __future__ import annotations

import torch


def target_seeds(rank: int, batch: int, base: int = 1000):
    """Seeds of the `batch` targets rank `rank` generates (weak scaling: every
    rank its own batch): base + rank * batch + b, disjoint across ranks."""
    return [base + rank * batch + b for b in range(batch)]


def shard(total: int, rank: int, world: int):
    """(start, count) of rank `rank`'s share of `total` targets split as
    evenly as possible (strong scaling): the first total % world ranks take
    one extra target.  Shares are contiguous and cover 0..total-1 once."""
    q, r = divmod(total, world)
    count = q + (1 if rank < r else 0)
    start = rank * q + min(rank, r)
    return start, count


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks (1 rank: value itself)."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_rows(t: torch.Tensor, counts):
    """Concatenation in rank order of every rank's `t` ([count_r][...], the
    same trailing shape on every rank, count_r = counts[r]); returned on all
    ranks.  Used once, after the runs, to collect per-target outputs."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return t
    world = dist.get_world_size()
    m = max(counts)
    pad = torch.zeros((m,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
    pad[: t.shape[0]] = t
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    return torch.cat([parts[r][: counts[r]] for r in range(world)])


def average_over_ranks(t: torch.Tensor) -> torch.Tensor:
    """In place: t becomes the mean of every rank's t (an all-reduce), the
    exchange of data-parallel training (each rank's gradient of its shard's
    mean loss; equal shards make the mean of the means the whole batch's)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        t.div_(dist.get_world_size())
    return t


def weak_scaling_rate(world: int, units_per_rank: float, max_seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    return world * units_per_rank / max_seconds
