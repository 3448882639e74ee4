"""Multi-GPU helpers: shots are independent, so ranks shard them with no data-path collective.

Only host-side bookkeeping lives here: which shots or seed stream a rank owns, and the reductions of
timing and integer counters after the decode (a max of elapsed times, a sum of counters).
"""
from __future__ import annotations


def shard_range(total: int, rank: int, world: int):
    """Contiguous [lo, hi) slice of `total` shots owned by `rank` (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of a rank's own synthetic shot stream (weak scaling: every rank decodes a full batch)."""
    return base_seed + 1000 * rank


def reduce_max(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum_counters(counters, device=None):
    """Sum an int64 counter vector (torch tensor or sequence) over ranks; returns a list of ints."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(counters, dtype=torch.int64, device=device).clone()
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [int(x) for x in t.cpu().tolist()]
