"""Shot-parallel runs over several processes (one GPU each).

Shots are independent (Sec. 2.5 / 3.2: every worker computes whole shot
gradients and the gradients are summed), so a multi-GPU run shards the shots
and has a single exchange: the sum of the per-rank gradients and misfits.
"""
from __future__ import annotations


def shard(nshots: int, rank: int, world: int) -> range:
    """Contiguous block of shot indices of `rank` (sizes differ by at most 1)."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    base, extra = divmod(nshots, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def sum_over_ranks(grad, misfit: float):
    """All-reduce (sum) of a gradient tensor (in place) and a misfit; returns
    the total misfit.  Works with any initialised torch.distributed backend."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return misfit
    dist.all_reduce(grad, op=dist.ReduceOp.SUM)
    J = torch.tensor([misfit], dtype=torch.float64, device=grad.device)
    dist.all_reduce(J, op=dist.ReduceOp.SUM)
    return float(J.item())
