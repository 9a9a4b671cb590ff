"""Aggregation of independent replica solves across ranks (one GPU each).

The solver does not shard a single feeder across GPUs; N ranks solve N
independent copies of the workload (weak scaling, no data-path
collective).  The job's time is the slowest rank's, and its work is the sum
over ranks -- the only cross-rank communication is this reduction of two
numbers after the timed region.
"""
from __future__ import annotations


def aggregate(seconds: float, iterations: float, device=None):
    """(max over ranks of seconds, sum over ranks of iterations); identity
    when torch.distributed is not initialized."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds), float(iterations)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([float(iterations)], dtype=torch.float64, device=device)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())
