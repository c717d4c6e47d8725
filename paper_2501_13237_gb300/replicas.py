"""Replicas across GPUs (one process per GPU): the hot path shards by whole
jobs, so ranks share no data; each rank runs its own job (its own circuit
seed) and only the timing and the work done are combined.

The job time is the slowest rank's (a barrier precedes and follows the timed
steps), the work is the sum over ranks.  The combination uses
torch.distributed with whichever backend the caller initialised (NCCL on
GPUs; gloo on CPUs for the tests).
"""
from __future__ import annotations


def replica_seed(rank: int, base: int = 0) -> int:
    """Circuit seed of a rank: ranks run different, reproducible jobs."""
    return base + rank


def aggregate(ms: float, units: float, dist=None, device=None):
    """(max of ms over ranks, sum of units over ranks); identity without dist."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms), float(units)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
