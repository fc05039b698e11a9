"""Aggregation of independent per-rank replicas (weak scaling).

Every rank builds and solves its own problem; nothing is exchanged on the
data path.  The only cross-rank steps are a barrier before the timed region
and two reductions after it: the maximum of the per-rank timed durations and
the sum of the units processed.  Works with any torch.distributed backend
(NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations


def aggregate(units: float, ms: float, device=None):
    """(total units over ranks, max ms over ranks); identity when not distributed."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(units), float(ms)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


def throughput(units: float, ms: float, device=None) -> float:
    """Whole-job throughput: units of all ranks over the slowest rank's time."""
    total, mx = aggregate(units, ms, device)
    return total / (mx / 1e3)
