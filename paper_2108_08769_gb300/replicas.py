"""Whole-job throughput of independent replicas, one process per GPU.

A tank does not shard across GPUs here: under torchrun every rank advances
its own replica and there is no data-path collective.  The only exchange is
this aggregation of the timing: the job's rate is the units every rank
processed divided by the slowest rank's device time.
"""
from __future__ import annotations

from typing import Tuple


def aggregate(units: float, ms: float, device=None) -> Tuple[float, float, float]:
    """Return (total units over ranks, max ms over ranks, units per second).

    Works on one process (no process group) and on any initialised
    torch.distributed group: gloo with CPU tensors, nccl with tensors on
    ``device``.
    """
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(units), float(ms), float(units) / (ms * 1e-3)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item()), float(u.item()) / (float(t.item()) * 1e-3)
