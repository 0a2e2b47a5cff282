"""Whole-job accounting for N independent replicas of the solve (one process per GPU).

The fermion solve of one lattice is not sharded here: every rank solves its own
system, so the job's time is the slowest rank's and its work is the sum over
ranks (weak scaling).  Nothing on the data path is communicated.
"""
from __future__ import annotations


def replica_reduce(local_ms: float, local_units: float, dist=None, device=None):
    """(max over ranks of local_ms, sum over ranks of local_units); identity without a group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(local_ms), float(local_units)
    import torch

    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.barrier()
    return float(t.item()), float(u.item())
