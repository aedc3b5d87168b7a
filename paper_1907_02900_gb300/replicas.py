"""Replica runs: every rank builds and probes its own independent table (the
path needs no exchange between tables), and the whole job's rate is the
units all ranks processed over the slowest rank's time."""
from __future__ import annotations


def whole_job_rate(units_local: float, elapsed_ms_local: float, device=None) -> tuple[float, float]:
    """(units per second summed over ranks, max elapsed ms over ranks).

    Without an initialised process group this is the local rate.  `device`
    is where the reduction tensors live (CPU for gloo, the rank's GPU for
    NCCL)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return units_local / (elapsed_ms_local * 1e-3), elapsed_ms_local
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    t = torch.tensor([float(elapsed_ms_local)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()) / (float(t.item()) * 1e-3), float(t.item())
