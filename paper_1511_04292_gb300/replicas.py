"""Multi-GPU replicas: every rank solves its own problem; no data-path collective.

SRJ sweeps need no exchange between independent problems, so N GPUs run N
independent solves (weak scaling).  The only collectives are the timing ones:
a barrier before and after the timed region and a MAX reduction of the elapsed
time, so the reported throughput is (sum of the ranks' work) / (slowest rank).
"""
from __future__ import annotations

import torch


def world():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def aggregate(elapsed_ms: float, updates: float, device=None):
    """Return (max elapsed ms over ranks, total updates over ranks, world size)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return elapsed_ms, updates, 1
    t = torch.tensor([elapsed_ms, updates], dtype=torch.float64, device=device)
    mx = t[:1].clone()
    sm = t[1:].clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx.item()), float(sm.item()), dist.get_world_size()


def throughput(elapsed_ms: float, updates: float, device=None):
    """Whole-job Gupdates/s over all ranks: total updates / slowest rank's time."""
    mx, total, n = aggregate(elapsed_ms, updates, device)
    return total / (mx / 1e3) / 1e9, mx, n
