"""Multi-GPU use of the rasterizer: replicas, one process per GPU.

Views are independent (each view is binned, sorted and composited on its own), so several GPUs
render several views with no data-path exchange: every rank holds the scene and renders its own
share of the views (weak scaling).  The only collectives are on the host side of a measurement:
a barrier around the timed region and the maximum of the ranks' times.  These helpers work on any
torch.distributed backend (NCCL on GPUs, gloo in the CPU tests).
"""
from __future__ import annotations

import os
from typing import Optional, Sequence


def dist_env() -> tuple:
    """(world size, rank, local rank) from the launcher's environment (1, 0, 0 when absent)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def views_for_rank(views: Sequence, rank: int, world_size: int) -> list:
    """The cycle of views rank `rank` renders: views rank, rank + N, rank + 2N, ... (wrapping), as
    many as there are views, so that every rank does the same amount of work per step and, when
    N divides the number of views, the ranks' views are disjoint."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("need 0 <= rank < world_size")
    n = len(views)
    return [views[(rank + i * world_size) % n] for i in range(n)]


def max_over_ranks(x: float, device=None) -> float:
    """The largest of the ranks' values (the job's time is its slowest rank's); x itself on one
    process or without an initialised process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device=None):
    """Host barrier across the ranks (a no-op on one process); synchronises the device first."""
    import torch
    import torch.distributed as dist
    if device is not None and torch.cuda.is_available() and getattr(device, "type", "") == "cuda":
        torch.cuda.synchronize(device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
    if device is not None and torch.cuda.is_available() and getattr(device, "type", "") == "cuda":
        torch.cuda.synchronize(device)


def job_throughput(units_per_rank: float, world_size: int, ms_total_max: Optional[float]) -> float:
    """Whole-job rate: the units all ranks processed divided by the slowest rank's time (per s)."""
    if not ms_total_max or ms_total_max <= 0:
        return 0.0
    return world_size * units_per_rank / (ms_total_max / 1e3)
