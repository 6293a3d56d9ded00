"""Multi-GPU helpers.  The instances of a batch are independent (Sec. 3),
so a batch shards over ranks with no data-path exchange: every rank solves
its own slice, and the only collective is the MAX of the step time that the
benchmark reports.  The helpers take the process group as an argument, so the
same code runs on NCCL (one GPU per rank) and on gloo (CPU tests)."""
from __future__ import annotations

from typing import Optional, Tuple

import torch
import torch.distributed as dist


def shard(n_total: int, rank: int, world: int) -> Tuple[int, int]:
    """[start, stop) of rank's contiguous share of n_total instances (the
    first n_total % world ranks take one more)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def max_over_ranks(x: float, device: Optional[torch.device] = None, group=None) -> float:
    """MAX of a per-rank scalar (e.g. the timed region's milliseconds)."""
    if not dist.is_available() or not dist.is_initialized():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sum_over_ranks(x: float, device: Optional[torch.device] = None, group=None) -> float:
    """SUM of a per-rank scalar (e.g. the instance-steps each rank processed)."""
    if not dist.is_available() or not dist.is_initialized():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())
