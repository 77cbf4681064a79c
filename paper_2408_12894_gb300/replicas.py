"""Multi-GPU use of the path: independent replicas, one process per GPU.

Rendering and differentiating different views are independent, so ranks need no data
exchange: each rank renders its own share of the views (``shard``), and the only collective
is the benchmark's reduction of per-rank times (``max_over_ranks``). Training with shared
parameters would add one gradient all-reduce per step; that exchange is not part of this
module."""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def world() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the torchrun environment (1 process if unset)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(items, rank: int, world_size: int):
    """Round-robin share of ``items`` for ``rank``: every item lands on exactly one rank."""
    return list(items)[rank::world_size]


def max_over_ranks(values, device=None):
    """Element-wise maximum over all ranks (identity without a process group)."""
    vals = [float(v) for v in values]
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return vals
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def barrier(device_sync: bool = True):
    if dist.is_available() and dist.is_initialized():
        dist.barrier()
    if device_sync and torch.cuda.is_available():
        torch.cuda.synchronize()
