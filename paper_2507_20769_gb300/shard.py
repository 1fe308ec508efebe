"""Multi-process helpers: one process per GPU, nodes sharded across ranks.

Subdomains and nodes are independent (Section 3.1), so a batch of nodes is
split into contiguous shards with no collective on the data path; only the
timing (max over ranks) and, when a caller wants the whole batch's results on
every rank, one all-gather of the per-node results cross process boundaries.
"""
from __future__ import annotations

import os

import numpy as np


def rank_world():
    """(rank, world_size, local_rank) from the torchrun environment"""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_range(n_items: int, rank: int, world: int):
    """contiguous [begin, end) of n_items for this rank (sizes differ by <= 1)"""
    base, extra = divmod(n_items, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    """maximum of a float over all ranks (identity without a process group)"""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def gather_node_results(local: np.ndarray, n_items: int, device=None) -> np.ndarray:
    """concatenate every rank's shard (rank order) of a per-node result array"""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return local
    world = dist.get_world_size()
    sizes = [shard_range(n_items, r, world) for r in range(world)]
    width = max(e - b for b, e in sizes)
    trail = local.shape[1:]
    buf = torch.zeros((width,) + trail, dtype=torch.float64, device=device)
    buf[: local.shape[0]] = torch.as_tensor(local, dtype=torch.float64, device=device)
    outs = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(outs, buf)
    parts = [o[: e - b].cpu().numpy() for o, (b, e) in zip(outs, sizes)]
    return np.concatenate(parts, axis=0)
