"""Multi-GPU runs: independent replicas and cell shards, no collective on the data path.

Interference is a property of one GPU, so a sweep never spans GPUs.  With N ranks
(one process per GPU, torch.distributed initialised by torchrun) the work splits
round-robin — whole victims for a sweep, or whole cells — and only three host-side
exchanges remain: a barrier around the timed region, the maximum of the ranks'
times, and a gather of the result rows onto rank 0.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def world():
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(), dist.get_rank()
    return 1, 0


def shard(items, world_size: int, rank: int):
    """Round-robin share of `items` for `rank` (items rank, rank + N, ...)."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("bad rank %d of %d" % (rank, world_size))
    return list(items)[rank::world_size]


def max_over_ranks(values, device=None):
    """Element-wise maximum of a list of floats over all ranks."""
    n, _ = world()
    if n == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def gather_rows(rows):
    """All ranks' result rows (any picklable objects), concatenated in rank order;
    returned on every rank."""
    n, _ = world()
    if n == 1:
        return list(rows)
    parts = [None] * n
    dist.all_gather_object(parts, list(rows))
    return [r for p in parts for r in p]


def barrier():
    n, _ = world()
    if n > 1:
        dist.barrier()
