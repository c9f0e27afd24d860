"""Sharding of batched work across GPUs, one process per GPU.

The problems of a batch are independent (the paper's method solves one grid;
a batch is many such solves), so they split across ranks by problem with no
exchange during the solve: rank r takes problems r, r + N, r + 2N, ... of N
ranks.  The one step that combines problems is the tomography gradient, the
sum over sources of each source's d(loss)/d(slowness).  To give the same
bits on any number of ranks, the per-source gradients are gathered on one
rank and summed there in source order (eik_sum_ordered: +0 + g_0 + g_1 + ...,
each addition rounded to nearest), exactly as a single GPU sums them.

Only torch.distributed collectives are used here (gather, all_reduce); they
carry results between ranks and do no arithmetic of the method.
"""
from __future__ import annotations


def problem_shard(n_items: int, rank: int, world: int) -> list[int]:
    """The items rank `rank` of `world` takes: rank, rank + world, ..."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of {world}")
    return list(range(rank, n_items, world))


def shard_sizes(n_items: int, world: int) -> list[int]:
    return [len(problem_shard(n_items, r, world)) for r in range(world)]


def gather_items(local, n_items: int, rank: int, world: int, dist, dst: int = 0):
    """Gather per-item arrays on rank `dst`.

    local: tensor (k, *shape) holding this rank's items in shard order
    (k = len(problem_shard(n_items, rank, world))).  Returns, on rank dst, a
    tensor (n_items, *shape) with item i in row i; None on the other ranks.
    Shards of unequal size are padded to the largest for the collective."""
    import torch
    k = len(problem_shard(n_items, rank, world))
    if local.shape[0] != k:
        raise ValueError(f"rank {rank} holds {local.shape[0]} items, its shard has {k}")
    kmax = -(-n_items // world)
    buf = torch.zeros((kmax,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    buf[:k] = local
    bufs = [torch.empty_like(buf) for _ in range(world)] if rank == dst else None
    dist.gather(buf, bufs, dst=dst)
    if rank != dst:
        return None
    out = torch.empty((n_items,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    for r in range(world):
        ids = problem_shard(n_items, r, world)
        if ids:
            out[ids] = bufs[r][:len(ids)]
    return out
