"""Slab decomposition of one grid across ranks (one slab per rank).

The domain decomposition the paper leaves to future work (Introduction): the
grid's outermost axis is split into `world` slabs; rank r solves its slab,
extended by one ghost row on each side it shares with a neighbour, by epochs.
In every epoch the ghost rows hold the neighbour's boundary values from the
previous epoch as fixed sources (finite values only; cells the neighbour has
not reached stay free and can only give upper bounds).  After the solve each
rank sends its first and last own rows to its neighbours (an all-gather of
the boundary rows), and the epochs stop when no rank's ghost rows changed (an
all-reduce of one flag: the global AND).  Ghost values only decrease, so the
loop ends, and then every cell satisfies the local update with its
neighbours' final values: the slabs together hold the unique fixed point of
the whole grid (Theorem 1), bit for bit.

`eik_solve_slabs` runs the same decomposition with every slab on one device;
this module is the mapping onto ranks, with the per-slab solve passed in (on
a GPU: the library's `solve`).  Only torch.distributed collectives cross
ranks; no kernel waits on another rank.
"""
from __future__ import annotations

import math

import numpy as np


def slab_rows(L: int, world: int) -> list[int]:
    """Row boundaries lo[0..world] of `world` near-equal slabs of L rows."""
    if not 1 <= world <= L:
        raise ValueError(f"{world} slabs for {L} rows")
    return [k * L // world for k in range(world + 1)]


def extended_rows(L: int, world: int, rank: int) -> tuple[int, int, int, int]:
    """(glo, lo, hi, ghi): the slab's own rows [lo, hi) and, with its ghost rows,
    the extended rows [glo, ghi)."""
    lo = slab_rows(L, world)
    a, b = lo[rank], lo[rank + 1]
    return (a - 1 if a > 0 else 0), a, b, (b + 1 if b < L else L)


def solve_slab(rank: int, world: int, speed_ext: np.ndarray, h: float, L: int,
               sources, src_t, solve, dist, max_epochs: int | None = None):
    """Solve rank `rank`'s slab of a grid of L rows along its outermost axis.

    speed_ext: this slab's speeds over its extended rows [glo, ghi) (C order,
    outermost axis first); sources / src_t: the grid's sources as flat indices
    of the whole grid and their times (every rank passes the same lists);
    solve(speed, h, src_idx, src_t) -> arrival times (numpy, the speed's
    shape): the per-slab solver; dist: torch.distributed with an initialised
    process group of `world` ranks.  Returns (times of the own rows [lo, hi),
    number of epochs)."""
    import torch
    glo, lo, hi, ghi = extended_rows(L, world, rank)
    speed_ext = np.ascontiguousarray(speed_ext, dtype=np.float64)
    if speed_ext.shape[0] != ghi - glo:
        raise ValueError(f"rank {rank}: speed has {speed_ext.shape[0]} rows, the slab {ghi - glo}")
    plane = int(np.prod(speed_ext.shape[1:]))
    src = np.asarray(sources, dtype=np.int64).reshape(-1)
    t0 = np.zeros(src.size) if src_t is None else np.asarray(src_t, np.float64).reshape(-1)
    own = (src // plane >= lo) & (src // plane < hi)
    own_idx = src[own] - glo * plane
    own_t0 = t0[own]
    top = np.full(plane, math.inf)       # ghost row glo (rank - 1's last own row)
    bottom = np.full(plane, math.inf)    # ghost row ghi - 1 (rank + 1's first own row)
    limit = max_epochs or (64 + 8 * world)
    for epoch in range(1, limit + 1):
        idx, tt = [own_idx], [own_t0]
        if rank > 0:
            f = np.isfinite(top)
            idx.append(np.nonzero(f)[0].astype(np.int64))
            tt.append(top[f])
        if rank + 1 < world:
            f = np.isfinite(bottom)
            idx.append((ghi - 1 - glo) * plane + np.nonzero(f)[0].astype(np.int64))
            tt.append(bottom[f])
        t = np.asarray(solve(speed_ext, h, np.concatenate(idx), np.concatenate(tt)))
        rows = t.reshape(ghi - glo, plane)
        mine = torch.from_numpy(np.stack([rows[lo - glo], rows[hi - 1 - glo]]).copy())
        every = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(every, mine)
        new_top = every[rank - 1][1].numpy() if rank > 0 else top
        new_bottom = every[rank + 1][0].numpy() if rank + 1 < world else bottom
        changed = not (np.array_equal(new_top, top) and np.array_equal(new_bottom, bottom))
        flag = torch.tensor([1 if changed else 0], dtype=torch.int64)
        dist.all_reduce(flag, op=dist.ReduceOp.MAX)
        top, bottom = new_top.copy(), new_bottom.copy()
        if int(flag.item()) == 0:
            return rows[lo - glo:hi - glo].reshape((hi - lo,) + speed_ext.shape[1:]).copy(), epoch
    raise RuntimeError(f"slab {rank}: boundary values still changing after {limit} epochs")
