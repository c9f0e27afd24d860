"""Slab decomposition across ranks (world size 2 and 3, gloo, CPU): each rank
solves its slab of the grid by epochs, exchanging boundary rows with its
neighbours, with the CPU oracle as the per-slab solver; the slabs put
together equal the oracle's solve of the whole grid bit for bit, on a random
2D grid with sources in several slabs, on a 3D grid, and on a grid whose
fastest path leaves a slab and comes back (several epochs)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402
from paper_2103_05694_gb300 import slabs  # noqa: E402


def _winding():
    ny, nx = 24, 60
    speed = np.full((ny, nx), 1.0)
    speed[14, :] = 50.0
    speed[2:15, 2] = 50.0
    speed[2:15, nx - 3] = 50.0
    return synth.Problem("winding", speed, 1.0, np.array([2 * nx + 2], dtype=np.int64),
                         np.zeros(1), {})


def _case(name):
    if name == "random2d":
        return synth.random_problem(3, (29, 17), n_src=3, contrast=10.0, h=0.6, src_t_max=0.3)
    if name == "random3d":
        return synth.random_problem(4, (11, 7, 9), n_src=2, contrast=6.0, h=0.8)
    return _winding()


def _worker(rank, world, port, name, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = _case(name)
        L = p.speed.shape[0]
        glo, lo, hi, ghi = slabs.extended_rows(L, world, rank)

        def solve(speed, h, src, t0):
            return oracle.fmm(speed, h, src, t0).t
        t, epochs = slabs.solve_slab(rank, world, p.speed[glo:ghi], p.h, L, p.sources, p.src_t,
                                     solve, dist)
        q.put((rank, lo, hi, t, epochs))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_slab_rows():
    assert slabs.slab_rows(10, 3) == [0, 3, 6, 10]
    assert slabs.extended_rows(10, 3, 0) == (0, 0, 3, 4)
    assert slabs.extended_rows(10, 3, 1) == (2, 3, 6, 7)
    assert slabs.extended_rows(10, 3, 2) == (5, 6, 10, 10)
    with pytest.raises(ValueError):
        slabs.slab_rows(3, 4)


@pytest.mark.parametrize("name,world", [("random2d", 2), ("random2d", 3), ("random3d", 2),
                                        ("winding", 2)])
def test_ranks_reach_the_oracle_fixed_point(name, world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, name, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    prob = _case(name)
    ref = oracle.fmm(prob.speed, prob.h, prob.sources, prob.src_t).t
    got = np.empty_like(ref)
    epochs = set()
    for rank, lo, hi, t, ep in parts:
        got[lo:hi] = t
        epochs.add(ep)
    assert len(epochs) == 1                     # every rank stops at the same epoch
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
    if name == "winding":
        assert epochs.pop() >= 3
