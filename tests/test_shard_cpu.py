"""Sharding of a batch across ranks (world size 2, gloo, CPU): the problem
assignment, the gather of per-item arrays to rank 0, and the ordered sum of
gathered per-source gradients, whose bits equal the single-rank sum."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2103_05694_gb300 import shard  # noqa: E402

N_SRC, SHAPE = 7, (5, 6)


def _items():
    rng = np.random.Generator(np.random.PCG64(11))
    # per-source gradients with mixed magnitudes and signs (the sum's bits then
    # depend on the order of the additions)
    return rng.standard_normal((N_SRC,) + SHAPE) * 10.0 ** rng.integers(-8, 8, (N_SRC,) + SHAPE)


def _ordered_sum(items):
    acc = np.zeros(SHAPE)
    for g in items:               # +0 + g_0 + g_1 + ... in source order
        acc = acc + g
    return acc


def test_problem_shard_covers_every_item_once():
    for n in (0, 1, 5, 88, 32):
        for world in (1, 2, 3, 8):
            got = sorted(i for r in range(world) for i in shard.problem_shard(n, r, world))
            assert got == list(range(n))
            assert shard.shard_sizes(n, world) == [len(range(r, n, world)) for r in range(world)]
    assert shard.problem_shard(88, 3, 8) == list(range(3, 88, 8))
    with pytest.raises(ValueError):
        shard.problem_shard(4, 2, 2)


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        items = _items()
        mine = shard.problem_shard(N_SRC, rank, world)
        local = torch.from_numpy(items[mine]) if mine else torch.zeros((0,) + SHAPE, dtype=torch.float64)
        got = shard.gather_items(local, N_SRC, rank, world, dist, dst=0)
        if rank == 0:
            q.put(("gathered", got.numpy()))
            q.put(("sum", _ordered_sum(got.numpy())))
        else:
            q.put(("none", got is None))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_gather_and_ordered_sum_match_single_rank(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world + 1):
        k, v = q.get(timeout=120)
        res.setdefault(k, []).append(v)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    items = _items()
    assert np.array_equal(res["gathered"][0].view(np.uint64), items.view(np.uint64))
    want = _ordered_sum(items)
    assert np.array_equal(res["sum"][0].view(np.uint64), want.view(np.uint64))
    assert all(res["none"])
    # the order matters for these inputs: another order gives other bits
    assert not np.array_equal(_ordered_sum(items[::-1]).view(np.uint64), want.view(np.uint64))
