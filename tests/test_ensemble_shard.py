"""Sharding of an ensemble across ranks (host logic of the multi-GPU path):
world_size-2 gloo process group on CPU. Every rank computes its shard on its
own; the gathered shards must partition the replicates, agree across ranks
and balance the particle counts; the timing reduction is a max over ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1805_11007_gb300 import ensemble as en
from paper_1805_11007_gb300 import workloads as wl


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, sizes, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = en.shard_replicates(sizes, world)[rank]
        shards = [None] * world
        dist.all_gather_object(shards, mine)
        # the step time of a rank grows with its particles: max over ranks
        t = torch.tensor([float(np.asarray(sizes)[mine].sum())], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        q.put((rank, shards, float(t.item())))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_shards_partition_and_balance(world):
    _, sizes, _, _ = wl.ensemble_state(replicates=64)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, sizes.tolist(), q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shards = got[0][1]
    assert all(g[1] == shards for g in got)  # every rank sees the same split
    flat = sorted(r for s in shards for r in s)
    assert flat == list(range(len(sizes)))  # a partition
    loads = [int(sizes[s].sum()) for s in shards]
    assert max(loads) - min(loads) <= int(sizes.max())  # greedy bound
    assert all(g[2] == max(loads) for g in got)


def test_shard_single_rank_and_empty():
    assert en.shard_replicates([5, 1, 3], 1) == [[0, 1, 2]]
    assert en.shard_replicates([], 3) == [[], [], []]
    s = en.shard_replicates([10, 10, 10, 10], 4)
    assert sorted(len(v) for v in s) == [1, 1, 1, 1]


def test_split_and_take_roundtrip():
    p, sizes, pos, sp = wl.ensemble_state(sizes=[3, 0, 5, 1])
    parts = en.split(pos, sizes)
    assert [len(x) for x in parts] == [3, 0, 5, 1]
    s2, p2, sp2 = en.take(pos, sp, sizes, [2, 0])
    assert s2.tolist() == [5, 3]
    np.testing.assert_array_equal(p2, np.concatenate([parts[2], parts[0]]))


def _gather_worker(rank, world, port, sizes, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = en.shard_replicates(sizes, world)[rank]
        # stand-in observables of this rank's replicates: (replicate, size, rank)
        rows = np.array([[r, sizes[r], rank] for r in mine], dtype=np.float64).reshape(-1, 3)
        allr = en.gather_replicates(rows, sizes, world, rank, dist.all_gather_object)
        q.put((rank, allr))
    finally:
        dist.destroy_process_group()


def test_gather_replicates_in_global_order():
    """The final exchange of a sharded ensemble: every rank ends with every
    replicate's row, in global replicate order, from the rank that ran it."""
    _, sizes, _, _ = wl.ensemble_state(replicates=37)
    sizes = sizes.tolist()
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gather_worker, args=(r, world, port, sizes, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shards = en.shard_replicates(sizes, world)
    owner = {r: k for k, s in enumerate(shards) for r in s}
    for rank in range(world):
        rows = got[rank]
        assert rows.shape == (len(sizes), 3)
        np.testing.assert_array_equal(rows[:, 0], np.arange(len(sizes)))
        np.testing.assert_array_equal(rows[:, 1], np.asarray(sizes, np.float64))
        np.testing.assert_array_equal(rows[:, 2], [owner[r] for r in range(len(sizes))])
    # one rank: no process group needed
    one = en.gather_replicates(np.arange(len(sizes))[:, None], sizes, 1, 0)
    np.testing.assert_array_equal(one[:, 0], np.arange(len(sizes)))
