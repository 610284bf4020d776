"""The z-slab decomposition across processes: two ranks of a gloo group on
the one GPU, each holding one sub-domain, the messages exchanged by
DistExchange (staged through host memory by gloo; with NCCL on several GPUs
the same calls send device buffers). Every step of the gathered run is
checked against the FP64 oracle's step from the previous gathered state.
The exchange waits on the host only: no kernel of one rank waits on the
other's."""
import datetime
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import chemo_oracle as orc
from paper_1805_11007_gb300 import chemo
from paper_1805_11007_gb300 import workloads as wl
from parity_util import assert_step_matches

pytestmark = pytest.mark.gpu

NSTEPS = 3


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, p, pos, sp, c0, q):
    import torch
    import torch.distributed as dist
    from paper_1805_11007_gb300 import slabs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=180))
    try:
        torch.cuda.set_device(0)
        layout = slabs.SlabLayout(p, world, z=pos[:, 2])
        recs = slabs.initial_records(layout, pos, sp)
        sub = slabs.Subdomain(layout, rank, pos.shape[0], stream=torch.cuda.Stream())
        try:
            chemo.chemo_slab_ingest(sub.sim, recs[rank], stream=sub.stream)
            q0, q1 = layout.local_planes(rank)
            sub.write_field(c0[q0:q1 + 1])
            torch.cuda.synchronize()
            run = slabs.SlabRun(layout, {rank: sub}, slabs.DistExchange({rank: sub}), pos.shape[0])
            states = []
            for _ in range(NSTEPS):
                run.step()
                states.append((sub.read_own_cells(), sub.read_own_field()))
            sub.check()
            parts = [None] * world
            dist.all_gather_object(parts, (layout.P, states))
            if rank == 0:
                q.put(parts)
        finally:
            sub.close()
    finally:
        dist.destroy_process_group()


def test_two_ranks_on_one_gpu_match_oracle_every_step():
    p, pos, sp = wl.initial_state("clumps_grid_3d", n=100000, grid=[64, 64, 64])
    c0 = wl.random_field(p, seed=7, scale=0.3)
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, p, pos, sp, c0, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    parts = q.get(timeout=600)
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    cuts = parts[0][0]
    assert parts[1][0] == cuts and len(cuts) == world + 1
    orc.set_threads(max(1, orc.get_threads()))
    x, s, c = pos, sp, c0
    for n in range(NSTEPS):
        recs = np.concatenate([parts[r][1][n][0] for r in range(world)])
        ids = recs["tag"] & np.uint32(chemo.GHOST_ID)
        np.testing.assert_array_equal(np.sort(ids), np.arange(pos.shape[0], dtype=np.uint32))  # every cell, once
        r = recs[np.argsort(ids)]
        x1 = np.stack([r["x"], r["y"], r["z"]], axis=1)
        s1 = (r["tag"] >> np.uint32(chemo.SPECIES_SHIFT)).astype(np.uint8)
        c1 = np.concatenate([parts[k][1][n][1] for k in range(world)])
        assert c1.shape == c0.shape
        assert_step_matches(p, x, s, c, x1, s1, c1, step_index=n)
        x, s, c = x1, s1, c1
