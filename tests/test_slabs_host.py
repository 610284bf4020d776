"""Host logic of the z-slab decomposition (paper_1805_11007_gb300/slabs.py),
no GPU: the layout (planes, ranges, halo, the sub-domains' parameters), the
first distribution of the cells, and the step's exchange protocol run over a
CPU stand-in of the sub-domains (tests/slab_fake.py) -- in one process
(LocalExchange) and as world_size-2 and -3 gloo groups (DistExchange) --
against the same toy step on one domain."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1805_11007_gb300 import chemo
from paper_1805_11007_gb300 import slabs
from paper_1805_11007_gb300 import workloads as wl
from slab_fake import fake_run


def _params(substeps=0, gz=40):
    p = dict(wl.params("clumps_grid_3d"))
    p.update(grid=[4, 4, gz], diameter=[0.03, 0.03], D=[1e-4, 1e-4], dt=1e-4, pde_substeps=substeps)
    return p


def _cells(n=1500, seed=3):
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)).astype(np.float32)
    sp = rng.integers(0, 2, n).astype(np.uint8)
    return pos, sp


# ---------------------------------------------------------------------------
# Layout
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("K", [1, 2, 3, 5])
def test_layout_partitions_planes_and_space(K):
    p = _params()
    L = slabs.SlabLayout(p, K)
    g = L.g
    owned = [L.owned_planes(k) for k in range(K)]
    assert owned[0][0] == 0 and owned[-1][1] == g
    assert all(owned[k][1] == owned[k + 1][0] for k in range(K - 1))
    rng = [L.own_range(k) for k in range(K)]
    assert rng[0][0] == -np.inf and rng[-1][1] == np.inf
    assert all(rng[k][1] == rng[k + 1][0] for k in range(K - 1))  # the same float on both sides of a face
    for k in range(K):
        q0, q1 = L.local_planes(k)
        a, b = owned[k]
        assert q0 == max(0, a - L.H) and q1 == (g - 1 if k == K - 1 else b - 1 + L.H)
        lp = L.local_params(k)
        assert lp["grid"][2] == q1 - q0 + 1 and lp["grid"][:2] == p["grid"][:2]
        h = (lp["hi"][2] - lp["lo"][2]) / (lp["grid"][2] - 1)
        assert abs(h - L.h) <= 1e-14 * L.h
        assert abs(lp["lo"][2] - (L.lo + q0 * L.h)) <= 1e-15
        o = L.open_faces(k)
        assert bool(o & chemo.OPEN_ZLO) == (k > 0) and bool(o & chemo.OPEN_ZHI) == (k < K - 1)
        for j in L.neighbours(k):
            # the planes of k's grid that j owns are k's halo toward j: H of them
            s0, s1 = L.shared(k, j)
            assert s1 - s0 == L.H
            assert (s1 <= a) if j < k else (s0 >= b)
            # the ghost band fits in k's box
            z0, z1 = L.select_range(k)
            if j < k:
                assert z0 >= L.lo + q0 * L.h
            else:
                assert z1 <= L.lo + q1 * L.h


def test_layout_rejects_what_it_cannot_decompose():
    p = _params()
    with pytest.raises(ValueError):
        slabs.SlabLayout(p, 20)  # slabs thinner than the halo
    with pytest.raises(ValueError):
        slabs.SlabLayout(p, 2, halo_planes=1)
    with pytest.raises(ValueError):
        slabs.SlabLayout(dict(p, boundary=1, pde_bc=2), 2)
    with pytest.raises(ValueError):
        slabs.SlabLayout(dict(wl.params("walls_grid_2d")), 2)
    with pytest.raises(ValueError):
        slabs.SlabLayout(p, 3, planes=[10])  # one cut for three slabs


def test_substeps_and_drift_widen_the_halo():
    L = slabs.SlabLayout(_params(substeps=6), 2)
    assert L.substeps == 6 and L.H >= 6
    a = slabs.SlabLayout(_params(), 2)
    b = slabs.SlabLayout(_params(), 2, max_drift=0.1)
    assert (b.H - 1) * b.h >= 0.1 and b.H > a.H


def test_balanced_cuts_follow_the_cells():
    p = _params(gz=200)
    rng = np.random.default_rng(1)
    z = np.clip(rng.normal(0.4, 0.15, 20000), 0, 1)
    L = slabs.SlabLayout(p, 4, z=z)
    counts = [np.sum((z >= L.lo + L.P[k] * L.h) & (z < (L.lo + L.P[k + 1] * L.h if k < 3 else 2.0)))
              for k in range(4)]
    # each cut is the nearest plane to a quantile: half a plane of cells off
    # at most, two cuts per slab
    per_plane = 20000 * (L.h / (0.15 * np.sqrt(2 * np.pi)))  # cells in the densest plane
    assert max(abs(c - 5000) for c in counts) <= per_plane
    # cuts closer than the halo are pushed apart: every slab keeps H planes
    L2 = slabs.SlabLayout(p, 4, z=np.clip(rng.normal(0.3, 0.02, 20000), 0, 1))
    assert min(np.diff(L2.P)) >= L2.H


def test_initial_records_own_each_cell_once_and_ghost_the_bands():
    p = _params()
    pos, sp = _cells()
    L = slabs.SlabLayout(p, 3)
    recs = slabs.initial_records(L, pos, sp)
    owner = np.full(pos.shape[0], -1)
    for k, r in enumerate(recs):
        ids = r["tag"] & np.uint32(chemo.GHOST_ID)
        own = ids != chemo.GHOST_ID
        assert np.all(owner[ids[own]] == -1)
        owner[ids[own]] = k
        np.testing.assert_array_equal(r["tag"][own] >> np.uint32(29), sp[ids[own]])
        z0, z1 = L.own_range(k)
        assert np.all((r["z"][own] >= z0) & (r["z"][own] < z1))
        # ghosts: exactly the other slabs' cells within the ghost width of this slab
        s0, s1 = L.select_range(k)
        z = pos[:, 2]
        want = np.sort(z[(z >= s0) & (z < s1) & ~((z >= z0) & (z < z1))])
        np.testing.assert_array_equal(np.sort(r["z"][~own]), want)
    assert np.all(owner >= 0)


# ---------------------------------------------------------------------------
# The step's exchanges over the CPU stand-in
# ---------------------------------------------------------------------------
NSTEPS = 6


def _reference(p, pos, sp, c0):
    run = fake_run(slabs.SlabLayout(p, 1), pos, sp, c0, pos.shape[0], slabs.LocalExchange)
    run.step_n(NSTEPS)
    return _gather(run)


def _gather(run):
    recs = np.concatenate([run.subs[k].read_own_cells() for k in sorted(run.subs)])
    ids = recs["tag"] & np.uint32(chemo.GHOST_ID)
    r = recs[np.argsort(ids)]
    field = np.concatenate([run.subs[k].read_own_field() for k in sorted(run.subs)])
    return np.sort(ids), np.stack([r["x"], r["y"], r["z"]], 1), r["dz"], field


def _compare(got, ref):
    ids, pos, dz, field = got
    rids, rpos, rdz, rfield = ref
    np.testing.assert_array_equal(ids, rids)  # every cell, once
    np.testing.assert_array_equal(pos, rpos)  # the same moves: ghosts were complete
    np.testing.assert_array_equal(dz, rdz)
    np.testing.assert_allclose(field, rfield, rtol=1e-12, atol=1e-12 * np.abs(rfield).max())


@pytest.mark.parametrize("K,substeps", [(2, 1), (3, 1), (3, 2)])
def test_local_exchange_matches_one_domain(K, substeps):
    p = _params(substeps=substeps)
    pos, sp = _cells()
    c0 = np.linspace(0.0, 1.0, p["grid"][2])
    ref = _reference(p, pos, sp, c0)
    L = slabs.SlabLayout(p, K)
    run = fake_run(L, pos, sp, c0, pos.shape[0], slabs.LocalExchange)
    start = {k: set((run.subs[k].read_own_cells()["tag"] & np.uint32(chemo.GHOST_ID)).tolist()) for k in run.subs}
    run.step_n(NSTEPS)
    _compare(_gather(run), ref)
    end = {k: set((run.subs[k].read_own_cells()["tag"] & np.uint32(chemo.GHOST_ID)).tolist()) for k in run.subs}
    assert any(start[k] != end[k] for k in run.subs)  # cells migrated


def test_missing_ghosts_are_seen():
    # the same run with ghost bands cut to nothing must not match: the
    # comparison above sees the ghosts' part of the step
    p = _params()
    pos, sp = _cells()
    c0 = np.linspace(0.0, 1.0, p["grid"][2])
    ref = _reference(p, pos, sp, c0)
    L = slabs.SlabLayout(p, 2)
    L.select_range = L.own_range
    run = fake_run(L, pos, sp, c0, pos.shape[0], slabs.LocalExchange)
    run.step_n(NSTEPS)
    with pytest.raises(AssertionError):
        _compare(_gather(run), ref)


def test_capacity_overflow_is_reported():
    p = _params()
    pos, sp = _cells()
    c0 = np.zeros(p["grid"][2])
    run = fake_run(slabs.SlabLayout(p, 2), pos, sp, c0, 800, slabs.LocalExchange)
    with pytest.raises(chemo.ChemoError) as ei:
        run.step()
    assert ei.value.status == chemo.EOVERFLOW


def test_a_lost_cell_is_reported():
    p = _params()
    pos, sp = _cells()
    c0 = np.zeros(p["grid"][2])
    run = fake_run(slabs.SlabLayout(p, 2), pos, sp, c0, pos.shape[0], slabs.LocalExchange)
    run.total += 1  # one cell more than the sub-domains hold
    with pytest.raises(chemo.ChemoError) as ei:
        run.step()
    assert ei.value.status == chemo.EDOMAIN


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, p, pos, sp, c0, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        L = slabs.SlabLayout(p, world)
        run = fake_run(L, pos, sp, c0, pos.shape[0], slabs.DistExchange, ranks=[rank])
        run.step_n(NSTEPS)
        mine = (run.subs[rank].read_own_cells(), run.subs[rank].read_own_field())
        parts = [None] * world
        dist.all_gather_object(parts, mine)
        q.put((rank, parts))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,substeps", [(2, 1), (3, 2)])
def test_dist_exchange_over_gloo_matches_one_domain(world, substeps):
    p = _params(substeps=substeps)
    pos, sp = _cells()
    c0 = np.linspace(0.0, 1.0, p["grid"][2])
    ref = _reference(p, pos, sp, c0)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, p, pos, sp, c0, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = [q.get(timeout=180) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    parts = got[0][1]
    recs = np.concatenate([c for c, _ in parts])
    ids = recs["tag"] & np.uint32(chemo.GHOST_ID)
    r = recs[np.argsort(ids)]
    field = np.concatenate([f for _, f in parts])
    _compare((np.sort(ids), np.stack([r["x"], r["y"], r["z"]], 1), r["dz"], field), ref)
