"""The z-slab decomposition on one GPU (sub-domains on their own streams,
paper_1805_11007_gb300/slabs.py over chemo_create_subdomain and the slab
calls of include/chemo.h).

* every step of a free-running decomposed run of the 1M-cell 3D clump
  workload against the FP64 oracle's step from the gathered state (the
  tolerance of the single-domain parity tests), and its first step against
  the single-domain GPU run;
* the device exchange (selection, migration, ghosts, halo planes) builds
  exactly the sub-domains that the host distribution builds from the same
  state: the next steps agree bit for bit;
* model variants (reactions, several PDE substeps, Dirichlet walls, tamed
  move with displacement) against the oracle;
* an empty slab, a halo too thin for a move, capacities, the calls a
  sub-domain refuses, and the plane and selection calls alone.
"""
import numpy as np
import pytest
import torch

from oracle import chemo_oracle as orc
from paper_1805_11007_gb300 import chemo
from paper_1805_11007_gb300 import slabs
from paper_1805_11007_gb300 import workloads as wl
from parity_util import assert_step_matches, increment_terms, make_sim, ulp32

pytestmark = pytest.mark.gpu


def _gather(run):
    pos, sp, disp, ids = slabs.gather_state(run)
    np.testing.assert_array_equal(ids, np.arange(run.total, dtype=np.uint32))  # every cell, once
    return pos, sp, disp, slabs.gather_field(run)


def _own_ids(run):
    return {k: np.sort(run.subs[k].read_own_cells()["tag"] & np.uint32(chemo.GHOST_ID)) for k in run.subs}


def _check_owners(run):
    """Each own cell lies in its slab's range after the exchange."""
    for k, sub in run.subs.items():
        z = sub.read_own_cells()["z"]
        z0, z1 = run.layout.own_range(k)
        assert np.all((z >= z0) & (z < z1)), k


def _cuts(run):
    return np.array([run.layout.own_range(k)[0] for k in range(1, run.layout.K)], np.float32)


@pytest.mark.parametrize("K,nsteps", [(2, 10), (3, 4)])
def test_decomposed_clump_run_matches_oracle_every_step(K, nsteps):
    p, pos, sp = wl.initial_state("clumps_grid_3d")
    c0 = wl.random_field(p, seed=7, scale=0.05)
    run = slabs.create_local(p, pos, sp, K, c0=c0)
    orc.set_threads(max(1, orc.get_threads()))
    try:
        assert run.layout.K == K and all(s.sim.n > 0 for s in run.subs.values())
        x, s, c = pos, sp, c0
        moved = 0
        for n in range(nsteps):
            run.step()
            x1, s1, _, c1 = _gather(run)
            _check_owners(run)
            assert_step_matches(p, x, s, c, x1, s1, c1, step_index=n)
            moved += int(np.sum(np.searchsorted(_cuts(run), x[:, 2], side="right")
                                != np.searchsorted(_cuts(run), x1[:, 2], side="right")))
            x, s, c = x1, s1, c1
        for sub in run.subs.values():
            sub.check()
        assert moved > 0  # cells crossed slab faces
    finally:
        slabs.close_run(run)


def test_first_decomposed_step_equals_single_domain_step():
    """From the same state both runs add the same exact pair sums and the same
    noise; they differ only in the rounding of the grid coordinates of a
    sub-domain and of the deposit's float additions."""
    p, pos, sp = wl.initial_state("clumps_grid_3d")
    c0 = wl.random_field(p, seed=7, scale=0.05)
    with make_sim(p, pos, sp, c0) as sim:
        chemo.chemo_step(sim)
        xs, ss, _ = chemo.read_state_host(sim)
        cs = chemo.read_field_host(sim)
    run = slabs.create_local(p, pos, sp, 2, c0=c0)
    try:
        run.step()
        x, s, _, c = _gather(run)
    finally:
        slabs.close_run(run)
    np.testing.assert_array_equal(s, ss)
    inc = increment_terms(p, pos, sp, c0)
    d = np.abs(x.astype(np.float64) - xs)
    assert np.all(d <= 1e-5 * inc + 2.0 * ulp32(xs))
    assert np.abs(c.astype(np.float64) - cs).max() <= 1e-5 * np.abs(cs).max()


def _equal_sets(u, v):
    return all(np.array_equal(u[k], v[k]) for k in u)


def test_device_exchange_builds_the_host_distribution():
    """Run A exchanges on the device; run B is rebuilt before every step from
    A's gathered state by the host distribution (initial_records). Their
    steps agree bit for bit, so A's selection, migration, ghosts and halo
    planes are those of the host logic."""
    p, pos, sp = wl.initial_state("clumps_grid_3d", n=200000, grid=[128, 128, 128])
    c0 = wl.random_field(p, seed=3, scale=0.3)
    a = slabs.create_local(p, pos, sp, 3, c0=c0)
    b = slabs.create_local(p, pos, sp, 3, c0=c0, planes=a.layout.P[1:-1])
    try:
        for n in range(10):
            x, s, d, ids = slabs.gather_state(a)
            c = slabs.gather_field(a)
            recs = slabs.initial_records(b.layout, x, s, disp=d, ids=ids)
            for k, sub in b.subs.items():
                chemo.chemo_slab_ingest(sub.sim, recs[k], stream=sub.stream)
                q0, q1 = b.layout.local_planes(k)
                sub.write_field(c[q0:q1 + 1])
                chemo.chemo_set_step_index(sub.sim, n, stream=sub.stream)
            torch.cuda.synchronize()
            assert _equal_sets(_own_ids(a), _own_ids(b))
            a.step()
            b.step()
            xa, sa, _, _ = slabs.gather_state(a)
            xb, sb, _, _ = slabs.gather_state(b)
            np.testing.assert_array_equal(xa, xb)
            np.testing.assert_array_equal(sa, sb)
            np.testing.assert_allclose(slabs.gather_field(a), slabs.gather_field(b), rtol=0,
                                       atol=1e-6 * np.abs(c).max() + 1e-30)
    finally:
        slabs.close_run(a)
        slabs.close_run(b)


VARIANTS = [
    ("reactions", dict(reactions=1, react_k0=[20.0, 5.0], react_kc=[0.0, 50.0], react_to=[1, 0]), 2),
    ("substeps", dict(Dc=25.0, dt=2e-5), 3),
    ("dirichlet", dict(pde_bc=1), 2),
    # four times the workload's force: a tamed drift of up to 0.026 per step
    # (the oracle's pair force at the initial state), given to the layout as
    # max_drift so that the halo reaches beyond it
    ("tamed_displacement", dict(move_scheme=1, track_displacement=1, inter=4.0), 3),
]


@pytest.mark.parametrize("name,over,K", VARIANTS, ids=[v[0] for v in VARIANTS])
def test_decomposed_variants_match_oracle(name, over, K):
    base = dict(grid=[48, 48, 48], diameter=[0.02, 0.03], dt=1e-5)
    base.update(over)
    p, pos, sp = wl.initial_state("clumps_grid_3d", n=30000, **base)
    c0 = wl.random_field(p, seed=5, scale=0.3)
    run = slabs.create_local(p, pos, sp, K, c0=c0, max_drift=0.03 if name == "tamed_displacement" else 0.0)
    try:
        if name == "substeps":
            assert run.layout.substeps > 1
        x, s, c = pos, sp, c0
        for n in range(3):
            run.step()
            x1, s1, d1, c1 = _gather(run)
            if not p.get("track_displacement") or n > 0:
                assert_step_matches(p, x, s, c, x1, s1, c1, step_index=n)
            else:  # the first step's displacement (later ones carry the sum's rounding)
                assert_step_matches(p, x, s, c, x1, s1, c1, disp_g=d1, step_index=n)
            x, s, c = x1, s1, c1
        for sub in run.subs.values():
            sub.check()
    finally:
        slabs.close_run(run)


def test_an_empty_slab_takes_part():
    p, pos, sp = wl.initial_state("clumps_grid_3d", n=20000, grid=[48, 48, 48], diameter=[0.02, 0.03], dt=1e-5)
    pos[:, 2] *= 0.3  # every cell in the lower third of the box
    c0 = wl.random_field(p, seed=5, scale=0.3)
    run = slabs.create_local(p, pos, sp, 2, c0=c0, planes=[30], balance=False)
    try:
        assert run.subs[1].read_own_cells().shape[0] == 0
        x, s, c = pos, sp, c0
        for n in range(2):
            run.step()
            x1, s1, _, c1 = _gather(run)
            assert_step_matches(p, x, s, c, x1, s1, c1, step_index=n)
            x, s, c = x1, s1, c1
    finally:
        slabs.close_run(run)


def test_an_empty_slab_receives_deposits():
    # a grid coarser than the ghost width: cells 0.012 - 0.02 below the cut
    # (more than 5.6 noise amplitudes beyond the 0.004 ghost band) are no
    # ghosts of the upper slab, which holds no cell at all, yet they deposit
    # on its first plane (within one node spacing, 0.0213, of the cut); its
    # sources are folded in every step and must be cleared every step
    # although it has no particle kernel to run
    p, pos, sp = wl.initial_state("clumps_grid_3d", n=5000, grid=[48, 48, 48], dt=1e-6)
    cut = 30
    z_cut = np.float32(cut / 47.0)
    rng = np.random.default_rng(4)
    # spread in x and y so that the band is dilute (mean spacing 0.012, three
    # times the cutoff): no pair force pushes a cell across the gap
    pos[:, :2] = rng.random((pos.shape[0], 2)).astype(np.float32)
    pos[:, 2] = (z_cut - rng.uniform(0.012, 0.02, pos.shape[0])).astype(np.float32)
    c0 = wl.random_field(p, seed=5, scale=0.3)
    run = slabs.create_local(p, pos, sp, 2, c0=c0, planes=[cut], balance=False)
    try:
        assert run.subs[1].sim.n == 0
        x, s, c = pos, sp, c0
        for n in range(4):
            run.step()
            assert run.subs[1].sim.n == 0
            x1, s1, _, c1 = _gather(run)
            assert_step_matches(p, x, s, c, x1, s1, c1, step_index=n)
            x, s, c = x1, s1, c1
    finally:
        slabs.close_run(run)


def test_a_halo_too_thin_for_a_move_is_latched():
    # noise of 0.05 per step against a box that reaches two planes of 1/47
    # beyond a face: some own cells step out of their sub-domain's box; they
    # are clamped and the step reports EDOMAIN
    p, pos, sp = wl.initial_state("clumps_grid_3d", n=20000, grid=[48, 48, 48], diameter=[0.02, 0.03],
                                  D=[125.0, 125.0], dt=1e-5)
    run = slabs.create_local(p, pos, sp, 2, halo_planes=3)
    try:
        with pytest.raises(chemo.ChemoError) as ei:
            run.step_n(1)
        assert ei.value.status == chemo.EDOMAIN
    finally:
        slabs.close_run(run)


def test_selection_past_capacity_and_ingest_beyond_capacity():
    p, pos, sp = wl.initial_state("clumps_grid_3d", n=20000, grid=[48, 48, 48], diameter=[0.02, 0.03], dt=1e-5)
    layout = slabs.SlabLayout(p, 2, z=pos[:, 2])
    run = slabs.create_local(p, pos, sp, 2, planes=layout.P[1:-1])
    try:
        sub = run.subs[0]
        guard = torch.full((4, chemo.CELL_FLOATS), 7.0, device="cuda")
        out = torch.cat([torch.zeros((5, chemo.CELL_FLOATS), device="cuda"), guard])
        cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
        chemo.chemo_slab_select(sub.sim, [(-np.inf, np.inf, -np.inf, np.inf, out[:5], cnt)], stream=sub.stream)
        torch.cuda.synchronize()
        assert int(cnt[0]) > 5 and int(cnt[1]) == int(cnt[0])  # counted past the capacity ...
        assert torch.all(out[5:] == 7.0)                       # ... and nothing written there
    finally:
        slabs.close_run(run)
    # each slab owns about half of the 20000 cells: 9000 records cannot hold
    # the first ingest, and the sub-domains already made are given back
    with pytest.raises(chemo.ChemoError) as ei:
        slabs.create_local(p, pos, sp, 2, planes=layout.P[1:-1], capacity=9000)
    assert ei.value.status == chemo.EINVAL


def test_subdomain_refuses_calls_by_id_and_checks_its_arguments():
    p, pos, sp = wl.initial_state("clumps_grid_3d", n=5000, grid=[48, 48, 48], diameter=[0.02, 0.03], dt=1e-5)
    run = slabs.create_local(p, pos, sp, 2)
    sim = run.subs[0].sim
    try:
        for call in (lambda: chemo.read_state_host(sim), lambda: chemo.chemo_observables(sim),
                     lambda: chemo.chemo_record(sim, 2, 1),
                     lambda: chemo.chemo_write_state(sim, pos[:10], sp[:10])):
            with pytest.raises(chemo.ChemoError) as ei:
                call()
            assert ei.value.status == chemo.ENOTSUP
        with pytest.raises(chemo.ChemoError) as ei:
            chemo.chemo_slab_ingest(sim, np.zeros(run.subs[0].capacity + 1, chemo.CELL_DTYPE))
        assert ei.value.status == chemo.EINVAL
        g = sim.params["grid"][2]
        buf = torch.zeros((4, 48 * 48), device="cuda")
        with pytest.raises(chemo.ChemoError) as ei:
            chemo.chemo_slab_planes(sim, 0, chemo.PLANES_READ, g - 2, 4, buf)
        assert ei.value.status == chemo.EINVAL
        with pytest.raises(chemo.ChemoError) as ei:
            chemo.chemo_slab_planes(sim, 3, chemo.PLANES_READ, 0, 1, buf)
        assert ei.value.status == chemo.EINVAL
        with pytest.raises(chemo.ChemoError) as ei:  # an ordinary simulation has no slab calls
            with make_sim(p, pos, sp) as one:
                chemo.chemo_step_particles(one)
        assert ei.value.status == chemo.ENOTSUP
    finally:
        slabs.close_run(run)


def test_planes_read_write_add():
    p, pos, sp = wl.initial_state("clumps_grid_3d", n=5000, grid=[48, 48, 48], diameter=[0.02, 0.03], dt=1e-5)
    run = slabs.create_local(p, pos, sp, 2, streams=False)
    sub = run.subs[1]
    try:
        gz = sub.sim.params["grid"][2]
        c = torch.arange(gz * 48 * 48, dtype=torch.float32, device="cuda").reshape(gz, 48 * 48)
        chemo.chemo_write_field(sub.sim, c)
        buf = torch.empty((3, 48 * 48), device="cuda")
        chemo.chemo_slab_planes(sub.sim, 0, chemo.PLANES_READ, 2, 3, buf)
        assert torch.equal(buf, c[2:5])
        chemo.chemo_slab_planes(sub.sim, 0, chemo.PLANES_ADD, 5, 3, buf)
        minus = torch.full((2, 48 * 48), -1.0, device="cuda")
        chemo.chemo_slab_planes(sub.sim, 0, chemo.PLANES_WRITE, 0, 2, minus)
        out = torch.empty_like(c)
        chemo.chemo_read_field(sub.sim, out)
        want = c.clone()
        want[5:8] += c[2:5]
        want[0:2] = -1
        assert torch.equal(out, want)
        # the source grid: written, read by the field step (a constant field
        # has no Laplacian, so one substep adds S and decays by dt gamma c),
        # cleared by the next particle step before its deposit
        chemo.chemo_write_field(sub.sim, torch.ones_like(c))
        src = torch.full((gz, 48 * 48), 0.25, device="cuda")
        chemo.chemo_slab_planes(sub.sim, 1, chemo.PLANES_WRITE, 0, gz, src)
        chemo.chemo_step_field(sub.sim)
        after = torch.empty_like(c)
        chemo.chemo_read_field(sub.sim, after)
        torch.cuda.synchronize()
        want_c = 1.0 + 0.25 - p["dt"] * p["gamma"]
        assert torch.allclose(after, torch.full_like(after, want_c), rtol=0, atol=1e-5)
        zero_cells = np.zeros(0, chemo.CELL_DTYPE)  # no cells: nothing is deposited again
        chemo.chemo_slab_ingest(sub.sim, zero_cells)
        chemo.chemo_step_particles(sub.sim)
        chemo.chemo_slab_planes(sub.sim, 1, chemo.PLANES_READ, 0, gz, src)
        torch.cuda.synchronize()
        assert torch.count_nonzero(src) == 0
    finally:
        slabs.close_run(run)
