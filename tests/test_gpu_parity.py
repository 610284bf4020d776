"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on
identical seeded inputs, row by row of the step and for whole steps.

Rows: a1 bins (bit-exact), a2 counting sort (valid permutation, bins in
order), a3 pair force and neighbour sets, a4 gradient interpolation, a5 move
and boundary, a6 deposit, a7 PDE; whole steps at sizes that span many tiles
with ragged tails, the full-size 3D clump workload, and edge cases.
"""
import numpy as np
import pytest
import torch

from oracle import chemo_oracle as orc
from paper_1805_11007_gb300 import chemo
from paper_1805_11007_gb300 import workloads as wl
from parity_util import (assert_forces_match, assert_step_matches, gpu_forces, make_sim, position_tolerance)

pytestmark = pytest.mark.gpu


# ---------------------------------------------------------------------------
# Philox: device generator == oracle generator, all four counter words
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 7, 0xDEADBEEFCAFEF00D])
def test_device_philox_matches_oracle(seed):
    rng = np.random.default_rng(seed & 0xFFFF)
    ctr = rng.integers(0, 2 ** 32, size=(5003, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:3] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4]]
    out = np.zeros_like(ctr)
    chemo.chemo_philox(seed, ctr, out)
    np.testing.assert_array_equal(out, orc.philox(ctr, seed))


# ---------------------------------------------------------------------------
# a1 / a2: bins and counting sort
# ---------------------------------------------------------------------------
BIN_CASES = [
    # (workload, overrides, n)
    ("walls_grid_2d", dict(bin_side=0.0101, search_mode=1), 20011),
    ("walls_grid_2d", dict(bin_side=0.0203, search_mode=2), 20011),
    ("periodic_fixed_gradient_2d", dict(bin_side=0.0125, search_mode=1), 1000),
    ("clumps_grid_3d", dict(bin_side=0.0041, search_mode=1, grid=[32, 32, 32]), 60001),
    ("clumps_grid_3d", dict(bin_side=0.0081, search_mode=2, grid=[32, 32, 32]), 60001),
]


@pytest.mark.parametrize("name,over,n", BIN_CASES)
def test_bins_exact_and_sort_valid(name, over, n):
    p, pos, sp = wl.initial_state(name, n=n, **over)
    pos[:7, 0] = 0.0
    if p["boundary"] == 0:
        pos[7:14, 1] = 1.0
    with make_sim(p, pos, sp) as sim:
        info = chemo.chemo_get_info(sim)
        cells = np.zeros((n, p["dim"]), np.int32)
        chemo.chemo_stage_bins(sim, cells)
        ref, nb = orc.bins_f32(p, p["bin_side"], pos)
        assert tuple(info["nbins"][: p["dim"]]) == nb[: p["dim"]]
        np.testing.assert_array_equal(cells, ref)
        ids = np.zeros(n, np.uint32)
        start = np.zeros(info["bin_slots"] + 1, np.uint32)
        chemo.chemo_stage_sort(sim, ids, start)
    assert np.array_equal(np.sort(ids), np.arange(n, dtype=np.uint32))  # permutation
    assert start[0] == 0 and start[-1] == n and np.all(np.diff(start.astype(np.int64)) >= 0)
    # row-major bins, rows padded to the pitch
    pitch = info["bin_pitch"]
    assert pitch % 8 == 0 and pitch >= nb[0]
    key = ref[:, 0].astype(np.int64)
    if p["dim"] == 3:
        key = key + pitch * (ref[:, 1] + nb[1] * ref[:, 2].astype(np.int64))
    else:
        key = key + pitch * ref[:, 1].astype(np.int64)
    k_sorted = key[ids].astype(np.int64)
    j = np.arange(n)
    assert np.all(start[k_sorted] <= j) and np.all(j < start[k_sorted + 1])


# ---------------------------------------------------------------------------
# a3: pair force and neighbour sets
# ---------------------------------------------------------------------------
FORCE_CASES = [
    ("periodic_fixed_gradient_2d", dict(), 1000),
    ("periodic_fixed_gradient_2d", dict(diameter=[0.03], search_mode=2), 3001),
    ("walls_grid_2d", dict(diameter=[0.01, 0.02], grid=[64, 64, 1]), 30007),
    ("walls_grid_2d", dict(diameter=[0.01, 0.02], grid=[64, 64, 1], search_mode=2), 30007),
    ("walls_grid_2d", dict(diameter=[0.01, 0.02], grid=[64, 64, 1], cutoff_mode=1, cutoff_factor=1.5,
                           inter=2.5), 30007),
    ("clumps_grid_3d", dict(diameter=[0.01, 0.02], grid=[16, 16, 16]), 80021),
    ("clumps_grid_3d", dict(diameter=[0.01, 0.02], grid=[16, 16, 16], search_mode=2), 80021),
    ("clumps_grid_3d", dict(diameter=[0.01, 0.03], grid=[16, 16, 16], search_mode=2, boundary=1, pde_bc=2), 40009),
    ("clumps_grid_3d", dict(diameter=[0.02, 0.03], grid=[16, 16, 16], boundary=1, pde_bc=2), 40009),
]


@pytest.mark.parametrize("name,over,n", FORCE_CASES)
def test_pair_forces_match_oracle(name, over, n):
    p, pos, sp = wl.initial_state(name, n=n, **over)
    with make_sim(p, pos, sp) as sim:
        F, cnt, ids = gpu_forces(sim)
    ex = assert_forces_match(p, F, cnt, ids, pos, sp)
    assert ex["count"].sum() > 0.3 * n  # real neighbourhoods


def test_dense_cluster_single_bin():
    # 3000 cells inside one bin: long candidate lists, heavy overlap
    p = wl.params("walls_grid_2d", diameter=[0.02, 0.02], grid=[16, 16, 1])
    rng = np.random.default_rng(0)
    pos = (0.5 + 0.004 * rng.random((3000, 2))).astype(np.float32)
    sp = wl.half_species(3000, 2)
    with make_sim(p, pos, sp) as sim:
        F, cnt, ids = gpu_forces(sim)
    assert_forces_match(p, F, cnt, ids, pos, sp)


# ---------------------------------------------------------------------------
# a4: gradient interpolation
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,over,n", [
    ("walls_grid_2d", dict(grid=[97, 65, 1]), 20011),
    ("clumps_grid_3d", dict(grid=[33, 29, 31]), 30011),
    ("walls_grid_2d", dict(grid=[64, 48, 1], boundary=1, pde_bc=2, diameter=[0.004, 0.004]), 20011),
])
def test_drift_matches_oracle(name, over, n):
    p, pos, sp = wl.initial_state(name, n=n, chi=1.7, **over)
    pos[:5, 0] = p["lo"][0]
    c0 = wl.random_field(p, seed=11)
    with make_sim(p, pos, sp, c0) as sim:
        d = torch.zeros((n, p["dim"]), dtype=torch.float32, device="cuda")
        chemo.chemo_stage_drift(sim, d)
        d = d.cpu().numpy().astype(np.float64)
    ref = orc.drift(p, pos.astype(np.float64), sp, c0.astype(np.float64))
    scale = np.abs(ref).max()
    assert scale > 0
    assert np.abs(d - ref).max() <= 1e-5 * scale


# ---------------------------------------------------------------------------
# a6: deposit
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,over,n", [
    ("walls_grid_2d", dict(grid=[129, 97, 1], consume=[0.0, 0.3]), 40009),
    ("clumps_grid_3d", dict(grid=[40, 36, 33], consume=[0.0, 0.3]), 50021),
    ("walls_grid_2d", dict(grid=[64, 64, 1], boundary=1, pde_bc=2, diameter=[0.004, 0.004]), 20011),
])
def test_deposit_matches_oracle(name, over, n):
    p, pos, sp = wl.initial_state(name, n=n, **over)
    pos[:5, 0] = p["lo"][0]
    if p["boundary"] == 0:
        pos[5:10, 1] = p["hi"][1]
    shape = orc.grid_shape(p)
    with make_sim(p, pos, sp) as sim:
        S = np.zeros(shape, np.float32)
        R = np.zeros(shape, np.float32)
        chemo.chemo_stage_deposit(sim, S, R)
    Sr, Rr = orc.deposit(p, pos.astype(np.float64), sp)
    assert np.abs(S - Sr).max() <= 1e-5 * np.abs(Sr).max()
    if np.abs(Rr).max() > 0:
        assert np.abs(R - Rr).max() <= 1e-5 * np.abs(Rr).max()


# ---------------------------------------------------------------------------
# a5 + a7: whole steps
# ---------------------------------------------------------------------------
STEP_CASES = [
    # fixed gradient, periodic, displacement tracking (the MSD set-up)
    ("periodic_fixed_gradient_2d", dict(), 1000, 0),
    # grid with one fused substep (PDE concurrent with the particle kernel)
    ("walls_grid_2d", dict(grid=[128, 128, 1]), 20011, 3),
    # many substeps (separate source grid)
    ("walls_grid_2d", dict(grid=[512, 512, 1]), 20011, 0),
    # consumption, fused and not fused
    ("walls_grid_2d", dict(grid=[128, 128, 1], consume=[0.0, 0.5]), 20011, 0),
    ("walls_grid_2d", dict(grid=[256, 256, 1], consume=[0.0, 0.5]), 20011, 0),
    # Dirichlet walls (held), periodic grid
    ("walls_grid_2d", dict(grid=[96, 80, 1], pde_bc=1), 12007, 0),
    ("walls_grid_2d", dict(grid=[96, 80, 1], boundary=1, pde_bc=2, diameter=[0.004, 0.008]), 12007, 0),
    # 3D, clumps, 7-point stencil
    ("clumps_grid_3d", dict(grid=[48, 48, 48], diameter=[0.01, 0.02]), 60013, 0),
    ("clumps_grid_3d", dict(grid=[40, 44, 36], diameter=[0.01, 0.02], search_mode=2), 60013, 5),
    # large steps that reflect more than once
    ("walls_grid_2d", dict(grid=[64, 64, 1], D=[3000.0, 2000.0], dt=1e-4), 5003, 0),
    # half-window pair search (each pair once, integer atomics for the partner)
    ("walls_grid_2d", dict(grid=[128, 128, 1], search_mode=4), 20011, 2),
    ("walls_grid_2d", dict(grid=[96, 80, 1], boundary=1, pde_bc=2, diameter=[0.004, 0.008], search_mode=4), 12007, 0),
    ("clumps_grid_3d", dict(grid=[48, 48, 48], diameter=[0.01, 0.02], search_mode=4), 60013, 0),
]


@pytest.mark.parametrize("name,over,n,step0", STEP_CASES)
def test_step_matches_oracle(name, over, n, step0):
    p, pos, sp = wl.initial_state(name, n=n, **over)
    c0 = wl.random_field(p, seed=5, scale=0.3) if p["chem_mode"] == 0 else None
    with make_sim(p, pos, sp, c0) as sim:
        if step0:
            chemo.chemo_set_step_index(sim, step0)
        chemo.chemo_step(sim)
        assert chemo.chemo_step_index(sim) == step0 + 1
        pos_g, sp_g, disp_g = chemo.read_state_host(sim)
        c_g = chemo.read_field_host(sim) if c0 is not None else None
    assert_step_matches(p, pos, sp, c0, pos_g, sp_g, c_g, disp_g, step_index=step0)


def test_reactions_step_matches_oracle():
    p, pos, sp = wl.initial_state("walls_grid_2d", n=40009, grid=[128, 128, 1], reactions=1,
                                  react_k0=[3000.0, 0.0], react_kc=[0.0, 2000.0], react_to=[1, 0])
    c0 = wl.random_field(p, seed=9, scale=2.0)
    with make_sim(p, pos, sp, c0) as sim:
        chemo.chemo_step(sim)
        pos_g, sp_g, _ = chemo.read_state_host(sim)
        c_g = chemo.read_field_host(sim)
    pos_r, sp_r, c_r, _ = orc.step(p, pos, sp, c0.astype(np.float64))
    # the switching decision compares u with (k0 + kc c(X)) dt; c(X) differs
    # between FP32 and FP64 by rounding, so cells within 1e-6 of a tie may
    # differ. All others must agree.
    conc = orc.conc(p, pos.astype(np.float64), c0.astype(np.float64))
    ctr = np.zeros((pos.shape[0], 4), np.uint32)
    ctr[:, 0] = np.arange(pos.shape[0])
    ctr[:, 2] = orc.TAG_REACT
    u = (orc.philox(ctr, p["seed"])[:, 0].astype(np.float64) + 0.5) / 2 ** 32
    k0 = np.array([np.float32(3000.0), 0.0])[sp]
    kc = np.array([0.0, np.float32(2000.0)])[sp]
    prop = (k0 + kc * conc) * p["dt"]
    tie = np.abs(u - prop) <= 1e-6 * np.maximum(prop, 1e-30) + 1e-12
    assert (sp_r != sp).sum() > 100
    np.testing.assert_array_equal(sp_g[~tie], sp_r[~tie])
    _, ex = orc.pair_forces(p, pos.astype(np.float64), sp, method=1, extras=True)
    tol = position_tolerance(p, pos, sp, c0, pos_r, ex["border"])
    assert (np.abs(pos_g - pos_r) <= tol).all()
    assert np.abs(c_g - c_r).max() <= 1e-4 * np.abs(c_r).max()  # deposit differs only on tie cells


def test_step_n_equals_repeated_steps_and_oracle():
    # force shifted to zero at the cutoff: the float atomics of the deposit
    # make c differ in its last bits between runs, and with a hard cutoff a
    # pair within an ulp of r_c could then switch its force on or off
    p, pos, sp = wl.initial_state("walls_grid_2d", n=20011, grid=[128, 128, 1], cutoff_mode=1)
    c0 = wl.random_field(p, seed=5, scale=0.3)
    k = 21  # exercises the 16-step graph, the 2-step graph and a direct step
    with make_sim(p, pos, sp, c0) as a, make_sim(p, pos, sp, c0) as b:
        chemo.chemo_step_n(a, k)
        for _ in range(k):
            chemo.chemo_step(b)
        pa, _, _ = chemo.read_state_host(a)
        pb, _, _ = chemo.read_state_host(b)
        ca = chemo.read_field_host(a)
        cb = chemo.read_field_host(b)
        assert chemo.chemo_step_index(a) == k
    # same kernels, same inputs; the float atomics of the deposit make c
    # differ in its last bits between runs (no bitwise reproducibility), so
    # the two trajectories agree to the single-step tolerance
    assert np.abs(pa - pb).max() <= 1e-5
    assert np.abs(ca - cb).max() <= 1e-5 * np.abs(ca).max()
    pr, _, cr, _ = orc.run(p, pos, sp, c0.astype(np.float64), nsteps=k)
    # k steps: per-step errors add up; allow k times the single-step tolerance
    assert np.abs(pa - pr).max() <= k * 1e-5
    assert np.abs(ca - cr).max() <= k * 1e-5 * np.abs(cr).max()


def test_hard_cutoff_multi_step_against_oracle():
    # with the paper's hard cutoff, FP32 and FP64 trajectories agree until a
    # pair sits within rounding of r_c; over 10 steps nearly every cell must
    # still match, and the few that do not may only be off by the force jump
    p, pos, sp = wl.initial_state("walls_grid_2d", n=20011, grid=[128, 128, 1])
    c0 = wl.random_field(p, seed=6, scale=0.3)
    k = 10
    with make_sim(p, pos, sp, c0) as a:
        chemo.chemo_step_n(a, k)
        pa, _, _ = chemo.read_state_host(a)
    pr, _, _, _ = orc.run(p, pos, sp, c0.astype(np.float64), nsteps=k)
    err = np.abs(pa - pr).max(axis=1)
    assert (err > k * 1e-5).mean() <= 1e-2
    jump = k * p["dt"] * (1.0 / float(np.float32(0.005))) * np.exp(-1.0) * 10
    assert err.max() <= jump


# ---------------------------------------------------------------------------
# Full-size workloads, in the launch configuration the benchmark times
# ---------------------------------------------------------------------------
def test_full_size_clumps_3d_step():
    p, pos, sp = wl.initial_state("clumps_grid_3d")
    c0 = wl.random_field(p, seed=7, scale=0.05)
    with make_sim(p, pos, sp, c0) as sim:
        info = chemo.chemo_get_info(sim)
        assert info["pde_substeps"] == 1
        chemo.chemo_step_n(sim, 1)
        pos_g, sp_g, _ = chemo.read_state_host(sim)
        c_g = chemo.read_field_host(sim)
    orc.set_threads(max(1, orc.get_threads()))
    assert_step_matches(p, pos, sp, c0, pos_g, sp_g, c_g)


def test_full_size_graph_steps_equal_direct_steps():
    """The bench replays its steps as CUDA graphs (chemo_step_n: 2- and
    16-step graphs of the overlapped step); at full size two graph-replayed
    steps equal two directly enqueued steps, the path the oracle checks
    above: species bit for bit, positions within 1e-6 of the unit box (the
    second step's gradient reads a field whose deposit's float atomics
    round in any order), the field within that rounding."""
    p, pos, sp = wl.initial_state("clumps_grid_3d")
    c0 = wl.random_field(p, seed=7, scale=0.05)
    with make_sim(p, pos, sp, c0) as sim:
        chemo.chemo_step_n(sim, 2)  # one 2-step graph
        xa, sa, _ = chemo.read_state_host(sim)
        ca = chemo.read_field_host(sim)
    with make_sim(p, pos, sp, c0) as sim:
        chemo.chemo_step(sim)
        chemo.chemo_step(sim)
        chemo.chemo_check(sim)
        xb, sb, _ = chemo.read_state_host(sim)
        cb = chemo.read_field_host(sim)
    np.testing.assert_array_equal(sa, sb)
    assert np.abs(xa - xb).max() <= 1e-6
    assert np.abs(ca - cb).max() <= 1e-5 * np.abs(cb).max()


def test_full_size_walls_2d_step():
    p, pos, sp = wl.initial_state("walls_grid_2d")
    c0 = wl.random_field(p, seed=8, scale=0.1)
    with make_sim(p, pos, sp, c0) as sim:
        assert chemo.chemo_get_info(sim)["pde_substeps"] == 12
        chemo.chemo_step_n(sim, 1)
        pos_g, sp_g, _ = chemo.read_state_host(sim)
        c_g = chemo.read_field_host(sim)
    assert_step_matches(p, pos, sp, c0, pos_g, sp_g, c_g)


def test_full_size_deposit_conserves_mass():
    # property at any size: the trapezoid integral of the deposited source is
    # dt * sum_i k_{s_i}
    p, pos, sp = wl.initial_state("clumps_grid_3d")
    with make_sim(p, pos, sp) as sim:
        S = torch.zeros(orc.grid_shape(p), dtype=torch.float32, device="cuda")
        chemo.chemo_stage_deposit(sim, S, None)
        S = S.double()
    h = 1.0 / 255
    w = torch.ones(256, dtype=torch.float64, device="cuda")
    w[0] = w[-1] = 0.5
    mass = torch.einsum("zyx,z,y,x->", S, w, w, w).item() * h ** 3
    expect = p["dt"] * float(np.float32(0.1)) * (sp == 0).sum()
    assert abs(mass - expect) <= 1e-5 * expect


# ---------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------
def test_empty_and_single_particle():
    p = wl.params("walls_grid_2d", grid=[33, 33, 1])
    with make_sim(p, np.zeros((0, 2), np.float32), np.zeros(0, np.uint8)) as sim:
        chemo.chemo_step_n(sim, 3)
        c = chemo.read_field_host(sim)
        assert np.all(c == 0.0)
        chemo.chemo_check(sim)
    pos = np.array([[0.5, 0.5]], np.float32)
    sp = np.array([0], np.uint8)
    with make_sim(p, pos, sp) as sim:
        chemo.chemo_step(sim)
        pos_g, sp_g, _ = chemo.read_state_host(sim)
        c_g = chemo.read_field_host(sim)
    assert_step_matches(p, pos, sp, np.zeros(orc.grid_shape(p), np.float32), pos_g, sp_g, c_g)


def test_host_buffers_round_trip():
    p, pos, sp = wl.initial_state("walls_grid_2d", n=1025, grid=[33, 33, 1])
    sim = chemo.chemo_create(p, pos, sp)  # host memory
    try:
        pos_g, sp_g, _ = chemo.read_state_host(sim)
        np.testing.assert_array_equal(pos_g, pos)
        np.testing.assert_array_equal(sp_g, sp)
        pos2 = np.ascontiguousarray(pos[::-1])
        chemo.chemo_write_state(sim, pos2, sp)
        pos_g, _, _ = chemo.read_state_host(sim)
        np.testing.assert_array_equal(pos_g, pos2)
    finally:
        sim.close()


@pytest.mark.parametrize("fault", ["nan", "outside", "species"])
def test_bad_device_input_is_latched(fault):
    """Device-side checks of the input (the host cannot see device buffers):
    a non-finite position, a position outside the box and a species value
    out of range are latched, reported once by chemo_check, and the state
    stays usable (clamped to the box, species 0)."""
    p = wl.params("walls_grid_2d", grid=[33, 33, 1])
    pos = np.full((10, 2), 0.5, np.float32)
    sp = np.zeros(10, np.uint8)
    want = {"nan": chemo.ENONFINITE, "outside": chemo.EDOMAIN, "species": chemo.EINVAL}[fault]
    if fault == "nan":
        pos[3, 0] = np.nan
    elif fault == "outside":
        pos[3, 1] = 1.5
    else:
        sp[4] = 7
    with make_sim(p, pos, sp) as sim:
        with pytest.raises(chemo.ChemoError) as ei:
            chemo.chemo_check(sim)
        assert ei.value.status == want
        chemo.chemo_check(sim)  # cleared
        x, s, _ = chemo.read_state_host(sim)
        assert np.isfinite(x).all() and (x >= 0).all() and (x <= 1).all() and (s < 2).all()
        chemo.chemo_step_n(sim, 3)
        chemo.chemo_check(sim)


def test_scan_wait_that_runs_out_is_latched_and_the_next_step_is_normal():
    """The one device-side wait (the scan's look-back) is bounded: a scan
    whose tiles wait on a predecessor that no block publishes gives up after
    its poll limit, latches ETIMEOUT (reported once by chemo_check) and
    leaves the context and the simulation usable: the next step still
    matches the oracle."""
    # bins of 0.002 on the unit square: 504 x 500 bins, 8 scan tiles
    p, pos, sp = wl.initial_state("walls_grid_2d", n=20011, grid=[128, 128, 1], diameter=[0.001, 0.002])
    c0 = wl.random_field(p, seed=5, scale=0.3)
    with make_sim(p, pos, sp, c0) as sim:
        chemo.chemo_check(sim)
        for spins in (1024, 1):
            chemo.chemo_stall_scan(sim, spins)
            with pytest.raises(chemo.ChemoError) as ei:
                chemo.chemo_check(sim)
            assert ei.value.status == chemo.ETIMEOUT
            chemo.chemo_check(sim)  # cleared
        chemo.chemo_step(sim)
        chemo.chemo_check(sim)
        pos_g, sp_g, _ = chemo.read_state_host(sim)
        c_g = chemo.read_field_host(sim)
    assert_step_matches(p, pos, sp, c0, pos_g, sp_g, c_g)


def test_stall_scan_needs_two_tiles():
    p, pos, sp = wl.initial_state("walls_grid_2d", n=1000, grid=[33, 33, 1])
    with make_sim(p, pos, sp) as sim:
        with pytest.raises(chemo.ChemoError) as ei:
            chemo.chemo_stall_scan(sim, 1024)
        assert ei.value.status == chemo.EINVAL


def test_set_params_changes_model_constants():
    p, pos, sp = wl.initial_state("walls_grid_2d", n=5003, grid=[64, 64, 1])
    with make_sim(p, pos, sp) as sim:
        q = dict(p, chi=3.0, D=[0.5, 0.25], inter=2.0)
        chemo.chemo_set_params(sim, q)
        chemo.chemo_step(sim)
        pos_g, sp_g, _ = chemo.read_state_host(sim)
        c_g = chemo.read_field_host(sim)
        with pytest.raises(chemo.ChemoError):
            chemo.chemo_set_params(sim, dict(p, grid=[65, 64, 1]))
    assert_step_matches(q, pos, sp, np.zeros(orc.grid_shape(p), np.float32), pos_g, sp_g, c_g)


@pytest.mark.parametrize("name,over", [
    ("walls_grid_2d", dict(grid=[64, 64, 1])),
    ("walls_grid_2d", dict(boundary=1, pde_bc=2, grid=[64, 64, 1])),
    ("clumps_grid_3d", dict(grid=[32, 32, 32])),
    ("clumps_grid_3d", dict(grid=[32, 32, 32], boundary=1, pde_bc=2)),
])
def test_warp_and_lane_search_agree_bitwise(name, over):
    """The warp-cooperative 3^d search, the per-lane 2^d and 3^d searches and
    the half window (each pair once, the partner's share by integer atomics)
    round every pair term the same way and sum exactly: identical forces,
    counts and neighbour id sums."""
    p, pos, sp = wl.initial_state(name, n=30011, **over)
    outs = []
    # 2^d per lane; 3^d warp search always; 3^d hybrid; 3^d per lane; half window
    for mode, runs in ((2, 0), (1, 32), (1, 0), (3, 0), (4, 0)):
        with make_sim(dict(p, search_mode=mode, warp_runs=runs), pos, sp) as sim:
            assert chemo.chemo_get_info(sim)["search_mode"] == mode
            outs.append(gpu_forces(sim))
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            np.testing.assert_array_equal(a, b)
    assert_forces_match(p, outs[0][0], outs[0][1], outs[0][2], pos, sp)


def test_warp_search_dense_cluster_bitwise():
    """Thousands of cells in a few bins (runs of 32, windows of thousands of
    candidates, queue flushes mid-run): the warp search equals the per-lane
    search bit for bit."""
    p = wl.params("walls_grid_2d", grid=[16, 16, 1])
    rng = np.random.default_rng(7)
    pos = (0.5 + 0.004 * rng.standard_normal((4000, 2))).astype(np.float32)
    sp = wl.half_species(4000, 2)
    outs = []
    for mode, runs in ((3, 0), (1, 32), (4, 0)):
        with make_sim(dict(p, search_mode=mode, warp_runs=runs), pos, sp) as sim:
            outs.append(gpu_forces(sim))
    for a, b in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(a, b)
    assert_forces_match(p, outs[1][0], outs[1][1], outs[1][2], pos, sp)


@pytest.mark.parametrize("name,over", [
    ("walls_grid_2d", dict(grid=[64, 64, 1])),
    ("walls_grid_2d", dict(boundary=1, pde_bc=2, grid=[64, 64, 1])),
    ("clumps_grid_3d", dict(grid=[32, 32, 32], diameter=[0.01, 0.02])),
    ("clumps_grid_3d", dict(grid=[32, 32, 32], diameter=[0.01, 0.03], boundary=1, pde_bc=2)),
])
def test_half_window_step_bitwise(name, over):
    """A whole step with the half window equals the per-lane 3^d search's bit
    for bit (the forces are the same integers); the partner sums are cleared
    by the step, so a second step agrees too."""
    p, pos, sp = wl.initial_state(name, n=30011, **over)
    c0 = wl.random_field(p, seed=3, scale=0.3) if p["chem_mode"] == 0 else None
    outs = []
    for mode in (3, 4):
        with make_sim(dict(p, search_mode=mode), pos, sp, c0) as sim:
            info = chemo.chemo_get_info(sim)
            assert info["search_mode"] == mode
            chemo.chemo_step(sim)
            outs.append(chemo.read_state_host(sim)[0])
            chemo.chemo_step(sim)
            chemo.chemo_check(sim)
            outs.append(chemo.read_state_host(sim)[0])
    np.testing.assert_array_equal(outs[0], outs[2])
    assert np.abs(outs[1] - outs[3]).max() <= 1e-6  # the deposit's float atomics round in any order


@pytest.mark.parametrize("name,over", [
    ("walls_grid_2d", dict(grid=[64, 64, 1])),
    ("clumps_grid_3d", dict(grid=[32, 32, 32], diameter=[0.01, 0.02])),
    ("clumps_grid_3d", dict(grid=[32, 32, 32], diameter=[0.01, 0.03], boundary=1, pde_bc=2)),
])
def test_block_shapes_give_identical_steps(name, over):
    """128, 256 and 512 threads per block of the half-window pair and move
    kernels (the autotuner's block-shape choice): forces and whole steps bit
    for bit the same."""
    p, pos, sp = wl.initial_state(name, n=30011, **over)
    c0 = wl.random_field(p, seed=3, scale=0.3) if p["chem_mode"] == 0 else None
    forces, states = [], []
    for bt in (0, 128, 256, 512):
        with make_sim(dict(p, search_mode=4, block_threads=bt), pos, sp, c0) as sim:
            forces.append(gpu_forces(sim)[0])
            chemo.chemo_step_n(sim, 3)
            states.append(chemo.read_state_host(sim)[0])
    for f, x in zip(forces[1:], states[1:]):
        np.testing.assert_array_equal(f, forces[0])
        if c0 is None:
            np.testing.assert_array_equal(x, states[0])
        else:  # the deposit's float atomics round in any order
            assert np.abs(x - states[0]).max() <= 1e-6


def test_half_window_many_steps_fixed_gradient_bitwise():
    """No chemical field (fixed gradient): every step is exact integer force
    sums and counter-based noise, so 37 graph-replayed steps of the half
    window repeat the per-lane search bit for bit, and a dense cluster of
    thousands of cells in a few bins (long lists, many atomics on the same
    partners) gives the same force as the per-lane search."""
    p, pos, sp = wl.initial_state("periodic_fixed_gradient_2d", n=20011)
    outs = []
    for mode in (3, 4):
        with make_sim(dict(p, search_mode=mode), pos, sp) as sim:
            chemo.chemo_step_n(sim, 37)
            outs.append(chemo.read_state_host(sim)[0])
    np.testing.assert_array_equal(outs[0], outs[1])
    q = wl.params("walls_grid_2d", grid=[16, 16, 1], chem_mode=1, fixed_grad=[1.0, 0.0, 0.0])
    rng = np.random.default_rng(11)
    pos = np.clip(0.5 + 0.004 * rng.standard_normal((4000, 2)), 0.0, 1.0).astype(np.float32)
    sp = wl.half_species(4000, 2)
    outs = []
    for mode in (3, 4):
        with make_sim(dict(q, search_mode=mode), pos, sp) as sim:
            chemo.chemo_step_n(sim, 3)
            outs.append(chemo.read_state_host(sim)[0])
    np.testing.assert_array_equal(outs[0], outs[1])


def test_profile_counts_pairs_and_candidate_tests():
    """The profiling pass counts every in-cutoff pair for both of its cells
    (the same total for the half and the full window) and, for the half
    window, the candidates it tested (at least one per pair found)."""
    p, pos, sp = wl.initial_state("walls_grid_2d", n=20011, grid=[64, 64, 1], chem_mode=1,
                                  fixed_grad=[1.0, 0.0, 0.0])
    prof = {}
    for mode in (3, 4):
        with make_sim(dict(p, search_mode=mode), pos, sp) as sim:
            prof[mode] = chemo.chemo_profile_steps(sim, 1)
    assert prof[3]["pairs_per_step"] == prof[4]["pairs_per_step"] > 0
    assert prof[3]["tests_per_step"] == 0.0
    assert prof[4]["tests_per_step"] >= 0.5 * prof[4]["pairs_per_step"]
    # the half window visits each unordered pair of cells at most once
    n = pos.shape[0]
    assert prof[4]["tests_per_step"] <= n * (n - 1) / 2


def test_time_step_rule_is_reported():
    """The paper's rule of thumb (a step moves a cell less than the
    interaction range): chemo_info.step_ratio is the largest
    sqrt(2 (D_i + D_j) dt) / eps_ij, and the binding warns above 1."""
    p, pos, sp = wl.initial_state("walls_grid_2d", n=2000, grid=[32, 32, 1])
    want = max(np.sqrt(2.0 * (p["D"][a] + p["D"][b]) * p["dt"]) / (0.5 * (p["diameter"][a] + p["diameter"][b]))
               for a in range(2) for b in range(2))
    with pytest.warns(UserWarning, match="dt is large"):
        sim = make_sim(p, pos, sp)
    with sim:
        assert chemo.chemo_get_info(sim)["step_ratio"] == pytest.approx(want, rel=1e-6)
    q = dict(p, dt=p["dt"] / 100.0)
    with make_sim(q, pos, sp) as sim:
        assert chemo.chemo_get_info(sim)["step_ratio"] == pytest.approx(want / 10.0, rel=1e-6)


def test_time_step_rule_of_the_paper_figure():
    """Fig. 1 of the paper picks dt = (0.23 epsilon)^2 / (4 D_beta)
    (tests/golden/paper_parameters.txt): its step moves a beta cell 0.23 of
    the interaction range, the largest ratio over the species pairs."""
    gold = {}
    for line in open(__file__.replace("test_gpu_parity.py", "golden/paper_parameters.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()[:2]
            gold[k] = float(v)
    eps, dt = gold["fig1_epsilon"], gold["fig1_dt"]
    p = wl.params("walls_grid_2d", grid=[32, 32, 1], diameter=[eps, eps], D=[gold["fig1_D_alpha"], gold["fig1_D_beta"]],
                  dt=dt)
    pos = np.random.default_rng(3).uniform(0.1, 0.9, (500, 2)).astype(np.float32)
    with make_sim(p, pos, wl.half_species(500, 2)) as sim:
        assert chemo.chemo_get_info(sim)["step_ratio"] == pytest.approx(0.23, rel=2e-3)


@pytest.mark.parametrize("dim,boundary", [(2, 0), (2, 1), (3, 0)])
def test_init_positions_match_oracle(dim, boundary):
    """The paper's initial state drawn on the device (chemo_init_positions)
    against the oracle's FP64 draw from the same Philox words: species
    exactly, positions within the single-precision Box-Muller error."""
    p = wl.params("walls_grid_2d" if dim == 2 else "clumps_grid_3d", boundary=boundary,
                  pde_bc=2 if boundary else 0, seed=21)
    n, na = 30011, 12001
    pos_h, sp_h = chemo.chemo_init_positions(p, n, na, 0.1)           # host buffers
    pos_d = torch.zeros((n, dim), dtype=torch.float32, device="cuda")
    sp_d = torch.zeros(n, dtype=torch.uint8, device="cuda")
    chemo.chemo_init_positions(p, n, na, 0.1, pos_d, sp_d)             # device buffers
    np.testing.assert_array_equal(pos_d.cpu().numpy(), pos_h)
    np.testing.assert_array_equal(sp_d.cpu().numpy(), sp_h)
    ref, sref = orc.init_positions(p, n, na, 0.1)
    np.testing.assert_array_equal(sp_h, sref)
    L = max(p["hi"][a] - p["lo"][a] for a in range(dim))
    assert np.abs(pos_h.astype(np.float64) - ref).max() <= 2e-6 * L
    # and it is a valid state for a simulation
    with make_sim(p, pos_h, sp_h) as sim:
        chemo.chemo_step(sim)
        chemo.chemo_check(sim)
