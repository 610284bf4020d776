"""The variants (tamed Euler, hard-sphere overlap correction, Gaussian
kernel density deposit) through the C ABI against the FP64 oracle, with the
tolerances of the step tests (positions 1e-5 L, field 1e-5 max |c|)."""
import numpy as np
import pytest

from oracle import chemo_oracle as orc
from paper_1805_11007_gb300 import chemo
from paper_1805_11007_gb300 import ensemble as en
from paper_1805_11007_gb300 import workloads as wl
from parity_util import assert_step_matches, dev, make_sim

pytestmark = pytest.mark.gpu

CASES_2D = [dict(), dict(boundary=1, pde_bc=2)]


def _state(name, n, seed_field=5, **over):
    p, pos, sp = wl.initial_state(name, n=n, **over)
    c0 = wl.random_field(p, seed=seed_field, scale=0.3) if p.get("chem_mode", 0) == 0 else None
    return p, pos, sp, c0


def _gpu_step(p, pos, sp, c0, k=1):
    with make_sim(p, pos, sp, c0) as sim:
        chemo.chemo_step_n(sim, k) if k > 1 else chemo.chemo_step(sim)
        pg, spg, dg = chemo.read_state_host(sim)
        cg = chemo.read_field_host(sim) if c0 is not None else None
    return pg, spg, cg, dg


# ----------------------------------------------------------------- tamed Euler
@pytest.mark.parametrize("over", CASES_2D)
def test_tamed_step_matches_oracle(over):
    p, pos, sp, c0 = _state("walls_grid_2d", 20011, grid=[128, 128, 1], move_scheme=1, **over)
    pg, spg, cg, _ = _gpu_step(p, pos, sp, c0)
    assert_step_matches(p, pos, sp, c0, pg, spg, cg)


def test_tamed_step_3d_and_strong_force():
    p, pos, sp, c0 = _state("clumps_grid_3d", 20011, grid=[32, 32, 32], move_scheme=1, inter=50.0, dt=1e-5)
    pg, spg, cg, _ = _gpu_step(p, pos, sp, c0)
    assert_step_matches(p, pos, sp, c0, pg, spg, cg)
    pe, _, _, _ = _gpu_step(dict(p, move_scheme=0), pos, sp, c0)
    assert np.abs(pe - pg).max() > 1e-4  # the taming is in effect at this force


# ------------------------------------------------------------ hard spheres
def _hs_sensitivity(p, pos, sp, delta=1e-6):
    """Bound on how far an FP32 error delta in the moved positions can carry
    a cell's correction: the line of centres of a pair at distance r turns by
    up to 2 delta / r, and the correction along it is at most twice the
    contact distance. Summed over the pairs overlapping after the move (the
    oracle's moved positions without the correction)."""
    from scipy.spatial import cKDTree
    xs, _, _, _ = orc.step(dict(p, hard_sphere=0, Dc=0.0), pos.astype(np.float64), sp)
    L = np.array(p["hi"][: p["dim"]]) - np.array(p["lo"][: p["dim"]])
    box = L if p.get("boundary") == 1 else None
    diam = np.asarray(p["diameter"][: p["n_species"]], np.float64)
    tree = cKDTree(xs - np.array(p["lo"][: p["dim"]]), boxsize=box)
    pairs = tree.query_pairs(float(diam.max()), output_type="ndarray")
    sens = np.zeros(len(pos))
    if len(pairs):
        dd = xs[pairs[:, 0]] - xs[pairs[:, 1]]
        if box is not None:
            dd -= box * np.round(dd / box)
        r = np.linalg.norm(dd, axis=1)
        contact = 0.5 * (diam[sp[pairs[:, 0]]] + diam[sp[pairs[:, 1]]])
        on = (r < contact) & (r > 0)
        v = np.where(on, 2.0 * contact * 2.0 * delta / np.maximum(r, 1e-30), 0.0)
        np.add.at(sens, pairs[:, 0], v)
        np.add.at(sens, pairs[:, 1], v)
    return sens


@pytest.mark.parametrize("over", [dict(), dict(inter=0.0), dict(boundary=1, pde_bc=2, track_displacement=1)])
def test_hard_sphere_step_matches_oracle(over):
    p, pos, sp, c0 = _state("walls_grid_2d", 8000, grid=[64, 64, 1], hard_sphere=1, diameter=[0.012, 0.02],
                            **over)
    pg, spg, cg, dg = _gpu_step(p, pos, sp, c0)
    disp = np.zeros(pos.shape) if p.get("track_displacement") else None
    pos_r, _, c_r, disp_r = orc.step(p, pos.astype(np.float64), sp, c0.astype(np.float64), disp=disp)
    tol = 1e-5 + _hs_sensitivity(p, pos, sp)[:, None]
    d = np.abs(pg - pos_r)
    if p.get("boundary") == 1:
        d = np.minimum(d, 1.0 - d)
    assert np.all(d <= tol), (d.max(), np.argwhere(d > tol)[:3])
    np.testing.assert_array_equal(spg, sp)
    assert np.abs(cg - c_r).max() <= 1e-5 * np.abs(c_r).max()
    if disp is not None:
        assert np.all(np.abs(dg - disp_r) <= tol)
    # the correction was active: overlaps existed before it
    _, ex = orc.pair_forces(dict(p, cutoff_factor=1.0), pos.astype(np.float64), sp, method=1, extras=True)
    assert ex["count"].sum() > 100


def test_hard_sphere_3d_and_multi_step():
    p, pos, sp, c0 = _state("clumps_grid_3d", 20011, grid=[32, 32, 32], hard_sphere=1, cutoff_mode=1)
    pg, spg, cg, _ = _gpu_step(p, pos, sp, c0)
    pos_r, _, c_r, _ = orc.step(p, pos.astype(np.float64), sp, c0.astype(np.float64))
    assert np.abs(pg - pos_r).max() <= 1e-5
    k = 9
    pk, _, ck, _ = _gpu_step(p, pos, sp, c0, k=k)
    pr, _, cr, _ = orc.run(p, pos.astype(np.float64), sp, c0.astype(np.float64), nsteps=k)
    assert np.abs(pk - pr).max() <= k * 1e-5
    assert np.abs(ck - cr).max() <= k * 1e-5 * np.abs(cr).max()


# --------------------------------------------------- kernel density deposit
@pytest.mark.parametrize("name,over", [
    ("walls_grid_2d", dict(grid=[128, 128, 1])),
    ("walls_grid_2d", dict(grid=[128, 128, 1], boundary=1, pde_bc=2, kde_range=4.0)),
    ("clumps_grid_3d", dict(grid=[48, 48, 48], diameter=[0.02, 0.03], consume=[0.0, 0.3])),
])
def test_kde_deposit_matches_oracle(name, over):
    p, pos, sp, _ = _state(name, 6000, deposit_kernel=1, **over)
    with make_sim(p, pos, sp) as sim:
        G = int(np.prod(p["grid"][: p["dim"]]))
        S = np.zeros(G, np.float32)
        R = np.zeros(G, np.float32)
        chemo.chemo_stage_deposit(sim, S, R)
    S_r, R_r = orc.kde_deposit(p, pos.astype(np.float64), sp)
    assert np.abs(S - S_r.reshape(-1)).max() <= 1e-5 * np.abs(S_r).max()
    if np.abs(R_r).max() > 0:
        assert np.abs(R - R_r.reshape(-1)).max() <= 1e-5 * np.abs(R_r).max()
    assert S_r.max() > 0


def test_kde_step_matches_oracle_and_is_bitwise_reproducible():
    p, pos, sp, c0 = _state("walls_grid_2d", 20011, grid=[128, 128, 1], deposit_kernel=1, cutoff_mode=1)
    pg, spg, cg, _ = _gpu_step(p, pos, sp, c0)
    assert_step_matches(p, pos, sp, c0, pg, spg, cg)
    # the density gather sums exactly: whole trajectories repeat bit for bit
    a = _gpu_step(p, pos, sp, c0, k=7)
    b = _gpu_step(p, pos, sp, c0, k=7)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[2], b[2])


def test_kde_in_an_ensemble():
    p, s, pos, sp = wl.ensemble_state(sizes=[700, 0, 1500], grid=[64, 64, 1], deposit_kernel=1)
    off = en.offsets(s)
    with chemo.chemo_create_batch(p, s, dev(pos), dev(sp)) as sim:
        S = np.zeros((3, 64, 64), np.float32)
        chemo.chemo_stage_deposit(sim, S, None)
    for r in range(3):
        S_r, _ = orc.kde_deposit(wl.replicate_params(p, r), pos[off[r]:off[r + 1]], sp[off[r]:off[r + 1]])
        assert np.abs(S[r] - S_r).max() <= 1e-5 * max(np.abs(S_r).max(), 1e-30)


def test_variants_have_no_adjoint():
    p, pos, sp, c0 = _state("walls_grid_2d", 100, grid=[32, 32, 1], move_scheme=1)
    with make_sim(p, pos, sp, c0) as sim:
        with pytest.raises(chemo.ChemoError) as ei:
            chemo.chemo_record(sim, 2, 1)
        assert ei.value.status == chemo.ENOTSUP
