"""Pins of the oracle's variants (no GPU): tamed Euler (Sect. 3.2, the tamed
scheme), the hard-sphere overlap correction (Sect. 3.2) and the Gaussian
kernel density estimate (Sect. 2.3; the density listing of Sect. 3). Each
pin is a property the paper or the mathematics fixes: agreement with
Euler-Maruyama to second order and a bounded step; the separation after a
correction and its split by diffusivity; unit mass and second moment d
sigma^2 of the kernel."""
import numpy as np
import pytest

from oracle import chemo_oracle as orc
from paper_1805_11007_gb300 import workloads as wl


def _one_step(p, pos, sp, c=None):
    pos_r, sp_r, c_r, _ = orc.step(p, np.asarray(pos, np.float64), np.asarray(sp, np.uint8),
                                   None if c is None else np.asarray(c, np.float64))
    return pos_r, c_r


# ---------------------------------------------------------------- tamed Euler
def _drift_only(**over):
    # fixed gradient, one chemotactic species, no noise, no pairs
    base = dict(dim=2, boundary=1, lo=[0, 0, 0], hi=[1, 1, 1], n_species=1, diameter=[0.0], D=[0.0],
                chemotactic=[1.0], secrete=[0.0], consume=[0.0], chi=1.0, inter=0.0, chem_mode=1,
                fixed_grad=[3.0, -4.0, 0.0], grid=[3, 3, 1], pde_bc=2, dt=1e-3, seed=3)
    base.update(over)
    return base


@pytest.mark.parametrize("dt", [1e-2, 1e-3, 1e-4])
def test_tamed_agrees_with_euler_to_second_order(dt):
    pos = np.array([[0.5, 0.5]])
    em, _ = _one_step(_drift_only(dt=dt), pos, [0])
    tm, _ = _one_step(_drift_only(dt=dt, move_scheme=1), pos, [0])
    d_em, d_tm = em - pos, tm - pos
    a = 5.0  # |grad| = |(3, -4)|
    assert np.linalg.norm(d_em - d_tm) <= (dt * a) ** 2 * (1 + 1e-9)
    assert np.linalg.norm(d_tm) > 0.0
    # same direction
    cos = float(d_em[0] @ d_tm[0]) / (np.linalg.norm(d_em) * np.linalg.norm(d_tm))
    assert cos == pytest.approx(1.0, abs=1e-12)


def test_tamed_step_is_bounded_for_a_singular_force():
    """Two almost coincident cells with a strong repulsion: Euler-Maruyama
    throws them far apart, the tamed step moves each by less than one."""
    p = dict(dim=2, boundary=0, lo=[0, 0, 0], hi=[100, 100, 1], n_species=1, diameter=[1.0], D=[0.0],
             chemotactic=[0.0], secrete=[0.0], consume=[0.0], chi=0.0, inter=1e6, chem_mode=1,
             fixed_grad=[0, 0, 0], grid=[3, 3, 1], dt=1e-2, seed=1)
    pos = np.array([[50.0, 50.0], [50.0 + 1e-3, 50.0]])
    em, _ = _one_step(p, pos, [0, 0])
    tm, _ = _one_step(dict(p, move_scheme=1), pos, [0, 0])
    assert np.linalg.norm(em - pos, axis=1).min() > 10.0
    step = np.linalg.norm(tm - pos, axis=1)
    assert np.all(step < 1.0) and np.all(step > 0.99)  # |dt f / (1 + dt |f|)| -> 1 from below
    # pushed apart along the line of centres, symmetric
    np.testing.assert_allclose(tm[0] - pos[0], -(tm[1] - pos[1]), rtol=0, atol=1e-12)
    assert tm[0, 0] < pos[0, 0] and tm[1, 0] > pos[1, 0]


# ---------------------------------------------------------- hard-sphere rule
def _hs_params(**over):
    # sizes are binary fractions: the oracle takes them in single precision
    base = dict(dim=2, boundary=0, lo=[0, 0, 0], hi=[1, 1, 1], n_species=2, diameter=[0.125, 0.125], D=[1.0, 1.0],
                chemotactic=[0, 0], secrete=[0, 0], consume=[0, 0], chi=0.0, inter=0.0, chem_mode=1,
                fixed_grad=[0, 0, 0], grid=[3, 3, 1], dt=1e-4, seed=1, hard_sphere=1)
    base.update(over)
    return base


def test_overlap_of_equal_cells_is_undone_twice_symmetrically():
    p = _hs_params()
    d = 0.09375  # contact 0.125: penetration 0.03125
    pos = np.array([[0.4, 0.5], [0.4 + d, 0.5]])
    out = orc.hard_sphere(p, pos, [0, 0])
    sep = out[1, 0] - out[0, 0]
    assert sep == pytest.approx(2 * 0.125 - d, abs=1e-14)  # moved apart by 2 d_p in total
    assert out[:, 0].mean() == pytest.approx(pos[:, 0].mean(), abs=1e-14)
    np.testing.assert_allclose(out[:, 1], pos[:, 1], atol=0)


def test_immobile_partner_leaves_the_whole_move_to_the_other():
    p = _hs_params(D=[0.0, 2.0], diameter=[0.125, 0.375])  # contact 0.25
    pos = np.array([[0.5, 0.5], [0.5, 0.5 + 0.1875]])
    out = orc.hard_sphere(p, pos, [0, 1])
    np.testing.assert_array_equal(out[0], pos[0])
    assert out[1, 1] - pos[1, 1] == pytest.approx(2 * (0.25 - 0.1875), abs=1e-14)


def test_split_follows_the_diffusivities():
    p = _hs_params(D=[1.0, 3.0])
    pos = np.array([[0.3, 0.3], [0.3 + 0.09, 0.3 + 0.12]])  # d = 0.15 > contact 0.125: no overlap
    np.testing.assert_array_equal(orc.hard_sphere(p, pos, [0, 1]), pos)
    pos = np.array([[0.3, 0.3], [0.3 + 0.03, 0.3 + 0.04]])  # d = 0.05, d_p = 0.075
    out = orc.hard_sphere(p, pos, [0, 1])
    d = np.linalg.norm(pos[0] - pos[1])
    u = (pos[0] - pos[1]) / d
    np.testing.assert_allclose(out[0] - pos[0], 2 * (0.125 - d) * 0.25 * u, atol=1e-14)
    np.testing.assert_allclose(out[1] - pos[1], -2 * (0.125 - d) * 0.75 * u, atol=1e-14)


def test_correction_reflects_at_walls_and_wraps_periodically():
    p = _hs_params()
    pos = np.array([[0.01, 0.5], [0.0725, 0.5]])  # d_p 0.0625: cell 0 pushed to -0.0525, reflected
    out = orc.hard_sphere(p, pos, [0, 0])
    assert out[0, 0] == pytest.approx(0.0525, abs=1e-14)
    q = _hs_params(boundary=1)
    pos = np.array([[0.98, 0.5], [0.02, 0.5]])  # 0.04 apart across the periodic edge, d_p 0.085
    out = orc.hard_sphere(q, pos, [0, 0])
    assert out[0, 0] == pytest.approx(0.98 - 0.085, abs=1e-12)
    assert out[1, 0] == pytest.approx(0.02 + 0.085, abs=1e-12)


def test_hard_sphere_step_is_move_then_correction():
    p = _hs_params(D=[0.0, 0.0])  # no noise, no force: the step is the correction alone
    pos = np.array([[0.4, 0.5], [0.45, 0.5], [0.8, 0.8]])
    out, _ = _one_step(p, pos, [0, 0, 1])
    np.testing.assert_allclose(out, orc.hard_sphere(p, pos, [0, 0, 1]), atol=1e-15)
    assert out[1, 0] - out[0, 0] == pytest.approx(0.2, abs=1e-14)  # 2 x 0.125 - 0.05


# --------------------------------------------------- kernel density estimate
def _kde_params(dim, sigma_h, rng_bw, boundary=0, **over):
    g = 41 if dim == 2 else 33
    base = dict(dim=dim, boundary=boundary, lo=[0, 0, 0], hi=[1, 1, 1], n_species=1, D=[0.0], chemotactic=[0.0],
                secrete=[2.0], consume=[0.5], chi=0.0, inter=0.0, grid=[g, g, g], Dc=0.0, gamma=0.0,
                pde_bc=2 if boundary else 0, dt=1e-3, seed=1, deposit_kernel=1, kde_range=rng_bw)
    h = 1.0 / (g if boundary else g - 1)
    base["diameter"] = [sigma_h * h]
    base.update(over)
    return base, h


@pytest.mark.parametrize("dim", [2, 3])
def test_kde_unit_mass_and_second_moment(dim):
    p, h = _kde_params(dim, 2.5 if dim == 2 else 2.0, 9.0)  # walls 8 bandwidths away
    X = np.array([[0.5 + 0.3 * h, 0.5 - 0.2 * h, 0.5 + 0.1 * h][:dim]])
    S, R = orc.kde_deposit(p, X, [0])
    rho = S / (p["dt"] * p["secrete"][0])
    np.testing.assert_allclose(R, p["consume"][0] * rho, rtol=1e-13, atol=0)
    assert rho.sum() * h ** dim == pytest.approx(1.0, abs=1e-9)
    axes = np.meshgrid(*[np.arange(s) * h for s in rho.shape], indexing="ij")  # [z][y][x] order
    coords = axes[::-1]  # x, y, (z)
    r2 = sum((coords[a] - X[0, a]) ** 2 for a in range(dim))
    sig = float(np.float32(p["diameter"][0]))
    assert (rho * r2).sum() * h ** dim == pytest.approx(dim * sig ** 2, rel=1e-8)


def test_kde_truncation_and_periodic_image():
    p, h = _kde_params(2, 2.0, 9.0, boundary=1)
    X = np.array([[0.0 + 0.4 * h, 1.0 - 0.3 * h]])  # next to the corner: the kernel wraps
    S, _ = orc.kde_deposit(p, X, [0])
    rho = S / (p["dt"] * p["secrete"][0])
    assert rho.sum() * h ** 2 == pytest.approx(1.0, abs=1e-9)
    q = dict(p, kde_range=1e-3)  # nothing within range of any node
    S0, _ = orc.kde_deposit(q, X, [0])
    assert S0.sum() == 0.0


def test_kde_step_adds_the_density_source():
    p, h = _kde_params(2, 2.0, 5.0)
    X = np.array([[0.31, 0.62], [0.7, 0.2]])
    c0 = wl.random_field(dict(p, grid=[41, 41, 1]), seed=2)
    S, R = orc.kde_deposit(p, X, [0, 0])
    _, c1 = _one_step(p, X, [0, 0], c0)
    # D_c = gamma = 0, one substep: c' = c + dt (-R c) + S
    np.testing.assert_allclose(c1, c0 + p["dt"] * (-R * c0) + S, rtol=1e-13, atol=1e-15)
