"""Pins of the oracle's full step: Euler-Maruyama move (Eq. (2) with the
drift of Eq. (1b)), boundary handling (Sect. 3.2 reflection, Sect. 4 periodic
displacement), reactions (Sect. 3.4) and the coupled PDE update.

* noise-free moves against closed forms: reflection as the triangle wave of
  period 2L, periodic wrap as x mod L;
* statistics of the MSD set-up of Sect. 4 (Fig. 3): E|dX|^2 = 2 d D t and
  E[dX] = chi g t for chemotactic cells, E[dX] = 0 for the others;
* the unwrapped displacement equals the positions' change modulo L;
* fixed-step reactions switch a fraction r dt of the cells per step and keep
  the total number of cells;
* the grid mass after a full step follows the discrete balance law.
"""
import numpy as np
import pytest
from scipy import stats

from oracle import chemo_oracle as orc
from paper_1805_11007_gb300 import workloads as wl


def _triangle(x, lo, hi):
    L = hi - lo
    y = np.mod(x - lo, 2 * L)
    return lo + np.where(y > L, 2 * L - y, y)


def test_noise_free_reflection_closed_form():
    # D = 0, no pair force: the move is dt * chi * g; reflect until inside
    p = wl.params("periodic_fixed_gradient_2d", boundary=0, D=[0.0], inter=0.0, dt=1e-3,
                  lo=[-0.5, 0.0, 0.0], hi=[0.5, 2.0, 1.0])
    rng = np.random.default_rng(0)
    for g in ([-1000.0, 300.0], [2500.0, -4100.0], [7.0, 0.5]):
        p["fixed_grad"] = g + [0.0]
        pos = np.column_stack([rng.uniform(-0.5, 0.5, 300), rng.uniform(0.0, 2.0, 300)])
        out, _, _, _ = orc.step(p, pos, np.zeros(300, np.uint8))
        gg = np.array([np.float32(v) for v in g]).astype(np.float64)
        x1 = pos + p["dt"] * gg
        expect = np.column_stack([_triangle(x1[:, 0], -0.5, 0.5), _triangle(x1[:, 1], 0.0, 2.0)])
        np.testing.assert_allclose(out, expect, atol=1e-12)


def test_noise_free_periodic_wrap_and_displacement():
    p = wl.params("periodic_fixed_gradient_2d", D=[0.0], inter=0.0, dt=1e-3,
                  fixed_grad=[1234.5, -777.0, 0.0])
    rng = np.random.default_rng(1)
    pos = rng.random((200, 2))
    disp = np.zeros_like(pos)
    out, _, _, d = orc.step(p, pos, np.zeros(200, np.uint8), disp=disp)
    step = p["dt"] * np.array([np.float32(1234.5), np.float32(-777.0)]).astype(np.float64)
    np.testing.assert_allclose(out, np.mod(pos + step, 1.0), atol=1e-12)
    np.testing.assert_allclose(d, np.tile(step, (200, 1)), atol=1e-15)


def test_noise_is_sqrt_2_D_dt_times_philox_normals():
    p = wl.params("periodic_fixed_gradient_2d", inter=0.0, chi=0.0, D=[0.37], seed=99)
    n = 500
    pos = np.full((n, 2), 0.5)
    ids = np.arange(n, dtype=np.uint32) * 7 + 3
    out, _, _, _ = orc.step(p, pos, np.zeros(n, np.uint8), step_index=41, ids=ids)
    xi = orc.normals(99, ids, 41)
    amp = np.sqrt(2 * float(np.float32(0.37)) * p["dt"])
    np.testing.assert_allclose(out - 0.5, amp * xi[:, :2], atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_free_diffusion_and_drift_msd(dim):
    # Sect. 4 / Fig. 3: periodic box, no pair force, species 1 chemotactic in
    # the fixed gradient g, species 0 not; MSD of species 0 is 2 d D t and the
    # mean displacement of species 1 is chi g t.
    chi = 50.0
    p = wl.params("walls_grid_2d", dim=dim, boundary=1, pde_bc=2, chem_mode=1, inter=0.0, chi=chi,
                  fixed_grad=[1.0, -0.5, 0.25], D=[1.0, 0.5], dt=1e-5, seed=7, grid=[4, 4, 4])
    n, steps = 4000, 60
    pos = wl.uniform_positions(n, dim, p["lo"], p["hi"], seed=3)
    sp = wl.half_species(n, 2)
    disp = np.zeros((n, dim))
    _, _, _, disp = orc.run(p, pos, sp, nsteps=steps, disp=disp)
    t = steps * p["dt"]
    a = sp == 0
    b = sp == 1
    D0, D1 = 1.0, 0.5
    msd0 = (disp[a] ** 2).sum(1)
    se0 = msd0.std() / np.sqrt(a.sum())
    assert abs(msd0.mean() - 2 * dim * D0 * t) < 5 * se0
    g = np.array([1.0, -0.5, 0.25][:dim])
    mean1 = disp[b].mean(0)
    se1 = np.sqrt(2 * D1 * t / b.sum())
    assert np.all(np.abs(mean1 - chi * g * t) < 5 * se1)
    assert np.all(np.abs(disp[a].mean(0)) < 5 * np.sqrt(2 * D0 * t / a.sum()))
    # the centred displacement of species 1 is Gaussian with variance 2 D t
    z = ((disp[b] - chi * g * t) / np.sqrt(2 * D1 * t)).ravel()
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_periodic_displacement_tracks_positions_with_forces():
    p, pos, sp = wl.initial_state("periodic_fixed_gradient_2d")
    disp = np.zeros(pos.shape)
    out, _, _, d = orc.run(p, pos, sp, nsteps=20, disp=disp)
    diff = out - pos.astype(np.float64) - d
    np.testing.assert_allclose(diff - np.round(diff), 0.0, atol=1e-12)


def test_walls_keep_particles_inside():
    p, pos, sp = wl.initial_state("walls_grid_2d", n=3000, grid=[33, 33, 1], D=[400.0, 200.0])
    out, _, _, _ = orc.run(p, pos, sp, nsteps=5)
    assert out.min() >= 0.0 and out.max() <= 1.0


def test_step_with_pair_force_noise_free_closed_form():
    # D = 0 and no chemical: X' = X + dt F(X) (Eq. (2) without noise)
    p = wl.params("walls_grid_2d", D=[0.0, 0.0], chi=0.0, secrete=[0.0, 0.0], grid=[5, 5, 1],
                  diameter=[0.05, 0.08], dt=1e-5)
    pos = np.array([[0.5, 0.5], [0.53, 0.5], [0.5, 0.54]])
    sp = np.array([0, 1, 1], np.uint8)
    out, _, _, _ = orc.step(p, pos, sp)
    eps = lambda i, j: 0.5 * (float(np.float32([0.05, 0.08][sp[i]])) + float(np.float32([0.05, 0.08][sp[j]])))
    expect = pos.copy()
    for i in range(3):
        for j in range(3):
            if i == j:
                continue
            d = pos[i] - pos[j]
            r = np.linalg.norm(d)
            e = eps(i, j)
            if r < e:
                expect[i] += p["dt"] * (1 / e) * np.exp(-r / e) * d / r
    np.testing.assert_allclose(out, expect, atol=1e-14)


def test_reactions_rate_and_conservation():
    # Sect. 3.4: a cell switches when a uniform falls below rate * dt
    p = wl.params("walls_grid_2d", reactions=1, react_k0=[2000.0, 0.0], react_kc=[0.0, 0.0],
                  react_to=[1, 0], grid=[9, 9, 1], chi=0.0, inter=0.0, secrete=[0.0, 0.0])
    n = 200_000
    pos = wl.uniform_positions(n, 2, p["lo"], p["hi"], seed=1)
    sp = np.zeros(n, np.uint8)
    _, sp1, _, _ = orc.step(p, pos, sp)
    frac = (sp1 == 1).mean()
    prob = float(np.float32(2000.0)) * p["dt"]
    assert abs(frac - prob) < 5 * np.sqrt(prob * (1 - prob) / n)
    assert sp1.size == n


def test_reaction_rate_follows_concentration():
    # beta -> alpha at rate r_beta * c (Eq. (1c)); with c = x the switching
    # probability of a cell at x is r_beta x dt.
    p = wl.params("walls_grid_2d", reactions=1, react_k0=[0.0, 0.0], react_kc=[0.0, 4000.0],
                  react_to=[1, 0], chem_mode=1, fixed_grad=[1.0, 0.0, 0.0], chi=0.0, inter=0.0,
                  secrete=[0.0, 0.0], grid=[9, 9, 1])
    n = 200_000
    pos = wl.uniform_positions(n, 2, p["lo"], p["hi"], seed=2)
    sp = np.ones(n, np.uint8)
    _, sp1, _, _ = orc.step(p, pos, sp)
    left = pos[:, 0] < 0.5
    pl = (sp1[left] == 0).mean()
    pr = (sp1[~left] == 0).mean()
    r = float(np.float32(4000.0)) * p["dt"]
    assert abs(pl - r * 0.25) < 5 * np.sqrt(r * 0.25 / left.sum())
    assert abs(pr - r * 0.75) < 5 * np.sqrt(r * 0.75 / (~left).sum())


def test_full_step_grid_mass_balance():
    p, pos, sp = wl.initial_state("walls_grid_2d", n=20000, grid=[65, 65, 1], dt=1e-4)
    c0 = wl.random_field(p, seed=5).astype(np.float64)
    out, _, c1, _ = orc.step(p, pos, sp, c0)
    dim = 2
    h = orc.grid_h(p, 0)
    tau = np.ones(orc.grid_shape(p))
    for ax in range(dim):
        sl = [slice(None)] * dim
        sl[ax] = 0
        tau[tuple(sl)] *= 0.5
        sl[ax] = -1
        tau[tuple(sl)] *= 0.5
    vol = tau * h * h
    s = orc.substeps(p)
    dts = p["dt"] / s
    g = float(np.float32(0.1))
    src = p["dt"] * float(np.float32(0.1)) * (sp == 0).sum()
    M = (c0 * vol).sum()
    for _ in range(s):
        M = M * (1 - g * dts) + src / s
    assert abs((c1 * vol).sum() - M) <= 1e-10 * M
