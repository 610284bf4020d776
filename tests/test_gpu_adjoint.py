"""The adjoint (chemo_record + chemo_gradient, through torch.autograd)
against FP64 central finite differences of the oracle, with the noise frozen
(same Philox counters): gradients of the differentiable workload's loss
(mean x-displacement + mean squared soft occupancy) with respect to chi, the
interaction strength and the diffusivities, and with respect to initial
positions."""
import numpy as np
import pytest
import torch

from oracle import chemo_oracle as orc
from paper_1805_11007_gb300 import adjoint as adj
from paper_1805_11007_gb300 import chemo
from paper_1805_11007_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

NB = 12  # analysis grid of the occupancy loss


def _setup(n=1500, grid=33, **over):
    p = wl.params("adjoint_2d", grid=[grid, grid, 1], **over)
    pos = wl.uniform_positions(n, 2, p["lo"], p["hi"], seed=21)
    sp = wl.half_species(n, 2)
    c0 = wl.random_field(p, seed=22, scale=0.3) if p["chem_mode"] == 0 else None
    return p, pos, sp, c0


def _gpu_grads(p, pos, sp, c0, nsteps, every, nb=NB):
    dpos = torch.from_numpy(pos).cuda()
    dsp = torch.from_numpy(sp).cuda()
    dc0 = torch.from_numpy(c0).cuda() if c0 is not None else None
    sim = chemo.chemo_create(p, dpos, dsp)
    try:
        theta = torch.tensor(adj.theta_of(p), dtype=torch.float64, requires_grad=True)
        x0 = dpos.clone().requires_grad_(True)
        xN = adj.ChemoRun.apply(theta, x0, sim, nsteps, every, dsp, dc0)
        L = adj.mean_x_displacement(xN, x0) + adj.occupancy_loss(xN, nb, p["lo"], p["hi"])
        L.backward()
        return float(L.item()), theta.grad.numpy().copy(), x0.grad.cpu().numpy().astype(np.float64)
    finally:
        sim.close()


def _oracle_loss(p, pos, sp, c0, nsteps, theta=None, pos0=None, nb=NB):
    q = adj.with_theta(p, theta) if theta is not None else p
    x0 = pos if pos0 is None else pos0
    xN, _, _, _ = orc.run(q, x0, sp, None if c0 is None else c0.astype(np.float64), nsteps=nsteps)
    return adj.loss_numpy(xN, x0, nb, p["lo"], p["hi"])


def _tangent_grads(p, pos, sp, c0, nsteps, nb=NB):
    """dL/dtheta of the oracle's own FP64 trajectory: the oracle's tangent
    (dX_N/dtheta, the step differentiated operation by operation) contracted
    with dL/dX_N (the loss differentiated by torch on the CPU in FP64)."""
    xN, _, _, dx, _ = orc.run_tangent(p, pos, sp, None if c0 is None else c0.astype(np.float64), nsteps=nsteps)
    xt = torch.from_numpy(xN).requires_grad_(True)
    x0 = torch.from_numpy(np.asarray(pos, np.float64))
    L = adj.mean_x_displacement(xt, x0) + adj.occupancy_loss(xt, nb, p["lo"], p["hi"])
    L.backward()
    return float(L.item()), np.einsum("ia,iak->k", xt.grad.numpy(), dx)


def _tangent_case(kind, over):
    if kind in ("full", "full7"):
        p, pos, sp = wl.initial_state("adjoint_2d")
        return p, pos, sp, None, 5 if kind == "full" else 7, 2, 64
    if kind == "3d":
        p = wl.params("clumps_grid_3d", grid=[17, 17, 17], dt=1e-5, diameter=[0.04, 0.06], cutoff_mode=1, **over)
        pos = wl.uniform_positions(700, 3, p["lo"], p["hi"], seed=31)
        return p, pos, wl.half_species(700, 2), wl.random_field(p, seed=32, scale=0.3), 12, 4, NB
    p, pos, sp, c0 = _setup(**over)
    return p, pos, sp, c0, 20, 5, NB


@pytest.mark.parametrize("kind,over", [
    ("full", dict()),
    ("full7", dict()),
    ("2d", dict()),
    ("2d", dict(chem_mode=1, fixed_grad=[3.0, -2.0, 0.0], boundary=1, pde_bc=2, diameter=[0.01, 0.02])),
    ("2d", dict(pde_substeps=3, Dc=20.0)),
    ("2d", dict(pde_substeps=5, Dc=20.0, boundary=1, pde_bc=2)),
    ("3d", dict()),
    ("3d", dict(boundary=1, pde_bc=2)),
])
def test_parameter_gradients_match_oracle_tangent(kind, over):
    """The adjoint against the oracle's own derivative (its forward-mode
    tangent along the FP64 trajectory, pinned against central differences
    and closed forms on the CPU) rather than differences with a step h: the
    differentiable workload at full density over 5 and 7 steps, the 2D
    cases over 20 steps and the 3D ones over 12. Measured on a GB300: the
    2D grid cases agree to 2e-5 of the largest component (central
    differences at h = 1e-4 were 2.5e-3 off, 3.6 % on dL/dD_0), the 3D ones
    to 1e-6, the full-density workload to 1.6e-3 over 5 steps and 4.2e-3
    over 7 (dL/dD_1 7.237e-3 against 7.268e-3; the differences, averaging a
    cutoff kink, give 6.945e-3), and the fixed gradient to 1e-3. Over 10
    steps the gap is 2.4 % of the largest component, over 15 steps 13 %:
    the FP32 path parts from the FP64 one."""
    p, pos, sp, c0, nsteps, every, nb = _tangent_case(kind, over)
    L_gpu, g, _ = _gpu_grads(p, pos, sp, c0, nsteps, every, nb=nb)
    L_t, g_t = _tangent_grads(p, pos, sp, c0, nsteps, nb=nb)
    assert abs(L_gpu - L_t) <= 1e-4 * abs(L_t)
    scale = np.abs(g_t).max()
    assert scale > 0
    assert np.all(np.abs(g - g_t) <= 0.01 * np.abs(g_t) + 0.005 * scale), (g, g_t)


def test_differentiable_workload_gradients_at_full_density():
    """The differentiable workload itself: 50,000 cells of the 2D walls
    physics on the 512^2 grid (12 PDE substeps), force shifted to zero at
    the cutoff, the loss on a 64^2 analysis grid, from its seeded initial
    state (c = 0), checkpointed every 2 steps. Over 5 steps the oracle's
    central differences at h = 1e-4 and h/2 agree to 6.5e-4, and the
    adjoint of the FP32 map matches them to 0.12 % of the largest component.
    Over 7 steps the differences still agree with each other but straddle a
    kink (a pair within h of its cutoff, where the shifted force's
    derivative jumps) and miss the slope at theta by 4 % on dL/dD_1; the
    7-step case is checked against the oracle's tangent instead; over 10
    steps the differences no longer converge
    (tests/golden/adjoint_fd_horizon.txt)."""
    p, pos, sp = wl.initial_state("adjoint_2d")
    assert pos.shape[0] == 50_000 and chemo.grid_shape(p) == (512, 512)
    nsteps, every, nb = 5, 2, 64
    L_gpu, g, _ = _gpu_grads(p, pos, sp, None, nsteps, every, nb=nb)
    L_orc = _oracle_loss(p, pos, sp, None, nsteps, nb=nb)
    assert abs(L_gpu - L_orc) <= 1e-4 * abs(L_orc)
    theta = np.array(adj.theta_of(p))
    h = 1e-4
    fd = np.zeros_like(theta)
    for k in range(theta.size):
        tp = theta.copy(); tp[k] += h
        tm = theta.copy(); tm[k] -= h
        fd[k] = (_oracle_loss(p, pos, sp, None, nsteps, tp, nb=nb) -
                 _oracle_loss(p, pos, sp, None, nsteps, tm, nb=nb)) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 0 and np.all(fd != 0.0)
    err = np.abs(g - fd)
    assert np.all(err <= 0.03 * np.abs(fd) + 0.01 * scale), (g, fd)


@pytest.mark.parametrize("over", [dict(), dict(chem_mode=1, fixed_grad=[3.0, -2.0, 0.0], boundary=1, pde_bc=2,
                                               diameter=[0.01, 0.02]),
                                  # several PDE substeps (one and two launches of the multi-substep kernel)
                                  dict(pde_substeps=3, Dc=20.0), dict(pde_substeps=14, Dc=50.0),
                                  dict(pde_substeps=5, Dc=20.0, boundary=1, pde_bc=2)])
def test_parameter_gradients_match_oracle_finite_differences(over):
    p, pos, sp, c0 = _setup(**over)
    nsteps, every = 20, 5
    L_gpu, g, _ = _gpu_grads(p, pos, sp, c0, nsteps, every)
    L_orc = _oracle_loss(p, pos, sp, c0, nsteps)
    assert abs(L_gpu - L_orc) <= 1e-4 * abs(L_orc)
    theta = np.array(adj.theta_of(p))
    h = 1e-4
    fd = np.zeros_like(theta)
    for k in range(theta.size):
        tp = theta.copy(); tp[k] += h
        tm = theta.copy(); tm[k] -= h
        fd[k] = (_oracle_loss(p, pos, sp, c0, nsteps, tp) - _oracle_loss(p, pos, sp, c0, nsteps, tm)) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 0
    err = np.abs(g - fd)
    assert np.all(err <= 0.03 * np.abs(fd) + 0.01 * scale), (g, fd)


def test_initial_position_gradient_matches_oracle_finite_differences():
    p, pos, sp, c0 = _setup(n=800)
    nsteps, every = 12, 4
    _, _, gx = _gpu_grads(p, pos, sp, c0, nsteps, every)
    rng = np.random.default_rng(3)
    pick = rng.choice(pos.shape[0], size=6, replace=False)
    h = 1e-5
    for i in pick:
        for a in range(2):
            xp = pos.astype(np.float64).copy(); xp[i, a] += h
            xm = pos.astype(np.float64).copy(); xm[i, a] -= h
            fd = (_oracle_loss(p, pos, sp, c0, nsteps, pos0=xp) - _oracle_loss(p, pos, sp, c0, nsteps, pos0=xm)) / (2 * h)
            assert abs(gx[i, a] - fd) <= 0.03 * abs(fd) + 2e-3 * np.abs(gx).max(), (i, a, gx[i, a], fd)


def _tangent_direction(p, pos, sp, c0, nsteps, v, nb=NB):
    """dL/dX_0 . v of the oracle's FP64 trajectory: a free tangent column
    seeded with v, contracted with dL/dX_N, plus the loss's own dL/dX_0 . v."""
    P = 2 + int(p["n_species"])
    d0 = np.zeros(pos.shape + (P + 1,))
    d0[:, :, P] = v
    x0 = np.asarray(pos, np.float64)
    xN, _, _, dx, _ = orc.run_tangent(p, x0, sp, None if c0 is None else c0.astype(np.float64), nsteps=nsteps,
                                      dpos=d0, extra=1)
    xt = torch.from_numpy(xN).requires_grad_(True)
    x0t = torch.from_numpy(x0).requires_grad_(True)
    L = adj.mean_x_displacement(xt, x0t) + adj.occupancy_loss(xt, nb, p["lo"], p["hi"])
    L.backward()
    return float((xt.grad.numpy() * dx[:, :, P]).sum() + (x0t.grad.numpy() * v).sum())


@pytest.mark.parametrize("kind,over", [("2d", dict()), ("2d", dict(pde_substeps=5, Dc=20.0, boundary=1, pde_bc=2)),
                                       ("3d", dict())])
def test_initial_position_gradient_matches_oracle_tangent(kind, over):
    """The gradient with respect to every initial position, projected on
    three random directions, against the oracle's directional derivative
    (its tangent seeded with the direction)."""
    p, pos, sp, c0, nsteps, every, nb = _tangent_case(kind, over)
    _, _, gx = _gpu_grads(p, pos, sp, c0, nsteps, every, nb=nb)
    rng = np.random.default_rng(11)
    for r in range(3):
        v = rng.standard_normal(pos.shape)
        want = _tangent_direction(p, pos, sp, c0, nsteps, v, nb=nb)
        got = float((gx * v).sum())
        assert abs(got - want) <= 2e-3 * abs(want), (r, got, want)


def test_record_leaves_final_state_and_gradient_restores_it():
    p, pos, sp, c0 = _setup(n=1000)
    dpos = torch.from_numpy(pos).cuda()
    dsp = torch.from_numpy(sp).cuda()
    with chemo.chemo_create(p, dpos, dsp) as a, chemo.chemo_create(p, dpos, dsp) as b:
        chemo.chemo_write_field(a, torch.from_numpy(c0).cuda())
        chemo.chemo_write_field(b, torch.from_numpy(c0).cuda())
        chemo.chemo_record(a, 10, 3)
        chemo.chemo_step_n(b, 10)
        pa, _, _ = chemo.read_state_host(a)
        pb, _, _ = chemo.read_state_host(b)
        assert np.abs(pa - pb).max() <= 1e-5
        g = torch.zeros((1000, 2), dtype=torch.float32, device="cuda")
        g[:, 0] = 1.0 / 1000
        dth = torch.zeros(4, dtype=torch.float32, device="cuda")
        chemo.chemo_gradient(a, g, dth)
        pa2, _, _ = chemo.read_state_host(a)
        np.testing.assert_array_equal(pa2, pa)
        assert chemo.chemo_step_index(a) == 10
        assert torch.isfinite(dth).all()
        # steps taken after the record do not change what the gradient
        # restores: the recorded run's final state and step index
        chemo.chemo_step_n(a, 4)
        dth2 = torch.zeros(4, dtype=torch.float32, device="cuda")
        chemo.chemo_gradient(a, g, dth2)
        pa3, _, _ = chemo.read_state_host(a)
        np.testing.assert_array_equal(pa3, pa)
        assert chemo.chemo_step_index(a) == 10
        torch.testing.assert_close(dth2, dth, rtol=1e-4, atol=1e-6 * float(dth.abs().max()))


@pytest.mark.parametrize("over", [dict(), dict(boundary=1, pde_bc=2), dict(pde_substeps=3, Dc=5.0)])
def test_parameter_gradients_3d_match_oracle_finite_differences(over):
    """The 3D adjoint (transposed 7-point stencil written out, trilinear
    interpolation Jacobian, 3^3 pair window) against FP64 central finite
    differences of the oracle."""
    p = wl.params("clumps_grid_3d", grid=[17, 17, 17], dt=1e-5, diameter=[0.04, 0.06], cutoff_mode=1, **over)
    pos = wl.uniform_positions(700, 3, p["lo"], p["hi"], seed=31)
    sp = wl.half_species(700, 2)
    c0 = wl.random_field(p, seed=32, scale=0.3)
    nsteps, every = 12, 4
    dpos = torch.from_numpy(pos).cuda()
    dsp = torch.from_numpy(sp).cuda()
    with chemo.chemo_create(p, dpos, dsp) as sim:
        theta = torch.tensor(adj.theta_of(p), dtype=torch.float64, requires_grad=True)
        x0 = dpos.clone().requires_grad_(True)
        xN = adj.ChemoRun.apply(theta, x0, sim, nsteps, every, dsp, torch.from_numpy(c0).cuda())
        L = adj.mean_x_displacement(xN, x0) + adj.occupancy_loss(xN, NB, p["lo"], p["hi"])
        L.backward()
        g = theta.grad.numpy().copy()

    def loss(th):
        q = adj.with_theta(p, th)
        xT, _, _, _ = orc.run(q, pos, sp, c0.astype(np.float64), nsteps=nsteps)
        return adj.loss_numpy(xT, pos, NB, p["lo"], p["hi"])

    theta_np = np.array(adj.theta_of(p))
    h = 1e-4
    fd = np.zeros_like(theta_np)
    for k in range(theta_np.size):
        tp = theta_np.copy(); tp[k] += h
        tm = theta_np.copy(); tm[k] -= h
        fd[k] = (loss(tp) - loss(tm)) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 0
    assert np.all(np.abs(g - fd) <= 0.03 * np.abs(fd) + 0.01 * scale), (g, fd)


def _segment_bytes(info, n, dim, every):
    """Device memory of one stored segment, from the layout chemo_record_stored
    documents (with the allocator's rounding)."""
    words = info["bin_slots"] // 2 + ((info["bin_slots"] // 8 + 1 + 3) & ~3)
    return every * (n * (8 * dim + 16) + 4 * info["grid_nodes"] + 4 * words) + n * 4 * dim + 6 * 256


@pytest.mark.parametrize("over", [dict(), dict(boundary=1, pde_bc=2, pde_substeps=5, Dc=20.0)])
def test_stored_segments_give_the_checkpointed_gradient(over):
    """Segments stored during the record (all of them, or the latest two that
    fit in a budget) give the gradient of the fully checkpointed run: the
    stored states are those the re-run computes (to the rounding of the
    deposit's float atomics)."""
    p, pos, sp, c0 = _setup(n=1200, **over)
    nsteps, every = 23, 4  # 6 segments, the last one short
    dpos = torch.from_numpy(pos).cuda()
    dsp = torch.from_numpy(sp).cuda()
    dc0 = torch.from_numpy(c0).cuda()
    out = []
    with chemo.chemo_create(p, dpos, dsp) as sim:
        seg = _segment_bytes(chemo.chemo_get_info(sim), dpos.shape[0], 2, every)
        for store in (0, -1, 2 * seg + seg // 2):
            chemo.chemo_write_state(sim, dpos, dsp)
            chemo.chemo_write_field(sim, dc0)
            chemo.chemo_set_step_index(sim, 0)
            chemo.chemo_record(sim, nsteps, every, store_bytes=store)
            xT = torch.zeros_like(dpos)
            chemo.chemo_read_state(sim, xT, None, None)
            g = torch.zeros_like(dpos)
            g[:, 0] = 1.0 / dpos.shape[0]
            g[:, 1] = torch.linspace(-1.0, 1.0, dpos.shape[0], device="cuda") / dpos.shape[0]
            dth = torch.zeros(4, dtype=torch.float32, device="cuda")
            dx0 = torch.zeros_like(dpos)
            chemo.chemo_gradient(sim, g, dth, None, dx0)
            assert chemo.chemo_step_index(sim) == nsteps
            out.append((xT.cpu().numpy(), dth.cpu().numpy().astype(np.float64), dx0.cpu().numpy().astype(np.float64)))
    for xT, dth, dx0 in out[1:]:
        assert np.abs(xT - out[0][0]).max() <= 1e-5
        np.testing.assert_allclose(dth, out[0][1], rtol=1e-3, atol=1e-6 * np.abs(out[0][1]).max())
        assert np.abs(dx0 - out[0][2]).max() <= 1e-3 * np.abs(out[0][2]).max() + 1e-9
