"""Pins of the oracle's tangent (forward-mode derivative of the step with
respect to theta = (chi, inter, D_0 .. D_{ns-1}), noise frozen): its
trajectory is run()'s bit for bit; its derivatives match FP64 central
differences of run() (steps exactly representable after the oracle's
single-precision rounding of the constants); and two closed forms, free
diffusion (dX/dD_s = sum_n dt / sqrt(2 D_s dt) xi_n) and drift in a fixed
gradient (dX/dchi = N dt chemotactic_s g)."""
import numpy as np
import pytest

from oracle import chemo_oracle as orc
from paper_1805_11007_gb300 import workloads as wl


def _with_theta(p, th):
    q = dict(p)
    q["chi"], q["inter"] = th[0], th[1]
    ns = int(p["n_species"])
    D = list(p["D"])
    D[:ns] = th[2:2 + ns]
    q["D"] = D
    return q


def _theta(p):
    return [float(p["chi"]), float(p["inter"])] + [float(v) for v in p["D"][:int(p["n_species"])]]


CASES = [
    ("2d walls, force shifted", "adjoint_2d", dict(grid=[33, 33, 1]), 2, 5),
    ("2d walls, hard cutoff", "walls_grid_2d", dict(grid=[33, 33, 1]), 2, 5),
    ("2d periodic, dense", "walls_grid_2d", dict(grid=[33, 33, 1], boundary=1, pde_bc=2, diameter=[0.03, 0.05]), 2, 5),
    ("2d fixed gradient", "walls_grid_2d", dict(chem_mode=1, fixed_grad=[3.0, -2.0, 0.0], boundary=1, pde_bc=2,
                                                diameter=[0.03, 0.05]), 2, 5),
    ("2d consumption, substeps", "walls_grid_2d", dict(grid=[33, 33, 1], consume=[0.0, 2.0], pde_substeps=3,
                                                       Dc=5.0, diameter=[0.03, 0.05]), 2, 5),
    ("3d walls", "clumps_grid_3d", dict(grid=[16, 16, 16], diameter=[0.04, 0.06], dt=1e-5), 3, 4),
    ("3d periodic", "clumps_grid_3d", dict(grid=[16, 16, 16], diameter=[0.04, 0.06], dt=1e-5, boundary=1,
                                           pde_bc=2), 3, 4),
]


def _case(name, over, dim):
    p = wl.params(name, **over)
    pos = wl.uniform_positions(400, dim, p["lo"], p["hi"], seed=5)
    sp = wl.half_species(400, int(p["n_species"]))
    c = wl.random_field(p, seed=6, scale=0.3) if p["chem_mode"] == 0 else None
    return p, pos, sp, c


@pytest.mark.parametrize("label,name,over,dim,steps", CASES)
def test_tangent_trajectory_is_run_bit_for_bit(label, name, over, dim, steps):
    p, pos, sp, c = _case(name, over, dim)
    x, s, cN, _ = orc.run(p, pos, sp, c, nsteps=steps)
    xt, st, ct, dx, dc = orc.run_tangent(p, pos, sp, c, nsteps=steps)
    np.testing.assert_array_equal(xt, x)
    np.testing.assert_array_equal(st, s)
    if cN is not None:
        np.testing.assert_array_equal(ct, cN)
        assert dc.shape == cN.shape + (len(_theta(p)),)
    assert dx.shape == (pos.shape[0], dim, len(_theta(p)))


@pytest.mark.parametrize("label,name,over,dim,steps", CASES)
def test_tangent_matches_central_differences(label, name, over, dim, steps):
    p, pos, sp, c = _case(name, over, dim)
    th = _theta(p)
    _, _, cN, dx, dc = orc.run_tangent(p, pos, sp, c, nsteps=steps)
    for k in range(len(th)):
        # positions: a small step (the derivative is smooth in theta); the
        # field depends on chi only through where the cells deposit, a
        # derivative of order 1e-8, so a larger step keeps its difference
        # above the rounding of c
        for h, field in ((2.0 ** -20, False), (2.0 ** -12, True)):
            if field and cN is None:
                continue
            tp, tm = list(th), list(th)
            tp[k] = float(np.float32(th[k] + h))
            tm[k] = float(np.float32(th[k] - h))
            xp, _, cp, _ = orc.run(_with_theta(p, tp), pos, sp, c, nsteps=steps)
            xm, _, cm, _ = orc.run(_with_theta(p, tm), pos, sp, c, nsteps=steps)
            den = tp[k] - tm[k]
            if field:
                fd = (cp - cm) / den
                assert np.abs(fd - dc[..., k]).max() <= 2e-4 * np.abs(fd).max(), (label, k)
            else:
                fd = (xp - xm) / den
                assert np.abs(fd - dx[:, :, k]).max() <= 2e-5 * np.abs(fd).max(), (label, k)


def test_tangent_free_diffusion_closed_form():
    # no interaction, no chemotaxis, cells far from the walls for a few
    # steps: X_N = X_0 + sum_n sqrt(2 D_s dt) xi_n, so
    # dX_N / dD_s = sum_n dt / sqrt(2 D_s dt) xi_n (the derivatives with
    # respect to inter and chi are not zero there: the unit pair force and
    # the gradient of the deposited field)
    p = wl.params("walls_grid_2d", grid=[17, 17, 1], inter=0.0, chi=0.0, dt=1e-6, D=[1.0, 0.5])
    rng = np.random.default_rng(9)
    n = 200
    pos = (0.3 + 0.4 * rng.random((n, 2))).astype(np.float32)
    sp = wl.half_species(n, 2)
    steps = 4
    _, _, _, dx, _ = orc.run_tangent(p, pos, sp, None, nsteps=steps)
    ids = np.arange(n, dtype=np.uint32)
    xi = sum(orc.normals(int(p["seed"]), ids, k)[:, :2] for k in range(steps))
    dt = float(p["dt"])  # the oracle keeps dt in double, the other constants in single precision
    for s, D in enumerate(p["D"]):
        amp = np.sqrt(2.0 * float(np.float32(D)) * dt)
        want = np.where((sp == s)[:, None], dt / amp * xi, 0.0)
        np.testing.assert_allclose(dx[:, :, 2 + s], want, rtol=1e-12, atol=1e-15)


def test_tangent_fixed_gradient_drift_closed_form():
    # fixed gradient g, no interaction, periodic box: the drift adds
    # dt chi chemotactic_s g every step, so dX_N / dchi = N dt chemotactic_s g
    g = [3.0, -2.0, 0.0]
    p = wl.params("walls_grid_2d", chem_mode=1, fixed_grad=g, boundary=1, pde_bc=2, inter=0.0, dt=1e-5)
    pos = wl.uniform_positions(300, 2, p["lo"], p["hi"], seed=4)
    sp = wl.half_species(300, 2)
    steps = 6
    _, _, _, dx, _ = orc.run_tangent(p, pos, sp, None, nsteps=steps)
    dt = float(p["dt"])
    kap = np.asarray(p["chemotactic"], np.float32).astype(np.float64)[sp]
    want = steps * dt * kap[:, None] * np.asarray([float(np.float32(v)) for v in g[:2]])[None, :]
    np.testing.assert_allclose(dx[:, :, 0], want, rtol=1e-12, atol=1e-18)


@pytest.mark.parametrize("label,name,over,dim,steps", [CASES[0], CASES[2], CASES[5]])
def test_tangent_direction_in_initial_positions(label, name, over, dim, steps):
    # a free column seeded with a direction v in the initial positions is the
    # directional derivative of the trajectory: central differences of run()
    # from X_0 +- h v
    p, pos, sp, c = _case(name, over, dim)
    P = 2 + int(p["n_species"])
    v = np.random.default_rng(8).standard_normal(pos.shape)
    d0 = np.zeros(pos.shape + (P + 1,))
    d0[:, :, P] = v
    x0 = pos.astype(np.float64)
    _, _, cN, dx, dc = orc.run_tangent(p, x0, sp, c, nsteps=steps, dpos=d0, extra=1)
    h = 2.0 ** -24
    xp, _, cp, _ = orc.run(p, x0 + h * v, sp, c, nsteps=steps)
    xm, _, cm, _ = orc.run(p, x0 - h * v, sp, c, nsteps=steps)
    fd = (xp - xm) / (2 * h)
    assert np.abs(fd - dx[:, :, P]).max() <= 1e-5 * np.abs(fd).max(), label
    if cN is not None:
        fdc = (cp - cm) / (2 * h)
        assert np.abs(fdc - dc[..., P]).max() <= 1e-4 * np.abs(fdc).max(), label


def _golden(name):
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    return os.path.join(here, name)


def test_tangent_growth_golden_reproduces_and_matches_differences():
    # tests/golden/adjoint_tangent_growth.txt: the exact gradient of the
    # differentiable workload's loss along the oracle trajectory against the
    # horizon K. Its first steps recompute exactly; up to K = 5 the central
    # differences of adjoint_fd_horizon.txt (their two steps agreeing within
    # 1 %) equal it; and it grows by many orders (the dynamics is chaotic
    # under frozen noise). At K = 7 the two differences still agree with
    # each other but not with the tangent (dL/dD_1 6.945e-3 against
    # 7.268e-3): a pair lies within the step of its cutoff, where the
    # shifted force's derivative jumps, so both differences straddle the
    # kink and average its two slopes, while the tangent is the slope at
    # theta itself
    import importlib.util
    tan = {}
    for line in open(_golden("adjoint_tangent_growth.txt")):
        if line.startswith("#"):
            continue
        f = line.split()
        tan[int(f[0])] = np.array([float(v) for v in f[1:5]])
    fd = {}
    for line in open(_golden("adjoint_fd_horizon.txt")):
        if line.startswith("#"):
            continue
        f = line.split()
        fd[int(f[0])] = (np.array([float(v) for v in f[7:11]]), float(f[12]))
    spec = importlib.util.spec_from_file_location("tangent_growth", _golden("adjoint_tangent_growth.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    p, x, sp = wl.initial_state("adjoint_2d")
    x0 = x.astype(np.float64)
    pos, _, _, dpos, _ = orc.run_tangent(p, x0, sp, np.zeros(orc.grid_shape(p)), nsteps=3)
    g = np.einsum("ia,iak->k", mod.loss_and_grad(pos, x0)[1], dpos)
    np.testing.assert_allclose(g, tan[3], rtol=1e-6, atol=1e-12)
    resolved = [k for k, (_, agree) in fd.items() if agree < 0.01 and k <= 5]
    assert len(resolved) == 4
    for k in resolved:
        g_fd, _ = fd[k]
        assert np.all(np.abs(g_fd - tan[k]) <= 5e-3 * (np.abs(tan[k]) + np.abs(tan[k]).max())), k
    assert np.abs(tan[200]).max() > 1e18 * np.abs(tan[5]).max()
