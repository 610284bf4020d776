"""Pins of the oracle's grid pieces: gradient interpolation (Sect. 2.3/3.6),
cloud-in-cell density estimate (Sect. 2.3), and the explicit PDE step of
Eq. (1d) (Sect. 3.5).

* multilinear fields: the interpolated central-difference gradient equals
  the analytic gradient (away from wall nodes) and the interpolated value
  equals the field;
* deposit: trapezoid-weighted mass and first moment of the particles are
  reproduced exactly; a particle on a node loads only that node;
* PDE: discrete mass balance with Neumann walls, eigen-decay of cosine and
  Fourier modes, uniform decay, and exact discrete steady states with
  Dirichlet ends (linear profile; A r1^k + B r2^k with decay).
"""
import os

import numpy as np
import pytest

from oracle import chemo_oracle as orc
from paper_1805_11007_gb300 import workloads as wl


def _nodes(p):
    dim = p["dim"]
    axes = [p["lo"][a] + orc.grid_h(p, a) * np.arange(p["grid"][a]) for a in range(dim)]
    mesh = np.meshgrid(*axes[::-1], indexing="ij")  # C-order: (z, y, x)
    return mesh[::-1]  # x, y, (z)


def _tau(p):
    dim = p["dim"]
    shape = orc.grid_shape(p)
    t = np.ones(shape)
    if p["pde_bc"] == 2:
        return t
    for a in range(dim):
        ax = dim - 1 - a
        sl = [slice(None)] * dim
        sl[ax] = 0
        t[tuple(sl)] *= 0.5
        sl[ax] = -1
        t[tuple(sl)] *= 0.5
    return t


@pytest.mark.parametrize("dim", [2, 3])
def test_multilinear_field_gradient_and_value_exact(dim):
    grid = [13, 9, 7][:dim] + [1] * (3 - dim)
    p = wl.params("walls_grid_2d", dim=dim, grid=grid, chi=1.7, chemotactic=[0.0, 2.0],
                  lo=[-0.5, 0.25, 0.0], hi=[0.5, 1.25, 2.0])
    rng = np.random.default_rng(1)
    coef = rng.standard_normal(8)
    X = _nodes(p)

    def field(*x):
        x = list(x) + [0 * x[0]] * (3 - len(x))
        out = 0 * x[0]
        for m in range(8):
            t = coef[m] * np.ones_like(x[0])
            for a in range(3):
                if (m >> a) & 1:
                    t = t * x[a]
            out = out + t
        return out

    def grad(x):
        x = list(x) + [0.0] * (3 - len(x))
        g = np.zeros(3)
        for m in range(8):
            for a in range(3):
                if (m >> a) & 1:
                    t = coef[m]
                    for b in range(3):
                        if b != a and (m >> b) & 1:
                            t *= x[b]
                    g[a] += t
        return g[:dim]

    c = field(*X)
    n = 400
    lo = np.array(p["lo"][:dim])
    hi = np.array(p["hi"][:dim])
    h = np.array([orc.grid_h(p, a) for a in range(dim)])
    # interior cells only: every corner node at least one node from the walls
    pos = lo + h + (hi - lo - 2 * h) * rng.random((n, dim))
    pos = np.clip(pos, lo + h * 1.0001, hi - h * 1.0001)
    sp = np.ones(n, dtype=np.uint8)
    sp[:50] = 0
    d = orc.drift(p, pos, sp, c)
    chi = float(np.float32(1.7)) * 2.0
    for i in range(n):
        expect = chi * grad(pos[i]) if sp[i] == 1 else np.zeros(dim)
        np.testing.assert_allclose(d[i], expect, rtol=1e-9, atol=1e-9)
    v = orc.conc(p, pos, c)
    np.testing.assert_allclose(v, field(*[pos[:, a] for a in range(dim)]), rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("dim", [2, 3])
def test_periodic_grid_gradient_wraps(dim):
    """Periodic grid (nodes k h, h = L/N): the central difference of a
    Fourier mode at every node, the wrapped ones included, is the derivative
    of the mode times sin(k h)/(k h) (for sin(k x): cos(k x_j) sin(k h)/h),
    and a cell in the last interval [L - h, L) interpolates between node N-1
    and node 0. Checked at random positions and in the last interval of
    every axis."""
    grid = [16, 12, 8][:dim] + [1] * (3 - dim)
    p = wl.params("walls_grid_2d", dim=dim, grid=grid, boundary=1, pde_bc=2, chi=1.3, chemotactic=[0.0, 1.0])
    X = _nodes(p)
    m = [1, 2, 1][:dim]
    kappa = [2 * np.pi * m[a] for a in range(dim)]
    # c = sin(k0 x) + cos(k1 y) (+ sin(k2 z))
    c = np.sin(kappa[0] * X[0]) + np.cos(kappa[1] * X[1]) + (np.sin(kappa[2] * X[2]) if dim == 3 else 0.0)
    h = [orc.grid_h(p, a) for a in range(dim)]

    def node_grad(a, j):  # central difference at node j of axis a, in closed form
        x = j * h[a]
        s = np.sin(kappa[a] * h[a]) / h[a]
        return -np.sin(kappa[a] * x) * s if a == 1 else np.cos(kappa[a] * x) * s

    rng = np.random.default_rng(3)
    pos = rng.random((300, dim))
    for a in range(dim):  # cells in the last interval of axis a
        pos[a * 20:(a + 1) * 20, a] = 1.0 - h[a] * rng.random(20)
    pos = pos.astype(np.float32).astype(np.float64)
    d = orc.drift(p, pos, np.ones(len(pos), np.uint8), c)
    chi = float(np.float32(1.3))
    for i in range(len(pos)):
        for a in range(dim):
            u = pos[i, a] / h[a]
            k = int(np.floor(u))
            f = u - k
            expect = (1 - f) * node_grad(a, k % grid[a]) + f * node_grad(a, (k + 1) % grid[a])
            assert abs(d[i, a] - chi * expect) <= 1e-9 * max(1.0, abs(chi * expect)), (i, a, d[i, a], chi * expect)


def test_wall_node_gradient_is_zero_normal_component():
    p = wl.params("walls_grid_2d", grid=[11, 11, 1])
    X = _nodes(p)
    c = X[0] ** 2 + 3 * X[1]
    pos = np.array([[0.0, 0.55], [1.0, 0.55]])
    d = orc.drift(p, pos, [1, 1], c)
    assert d[0, 0] == 0.0 and d[1, 0] == 0.0
    np.testing.assert_allclose(d[:, 1], 3.0 * float(np.float32(1.0)), rtol=1e-12)


def test_fixed_gradient_mode():
    p = wl.params("periodic_fixed_gradient_2d", chi=0.75, fixed_grad=[1.0, -2.0, 0.0])
    pos = np.random.default_rng(0).random((10, 2))
    d = orc.drift(p, pos, np.zeros(10, dtype=np.uint8))
    np.testing.assert_allclose(d, np.tile([0.75, -1.5], (10, 1)))


@pytest.mark.parametrize("dim,bc", [(2, 0), (3, 0), (2, 2), (3, 2)])
def test_deposit_mass_and_first_moment(dim, bc):
    grid = [17, 12, 9][:dim] + [1] * (3 - dim)
    p = wl.params("walls_grid_2d", dim=dim, grid=grid, pde_bc=bc, boundary=1 if bc == 2 else 0,
                  secrete=[0.3, 0.05], consume=[0.0, 0.2], dt=1e-3)
    n = 5000
    pos = wl.uniform_positions(n, dim, p["lo"], p["hi"], seed=2).astype(np.float64)
    pos[:10, 0] = 0.0
    if bc == 0:
        pos[10:20, 0] = 1.0
    sp = wl.half_species(n, 2)
    S, R = orc.deposit(p, pos, sp)
    hd = np.prod([orc.grid_h(p, a) for a in range(dim)])
    vol = _tau(p) * hd
    k = np.array([np.float32(0.3), np.float32(0.05)], dtype=np.float64)
    kap = np.array([0.0, np.float32(0.2)], dtype=np.float64)
    assert abs((S * vol).sum() - p["dt"] * k[sp].sum()) <= 1e-10 * n
    assert abs((R * vol).sum() - kap[sp].sum()) <= 1e-10 * n
    if bc == 0:  # first moment (linear weights reproduce x; no wrap)
        X = _nodes(p)
        for a in range(dim):
            m = (S * vol * X[a]).sum()
            assert abs(m - p["dt"] * (k[sp] * pos[:, a]).sum()) <= 1e-10 * n


def test_particle_on_node_loads_one_node():
    p = wl.params("walls_grid_2d", grid=[11, 11, 1], secrete=[2.0, 0.0], dt=0.5)
    h = orc.grid_h(p, 0)
    pos = np.array([[3 * h, 7 * h], [0.0, 5 * h], [1.0, 1.0]])
    S, _ = orc.deposit(p, pos, [0, 0, 0])
    # (x/h may round just below the node: allow weights at rounding level)
    assert np.count_nonzero(np.abs(S) > 1e-9 * np.abs(S).max()) == 3
    assert abs(S[7, 3] - 0.5 * 2.0 / h ** 2) < 1e-9 / h ** 2
    assert abs(S[5, 0] - 0.5 * 2.0 / (0.5 * h ** 2)) < 1e-9 / h ** 2
    assert abs(S[10, 10] - 0.5 * 2.0 / (0.25 * h ** 2)) < 1e-9 / h ** 2


@pytest.mark.parametrize("dim", [2, 3])
def test_pde_mass_balance_neumann(dim):
    grid = [33, 21, 17][:dim] + [1] * (3 - dim)
    p = wl.params("walls_grid_2d", dim=dim, grid=grid, Dc=0.7, gamma=0.3, dt=2e-5)
    rng = np.random.default_rng(4)
    c = rng.random(orc.grid_shape(p))
    S = rng.random(orc.grid_shape(p)) * 1e-3
    hd = np.prod([orc.grid_h(p, a) for a in range(dim)])
    vol = _tau(p) * hd
    s = 3
    out = orc.pde_substep(p, c, S, None, s)
    gam = float(np.float32(0.3))
    expect = (c * vol).sum() * (1 - gam * p["dt"] / s) + (S * vol).sum() / s
    assert abs((out * vol).sum() - expect) <= 1e-12 * (c * vol).sum()


@pytest.mark.parametrize("m", [1, 2, 5])
def test_pde_neumann_cosine_mode_decay(m):
    N = 41
    p = wl.params("walls_grid_2d", grid=[N, 9, 1], Dc=1.3, gamma=0.2, dt=1e-5)
    X = _nodes(p)
    L = 1.0
    c = np.cos(np.pi * m * X[0] / L)
    h = orc.grid_h(p, 0)
    s = 2
    dts = p["dt"] / s
    D = float(np.float32(1.3))
    g = float(np.float32(0.2))
    fac = 1 - dts * (g + 4 * D / h ** 2 * np.sin(np.pi * m * h / (2 * L)) ** 2)
    out = orc.pde_substep(p, c, None, None, s)
    np.testing.assert_allclose(out, fac * c, rtol=0, atol=1e-12)


def test_pde_periodic_fourier_mode_decay():
    N = 32
    p = wl.params("walls_grid_2d", dim=3, grid=[N, 8, 4], pde_bc=2, boundary=1, Dc=0.9, gamma=0.0,
                  dt=1e-5)
    X = _nodes(p)
    m = 3
    c = np.sin(2 * np.pi * m * X[0]) + 2.0
    h = orc.grid_h(p, 0)
    D = float(np.float32(0.9))
    fac = 1 - p["dt"] * 4 * D / h ** 2 * np.sin(np.pi * m / N) ** 2
    out = orc.pde_substep(p, c, None, None, 1)
    np.testing.assert_allclose(out - 2.0, fac * (c - 2.0), atol=1e-12)


@pytest.mark.parametrize("dim,bc", [(2, 0), (3, 0), (2, 2), (3, 2)])
def test_pde_separable_mode_on_every_axis(dim, bc):
    """A product of one eigenmode per axis on a grid whose spacing differs by
    axis decays by 1 - dt_s (gamma + sum_a 4 D_c / h_a^2 sin^2(theta_a / 2)),
    theta_a = pi m_a h_a / L_a (Neumann cosine) or 2 pi m_a / N_a (periodic):
    every axis's stencil and spacing enter, so a wrong h, a dropped axis or a
    transposed index shows."""
    grid = [13, 9, 7][:dim] + [1] * (3 - dim)
    over = dict(dim=dim, grid=grid, Dc=0.7, gamma=0.15, dt=2e-5)
    if bc == 2:
        over.update(pde_bc=2, boundary=1)
    p = wl.params("walls_grid_2d", **over)
    X = _nodes(p)
    m = [2, 1, 3][:dim]
    c = np.ones(orc.grid_shape(p))
    lam = 0.0
    for a in range(dim):
        h = orc.grid_h(p, a)
        L = p["hi"][a] - p["lo"][a]
        if bc == 2:
            c = c * np.cos(2 * np.pi * m[a] * (X[a] - p["lo"][a]) / L)
            theta = 2 * np.pi * m[a] / grid[a]
        else:
            c = c * np.cos(np.pi * m[a] * (X[a] - p["lo"][a]) / L)
            theta = np.pi * m[a] * h / L
        lam += 4 * float(np.float32(0.7)) / h ** 2 * np.sin(theta / 2) ** 2
    s = 3
    fac = 1 - p["dt"] / s * (float(np.float32(0.15)) + lam)
    out = orc.pde_substep(p, c, None, None, s)
    np.testing.assert_allclose(out, fac * c, rtol=0, atol=1e-12)


@pytest.mark.parametrize("s", [1, 4])
def test_pde_reaction_terms_per_node(s):
    """With no diffusion a substep acts node by node: c' = c (1 - dt_s
    (gamma + R)) + S / s, R the consumption density (kappa rho) and S the
    step's source split over the s substeps (Eq. (1d), Sect. 3.5)."""
    p = wl.params("walls_grid_2d", grid=[9, 7, 1], Dc=0.0, gamma=0.3, dt=1e-2)
    rng = np.random.default_rng(8)
    shape = orc.grid_shape(p)
    c = rng.random(shape) + 0.5
    R = 2.0 * rng.random(shape)
    S = 0.01 * rng.random(shape)
    dts = p["dt"] / s
    g = float(np.float32(0.3))
    out = orc.pde_substep(p, c, S, R, s)
    np.testing.assert_allclose(out, c * (1 - dts * (g + R)) + S / s, rtol=0, atol=1e-14)


def test_pde_uniform_decay():
    p = wl.params("clumps_grid_3d", grid=[9, 9, 9], gamma=0.1)
    c = np.full(orc.grid_shape(p), 3.0)
    out = orc.pde_substep(p, c, None, None, 1)
    np.testing.assert_allclose(out, 3.0 * (1 - float(np.float32(0.1)) * p["dt"]), rtol=1e-14)


def test_pde_dirichlet_linear_steady_state():
    p = wl.params("walls_grid_2d", grid=[21, 11, 1], pde_bc=1, gamma=0.0, Dc=1.0, dt=1e-5)
    X = _nodes(p)
    c = X[0].copy()
    out = orc.pde_substep(p, c, None, None, 1)
    np.testing.assert_allclose(out, c, atol=1e-13)


def test_pde_dirichlet_decay_steady_state():
    # c_{k+1} - 2 c_k + c_{k-1} = (gamma h^2 / D) c_k has the solution
    # A r1^k + B r2^k, r1 r2 = 1; with c_0 = 0 and c_{N-1} = 1 it is a fixed
    # point of the explicit step (constant along y with Neumann... held ends).
    N = 25
    p = wl.params("walls_grid_2d", grid=[N, 6, 1], pde_bc=1, gamma=4.0, Dc=0.5, dt=1e-6)
    h = orc.grid_h(p, 0)
    g = float(np.float32(4.0))
    D = float(np.float32(0.5))
    b = 2 + g * h * h / D
    r1 = (b + np.sqrt(b * b - 4)) / 2
    r2 = 1 / r1
    k = np.arange(N)
    # A + B = 0, A r1^(N-1) + B r2^(N-1) = 1
    A = 1 / (r1 ** (N - 1) - r2 ** (N - 1))
    prof = A * (r1 ** k - r2 ** k)
    c = np.tile(prof, (6, 1))
    # the y walls are Dirichlet too: hold them at the same profile
    out = orc.pde_substep(p, c, None, None, 1)
    np.testing.assert_allclose(out, c, atol=1e-12)


def test_substeps_match_stability_rule():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "substeps.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for name, dim, N, Dc, dt, _lam, s in rows:
        p = wl.params(name)
        assert p["dim"] == int(dim) and p["grid"][0] == int(N)
        assert float(p["Dc"]) == float(Dc) and float(p["dt"]) == float(dt)
        assert orc.substeps(p) == int(s), name
