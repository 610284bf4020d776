"""Statistics of long GPU runs against closed forms (Sect. 4): with no
interaction in a periodic box and the fixed gradient c = x, each cell's
unwrapped displacement after t = n dt has mean chi g t and variance
2 D t per axis (the MSD curves of the paper's Fig. 3 set-up), also for the
batched ensemble; and the 2D walls workload conserves its chemical mass
balance over many steps."""
import numpy as np
import pytest

from paper_1805_11007_gb300 import chemo
from paper_1805_11007_gb300 import workloads as wl
from parity_util import dev, make_sim

pytestmark = pytest.mark.gpu


def _check_moments(disp, chi_g, D, t):
    n = disp.shape[0]
    for a in range(disp.shape[1]):
        mean, var = disp[:, a].mean(), disp[:, a].var()
        se_mean = np.sqrt(2 * D * t / n)
        se_var = 2 * D * t * np.sqrt(2.0 / (n - 1))
        assert abs(mean - chi_g[a] * t) <= 4 * se_mean, (a, mean, chi_g[a] * t)
        assert abs(var - 2 * D * t) <= 4 * se_var, (a, var, 2 * D * t)


@pytest.mark.parametrize("chi", [0.0, 3.0])
def test_msd_and_drift_over_many_steps(chi):
    n, steps = 200_000, 400
    p = wl.params("periodic_fixed_gradient_2d", inter=0.0, chi=chi, fixed_grad=[2.0, -1.0, 0.0], dt=2e-5, D=[0.5])
    pos = wl.uniform_positions(n, 2, p["lo"], p["hi"], seed=41)
    sp = np.zeros(n, np.uint8)
    with make_sim(p, pos, sp) as sim:
        chemo.chemo_step_n(sim, steps)
        _, _, disp = chemo.read_state_host(sim)
    t = steps * p["dt"]
    _check_moments(disp.astype(np.float64), [chi * 2.0, -chi * 1.0], 0.5, t)


def test_msd_in_an_ensemble_of_replicates():
    """Every replicate of a batch has its own noise stream: pooled moments
    follow the closed forms and replicates are uncorrelated."""
    sizes = [30_000] * 8
    p, s, pos, sp = wl.ensemble_state(sizes=sizes, grid=[3, 3, 1], boundary=1, pde_bc=2, chem_mode=1,
                                      fixed_grad=[1.5, 0.0, 0.0], chi=1.0, chemotactic=[1.0, 1.0], inter=0.0,
                                      secrete=[0.0, 0.0], D=[0.5, 0.5], track_displacement=1, dt=2e-5)
    steps = 300
    with chemo.chemo_create_batch(p, s, dev(pos), dev(sp)) as sim:
        chemo.chemo_step_n(sim, steps)
        _, _, disp = chemo.read_state_host(sim)
    t = steps * p["dt"]
    _check_moments(disp.astype(np.float64), [1.5, 0.0], 0.5, t)
    # replicates with the same initial positions would move identically if
    # they shared a noise stream: their displacements must differ
    d = disp.reshape(8, 30_000, 2)
    assert np.corrcoef(d[0, :, 1], d[1, :, 1])[0, 1] < 0.05


def test_chemical_mass_balance_over_many_steps():
    """No consumption, Neumann walls: the trapezoid-weighted mass M of c
    follows M(t + dt) = (1 - gamma dt)^s-ish decay plus the deposited dt k
    per secreting cell per step; checked against the discrete recursion."""
    p, pos, sp = wl.initial_state("walls_grid_2d", n=20_000, grid=[128, 128, 1])
    h = 1.0 / 127
    tau = np.ones((128, 128))
    tau[0, :] *= 0.5
    tau[-1, :] *= 0.5
    tau[:, 0] *= 0.5
    tau[:, -1] *= 0.5
    nsec = int((sp == 0).sum())
    with make_sim(p, pos, sp, np.zeros((128, 128), np.float32)) as sim:
        s = chemo.chemo_get_info(sim)["pde_substeps"]
        M = 0.0
        for k in range(5):
            chemo.chemo_step_n(sim, 20)
            for _ in range(20):
                # one step: s substeps of decay, the deposit (dt k per cell)
                # split evenly over them
                add = p["dt"] * p["secrete"][0] * nsec / s
                for _ in range(s):
                    M = M * (1 - p["gamma"] * p["dt"] / s) + add
            c = chemo.read_field_host(sim).astype(np.float64)
            Mg = (c * tau).sum() * h * h
            assert Mg == pytest.approx(M, rel=2e-4)
