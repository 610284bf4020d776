"""Calibration of the whole-step parity check (CPU, no GPU).

The check of `parity_util.assert_step_matches` must accept the oracle's own
step rounded to single precision and must reject the plausible mistakes of
a GPU step that an absolute tolerance of 1e-5 L would let through at the
time steps of the 3D workloads: a step without the chemotactic drift
(chi = 0, Eq. (1b)) and a noise amplitude off by 0.1 % (Eq. (2)).
"""
import numpy as np
import pytest

from oracle import chemo_oracle as orc
from paper_1805_11007_gb300 import workloads as wl
from parity_util import assert_step_matches


def _case(name, n, **over):
    p, pos, sp = wl.initial_state(name, n=n, **over)
    c0 = wl.random_field(p, seed=5, scale=0.3) if p["chem_mode"] == 0 else None
    return p, pos, sp, c0


CASES = [
    ("clumps_grid_3d", 60013, dict(grid=[48, 48, 48], diameter=[0.01, 0.02])),
    ("clumps_grid_3d", 60013, dict(grid=[48, 48, 48], diameter=[0.01, 0.02], dt=1e-6)),
    ("walls_grid_2d", 20011, dict(grid=[128, 128, 1])),
    ("walls_grid_2d", 12007, dict(grid=[96, 80, 1], boundary=1, pde_bc=2, diameter=[0.004, 0.008])),
    ("periodic_fixed_gradient_2d", 1000, dict()),
]


def _oracle_f32(p, pos, sp, c0):
    pos_r, sp_r, c_r, _ = orc.step(p, pos.astype(np.float64), sp, None if c0 is None else c0.astype(np.float64))
    return pos_r.astype(np.float32), sp_r, None if c0 is None else c_r.astype(np.float32)


@pytest.mark.parametrize("name,n,over", CASES)
def test_check_accepts_the_oracle_rounded_to_single(name, n, over):
    p, pos, sp, c0 = _case(name, n, **over)
    pos_g, sp_g, c_g = _oracle_f32(p, pos, sp, c0)
    assert_step_matches(p, pos, sp, c0, pos_g, sp_g, c_g)


@pytest.mark.parametrize("name,n,over", CASES)
def test_check_rejects_a_step_without_chemotactic_drift(name, n, over):
    p, pos, sp, c0 = _case(name, n, **over)
    q = dict(p, chi=0.0)
    pos_g, sp_g, c_g = _oracle_f32(q, pos, sp, c0)
    with pytest.raises(AssertionError, match="position mismatch"):
        assert_step_matches(p, pos, sp, c0, pos_g, sp_g, c_g)


@pytest.mark.parametrize("name,n,over", CASES)
def test_check_rejects_noise_amplitude_off_by_a_tenth_of_a_percent(name, n, over):
    p, pos, sp, c0 = _case(name, n, **over)
    q = dict(p, D=[float(np.float32(d)) * 1.001 ** 2 for d in p["D"]])
    pos_g, sp_g, c_g = _oracle_f32(q, pos, sp, c0)
    with pytest.raises(AssertionError, match="position mismatch"):
        assert_step_matches(p, pos, sp, c0, pos_g, sp_g, c_g)
