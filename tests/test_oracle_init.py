"""Pins of the oracle's initial state (the paper's Sect. 3 set-up: alpha
cells normal around the centre with sigma = 0.1 of the width, beta cells
uniform), without a GPU: the species split, the box, the alpha moments and
normality, beta uniformity, determinism in the seed, and the reflection and
wrap of draws that leave the box."""
import numpy as np
import pytest
from scipy import stats

from oracle import chemo_oracle as orc
from paper_1805_11007_gb300 import workloads as wl


def _p(dim, boundary=0, seed=11):
    return wl.params("walls_grid_2d" if dim == 2 else "clumps_grid_3d", boundary=boundary,
                     pde_bc=2 if boundary else 0, seed=seed)


@pytest.mark.parametrize("dim", [2, 3])
def test_alpha_normal_beta_uniform(dim):
    p = _p(dim)
    n, na = 40000, 15000
    pos, sp = orc.init_positions(p, n, na, 0.1)
    assert pos.shape == (n, dim)
    np.testing.assert_array_equal(sp, np.r_[np.zeros(na), np.ones(n - na)])
    lo, hi = np.asarray(p["lo"])[:dim], np.asarray(p["hi"])[:dim]
    assert (pos >= lo).all() and (pos <= hi).all()
    L = hi - lo
    a = (pos[:na] - 0.5 * (lo + hi)) / (0.1 * L)  # standardised alpha coordinates
    for k in range(dim):
        assert abs(a[:, k].mean()) < 4.0 / np.sqrt(na)
        assert a[:, k].std() == pytest.approx(1.0, rel=0.03)
        assert stats.kstest(a[:, k], "norm").pvalue > 1e-3
        b = (pos[na:, k] - lo[k]) / L[k]
        assert stats.kstest(b, "uniform").pvalue > 1e-3
    # alpha axes are independent draws
    assert abs(np.corrcoef(a[:, 0], a[:, 1])[0, 1]) < 4.0 / np.sqrt(na)


def test_seed_and_counter_determinism():
    p = _p(2)
    a1, s1 = orc.init_positions(p, 1000, 400)
    a2, _ = orc.init_positions(p, 1000, 400)
    np.testing.assert_array_equal(a1, a2)
    b, _ = orc.init_positions(dict(p, seed=12), 1000, 400)
    assert np.abs(a1 - b).min() > 0.0
    # cell i depends only on its own counter: a prefix of a larger draw
    c, _ = orc.init_positions(p, 600, 400)
    np.testing.assert_array_equal(c, a1[:600])


def test_wide_alpha_reflects_or_wraps():
    """A wide alpha cloud (sigma = 2 widths) leaves the box often: walls fold
    it back (a triangle wave keeps it inside), a periodic box wraps it (the
    wrapped standardised coordinate is uniform)."""
    n = 20000
    for boundary in (0, 1):
        p = _p(2, boundary=boundary)
        pos, _ = orc.init_positions(p, n, n, 2.0)
        lo, hi = np.asarray(p["lo"])[:2], np.asarray(p["hi"])[:2]
        assert (pos >= lo).all() and (pos <= hi).all()
        if boundary == 1:
            assert (pos < hi).all()
            assert stats.kstest((pos[:, 0] - lo[0]) / (hi[0] - lo[0]), "uniform").pvalue > 1e-3
