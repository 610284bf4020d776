"""The seeded input generators hold the recipe of the synthetic workloads
(no arithmetic of the method): uniform cells strictly inside the box in
float32, the 3D clumps (2^d Gaussian clumps of std 0.05 at the corners of
{0.25, 0.75}^d, cell i in clump i mod 2^d), log-uniform ensemble sizes in
[1000, 64000] (about 3.9 M cells over 256 replicates), the species split
(alpha = the first half of the ids), and determinism in the seed."""
import numpy as np
import pytest

from paper_1805_11007_gb300 import workloads as wl


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_positions_inside_and_seeded(dim):
    lo, hi = [-1.0, 0.0, 2.0], [1.0, 0.5, 3.0]
    x = wl.uniform_positions(20000, dim, lo, hi, seed=4)
    assert x.dtype == np.float32 and x.shape == (20000, dim)
    assert np.all(x >= np.float32(lo[:dim])) and np.all(x < np.float32(hi[:dim]))
    u = (x.astype(np.float64) - lo[:dim]) / (np.array(hi[:dim]) - lo[:dim])
    assert np.abs(u.mean(0) - 0.5).max() < 0.01 and np.abs(u.var(0) - 1 / 12).max() < 0.003
    np.testing.assert_array_equal(x, wl.uniform_positions(20000, dim, lo, hi, seed=4))
    assert not np.array_equal(x, wl.uniform_positions(20000, dim, lo, hi, seed=5))


def test_clumps_of_the_3d_workload():
    n = 80000
    x = wl.clump_positions(n, 3, [0.0] * 3, [1.0] * 3, seed=1).astype(np.float64)
    assert np.all(x >= 0.0) and np.all(x < 1.0)
    for c in range(8):
        centre = np.array([0.25 if not (c >> a) & 1 else 0.75 for a in range(3)])
        xc = x[c::8]
        assert np.abs(xc.mean(0) - centre).max() < 0.002
        assert np.abs(xc.std(0) - 0.05).max() < 0.002


def test_ensemble_sizes_are_log_uniform():
    s = wl.ensemble_sizes(256, 1000, 64000, seed=1)
    assert s.min() >= 1000 and s.max() < 64000
    # E[N] = (b - a) / ln(b / a) = 15.1k per replicate, 3.9 M over 256
    expect = (64000 - 1000) / np.log(64.0)
    assert abs(s.mean() - expect) < 0.15 * expect
    p, sizes, pos, sp = wl.ensemble_state()
    assert len(sizes) == 256 and pos.shape == (int(sizes.sum()), 2) and sp.shape == (int(sizes.sum()),)
    assert 3.0e6 < sizes.sum() < 4.8e6


def test_initial_state_species_and_shapes():
    p, pos, sp = wl.initial_state("walls_grid_2d", n=1001)
    assert pos.shape == (1001, 2) and sp.dtype == np.uint8
    assert np.all(sp[:500] == 0) and np.all(sp[500:] == 1)
    p1, pos1, sp1 = wl.initial_state("periodic_fixed_gradient_2d", n=10)
    assert np.all(sp1 == 0) and p1["boundary"] == 1 and p1["chem_mode"] == 1
    p3, pos3, _ = wl.initial_state("clumps_grid_3d", n=4000)
    assert pos3.shape == (4000, 3) and p3["grid"] == [256, 256, 256]
