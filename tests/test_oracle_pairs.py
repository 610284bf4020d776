"""Pins of the oracle's cell list and pair force (Sect. 3.2 interaction loop,
Eq. (1a)/(1b) pair term).

* neighbour sets of the cell list equal an all-pairs numpy search (periodic
  minimum image and walls);
* the force of a pair is minus the derivative of the pair potential
  u(r) = inter * exp(-r/eps) (Sect. 3), checked by finite differences of the
  total potential energy, not by the force formula;
* Newton's third law (sum of forces 0), translation invariance under
  periodicity, and heterogeneous contact distance eps_ij = (s_i + s_j)/2.
"""
import numpy as np
import pytest

from oracle import chemo_oracle as orc
from paper_1805_11007_gb300 import workloads as wl


def _numpy_neighbours(p, pos):
    """All pairs within the cutoff by brute force (numpy), as per-particle
    (count, index sum, index xor)."""
    pos = np.asarray(pos, dtype=np.float64)
    n, dim = pos.shape
    L = np.array(p["hi"][:dim]) - np.array(p["lo"][:dim])
    d = pos[:, None, :] - pos[None, :, :]
    if p["boundary"] == 1:
        d -= L * np.round(d / L)
    r = np.sqrt((d ** 2).sum(-1))
    sp = np.asarray(p["_sp"])
    diam = np.asarray(p["diameter"], dtype=np.float32).astype(np.float64)
    eps = 0.5 * (diam[sp][:, None] + diam[sp][None, :])
    rc = float(np.float32(p.get("cutoff_factor", 1.0))) * eps
    m = (r > 0) & (r < rc)
    np.fill_diagonal(m, False)
    idx = np.arange(n, dtype=np.uint64)
    cnt = m.sum(1)
    s = (m * idx[None, :]).sum(1).astype(np.uint64)
    x = np.zeros(n, dtype=np.uint64)
    for i in range(n):
        js = idx[m[i]]
        if js.size:
            x[i] = np.bitwise_xor.reduce(js)
    border = np.abs(r ** 2 - rc ** 2) <= 1e-6 * rc ** 2
    np.fill_diagonal(border, False)
    return cnt, s, x, border.any(1)


@pytest.mark.parametrize("dim,boundary", [(2, 0), (2, 1), (3, 0), (3, 1)])
def test_cell_list_neighbours_equal_brute_force(dim, boundary):
    diam = [0.03, 0.06] if dim == 2 else [0.08, 0.12]
    p = wl.params("walls_grid_2d", dim=dim, boundary=boundary, diameter=diam, grid=[5, 5, 5])
    n = 1500 if dim == 2 else 2500
    pos = wl.uniform_positions(n, dim, p["lo"], p["hi"], seed=11 + dim + boundary)
    # put some particles exactly on the walls / periodic seam
    pos[:20, 0] = 0.0
    if boundary == 0:
        pos[20:40, 1] = 1.0
    sp = wl.half_species(n, 2)
    p["_sp"] = sp
    F1, e1 = orc.pair_forces(p, pos, sp, method=1, extras=True)
    F0, e0 = orc.pair_forces(p, pos, sp, method=0, extras=True)
    cnt, s, x, border = _numpy_neighbours(p, pos)
    ok = ~border
    assert cnt.sum() > 5 * n  # the test exercises real neighbourhoods
    for e in (e0, e1):
        np.testing.assert_array_equal(e["count"][ok], cnt[ok])
        np.testing.assert_array_equal(e["idsum"][ok], s[ok])
        np.testing.assert_array_equal(e["idxor"][ok], x[ok])
    np.testing.assert_allclose(F1, F0, rtol=1e-12, atol=1e-9)


def _energy(p, pos, sp):
    """Total potential energy sum_{i<j, r<rc} inter * exp(-r/eps_ij)."""
    pos = np.asarray(pos, dtype=np.float64)
    n, dim = pos.shape
    L = np.array(p["hi"][:dim]) - np.array(p["lo"][:dim])
    diam = np.asarray(p["diameter"], dtype=np.float32).astype(np.float64)
    inter = float(np.float32(p["inter"]))
    E = 0.0
    for i in range(n):
        for j in range(i + 1, n):
            d = pos[i] - pos[j]
            if p["boundary"] == 1:
                d -= L * np.round(d / L)
            r = np.sqrt((d ** 2).sum())
            eps = 0.5 * (diam[sp[i]] + diam[sp[j]])
            if 0 < r < eps * float(np.float32(p["cutoff_factor"])):
                E += inter * np.exp(-r / eps)
    return E


@pytest.mark.parametrize("dim,boundary", [(2, 0), (2, 1), (3, 1)])
def test_force_is_minus_gradient_of_potential(dim, boundary):
    p = wl.params("walls_grid_2d", dim=dim, boundary=boundary, diameter=[0.2, 0.3],
                  inter=2.5, cutoff_factor=1.7, grid=[5, 5, 5])
    rng = np.random.default_rng(3 + dim)
    n = 12
    pos = rng.random((n, dim)) * 0.3 + 0.05  # near the seam when periodic
    if boundary == 1:
        pos[::3, 0] = 0.97
    sp = np.arange(n) % 2
    F = orc.pair_forces(p, pos, sp, method=1)
    h = 1e-6
    for i in range(n):
        for a in range(dim):
            pp = pos.copy(); pp[i, a] += h
            pm = pos.copy(); pm[i, a] -= h
            g = (_energy(p, pp, sp) - _energy(p, pm, sp)) / (2 * h)
            assert abs(F[i, a] + g) <= 1e-6 * (1 + abs(g)), (i, a, F[i, a], -g)


def test_two_body_closed_form_and_contact_distance():
    # Sect. 3: u(r) = exp(-r/eps) with eps = 0.01; two cells of species (0,1)
    # with diameters 0.01 and 0.03 interact with eps_01 = 0.02.
    p = wl.params("walls_grid_2d", diameter=[0.01, 0.03], inter=1.0, grid=[5, 5, 1])
    pos = np.array([[0.5, 0.5], [0.5 + 0.012, 0.5]])
    F = orc.pair_forces(p, pos, [0, 1])
    mag = (1.0 / np.float32(0.02)) * np.exp(-0.012 / np.float64(np.float32(0.02)))
    # the value printed by hand: (1/0.02) * exp(-0.6) = 27.440581804701324
    assert abs(mag - 27.440581804701324) < 1e-4
    np.testing.assert_allclose(F[0], [-mag, 0.0], rtol=1e-6)
    np.testing.assert_allclose(F[1], [mag, 0.0], rtol=1e-6)
    # same species 0: eps = 0.01 < 0.012, out of range
    F = orc.pair_forces(p, pos, [0, 0])
    np.testing.assert_array_equal(F, 0.0)


def test_coincident_particles_and_self_get_no_force():
    p = wl.params("walls_grid_2d", grid=[5, 5, 1])
    pos = np.array([[0.3, 0.3], [0.3, 0.3], [0.9, 0.9]])
    F = orc.pair_forces(p, pos, [0, 1, 0])
    np.testing.assert_array_equal(F, 0.0)


@pytest.mark.parametrize("dim", [2, 3])
def test_newton_third_law_and_periodic_translation(dim):
    p = wl.params("walls_grid_2d", dim=dim, boundary=1, diameter=[0.04, 0.07], grid=[5, 5, 5])
    n = 3000
    pos = wl.uniform_positions(n, dim, p["lo"], p["hi"], seed=5).astype(np.float64)
    sp = wl.half_species(n, 2)
    F, e = orc.pair_forces(p, pos, sp, extras=True)
    assert np.abs(F.sum(0)).max() <= 1e-10 * e["fabs"].sum()
    shift = np.array([0.37, 0.81, 0.13][:dim])
    pos2 = (pos + shift) % 1.0
    F2 = orc.pair_forces(p, pos2, sp)
    np.testing.assert_allclose(F2, F, rtol=1e-9, atol=1e-9 * e["fabs"].max())


def test_force_shifted_mode_vanishes_at_cutoff():
    p = wl.params("walls_grid_2d", diameter=[0.02, 0.02], cutoff_mode=1, cutoff_factor=1.5,
                  grid=[5, 5, 1])
    eps = float(np.float32(0.02))
    rc = float(np.float32(1.5)) * eps
    for r, expect in [(rc * (1 - 1e-9), 0.0), (0.5 * eps, (1 / eps) * (np.exp(-0.5) - np.exp(-1.5)))]:
        pos = np.array([[0.5, 0.5], [0.5 + r, 0.5]])
        F = orc.pair_forces(p, pos, [0, 0])
        assert abs(-F[0, 0] - expect) <= 1e-6 * (1 + expect)


def test_bins_f32_rule():
    p = wl.params("clumps_grid_3d")
    rng = np.random.default_rng(0)
    pos = rng.random((10000, 3)).astype(np.float32)
    pos[0] = [0.0, 0.5, 1.0]
    pos[1] = [np.float32(0.25), np.float32(0.75), np.nextafter(np.float32(0.25), np.float32(0))]
    cells, nb = orc.bins_f32(p, 1.0 / 128, pos)
    assert nb == (128, 128, 128)
    # nb/L = 128 is a power of two: the FP32 product is exact and the bin is
    # floor(128 x), clamped to the last bin at x = 1
    ref = np.minimum(np.floor(pos.astype(np.float64) * 128), 127).astype(np.int32)
    np.testing.assert_array_equal(cells, ref)
    assert tuple(cells[1]) == (32, 96, 31)
    # non power of two: bins agree with IEEE single-precision numpy arithmetic
    cells, nb = orc.bins_f32(p, 0.004, pos)
    inv = np.float32(nb[0] / 1.0)
    ref = np.clip(np.floor((pos - np.float32(0.0)) * inv), 0, nb[0] - 1).astype(np.int32)
    np.testing.assert_array_equal(cells, ref)
