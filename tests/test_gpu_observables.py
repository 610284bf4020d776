"""Observables reduced on the device (chemo_observables, chemo_histogram)
against numpy on the state read back by id: cells per species, mean and
mean-square unwrapped displacement per species, the chemical mass by the
trapezoid rule, and occupancy histograms, per replicate of an ensemble."""
import numpy as np
import pytest

from paper_1805_11007_gb300 import chemo
from paper_1805_11007_gb300 import ensemble as en
from paper_1805_11007_gb300 import workloads as wl
from parity_util import dev, make_sim

pytestmark = pytest.mark.gpu


def _mass(p, c):
    """h^d sum tau_k c_k with tau = 1/2 per wall axis at boundary nodes."""
    w = np.ones_like(c, dtype=np.float64)
    dim = p["dim"]
    h = 1.0
    for a in range(dim):
        n = p["grid"][a]
        L = p["hi"][a] - p["lo"][a]
        periodic = p["pde_bc"] == 2
        h *= L / n if periodic else L / (n - 1)
        if not periodic:
            ax = dim - 1 - a  # C-order: x is the last axis
            idx = [slice(None)] * dim
            idx[ax] = 0
            w[tuple(idx)] *= 0.5
            idx[ax] = n - 1
            w[tuple(idx)] *= 0.5
    return h * float((w * c).sum())


def _expect(p, x, sp, d):
    ns = p["n_species"]
    cnt = np.array([(sp == s).sum() for s in range(ns)], np.float64)
    md = np.zeros((ns, 3))
    msd = np.zeros(ns)
    for s in range(ns):
        m = sp == s
        if m.any() and d is not None:
            dd = d[m].astype(np.float64)
            md[s, :dd.shape[1]] = dd.mean(axis=0)
            msd[s] = (dd ** 2).sum(axis=1).mean()
    return cnt, md, msd


@pytest.mark.parametrize("name,over", [
    ("walls_grid_2d", dict(grid=[64, 64, 1], track_displacement=1)),
    ("walls_grid_2d", dict(grid=[64, 48, 1], boundary=1, pde_bc=2, track_displacement=1)),
    ("clumps_grid_3d", dict(grid=[24, 24, 24], diameter=[0.01, 0.02], track_displacement=1)),
])
def test_observables_match_numpy(name, over):
    p, pos, sp = wl.initial_state(name, n=30011, **over)
    c0 = wl.random_field(p, seed=8, scale=0.3)
    with make_sim(p, pos, sp, c0) as sim:
        chemo.chemo_step_n(sim, 7)
        obs = chemo.chemo_observables(sim)
        x, s, d = chemo.read_state_host(sim)
        c = chemo.read_field_host(sim)
        shape = [7, 5, 3][:p["dim"]]
        hist = chemo.chemo_histogram(sim, shape)
    assert len(obs) == 1
    cnt, md, msd = _expect(p, x, s, d)
    np.testing.assert_array_equal(obs[0]["count"], cnt)
    np.testing.assert_allclose(obs[0]["mean_disp"], md, rtol=1e-4, atol=1e-7 * np.abs(d).max())
    np.testing.assert_allclose(obs[0]["msd"], msd, rtol=1e-4)
    assert obs[0]["c_mass"] == pytest.approx(_mass(p, c.astype(np.float64)), rel=1e-5)
    # the histogram: cells per part of the box, species-resolved, C-order
    for sp_ in range(p["n_species"]):
        xs = x[s == sp_]
        # the kernel's single-precision rule: floor(((x - lo) / (hi - lo)) * shape)
        lo = np.float32(p["lo"]) if np.ndim(p["lo"]) == 0 else np.asarray(p["lo"], np.float32)
        hi = np.asarray(p["hi"], np.float32)
        k = [np.clip(np.floor(((xs[:, a] - lo[a]) / (hi[a] - lo[a])) * np.float32(shape[a])), 0, shape[a] - 1)
             .astype(int) for a in range(p["dim"])]
        ref = np.zeros(list(reversed(shape)))
        np.add.at(ref, tuple(reversed(k)), 1.0)
        np.testing.assert_array_equal(hist[0, sp_], ref)
    assert hist.sum() == x.shape[0]


def test_observables_per_replicate():
    sizes = [37, 0, 1, 600, 2500, 257]
    p, s, pos, sp = wl.ensemble_state(sizes=sizes, grid=[32, 32, 1], track_displacement=1)
    off = en.offsets(s)
    with chemo.chemo_create_batch(p, s, dev(pos), dev(sp)) as sim:
        chemo.chemo_step_n(sim, 5)
        obs = chemo.chemo_observables(sim)
        x, spg, d = chemo.read_state_host(sim)
        c = chemo.read_field_host(sim)
        hist = chemo.chemo_histogram(sim, [4, 6])
    assert len(obs) == len(sizes)
    for r in range(len(sizes)):
        a, b = off[r], off[r + 1]
        q = wl.replicate_params(p, r)
        cnt, md, msd = _expect(q, x[a:b], spg[a:b], d[a:b])
        np.testing.assert_array_equal(obs[r]["count"], cnt)
        if b > a:
            np.testing.assert_allclose(obs[r]["msd"], msd, rtol=1e-4, atol=1e-12)
        assert obs[r]["c_mass"] == pytest.approx(_mass(q, c[r].astype(np.float64)), rel=1e-5, abs=1e-12)
        assert hist[r].sum() == b - a
