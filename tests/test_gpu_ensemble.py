"""Batched ensembles (chemo_create_batch): replicates of uneven size stacked
in one simulation, against the FP64 oracle run replicate by replicate (seed +
r) and against single GPU simulations of each replicate."""
import numpy as np
import pytest

from oracle import chemo_oracle as orc
from paper_1805_11007_gb300 import chemo
from paper_1805_11007_gb300 import ensemble as en
from paper_1805_11007_gb300 import workloads as wl
from parity_util import assert_step_matches, dev

pytestmark = pytest.mark.gpu

SIZES = [37, 0, 1, 600, 2500, 257]  # ragged, an empty and a one-cell replicate
DENSE = dict(diameter=[0.03, 0.05])  # more pairs per cell in small boxes of cells
PERIODIC = dict(boundary=1, pde_bc=2, diameter=[0.03, 0.05])


def _ens(sizes, grid=128, **over):
    p, s, pos, sp = wl.ensemble_state(sizes=sizes, grid=[grid, grid, 1], **over)
    c0 = np.stack([wl.random_field(wl.replicate_params(p, r), seed=50 + r, scale=0.3) for r in range(len(s))])
    return p, s, pos, sp, c0.astype(np.float32)


def _batch(p, s, pos, sp, c0):
    sim = chemo.chemo_create_batch(p, s, dev(pos), dev(sp))
    if c0 is not None:
        chemo.chemo_write_field(sim, dev(c0))
    return sim


@pytest.mark.parametrize("over", [dict(), DENSE, PERIODIC])
def test_batch_step_matches_oracle_per_replicate(over):
    p, s, pos, sp, c0 = _ens(SIZES, **over)
    with _batch(p, s, pos, sp, c0) as sim:
        info = chemo.chemo_get_info(sim)
        assert info["layers"] == len(SIZES)
        assert info["grid_nodes"] == len(SIZES) * 128 * 128
        chemo.chemo_step(sim)
        pg, spg, _ = chemo.read_state_host(sim)
        cg = chemo.read_field_host(sim)
    off = en.offsets(s)
    for r in range(len(s)):
        a, b = off[r], off[r + 1]
        assert_step_matches(wl.replicate_params(p, r), pos[a:b], sp[a:b], c0[r], pg[a:b], spg[a:b], cg[r])


@pytest.mark.parametrize("over", [dict(), PERIODIC])
def test_batch_equals_single_simulations(over):
    """Replicate r of the batch is the simulation of its own cells with seed
    + r: bitwise for the particles after one step (forces are exact sums),
    within the single-step tolerance after several (float atomics of the
    deposit round differently)."""
    p, s, pos, sp, c0 = _ens(SIZES, **over)
    off = en.offsets(s)
    with _batch(p, s, pos, sp, c0) as sim:
        chemo.chemo_step(sim)
        pg1, _, _ = chemo.read_state_host(sim)
        chemo.chemo_step_n(sim, 5)
        pg6, _, _ = chemo.read_state_host(sim)
    for r in range(len(s)):
        a, b = off[r], off[r + 1]
        q = wl.replicate_params(p, r)
        with chemo.chemo_create(q, dev(pos[a:b]), dev(sp[a:b])) as one:
            chemo.chemo_write_field(one, dev(c0[r]))
            chemo.chemo_step(one)
            p1, _, _ = chemo.read_state_host(one)
            chemo.chemo_step_n(one, 5)
            p6, _, _ = chemo.read_state_host(one)
        np.testing.assert_array_equal(pg1[a:b], p1)
        assert (np.abs(pg6[a:b] - p6).max() if b > a else 0.0) <= 6e-5


def test_batch_bins_exact_and_sort_layer_major():
    p, s, pos, sp, c0 = _ens(SIZES, bin_side=1.0 / 16, **DENSE)
    off = en.offsets(s)
    with _batch(p, s, pos, sp, c0) as sim:
        info = chemo.chemo_get_info(sim)
        assert info["nbins"] == [16, 16, len(SIZES)]
        n = sim.n
        cells = np.zeros((n, 2), np.int32)
        chemo.chemo_stage_bins(sim, cells)
        ids = np.zeros(n, np.uint32)
        chemo.chemo_stage_sort(sim, ids)
    for r in range(len(s)):
        a, b = off[r], off[r + 1]
        if b > a:
            ref, nb = orc.bins_f32(p, p["bin_side"], pos[a:b])
            assert nb[:2] == (16, 16)
            np.testing.assert_array_equal(cells[a:b], ref[:, :2])
    # sorted order: a permutation, layer-major, then by bin key inside a layer
    assert sorted(ids.tolist()) == list(range(n))
    layer = np.searchsorted(off, ids, side="right") - 1
    key = cells[ids, 0] + info["bin_pitch"] * (cells[ids, 1] + info["nbins"][1] * layer)
    assert np.all(np.diff(layer) >= 0)
    assert np.all(np.diff(key.astype(np.int64)) >= 0)


def test_batch_multi_step_matches_oracle():
    p, s, pos, sp, c0 = _ens([1500, 40, 3000], cutoff_mode=1, **DENSE)
    k = 19  # 16-step graph, 2-step graph, one direct step
    off = en.offsets(s)
    with _batch(p, s, pos, sp, c0) as sim:
        chemo.chemo_step_n(sim, k)
        pg, _, _ = chemo.read_state_host(sim)
        cg = chemo.read_field_host(sim)
    for r in range(len(s)):
        a, b = off[r], off[r + 1]
        pr, _, cr, _ = orc.run(wl.replicate_params(p, r), pos[a:b], sp[a:b], c0[r].astype(np.float64), nsteps=k)
        assert np.abs(pg[a:b] - pr).max() <= k * 1e-5
        assert np.abs(cg[r] - cr).max() <= k * 1e-5 * np.abs(cr).max()


def test_full_size_ensemble_sampled_replicates():
    """The 256-replicate ensemble (log-uniform sizes 1e3..6.4e4, 128^2 grid
    each) in the launch configuration of the bench: one step, the smallest,
    median and largest replicates against the oracle."""
    p, s, pos, sp = wl.ensemble_state()
    off = en.offsets(s)
    with chemo.chemo_create_batch(p, s, dev(pos), dev(sp)) as sim:
        chemo.chemo_step(sim)
        pg, spg, _ = chemo.read_state_host(sim)
        cg = chemo.read_field_host(sim)
        chemo.chemo_step_n(sim, 4)
        chemo.chemo_check(sim)
    order = np.argsort(s)
    for r in (int(order[0]), int(order[len(s) // 2]), int(order[-1])):
        a, b = off[r], off[r + 1]
        assert_step_matches(wl.replicate_params(p, r), pos[a:b], sp[a:b], np.zeros((128, 128), np.float32),
                            pg[a:b], spg[a:b], cg[r])


def test_all_empty_and_host_round_trip():
    p, s, pos, sp, c0 = _ens([0, 0, 0])
    with chemo.chemo_create_batch(p, s, pos, sp) as sim:
        chemo.chemo_step_n(sim, 3)
        chemo.chemo_check(sim)
        assert chemo.chemo_step_index(sim) == 3
    p, s, pos, sp, c0 = _ens([5, 0, 9])
    with chemo.chemo_create_batch(p, s, pos, sp) as sim:  # host buffers
        pg, spg, _ = chemo.read_state_host(sim)
        np.testing.assert_array_equal(pg, pos)
        np.testing.assert_array_equal(spg, sp)
        chemo.chemo_write_field(sim, c0)
        np.testing.assert_array_equal(chemo.read_field_host(sim), c0)


def _record_and_gradient(sim, nsteps, every, wpos, wc, npar):
    """dL/d(chi, inter, D_s) and dL/dX(0) of L = sum wpos . X(T) + sum wc c(T)."""
    chemo.chemo_record(sim, nsteps, every)
    dpar = np.zeros(npar, np.float32)
    dx0 = np.zeros_like(wpos)
    chemo.chemo_gradient(sim, np.ascontiguousarray(wpos), dpar, dL_dc_final=np.ascontiguousarray(wc), dL_dpos0=dx0)
    chemo.chemo_check(sim)
    return dpar.astype(np.float64), dx0.astype(np.float64)


def test_batch_gradient_is_the_sum_of_replicate_gradients():
    """The adjoint of a batch. With a loss that sums per-replicate terms, the
    gradient with respect to the shared parameters is the sum of each
    replicate's gradient as its own simulation (seed + r: the same noise),
    and the gradient with respect to initial positions is each replicate's,
    block by block. Differences come only from the order of float atomics
    (deposit, the adjoint's field scatter, the pair term's partners)."""
    sizes = [300, 0, 700, 450]
    p, s, pos, sp, c0 = _ens(sizes, grid=33, cutoff_mode=1, **DENSE)
    off = en.offsets(s)
    n = int(sum(s))
    npar = 2 + int(p["n_species"])
    rng = np.random.default_rng(5)
    wpos = rng.standard_normal((n, 2)).astype(np.float32)
    wc = rng.standard_normal(c0.shape).astype(np.float32)
    nsteps, every = 8, 3
    with _batch(p, s, pos, sp, c0) as sim:
        dpar_b, dx0_b = _record_and_gradient(sim, nsteps, every, wpos, wc, npar)
    dpar_sum = np.zeros(npar)
    for r in range(len(s)):
        a, b = off[r], off[r + 1]
        if b == a:  # no cells: the field does not depend on the parameters
            continue
        q = wl.replicate_params(p, r)
        with chemo.chemo_create(q, dev(pos[a:b]), dev(sp[a:b])) as one:
            chemo.chemo_write_field(one, dev(c0[r]))
            dpar_r, dx0_r = _record_and_gradient(one, nsteps, every, wpos[a:b], wc[r], npar)
        dpar_sum += dpar_r
        np.testing.assert_allclose(dx0_b[a:b], dx0_r, rtol=1e-4, atol=1e-4 * np.abs(dx0_r).max())
    assert np.all(np.isfinite(dpar_b)) and np.abs(dpar_b).max() > 0
    np.testing.assert_allclose(dpar_b, dpar_sum, rtol=1e-4, atol=1e-5 * np.abs(dpar_sum).max())


def test_autotune_choice_leaves_particles_unchanged():
    """The tuned layout changes only the speed: particles after one step are
    bitwise those of the default layout."""
    p, s, pos, sp, c0 = _ens([3000, 5000, 800], **DENSE)
    best, ms = chemo.chemo_autotune(p, s, pos, sp, trial_steps=3)
    assert ms > 0.0
    assert best["search_mode"] in (1, 2, 3, 4)
    assert best["block_threads"] in (0, 128, 512)  # 0: the default 256 was fastest
    out = []
    for q in (p, best):
        with _batch(q, s, pos, sp, c0) as sim:
            chemo.chemo_step(sim)
            out.append(chemo.read_state_host(sim)[0])
    np.testing.assert_array_equal(out[0], out[1])
