"""Long GPU runs against the FP64 oracle, compared statistically: after 400
steps of the aggregation set-up of Sect. 3 (alpha cells secreting at the
centre, beta cells climbing the gradient, soft repulsion, the chemical on a
grid with walls), the radial profiles of both species, their mean squared
displacement curves and c at the centre agree between 64 GPU runs and 8 oracle
runs with other noise seeds: every observable's oracle mean lies within
Z_MAX = 6 standard errors of the GPU mean, the standard error taken from the
spread of the GPU runs. The initial state is drawn on each side by its own
initialiser; the GPU runs are one ensemble in 2D and single simulations in
3D. The calibration of the band (same-law samples inside it, planted
mistakes far outside) is the oracle-only test of the same statistics."""
import numpy as np
import pytest

import stats_util as su
from oracle import chemo_oracle as orc
from paper_1805_11007_gb300 import chemo
from parity_util import dev

pytestmark = pytest.mark.gpu

R_GPU = 64
ORACLE_SEEDS = range(5000, 5008)  # disjoint from the GPU runs' keys 1000 .. 1063
INIT_SEED = 7


def _oracle(dim):
    p = su.params(dim)
    pos0, sp = orc.init_positions(dict(p, seed=INIT_SEED), su.N_CELLS, su.N_ALPHA)
    pos0 = pos0.astype(np.float32).astype(np.float64)
    return su.oracle_runs(p, pos0, sp, ORACLE_SEEDS)


def _compare(dim, A, sp):
    B = _oracle(dim)
    z = su.zscores(A, B, su.floors([(sp == 0).sum(), (sp == 1).sum()]))
    assert np.all(np.isfinite(z)), np.round(z, 2)
    print(f"dim {dim}: largest |z| {np.abs(z).max():.2f} over {z.size} observables")
    assert np.abs(z).max() < su.Z_MAX, (dim, np.round(z, 2), np.round(A.mean(0), 4), np.round(B.mean(0), 4))


def test_ensemble_2d_long_run_matches_oracle_statistics():
    p = su.params(2, seed=1000)  # replicate r runs with key 1000 + r
    pos0, sp = chemo.chemo_init_positions(dict(p, seed=INIT_SEED), su.N_CELLS, su.N_ALPHA)
    sizes = [su.N_CELLS] * R_GPU
    traj = []
    with chemo.chemo_create_batch(p, sizes, dev(np.tile(pos0, (R_GPU, 1))), dev(np.tile(sp, R_GPU))) as sim:
        for _ in range(su.CHUNKS):
            chemo.chemo_step_n(sim, su.STEPS // su.CHUNKS)
            x, s, _ = chemo.read_state_host(sim)
            assert np.all((x >= 0.0) & (x <= 1.0))
            traj.append(x.reshape(R_GPU, su.N_CELLS, 2))
        c = chemo.read_field_host(sim)
    s = s.reshape(R_GPU, su.N_CELLS)
    assert np.all(s == sp[None, :])
    A = np.array([su.observables(pos0, [x[r] for x in traj], s[r], c[r]) for r in range(R_GPU)])
    _compare(2, A, sp)


def test_single_runs_3d_long_run_match_oracle_statistics():
    p = su.params(3)
    pos0, sp = chemo.chemo_init_positions(dict(p, seed=INIT_SEED), su.N_CELLS, su.N_ALPHA)
    rows = []
    for r in range(R_GPU):
        traj = []
        with chemo.chemo_create(dict(p, seed=1000 + r), dev(pos0), dev(sp)) as sim:
            for _ in range(su.CHUNKS):
                chemo.chemo_step_n(sim, su.STEPS // su.CHUNKS)
                x, s, _ = chemo.read_state_host(sim)
                assert np.all((x >= 0.0) & (x <= 1.0))
                traj.append(x)
            c = chemo.read_field_host(sim)
        rows.append(su.observables(pos0, traj, s, c))
    _compare(3, np.array(rows), sp)
