"""Long-run statistics of the aggregation set-up of Sect. 3, shared by the
oracle-only calibration test and the GPU test.

Set-up: 2,000 cells in the unit square (cube) with reflecting walls, 1,000
alpha cells (species 0) drawn normal around the centre with sigma = 0.1 and
1,000 beta cells (species 1) uniform; alpha cells secrete the chemical, beta
cells climb its gradient (chi = 1); soft repulsion with diameters 0.02 and
0.04 (so alpha cells at the centre push each other apart and beta cells pack
around them); chemical with D_c = 1 and gamma = 0.1 on a 33^2 (17^3) grid
with Neumann walls, starting from c = 0; dt = 5e-5, 400 steps. The
diameters are 4x the paper's so that dt can be 5x its value with the step
still shorter than the interaction range (the paper's rule of Sect. 3).

Observables of one run (a vector of 2 x 7 + 2 x 4 + 1 = 23 numbers): for
each species the fraction of its cells in the radial shells |x - centre| in
[0, 0.1), [0.1, 0.15), [0.15, 0.2), [0.2, 0.3), [0.3, 0.4), [0.4, 0.5),
[0.5, inf) at the end; the mean squared displacement curve of each species
(after 100, 200, 300 and 400 steps); c at the centre node at the end.

Comparison of two sets of independent runs (different noise streams, the
same initial state): for each observable z = (mean_B - mean_A) /
(s_A sqrt(1/R_A + 1/R_B)), s_A the standard deviation over the R_A runs of
set A (floored at one cell's share for the shell fractions). Two samples of
the same law keep every |z| below Z_MAX = 6 (23 observables: a false alarm
has a probability of about 5e-8 when the means are normal). A family-wise
level of 0.01 (Bonferroni over the 23) would put the band at 3.5; every GPU
run is a new sample (the float atomics of the deposit round in a different
order each time), so the band is set where a run of the same law practically
never leaves it, and the planted mistakes of the calibration land at
|z| >= 2 Z_MAX.
"""
from __future__ import annotations

import numpy as np

from oracle import chemo_oracle as orc
from paper_1805_11007_gb300 import workloads as wl

N_CELLS = 2000
N_ALPHA = 1000
STEPS = 400
CHUNKS = 4  # points of the MSD curves, STEPS // CHUNKS steps apart
EDGES = np.array([0.0, 0.1, 0.15, 0.2, 0.3, 0.4, 0.5, np.inf])
Z_MAX = 6.0


def params(dim: int, **overrides) -> dict:
    """Model parameters of the set-up (keys of chemo_params)."""
    grid = [33, 33, 1] if dim == 2 else [17, 17, 17]
    secrete = 0.05 if dim == 2 else 0.1  # 3D spreads the chemical over one more axis
    p = wl.params("walls_grid_2d", dim=dim, diameter=[0.02, 0.04], grid=grid, dt=5e-5,
                  secrete=[secrete, 0.0])
    p.update(overrides)
    return p


def observables(pos0, traj, species, c) -> np.ndarray:
    """Observable vector of one run from the initial positions, the positions
    after each chunk of steps (the last is the end state), the species and
    the final field: shell fractions per species at the end, the MSD curve
    per species, c at the centre node."""
    pos0 = np.asarray(pos0, np.float64)
    species = np.asarray(species)
    end = np.asarray(traj[-1], np.float64)
    r = np.linalg.norm(end - 0.5, axis=1)
    out = []
    for s in (0, 1):
        h, _ = np.histogram(r[species == s], EDGES)
        out += list(h / max(1, int((species == s).sum())))
    for s in (0, 1):
        for x in traj:
            d = np.asarray(x, np.float64)[species == s] - pos0[species == s]
            out.append(float((d * d).sum(axis=1).mean()))
    c = np.asarray(c, np.float64)
    out.append(float(c[tuple(k // 2 for k in c.shape)]))
    return np.array(out)


def floors(n_species_cells) -> np.ndarray:
    """Least standard deviation of each observable: one cell's share for the
    shell fractions, none for the rest."""
    f = []
    for m in n_species_cells:
        f += [1.0 / max(1, int(m))] * (len(EDGES) - 1)
    return np.array(f + [0.0] * (2 * CHUNKS + 1))


def oracle_runs(p: dict, pos0, species, seeds, steps: int = STEPS) -> np.ndarray:
    """Observable vectors of FP64 oracle runs, one per noise seed."""
    shape = orc.grid_shape(p)
    per = steps // CHUNKS
    rows = []
    for s in seeds:
        q = dict(p, seed=int(s))
        pos, sp, c = pos0, species, np.zeros(shape)
        traj = []
        for k in range(CHUNKS):
            pos, sp, c, _ = orc.run(q, pos, sp, c=c, step0=k * per, nsteps=per)
            traj.append(pos)
        rows.append(observables(pos0, traj, sp, c))
    return np.array(rows)


def zscores(A: np.ndarray, B: np.ndarray, floor: np.ndarray) -> np.ndarray:
    """z of each observable's mean of B against the mean of A, the spread
    taken from A."""
    s = np.maximum(A.std(axis=0, ddof=1), floor)
    se = s * np.sqrt(1.0 / A.shape[0] + 1.0 / B.shape[0])
    d = B.mean(axis=0) - A.mean(axis=0)
    return np.where(se > 0, d / np.where(se > 0, se, 1.0), np.where(d == 0, 0.0, np.inf))
