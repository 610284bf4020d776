"""The exact gradient of the differentiable workload's loss along the FP64
oracle's trajectory, as a function of the horizon K: the oracle's tangent
(the step differentiated operation by operation, the noise frozen) carried
for 200 steps from the seeded initial state (50,000 cells of the 2D walls
physics, 512^2 grid, 12 PDE substeps, force shifted to zero at the cutoff,
c = 0), contracted at each listed K with dL/dX_K. The loss is the
workload's: the mean x displacement plus the mean squared cloud-in-cell
occupancy of a 64^2 analysis grid (o_b = n_b B / N); its derivative is
written out below (the weights' derivatives). Writes
adjoint_tangent_growth.txt beside this file: per K, dL/d(chi, inter, D_0,
D_1) and the largest magnitude.

    python tests/golden/adjoint_tangent_growth.py [K ...]

Calls only the oracle, numpy and the seeded input generators (a few minutes
for 200 steps on 8 threads).
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import chemo_oracle as orc  # noqa: E402

from paper_1805_11007_gb300 import workloads as wl  # noqa: E402  (seeded inputs only)

NB = 64


def loss_and_grad(xN, x0):
    """L = mean x displacement + (1/B) sum_b o_b^2 on the unit box, and
    dL/dX_N (n x 2): (1/n) on x plus (2/N) sum_b o_b dw_b/dX."""
    n = xN.shape[0]
    B = NB * NB
    t = xN * (NB - 1)
    k0 = np.clip(np.floor(t), 0, NB - 2)
    f = t - k0
    k0 = k0.astype(np.int64)
    counts = np.zeros(B)
    idx, w, dw = [], [], []
    for bx in (0, 1):
        for by in (0, 1):
            wx = f[:, 0] if bx else 1.0 - f[:, 0]
            wy = f[:, 1] if by else 1.0 - f[:, 1]
            b = (k0[:, 0] + bx) + NB * (k0[:, 1] + by)
            np.add.at(counts, b, wx * wy)
            idx.append(b)
            dw.append(np.stack([(1.0 if bx else -1.0) * (NB - 1) * wy, (1.0 if by else -1.0) * (NB - 1) * wx], 1))
    occ = counts * (B / n)
    L = float((xN[:, 0] - x0[:, 0]).mean() + (occ ** 2).mean())
    g = np.zeros_like(xN)
    g[:, 0] += 1.0 / n
    for b, d in zip(idx, dw):
        g += (2.0 / n) * occ[b][:, None] * d
    return L, g


def main(ks):
    orc.build()
    orc.set_threads(len(os.sched_getaffinity(0)))
    p, x, sp = wl.initial_state("adjoint_2d")
    x0 = x.astype(np.float64)
    c = np.zeros(orc.grid_shape(p))
    lines = ["# K, then dL/d(chi, inter, D0, D1) along the FP64 oracle trajectory from its tangent,",
             "# and max |dL/dtheta| (the loss's own derivative contracted with dX_K/dtheta)"]
    pos, dpos, dc, done = x0, None, None, 0
    for k in sorted(ks):
        pos, _, c, dpos, dc = orc.run_tangent(p, pos, sp, c, step0=done, nsteps=k - done, dpos=dpos, dc=dc)
        done = k
        _, gx = loss_and_grad(pos, x0)
        g = np.einsum("ia,iak->k", gx, dpos)
        lines.append("%4d  %+.6e %+.6e %+.6e %+.6e  max %.3e" % ((k,) + tuple(g) + (float(np.abs(g).max()),)))
        print(lines[-1], flush=True)
    with open(os.path.join(HERE, "adjoint_tangent_growth.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [1, 2, 3, 5, 7, 10, 15, 20, 30, 40, 60, 80, 100, 120, 140, 160, 180, 200])
