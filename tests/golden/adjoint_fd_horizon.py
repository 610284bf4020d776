"""How far finite differences of the FP64 oracle resolve the gradient of the
differentiable workload (50,000 cells of the 2D walls physics, 512^2 grid,
12 PDE substeps, force shifted to zero at the cutoff), as a function of the
horizon K (steps from the seeded initial state, c = 0).

For every K, each parameter theta = (chi, inter, D_0, D_1) gets central
differences at h = 1e-4 and h/2; the loss is the workload's: the mean x
displacement plus the mean squared cloud-in-cell occupancy of a 64^2
analysis grid (o_b = n_b B / N). Writes adjoint_fd_horizon.txt beside this
file: per K, dL/dtheta at h and at h/2 and how well the two agree. The noise is the same Philox stream in every run (frozen), so the
differences measure the map's sensitivity, not sampling noise.

    python tests/golden/adjoint_fd_horizon.py [K ...]

Calls only the oracle, numpy and the seeded input generators; run on a multi-core host (about a minute
per 10 steps of horizon on 8 threads).
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


def loss(xN, x0):
    """Mean x displacement + (1/B) sum_b o_b^2, cloud-in-cell counts n_b on a
    node-centred NB x NB grid spanning the box, o_b = n_b B / N."""
    n = xN.shape[0]
    t = xN * (NB - 1)
    k0 = np.clip(np.floor(t), 0, NB - 2)
    f = t - k0
    k0 = k0.astype(np.int64)
    counts = np.zeros(NB * NB)
    for bx in (0, 1):
        for by in (0, 1):
            w = (f[:, 0] if bx else 1.0 - f[:, 0]) * (f[:, 1] if by else 1.0 - f[:, 1])
            np.add.at(counts, (k0[:, 0] + bx) + NB * (k0[:, 1] + by), w)
    occ = counts * (NB * NB / n)
    return float((xN[:, 0] - x0[:, 0]).mean() + (occ ** 2).mean())


def with_theta(theta):
    q = dict(wl.params("adjoint_2d"))
    q["chi"], q["inter"] = float(theta[0]), float(theta[1])
    q["D"] = [float(theta[2]), float(theta[3])]
    return q


def fd(theta, k, h, x0, sp):
    c0 = np.zeros(orc.grid_shape(wl.params("adjoint_2d")))
    out = np.zeros(4)
    for a in range(4):
        tp = np.array(theta, np.float64)
        tm = tp.copy()
        tp[a] += h
        tm[a] -= h
        lp = loss(orc.run(with_theta(tp), x0, sp, c0, nsteps=k)[0], x0)
        lm = loss(orc.run(with_theta(tm), x0, sp, c0, nsteps=k)[0], x0)
        out[a] = (lp - lm) / (2.0 * h)
    return out


def main(ks):
    orc.build()
    orc.set_threads(len(os.sched_getaffinity(0)))
    p, x, sp = wl.initial_state("adjoint_2d")
    x0 = x.astype(np.float64)
    theta = [p["chi"], p["inter"]] + list(p["D"][:2])
    lines = ["# K, then dL/d(chi, inter, D0, D1) by central differences at h = 1e-4 and at h/2, and",
             "# agree = max over the parameters of |g_h - g_h/2| / (|g_h| + max_b |g_h,b|)",
             "# (below 0.01: the finite difference resolves the derivative)"]
    for k in ks:
        g1 = fd(theta, k, 1e-4, x0, sp)
        g2 = fd(theta, k, 5e-5, x0, sp)
        agree = float(np.max(np.abs(g1 - g2) / (np.abs(g1) + np.abs(g1).max())))
        lines.append("%4d  h: %+.6e %+.6e %+.6e %+.6e  h/2: %+.6e %+.6e %+.6e %+.6e  agree %.3e"
                     % ((k,) + tuple(g1) + tuple(g2) + (agree,)))
        print(lines[-1], flush=True)
    with open(os.path.join(HERE, "adjoint_fd_horizon.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [1, 2, 3, 5, 7, 10, 15, 20, 30, 40, 60])
