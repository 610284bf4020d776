"""Helpers of the GPU parity tests: run the CUDA library through its C ABI
and the FP64 oracle on the same seeded inputs, and compare element by element.

Tolerances (single step, FP32 GPU against FP64 oracle):
  * pair force, per particle: |F_gpu - F_ref| <= 1e-5 * sum_j |f_ij| plus the
    magnitude of the pairs within 1e-6 r_c^2 of the cutoff (either
    classification is correct there), plus one fixed-point quantum of the
    GPU's exact force sum per neighbour (2^-25 of the largest pair force
    inter/eps, about half an FP32 ulp at that scale);
  * positions, per component: 1e-5 of the step's increment plus 2 single-
    precision ulps of the position (before a periodic wrap), plus dt times
    the borderline force magnitude. The increment is measured by the magnitudes of its terms,
    |dt F| + |dt chi_s grad c| + sqrt(2 D_s dt) |xi| from the oracle (FP32
    rounds each term relative to its own size, so cancelling terms do not
    make the bound smaller than the rounding); at dt = 1e-6 this resolves
    the chemotactic drift (~1e-6 per step) and a 0.1 % error in the noise
    amplitude, which an absolute 1e-5 L does not;
  * chemical field and deposit: 1e-5 * max |value| elementwise;
  * drift: 1e-5 * max |drift| elementwise.
"""
from __future__ import annotations

import numpy as np
import torch

from oracle import chemo_oracle as orc
from paper_1805_11007_gb300 import chemo


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def make_sim(p, pos, sp, c0=None):
    sim = chemo.chemo_create(p, dev(pos), dev(sp))
    if c0 is not None:
        chemo.chemo_write_field(sim, dev(c0))
    return sim


def gpu_forces(sim):
    n, d = sim.n, sim.dim
    F = torch.zeros((n, d), dtype=torch.float32, device="cuda")
    cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
    ids = torch.zeros(n, dtype=torch.int64, device="cuda")
    chemo.chemo_stage_forces(sim, F, cnt, ids)
    torch.cuda.synchronize()
    chemo.chemo_check(sim)
    return F.cpu().numpy().astype(np.float64), cnt.cpu().numpy(), ids.cpu().numpy().view(np.uint64)


def force_quantum(p):
    """Quantum of the GPU's fixed-point force sum: 2^-25 of max inter/eps."""
    ns = int(p["n_species"])
    diam = np.asarray(p["diameter"][:ns], dtype=np.float32).astype(np.float64)
    eps_min = diam.min() if ns else 1.0
    inter = abs(float(np.float32(p.get("inter", 1.0))))
    return inter / max(eps_min, 1e-30) * 2.0 ** -25


def min_image(d, p):
    d = np.array(d, dtype=np.float64)
    if p.get("boundary", 0) == 1:
        L = np.array(p["hi"][: d.shape[1]]) - np.array(p["lo"][: d.shape[1]])
        d -= L * np.round(d / L)
    return d


def assert_forces_match(p, F_gpu, cnt_gpu, ids_gpu, pos, sp):
    F, ex = orc.pair_forces(p, pos.astype(np.float64), sp, method=1, extras=True)
    border = ex["border"] > 0
    ok = ~border
    np.testing.assert_array_equal(cnt_gpu[ok], ex["count"][ok])
    np.testing.assert_array_equal(ids_gpu[ok], ex["idsum"][ok])
    err = np.linalg.norm(F_gpu - F, axis=1)
    tol = 1e-5 * ex["fabs"] + ex["border"] + force_quantum(p) * (ex["count"] + 1) * np.sqrt(3.0)
    bad = np.where(err > tol)[0]
    assert bad.size == 0, "force mismatch at %s: err %s tol %s" % (bad[:5], err[bad[:5]], tol[bad[:5]])
    return ex


def ulp32(x):
    """Spacing of single-precision numbers at |x| (elementwise)."""
    return np.spacing(np.abs(np.asarray(x, dtype=np.float64)).astype(np.float32)).astype(np.float64)


def increment_terms(p, pos0, sp0, c0=None, step_index=0, ids=None):
    """Per component, |dt F| + |dt chi_s grad c| + sqrt(2 D_s dt) |xi|: the
    sizes of the terms of the Euler-Maruyama increment (Eq. (2)) at the
    oracle's pair force, drift and normals."""
    pos = pos0.astype(np.float64)
    n, d = pos.shape
    F = orc.pair_forces(p, pos, sp0, method=1)
    dr = orc.drift(p, pos, sp0, None if c0 is None else np.asarray(c0, np.float64))
    ids = np.arange(n, dtype=np.uint32) if ids is None else ids
    xi = orc.normals(p["seed"], ids, step_index)[:, :d]
    D = np.array([np.float32(v) for v in p["D"]], dtype=np.float64)[np.asarray(sp0, np.int64)]
    amp = np.sqrt(2.0 * D * p["dt"])
    return p["dt"] * (np.abs(F) + np.abs(dr)) + amp[:, None] * np.abs(xi)


def position_tolerance(p, pos0, sp0, c0, pos_r, border, step_index=0):
    """Per-component bound of |x_gpu - x_ref| after one step (module doc).
    The ulps are those of the larger of the end point and the moved point
    before a periodic wrap (x0 + the minimum-image displacement): a cell
    that crosses the upper face is rounded near hi, then shifted by L."""
    inc = increment_terms(p, pos0, sp0, c0, step_index)
    x0 = pos0.astype(np.float64)
    moved = x0 + min_image(pos_r - x0, p)
    return 1e-5 * inc + 2.0 * np.maximum(ulp32(pos_r), ulp32(moved)) + p["dt"] * border[:, None]


def assert_step_matches(p, pos0, sp0, c0, pos_g, sp_g, c_g, disp_g=None, step_index=0):
    pos_r, sp_r, c_r, disp_r = orc.step(p, pos0.astype(np.float64), sp0,
                                        None if c0 is None else c0.astype(np.float64), step_index=step_index,
                                        disp=None if disp_g is None else np.zeros(pos0.shape))
    _, ex = orc.pair_forces(p, pos0.astype(np.float64), sp0, method=1, extras=True)
    d = np.abs(min_image(pos_g.astype(np.float64) - pos_r, p))
    tol = position_tolerance(p, pos0, sp0, c0, pos_r, ex["border"], step_index)
    bad = np.argwhere(d > tol)
    assert bad.size == 0, "position mismatch at %s: %s (tolerance %s)" % (bad[:5], d[tuple(bad[:5].T)],
                                                                          tol[tuple(bad[:5].T)])
    if p.get("reactions", 0):
        np.testing.assert_array_equal(sp_g, sp_r)
    else:
        np.testing.assert_array_equal(sp_g, sp0)
    if c_g is not None:
        scale = max(np.abs(c_r).max(), 1e-30)
        dc = np.abs(c_g.astype(np.float64) - c_r) / scale
        assert dc.max() <= 1e-5, "field mismatch: max rel %g at %s" % (dc.max(), np.unravel_index(dc.argmax(), dc.shape))
    if disp_g is not None:
        dd = np.abs(disp_g.astype(np.float64) - disp_r)
        assert (dd <= tol + 2.0 * ulp32(disp_r)).all()
    return pos_r, sp_r, c_r
