"""Differentiable trajectories: a ``torch.autograd.Function`` around the
library's recorded run (``chemo_record``) and its adjoint (``chemo_gradient``),
and the observables of the differentiable workload.

``ChemoRun.apply(theta, pos0, sim, nsteps, every, species, c0)`` returns the final positions
(by particle id) after ``nsteps`` steps from ``pos0`` with the parameters
``theta = [chi, inter, D_0, ..., D_{S-1}]`` (the other model parameters are
those the simulation was created with); its backward pass returns dL/dtheta
and dL/dpos0 from the hand-written adjoint kernels, with the noise frozen.

Observables (the loss of the differentiable workload):

* ``mean_x_displacement(pos, pos0)``: mean over cells of x(T) - x(0);
* ``occupancy_loss(pos, nb, lo, hi)``: mean squared occupancy of a fixed
  nb^d analysis grid, with occupancy o_b = n_b B / N (mean 1) and n_b the
  cloud-in-cell (bilinear) count of cells around node b, a piecewise-smooth
  stand-in for the count per bin so that it can be differentiated.
"""
from __future__ import annotations

import numpy as np
import torch

from . import chemo

PARAM_NAMES = ("chi", "inter")  # followed by D_0 .. D_{S-1}


def theta_of(params: dict) -> list:
    ns = int(params["n_species"])
    return [float(params["chi"]), float(params["inter"])] + [float(v) for v in params["D"][:ns]]


def with_theta(params: dict, theta) -> dict:
    q = dict(params)
    t = [float(v) for v in theta]
    q["chi"], q["inter"] = t[0], t[1]
    ns = int(params["n_species"])
    D = list(params["D"])
    D[:ns] = t[2:2 + ns]
    q["D"] = D
    return q


class ChemoRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, pos0, sim, nsteps, every, species, c0=None, step0=0, store_bytes=0):
        params = with_theta(sim.params, theta.detach().cpu().tolist())
        chemo.chemo_set_params(sim, params)
        chemo.chemo_write_state(sim, pos0.detach().contiguous(), species)
        if c0 is not None:
            chemo.chemo_write_field(sim, c0)
        chemo.chemo_set_step_index(sim, step0)
        chemo.chemo_record(sim, int(nsteps), int(every), store_bytes=int(store_bytes))
        out = torch.empty_like(pos0)
        chemo.chemo_read_state(sim, out, None, None)
        ctx.sim = sim
        ctx.ntheta = theta.numel()
        ctx.theta_dtype = theta.dtype
        ctx.theta_device = theta.device
        return out

    @staticmethod
    def backward(ctx, g):
        sim = ctx.sim
        dtheta = torch.zeros(ctx.ntheta, dtype=torch.float32, device=g.device)
        dpos0 = torch.zeros_like(g)
        chemo.chemo_gradient(sim, g.detach().contiguous().float(), dtheta, None, dpos0)
        return dtheta.to(device=ctx.theta_device, dtype=ctx.theta_dtype), dpos0, None, None, None, None, None, None, None


def mean_x_displacement(pos: torch.Tensor, pos0: torch.Tensor) -> torch.Tensor:
    return (pos[:, 0] - pos0[:, 0]).mean()


def occupancy_loss(pos: torch.Tensor, nb: int, lo, hi) -> torch.Tensor:
    """(1/B) sum_b o_b^2 with o_b = n_b B / N, n_b the cloud-in-cell count on
    the nb^d nodes of a regular grid spanning the box (node-centred)."""
    n, dim = pos.shape
    lo_t = torch.as_tensor(lo[:dim], dtype=pos.dtype, device=pos.device)
    hi_t = torch.as_tensor(hi[:dim], dtype=pos.dtype, device=pos.device)
    t = (pos - lo_t) / (hi_t - lo_t) * (nb - 1)
    k0 = torch.clamp(torch.floor(t.detach()), 0, nb - 2)
    f = t - k0
    k0 = k0.long()
    B = nb ** dim
    counts = torch.zeros(B, dtype=pos.dtype, device=pos.device)
    for m in range(1 << dim):
        w = torch.ones(n, dtype=pos.dtype, device=pos.device)
        idx = torch.zeros(n, dtype=torch.long, device=pos.device)
        stride = 1
        for a in range(dim):
            bit = (m >> a) & 1
            w = w * (f[:, a] if bit else 1.0 - f[:, a])
            idx = idx + (k0[:, a] + bit) * stride
            stride *= nb
        counts = counts.index_add(0, idx, w)
    occ = counts * (B / n)
    return (occ ** 2).mean()


def loss_numpy(pos: np.ndarray, pos0: np.ndarray, nb: int, lo, hi) -> float:
    """The same loss in FP64 numpy (for finite differences of the oracle)."""
    pos = np.asarray(pos, np.float64)
    pos0 = np.asarray(pos0, np.float64)
    n, dim = pos.shape
    lx = (pos[:, 0] - pos0[:, 0]).mean()
    lo_a = np.asarray(lo[:dim], np.float64)
    hi_a = np.asarray(hi[:dim], np.float64)
    t = (pos - lo_a) / (hi_a - lo_a) * (nb - 1)
    k0 = np.clip(np.floor(t), 0, nb - 2)
    f = t - k0
    k0 = k0.astype(np.int64)
    B = nb ** dim
    counts = np.zeros(B)
    for m in range(1 << dim):
        w = np.ones(n)
        idx = np.zeros(n, dtype=np.int64)
        stride = 1
        for a in range(dim):
            bit = (m >> a) & 1
            w = w * (f[:, a] if bit else 1.0 - f[:, a])
            idx = idx + (k0[:, a] + bit) * stride
            stride *= nb
        np.add.at(counts, idx, w)
    occ = counts * (B / n)
    return float(lx + (occ ** 2).mean())
