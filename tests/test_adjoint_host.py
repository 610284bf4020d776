"""Host-side pieces of the differentiable workload (no GPU): the parameter
vector theta = [chi, inter, D_0 .. D_{S-1}] and its round trip through the
parameter dict, and the loss of the adjoint workload (mean x displacement
plus the mean squared cloud-in-cell occupancy of an analysis grid): its
closed-form values on lattice and collapsed configurations, the agreement
of the torch and FP64 numpy forms, and its torch gradient against finite
differences (the loss is smooth inside each analysis cell)."""
import numpy as np
import pytest
import torch

from paper_1805_11007_gb300 import adjoint as adj
from paper_1805_11007_gb300 import workloads as wl


def test_theta_round_trip():
    p = wl.params("adjoint_2d")
    th = adj.theta_of(p)
    assert th == [p["chi"], p["inter"], p["D"][0], p["D"][1]]
    q = adj.with_theta(p, [0.5, 2.0, 0.3, 0.7])
    assert (q["chi"], q["inter"]) == (0.5, 2.0)
    assert q["D"][:2] == [0.3, 0.7] and list(q["D"][2:]) == list(p["D"][2:])
    assert adj.theta_of(q) == [0.5, 2.0, 0.3, 0.7]
    assert p["chi"] == th[0]  # the input dict is not changed


@pytest.mark.parametrize("dim", [2, 3])
def test_occupancy_of_one_cell_per_node_is_one(dim):
    """A cell on every node of the analysis grid: o_b = 1 everywhere, the
    smallest value the mean square can take (Jensen, mean o_b = 1)."""
    nb = 5
    axes = [np.linspace(0.0, 1.0, nb)] * dim
    pos = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, dim)
    lo, hi = [0.0] * 3, [1.0] * 3
    val = adj.occupancy_loss(torch.from_numpy(pos), nb, lo, hi)
    assert abs(float(val) - 1.0) < 1e-12
    # moving cells only raises it
    rng = np.random.default_rng(0)
    moved = np.clip(pos + 0.05 * rng.standard_normal(pos.shape), 0.0, 1.0)
    assert float(adj.occupancy_loss(torch.from_numpy(moved), nb, lo, hi)) > 1.0


def test_occupancy_of_a_collapsed_population_is_B():
    """Every cell on one node: n_b = N there, o_b = B, mean square B."""
    nb, dim = 6, 2
    pos = np.tile([0.4, 0.6], (100, 1))  # node (2, 3) of the 6 x 6 grid
    val = adj.occupancy_loss(torch.from_numpy(pos), nb, [0.0] * 3, [1.0] * 3)
    assert abs(float(val) - nb ** dim) < 1e-9


@pytest.mark.parametrize("dim", [2, 3])
def test_torch_and_numpy_losses_agree(dim):
    rng = np.random.default_rng(dim)
    lo, hi = [-0.5, 0.0, 1.0], [0.5, 2.0, 1.5]
    pos0 = np.array(lo[:dim]) + (np.array(hi[:dim]) - np.array(lo[:dim])) * rng.random((500, dim))
    pos = np.clip(pos0 + 0.02 * rng.standard_normal(pos0.shape), lo[:dim], hi[:dim])
    t = torch.from_numpy(pos)
    lt = float(adj.mean_x_displacement(t, torch.from_numpy(pos0)) + adj.occupancy_loss(t, 7, lo, hi))
    ln = adj.loss_numpy(pos, pos0, 7, lo, hi)
    assert abs(lt - ln) <= 1e-12 * max(1.0, abs(ln))


def test_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    pos0 = torch.from_numpy(0.05 + 0.9 * rng.random((60, 2)))
    pos = (pos0 + 0.01 * torch.from_numpy(rng.standard_normal((60, 2)))).requires_grad_(True)

    def loss(x):
        return adj.mean_x_displacement(x, pos0) + adj.occupancy_loss(x, 8, [0.0] * 3, [1.0] * 3)

    assert torch.autograd.gradcheck(loss, (pos,), eps=1e-7, atol=1e-6)
