"""Calibration of the long-run statistical comparison (the GPU test compares
its ensemble with oracle runs the same way): two sets of FP64 oracle runs
with different noise seeds agree within Z_MAX on every observable, and runs
of a model with a planted mistake (the sign of chi, no repulsion, the
species' diffusivities swapped, the wrong species secreting) are told apart
by far more than Z_MAX. Both dimensions, the paper's aggregation set-up of
Sect. 3 (alpha cells normal around the centre, beta cells uniform)."""
import numpy as np
import pytest

import stats_util as su
from oracle import chemo_oracle as orc

PLANTED = {
    "chi_sign": lambda p: dict(chi=-p["chi"]),
    "no_repulsion": lambda p: dict(inter=0.0),
    "diffusivities_swapped": lambda p: dict(D=list(reversed(p["D"][:2]))),
    "wrong_species_secretes": lambda p: dict(secrete=list(reversed(p["secrete"][:2]))),
}


@pytest.fixture(scope="module", params=[2, 3])
def reference(request):
    dim = request.param
    p = su.params(dim)
    pos0, sp = orc.init_positions(dict(p, seed=7), su.N_CELLS, su.N_ALPHA)
    pos0 = pos0.astype(np.float32).astype(np.float64)  # the state the GPU starts from
    A = su.oracle_runs(p, pos0, sp, range(100, 116))
    floor = su.floors([(sp == 0).sum(), (sp == 1).sum()])
    return dim, p, pos0, sp, A, floor


def test_same_model_other_seeds_within_band(reference):
    dim, p, pos0, sp, A, floor = reference
    B = su.oracle_runs(p, pos0, sp, range(200, 208))
    z = su.zscores(A, B, floor)
    assert np.all(np.isfinite(z))
    assert np.abs(z).max() < su.Z_MAX, (dim, np.round(z, 2))


@pytest.mark.parametrize("mistake", sorted(PLANTED))
def test_planted_mistake_is_detected(reference, mistake):
    dim, p, pos0, sp, A, floor = reference
    q = dict(p, **PLANTED[mistake](p))
    C = su.oracle_runs(q, pos0, sp, range(300, 304))
    z = su.zscores(A, C, floor)
    assert np.abs(z).max() > 2 * su.Z_MAX, (dim, mistake, np.round(z, 2))
