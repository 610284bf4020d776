"""The no-allocation pair-force entry point (chemo_forces_noalloc) against
the allocating path (chemo_create + chemo_stage_forces), through the C ABI.

Callers that cannot allocate device memory where they need forces use
chemo_forces_noalloc; its cell list lives in a static device array that every
call shares. This file is collected last so that a run stopping at its first
failure has already run every other test; it also passes on its own.
"""
import numpy as np
import pytest
import torch

from oracle import chemo_oracle as orc
from paper_1805_11007_gb300 import chemo
from paper_1805_11007_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _reference_forces(p, pos, sp):
    sim = chemo.chemo_create(p, torch.from_numpy(pos).cuda(), torch.from_numpy(sp).cuda())
    try:
        F = torch.zeros((pos.shape[0], p["dim"]), dtype=torch.float32, device="cuda")
        chemo.chemo_stage_forces(sim, F)
        torch.cuda.synchronize()
        return F.cpu().numpy().astype(np.float64)
    finally:
        sim.close()


@pytest.mark.parametrize("name,over,n", [
    ("walls_grid_2d", dict(diameter=[0.01, 0.02], grid=[16, 16, 1]), 30011),
    ("clumps_grid_3d", dict(diameter=[0.01, 0.02], grid=[16, 16, 16]), 65536),
    ("periodic_fixed_gradient_2d", dict(diameter=[0.03]), 4001),
])
def test_noalloc_forces_match_allocating_path_twice(name, over, n):
    p, pos, sp = wl.initial_state(name, n=n, **over)
    ref = _reference_forces(p, pos, sp)
    # the force tolerance of the parity tests: 1e-5 of the summed pair
    # magnitudes per particle (plus pairs at the cutoff, either way correct)
    _, ex = orc.pair_forces(p, pos.astype(np.float64), sp, extras=True)
    from parity_util import force_quantum
    tol = 1e-5 * ex["fabs"] + ex["border"] + force_quantum(p) * (ex["count"] + 1) * np.sqrt(3.0)
    dpos = torch.from_numpy(pos).cuda()
    dsp = torch.from_numpy(sp).cuda()
    for call in range(2):  # the second call starts from the first one's leftovers
        F = torch.full((n, p["dim"]), float("nan"), dtype=torch.float32, device="cuda")
        chemo.chemo_forces_noalloc(p, dpos, dsp, F)
        torch.cuda.synchronize()
        got = F.cpu().numpy().astype(np.float64)
        err = np.linalg.norm(got - ref, axis=1)
        assert np.all(np.isfinite(got)), call
        assert np.all(err <= tol), (call, int(np.argmax(err - tol)))


def test_noalloc_rejects_sizes_beyond_its_limit():
    p, pos, sp = wl.initial_state("walls_grid_2d", n=65537, diameter=[0.01, 0.02], grid=[16, 16, 1])
    F = torch.zeros((65537, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(chemo.ChemoError) as ei:
        chemo.chemo_forces_noalloc(p, torch.from_numpy(pos).cuda(), torch.from_numpy(sp).cuda(), F)
    assert ei.value.status == chemo.EINVAL
    assert "65536" in str(ei.value)
    # a cutoff far below the box size needs too many bins
    q = dict(p, diameter=[1e-4, 1e-4])
    pos2 = pos[:1000].copy()
    with pytest.raises(chemo.ChemoError) as ei:
        chemo.chemo_forces_noalloc(q, torch.from_numpy(pos2).cuda(), torch.from_numpy(sp[:1000]).cuda(), F[:1000])
    assert ei.value.status == chemo.EINVAL
