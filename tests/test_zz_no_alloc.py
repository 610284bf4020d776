"""The no-allocation pair-force entry point (chemo_forces_noalloc) through the
C ABI: bitwise against the allocating path (chemo_create +
chemo_stage_forces) and within the parity tolerance of the FP64 oracle.

Callers that cannot allocate device memory where they need forces (a fixed
device-memory budget set at start-up, a real-time loop that must not
synchronise the device, a plug-in inside another framework's allocator) use
chemo_forces_noalloc; its cell list lives in one static device array that
every call shares and that keeps the last call's contents. The tests
therefore chain calls of different sizes, boxes and bin counts on one
non-default stream and check each against a fresh allocating computation.
This file is collected last so that a run stopping at its first failure has
already run every other test; it also passes on its own.
"""
import numpy as np
import pytest
import torch

from oracle import chemo_oracle as orc
from paper_1805_11007_gb300 import chemo
from paper_1805_11007_gb300 import workloads as wl
from parity_util import force_quantum

pytestmark = pytest.mark.gpu

LIMIT = 65535  # largest 16-bit bin count: no bin can overflow below it


def _allocating_forces(p, pos, sp, stream):
    with torch.cuda.stream(stream):
        dpos = torch.from_numpy(pos).cuda()
        dsp = torch.from_numpy(sp).cuda()
        F = torch.zeros((pos.shape[0], p["dim"]), dtype=torch.float32, device="cuda")
    sim = chemo.chemo_create(p, dpos, dsp, stream=stream)
    try:
        chemo.chemo_stage_forces(sim, F, stream=stream)
        stream.synchronize()
        return F.cpu().numpy()
    finally:
        sim.close()


def _noalloc_forces(p, pos, sp, stream):
    with torch.cuda.stream(stream):
        dpos = torch.from_numpy(pos).cuda()
        dsp = torch.from_numpy(sp).cuda()
        F = torch.full((pos.shape[0], p["dim"]), float("nan"), dtype=torch.float32, device="cuda")
    chemo.chemo_forces_noalloc(p, dpos, dsp, F, stream=stream)
    stream.synchronize()
    return F.cpu().numpy()


def _assert_oracle_forces(p, pos, sp, F):
    """Parity tolerance of the force tests: 1e-5 of the summed pair
    magnitudes per particle, the pairs at the cutoff (either way correct) and
    one fixed-point quantum per neighbour."""
    Fr, ex = orc.pair_forces(p, pos.astype(np.float64), sp, method=1, extras=True)
    tol = 1e-5 * ex["fabs"] + ex["border"] + force_quantum(p) * (ex["count"] + 1) * np.sqrt(3.0)
    err = np.linalg.norm(F.astype(np.float64) - Fr, axis=1)
    assert np.all(err <= tol), int(np.argmax(err - tol))


CASES = [
    ("walls_grid_2d", dict(diameter=[0.01, 0.02], grid=[16, 16, 1]), 30011),
    ("clumps_grid_3d", dict(diameter=[0.01, 0.02], grid=[16, 16, 16]), LIMIT),
    ("periodic_fixed_gradient_2d", dict(diameter=[0.03]), 4001),
]


@pytest.mark.parametrize("name,over,n", CASES)
def test_noalloc_forces_match_allocating_path_and_oracle_twice(name, over, n):
    p, pos, sp = wl.initial_state(name, n=n, **over)
    stream = torch.cuda.Stream()
    ref = _allocating_forces(p, pos, sp, stream)
    for call in range(2):  # the second call starts from the first one's leftovers
        got = _noalloc_forces(p, pos, sp, stream)
        np.testing.assert_array_equal(got, ref, err_msg="call %d" % call)
    _assert_oracle_forces(p, pos, sp, got)


def test_noalloc_calls_of_different_sizes_in_a_row():
    # large 3D, then a small 2D set in another box with far fewer bins, then
    # the large one again: stale counts, tiles or offsets of an earlier call
    # would show in the next
    big = wl.initial_state("clumps_grid_3d", n=LIMIT, diameter=[0.01, 0.02], grid=[16, 16, 16])
    small = wl.initial_state("walls_grid_2d", n=3001, diameter=[0.05, 0.08], grid=[16, 16, 1],
                             lo=[-1.0, 0.5, 0.0], hi=[0.5, 1.25, 1.0])
    stream = torch.cuda.Stream()
    refs = [_allocating_forces(*case, stream) for case in (big, small)]
    for case, ref in ((big, refs[0]), (small, refs[1]), (big, refs[0])):
        got = _noalloc_forces(*case, stream)
        np.testing.assert_array_equal(got, ref)
    _assert_oracle_forces(*small, _noalloc_forces(*small, stream))


def test_noalloc_every_particle_in_one_bin_at_the_limit():
    # a cutoff as long as the box: one bin holds all LIMIT particles, the
    # largest count a 16-bit bin takes without wrapping into its neighbour
    p, pos, sp = wl.initial_state("walls_grid_2d", n=LIMIT, diameter=[1.0, 1.0], grid=[16, 16, 1])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = chemo.chemo_create(p, torch.from_numpy(pos).cuda(), torch.from_numpy(sp).cuda(), stream=stream)
    try:
        assert int(np.prod(chemo.chemo_get_info(sim)["nbins"][:2])) == 1
    finally:
        sim.close()
    ref = _allocating_forces(p, pos, sp, stream)
    got = _noalloc_forces(p, pos, sp, stream)
    np.testing.assert_array_equal(got, ref)
    # the sum over all particles of exact pair sums is zero up to the final
    # rounding of each particle's sum to single precision
    assert np.all(np.isfinite(got))
    assert np.abs(got.astype(np.float64).sum(axis=0)).max() <= 1e-6 * np.abs(got).sum()


def test_noalloc_rejects_sizes_beyond_its_limit():
    p, pos, sp = wl.initial_state("walls_grid_2d", n=LIMIT + 1, diameter=[0.01, 0.02], grid=[16, 16, 1])
    F = torch.zeros((LIMIT + 1, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(chemo.ChemoError) as ei:
        chemo.chemo_forces_noalloc(p, torch.from_numpy(pos).cuda(), torch.from_numpy(sp).cuda(), F)
    assert ei.value.status == chemo.EINVAL
    assert str(LIMIT) in str(ei.value)
    # a cutoff far below the box size needs too many bins
    q = dict(p, diameter=[1e-4, 1e-4])
    pos2 = pos[:1000].copy()
    with pytest.raises(chemo.ChemoError) as ei:
        chemo.chemo_forces_noalloc(q, torch.from_numpy(pos2).cuda(), torch.from_numpy(sp[:1000]).cuda(), F[:1000])
    assert ei.value.status == chemo.EINVAL
