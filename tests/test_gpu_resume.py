"""Checkpoint and resume through the C ABI: the state read back by id
(positions, species, unwrapped displacement), the field and the step index
restart a trajectory in a new simulation. The noise is keyed by (id,
absolute step) and the pair forces are exact integer sums, so without a
chemical field the resumed run repeats the uninterrupted one bit for bit;
with a field it agrees to the rounding of the deposit's float atomics."""
import numpy as np
import pytest

from paper_1805_11007_gb300 import chemo
from paper_1805_11007_gb300 import workloads as wl
from parity_util import dev, make_sim

pytestmark = pytest.mark.gpu


def _run_split(p, pos, sp, c0, k1, k2):
    with make_sim(p, pos, sp, c0) as a:
        chemo.chemo_step_n(a, k1 + k2)
        whole = chemo.read_state_host(a)
        cw = chemo.read_field_host(a) if c0 is not None else None
    with make_sim(p, pos, sp, c0) as b:
        chemo.chemo_step_n(b, k1)
        xs, ss, ds = chemo.read_state_host(b)
        cs = chemo.read_field_host(b) if c0 is not None else None
        step = chemo.chemo_step_index(b)
    assert step == k1
    # a new simulation from the saved checkpoint
    with make_sim(p, xs, ss) as r:
        if ds is not None:
            chemo.chemo_write_state(r, dev(xs), dev(ss), dev(ds))
        if cs is not None:
            chemo.chemo_write_field(r, dev(cs))
        chemo.chemo_set_step_index(r, step)
        chemo.chemo_step_n(r, k2)
        chemo.chemo_check(r)
        assert chemo.chemo_step_index(r) == k1 + k2
        resumed = chemo.read_state_host(r)
        cr = chemo.read_field_host(r) if c0 is not None else None
    return whole, resumed, cw, cr


@pytest.mark.parametrize("mode", [3, 4])
def test_resume_fixed_gradient_bitwise(mode):
    p, pos, sp = wl.initial_state("periodic_fixed_gradient_2d", n=20011, search_mode=mode)
    assert p["track_displacement"]
    whole, resumed, _, _ = _run_split(p, pos, sp, None, 13, 24)
    for a, b in zip(whole, resumed):
        np.testing.assert_array_equal(a, b)


def test_resume_with_field():
    p, pos, sp = wl.initial_state("walls_grid_2d", n=20011, grid=[128, 128, 1], cutoff_mode=1)
    c0 = wl.random_field(p, seed=4, scale=0.3)
    whole, resumed, cw, cr = _run_split(p, pos, sp, c0, 9, 11)
    np.testing.assert_array_equal(whole[1], resumed[1])
    assert np.abs(whole[0] - resumed[0]).max() <= 1e-5
    assert np.abs(cw - cr).max() <= 1e-5 * np.abs(cw).max()


def test_checkpoint_file_resumes_bitwise(tmp_path):
    """save_sim / load_sim: the same continuation through an .npz file."""
    from paper_1805_11007_gb300 import checkpoint as ck
    p, pos, sp = wl.initial_state("periodic_fixed_gradient_2d", n=5003)
    with make_sim(p, pos, sp) as a:
        chemo.chemo_step_n(a, 30)
        whole = chemo.read_state_host(a)
    with make_sim(p, pos, sp) as b:
        chemo.chemo_step_n(b, 17)
        ck.save_sim(b, tmp_path / "run.npz")
    with ck.load_sim(tmp_path / "run.npz") as r:
        assert chemo.chemo_step_index(r) == 17
        chemo.chemo_step_n(r, 13)
        resumed = chemo.read_state_host(r)
    for x, y in zip(whole, resumed):
        np.testing.assert_array_equal(x, y)


def test_checkpoint_file_of_an_ensemble(tmp_path):
    """An ensemble's checkpoint keeps its replicate sizes and every
    replicate's grid."""
    from paper_1805_11007_gb300 import checkpoint as ck
    p, s, pos, sp = wl.ensemble_state(sizes=[300, 0, 1200, 77], grid=[32, 32, 1], cutoff_mode=1)
    with chemo.chemo_create_batch(p, s, dev(pos), dev(sp)) as a:
        chemo.chemo_step_n(a, 5)
        ck.save_sim(a, tmp_path / "ens.npz")
        chemo.chemo_step_n(a, 6)
        whole = chemo.read_state_host(a)
        cw = chemo.read_field_host(a)
    with ck.load_sim(tmp_path / "ens.npz") as r:
        assert r.sizes == [300, 0, 1200, 77] and chemo.chemo_step_index(r) == 5
        chemo.chemo_step_n(r, 6)
        resumed = chemo.read_state_host(r)
        cr = chemo.read_field_host(r)
    np.testing.assert_array_equal(whole[1], resumed[1])
    assert np.abs(whole[0] - resumed[0]).max() <= 1e-5
    assert np.abs(cw - cr).max() <= 1e-5 * max(np.abs(cw).max(), 1e-30)
