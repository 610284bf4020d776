"""Device memory from a caller's allocator (chemo_set_allocator): every
buffer of a simulation, of a recorded run and of the host-buffer temporaries
comes from the callbacks and goes back through them with its size; a
simulation keeps the allocator it was created with; an allocator that fails
part-way leaves nothing behind; the results do not depend on where the
memory came from; PyTorch's caching allocator can back the library."""
import numpy as np
import pytest
import torch

from paper_1805_11007_gb300 import chemo
from paper_1805_11007_gb300 import workloads as wl
from parity_util import dev

pytestmark = pytest.mark.gpu


class Counting:
    """Allocator over PyTorch's caching allocator that records every buffer."""

    def __init__(self, fail_after=None):
        self.live = {}
        self.calls = 0
        self.released = 0
        self.bad = []
        self.fail_after = fail_after

    def alloc(self, nbytes):
        self.calls += 1
        if self.fail_after is not None and self.calls > self.fail_after:
            return 0
        ptr = torch.cuda.caching_allocator_alloc(nbytes)
        self.live[ptr] = nbytes
        return ptr

    def release(self, ptr, nbytes):
        if self.live.pop(ptr, None) != nbytes:
            self.bad.append((ptr, nbytes))
        torch.cuda.caching_allocator_delete(ptr)
        self.released += 1


@pytest.fixture
def counting():
    a = Counting()
    chemo.chemo_set_allocator(a.alloc, a.release)
    try:
        yield a
    finally:
        chemo.chemo_set_allocator(None, None)


def _fixed_gradient(n=5000):
    p = wl.params("periodic_fixed_gradient_2d", inter=1.0, diameter=[0.02])
    pos = wl.uniform_positions(n, 2, p["lo"], p["hi"], seed=5)
    return p, pos, np.zeros(n, np.uint8)


def test_simulation_buffers_come_from_the_allocator(counting):
    p, pos, sp = _fixed_gradient()
    a = chemo.chemo_create(p, dev(pos), dev(sp))
    chemo.chemo_set_allocator(None, None)  # later simulations: cudaMalloc; `a` keeps its allocator
    try:
        assert counting.calls >= 3 and counting.live
        assert sum(counting.live.values()) == chemo.chemo_get_info(a)["device_bytes"]
        n_calls = counting.calls
        with chemo.chemo_create(p, dev(pos), dev(sp)) as b:
            assert counting.calls == n_calls  # `b` takes nothing from it
            chemo.chemo_step_n(a, 20)
            chemo.chemo_step_n(b, 20)
            pa, _, da = chemo.read_state_host(a)
            pb, _, db = chemo.read_state_host(b)
            assert sum(counting.live.values()) == chemo.chemo_get_info(a)["device_bytes"]
        np.testing.assert_array_equal(pa, pb)  # no deposit: the steps are deterministic
        np.testing.assert_array_equal(da, db)
    finally:
        a.close()
    assert not counting.live and not counting.bad
    assert counting.released == counting.calls


def test_recorded_run_buffers_come_from_the_allocator(counting):
    p, pos, sp = wl.initial_state("adjoint_2d", n=1000, grid=[64, 64, 1])
    with chemo.chemo_create(p, dev(pos), dev(sp)) as sim:
        before = len(counting.live)
        chemo.chemo_record(sim, 8, 4)
        assert len(counting.live) > before  # checkpoints and segment buffers
        g = torch.zeros((1000, 2), dtype=torch.float32, device="cuda")
        g[:, 0] = 1.0 / 1000
        dth = torch.zeros(4, dtype=torch.float32, device="cuda")
        chemo.chemo_gradient(sim, g, dth)
        assert torch.isfinite(dth).all()
    assert not counting.live and not counting.bad


@pytest.mark.parametrize("fail_after", [0, 1, 3])
def test_failing_allocator_leaves_nothing_behind(fail_after):
    a = Counting(fail_after=fail_after)
    p, pos, sp = _fixed_gradient(1000)
    chemo.chemo_set_allocator(a.alloc, a.release)
    try:
        with pytest.raises(chemo.ChemoError) as e:
            chemo.chemo_create(p, dev(pos), dev(sp))
        assert e.value.status == chemo.ENOMEM
    finally:
        chemo.chemo_set_allocator(None, None)
    assert a.calls == fail_after + 1
    assert not a.live and not a.bad
    # the failure is the caller's allocator's, not the device's: it still works
    with chemo.chemo_create(p, dev(pos), dev(sp)) as sim:
        chemo.chemo_step(sim)
        chemo.chemo_check(sim)


def test_host_call_temporaries_come_from_the_allocator(counting):
    p = wl.params("walls_grid_2d")
    pos, sp = chemo.chemo_init_positions(p, 3000, 1500)
    assert counting.calls == 1 and not counting.live
    ctr = np.arange(64, dtype=np.uint32).reshape(16, 4)
    out = np.zeros_like(ctr)
    chemo.chemo_philox(7, ctr, out)
    assert counting.calls == 2 and not counting.live and not counting.bad
    assert pos.shape == (3000, 2) and int((sp == 0).sum()) == 1500 and out.any()


def test_torch_caching_allocator_backs_the_library():
    p, pos, sp = _fixed_gradient()
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    chemo.use_torch_allocator()
    try:
        sim = chemo.chemo_create(p, dev(pos), dev(sp))
    finally:
        chemo.chemo_set_allocator(None, None)
    held = chemo.chemo_get_info(sim)["device_bytes"]
    assert torch.cuda.memory_allocated() - base >= held
    chemo.chemo_step_n(sim, 10)
    x, _, _ = chemo.read_state_host(sim)
    assert np.all(np.isfinite(x))
    sim.close()
    assert torch.cuda.memory_allocated() - base < held
