"""Checkpoint files on the host (no GPU): a snapshot written by save comes
back from load with the same arrays, dtypes, step, replicate sizes and
parameters (numpy values included); optional arrays stay optional; restore
refuses an unknown format before creating anything."""
import numpy as np
import pytest

from paper_1805_11007_gb300 import checkpoint as ck
from paper_1805_11007_gb300 import workloads as wl


def _snap(with_optional):
    rng = np.random.default_rng(0)
    p = wl.params("walls_grid_2d", grid=[16, 16, 1], chi=np.float32(1.5), D=np.array([1.0, 0.5]))
    s = {"format": ck.FORMAT, "params": p, "sizes": [3, 0, 4], "step": 12345678901,
         "pos": rng.random((7, 2)).astype(np.float32), "species": np.array([0, 1, 0, 1, 1, 0, 0], np.uint8)}
    if with_optional:
        s["disp"] = rng.standard_normal((7, 2)).astype(np.float32)
        s["c"] = rng.random((3, 16, 16)).astype(np.float32)
    return s


@pytest.mark.parametrize("with_optional", [False, True])
def test_save_load_round_trip(tmp_path, with_optional):
    s = _snap(with_optional)
    path = tmp_path / "run.npz"
    ck.save(path, s)
    r = ck.load(path)
    assert r["format"] == ck.FORMAT and r["step"] == 12345678901 and r["sizes"] == [3, 0, 4]
    for k in ("pos", "species", "disp", "c"):
        if k in s:
            assert r[k].dtype == s[k].dtype
            np.testing.assert_array_equal(r[k], s[k])
        else:
            assert k not in r
    assert r["params"]["chi"] == pytest.approx(1.5) and r["params"]["D"] == [1.0, 0.5]
    assert {k: v for k, v in r["params"].items() if k not in ("chi", "D")} == \
        {k: v for k, v in s["params"].items() if k not in ("chi", "D")}


def test_restore_refuses_unknown_format():
    s = _snap(False)
    s["format"] = 99
    with pytest.raises(ValueError):
        ck.restore(s)
