"""Host pieces of the benchmark (no GPU): the clock record taken during the
timed region (median SM clock under load, the maximum clock, and every
throttle reason seen active, which decide whether a number is kept), the
per-pair flop count of the roofline, and the reference arm's rank rule."""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc = _Done()
    s.fh = tempfile.TemporaryFile(mode="w+")
    s.fh.write("\n".join(lines) + "\n")
    return s


def _row(util, mhz, reasons=("Not Active",) * 4, mx=2070):
    return ", ".join(["2026/01/01 00:00:00.000", "0", str(util), str(mhz), str(mx), "900.00", "0x0"] + list(reasons))


def test_clock_record_under_load():
    lines = [_row(0, 990)] + [_row(100, m) for m in (2070, 2070, 2055, 2070, 2040)] + [_row(3, 1200)]
    rec = _sampler(lines).stop()
    assert rec["sm_mhz"] == 2070 and rec["sm_max_mhz"] == 2070
    assert rec["reasons"] == [] and rec["samples"] == 7 and rec["samples_under_load"] == 5


def test_clock_record_counts_samples_inside_the_busy_windows():
    """A short run: nvidia-smi's utilisation (averaged over a longer time)
    stays low, but the samples taken while the kernels ran count."""
    import datetime

    def at(t, util, mhz):
        stamp = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return ", ".join([stamp, "0", str(util), str(mhz), "2070", "900.00", "0x0"] + ["Not Active"] * 4)

    t0 = 1.8e9
    lines = [at(t0 - 1.0, 0, 990), at(t0 + 0.02, 4, 2070), at(t0 + 0.04, 9, 2055), at(t0 + 0.5, 0, 1200),
             at(t0 + 0.62, 12, 2070)]
    rec = _sampler(lines).stop(windows=[(t0, t0 + 0.05), (t0 + 0.6, t0 + 0.7)])
    assert rec["samples"] == 5 and rec["samples_under_load"] == 3
    assert rec["sm_mhz"] == 2070


def test_clock_record_keeps_every_active_reason():
    act = "Active"
    lines = [_row(100, 2070), _row(100, 1800, ("Not Active", "Not Active", "Not Active", act)),
             _row(100, 1500, (act, "Not Active", act, "Not Active"))]
    rec = _sampler(lines).stop()
    assert rec["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert rec["sm_mhz"] == 1800


def test_clock_record_without_samples():
    s = bench.ClockSampler(0)
    assert s.stop() is None  # the sampler never started (no nvidia-smi)
    rec = _sampler([]).stop()
    assert rec["sm_mhz"] is None and rec["samples"] == 0


def test_flop_per_pair():
    assert bench.flop_per_pair(2) == 22 and bench.flop_per_pair(3) == 23
    assert bench.FLOP_PER_TEST == 8


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == ""


@pytest.mark.parametrize("flag", ["--steps", "--warmup"])
def test_arguments_parse(flag, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py", flag, "5"])
    args = bench.parse()
    assert getattr(args, flag[2:]) == 5 and args.gpus == 1 and args.impl == "gb300"
