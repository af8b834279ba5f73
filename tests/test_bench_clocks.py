"""bench.py host logic on CPU: the clock record of the timed region and the default step counts per arm."""
import sys

import pytest

pytest.importorskip("torch")
import bench  # noqa: E402


class _Proc:
    """Stands in for the nvidia-smi process: already finished."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _line(sm, smax, *reasons):
    flags = ["Active" if r else "Not Active" for r in reasons]
    return ", ".join(["0", str(sm), str(smax), "900.0", "0x0"] + flags)


def test_clock_record_keeps_the_samples_of_the_timed_region():
    cs = bench.ClockSampler(0)
    cs.proc = _Proc()
    # two samples before the timed region started (start() returns after the first one), three inside it
    cs.lines = [_line(1200, 2070, 0, 0, 0, 0), _line(1300, 2070, 0, 0, 0, 0),
                _line(2070, 2070, 0, 0, 0, 0), _line(2040, 2070, 0, 0, 0, 1), _line(2070, 2070, 0, 0, 0, 0)]
    cs.skip = 2
    rec = cs.stop()
    assert rec["samples"] == 3
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]


def test_clock_record_falls_back_to_every_sample_and_flags_slowdowns():
    cs = bench.ClockSampler(0)
    cs.proc = _Proc()
    cs.lines = [_line(1500, 2070, 1, 0, 0, 0), "garbled line", _line(1600, 2070, 0, 1, 1, 0)]
    cs.skip = 3  # no sample arrived after the region started: the record uses all of them
    rec = cs.stop()
    assert rec["samples"] == 2 and rec["sm_mhz"] == 1550.0
    assert rec["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_record_without_nvidia_smi():
    rec = bench.ClockSampler(0).stop()
    assert rec["samples"] == 0 and rec["reasons"] == ["nvidia-smi unavailable"]


@pytest.mark.parametrize("argv,steps", [([], 200), (["--impl", "reference"], 20), (["--steps", "7"], 7),
                                        (["--impl", "reference", "--steps", "3"], 3)])
def test_default_steps_per_arm(monkeypatch, argv, steps):
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    assert bench.parse().steps == steps
