"""bench.py's clock record (no GPU): the nvidia-smi samples taken during the
timed region are parsed into the median SM clock, the maximum clock and the
set of active throttle reasons that decide whether a run is kept."""

from __future__ import annotations

import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test",
                                                  os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _sampler(lines):
    b = _bench()
    s = b.ClockSampler(0)
    s.proc = _Done()  # as if nvidia-smi had run and been stopped
    s.lines = list(lines)
    return s.stop()


# index, clocks.sm, clocks.max.sm, power.draw, reasons.active, hw_slowdown,
# hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
def _line(sm, smax=2070, hw="Not Active", hwt="Not Active", swt="Not Active",
          cap="Not Active"):
    return f"0, {sm}, {smax}, 900.5, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}"


def test_clean_run():
    r = _sampler([_line(2070), _line(2070), _line(2055)])
    assert r["sm_mhz"] == 2070 and r["sm_max_mhz"] == 2070 and r["samples"] == 3
    assert r["reasons"] == []


def test_reasons_are_collected():
    r = _sampler([_line(1900, cap="Active"), _line(2070), _line(1500, hwt="Active"),
                  _line(1800, hw="Active", swt="Active")])
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap",
                            "sw_thermal_slowdown"]
    assert r["sm_mhz"] == (1800 + 1900) / 2


def test_unparsable_lines_are_skipped_and_no_samples_reported():
    r = _sampler(["", "garbage", "0, [N/A], 2070, 1, 0x0, x, x, x, x", _line(2000)])
    assert r["samples"] == 1 and r["sm_mhz"] == 2000
    r = _sampler(["garbage"])
    assert r["sm_mhz"] is None and r["reasons"] == ["no samples"]


def test_missing_nvidia_smi_is_reported():
    b = _bench()
    s = b.ClockSampler(0)  # never started: no process
    r = s.stop()
    assert r["sm_mhz"] is None and r["reasons"] == ["nvidia-smi unavailable"]
