"""Host logic of bench.py that needs no GPU: the clock sampler's reading of
nvidia-smi rows (median SM clock, the maximum, and which throttle reasons were
active), and the roofline entry's arithmetic."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc = _FakeProc()
    s.lines = list(lines)
    return s


def test_clock_rows_median_max_and_reasons():
    rows = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1201.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1180.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 10, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = _sampler(rows).stop()
    assert out["sm_mhz"] == 2070.0
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["samples"] == 3


def test_clock_rows_report_every_slowdown_kind():
    rows = ["0, 1500, 2070, 1300, 0x8, Active, Active, Active, Not Active"]
    out = _sampler(rows).stop()
    assert out["sm_mhz"] == 1500.0
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi():
    out = bench.ClockSampler(0).stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


def test_roofline_entry_arithmetic():
    pk = {"hbm_gbs": 7000.0}
    cells = 512 * 512
    ms = 0.1
    r = bench.roofline_entry("flux", ms, cells, pk, "test")
    fl = bench.FP64_FLOPS_PER_CELL["flux"]
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(fl * cells / (ms / 1e3) / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["traffic"] == bench.TRAFFIC_PER_LAUNCH["flux"]
    # an unknown kernel kind reports no figure rather than a made-up one
    u = bench.roofline_entry("unknown", ms, cells, pk, "test")
    assert u["achieved"] is None and u["frac"] is None
