"""Host logic of bench.py that decides whether a timed run is kept: the
nvidia-smi clock record read back into the line's `clocks` object."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _summary(tmp_path, lines):
    p = tmp_path / "clocks.csv"
    p.write_text("".join(line + "\n" for line in lines))
    c = bench.ClockSampler(0)
    c.path = str(p)
    return c.summary()


def test_clock_summary_median_max_and_reasons(tmp_path):
    s = _summary(tmp_path, [
        "0, 2032, 2032, 812.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2032, 1099.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2010, 2032, 950.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    ])
    assert s["sm_mhz"] == 2010.0 and s["sm_max_mhz"] == 2032.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    assert s["power_w_max"] == 1099.0
    assert not os.path.exists(tmp_path / "clocks.csv")  # the record is removed once read


def test_clock_summary_reports_throttle_reasons_by_name(tmp_path):
    s = _summary(tmp_path, [
        "0, 1500, 2032, 900.0, 0x0000000000000048, Active, Active, Not Active, Not Active",
        "0, 1400, 2032, 900.0, 0x0000000000000020, Not Active, Not Active, Active, Not Active",
    ])
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples_or_power(tmp_path):
    s = _summary(tmp_path, ["No devices were found", ""])
    assert s["samples"] == 0 and s["reasons"] == ["unsampled"] and s["sm_mhz"] is None
    s = _summary(tmp_path, ["0, 2032, 2032, [N/A], 0x0, Not Active, Not Active, Not Active, Not Active"])
    assert s["samples"] == 1 and s["power_w_max"] is None
