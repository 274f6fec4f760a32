"""Host-side logic of bench.py that decides whether a run is kept: the clock
record taken during the timed region (median SM clock, maximum, throttle
reasons) and the whole-job aggregation in a single process.  No GPU."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _row(sm, mx, hw="Not Active", thermal="Not Active", sw_thermal="Not Active", cap="Not Active"):
    # index, clocks.sm, clocks.max.sm, power.draw, active mask, then the four reasons
    return ["0", str(sm), str(mx), "900.0", "0x0", hw, thermal, sw_thermal, cap]


def test_clock_summary_median_max_and_no_reasons():
    s = bench.ClockSampler(0)
    s.samples = [_row(2032, 2032), _row(2017, 2032), _row(1990, 2032), _row(2032, 2032), _row(2025, 2032)]
    out = s.summary()
    assert out["sm_mhz"] == 2025.0
    assert out["sm_max_mhz"] == 2032.0
    assert out["reasons"] == []
    assert out["samples"] == 5


def test_clock_summary_collects_every_active_reason_once():
    s = bench.ClockSampler(0)
    s.samples = [_row(1800, 2032, cap="Active"), _row(1700, 2032, hw="Active", cap="Active"),
                 _row(2032, 2032, thermal="Active"), _row(2032, 2032, sw_thermal="Active")]
    out = s.summary()
    assert out["reasons"] == sorted(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                     "sw_power_cap"])


def test_clock_summary_skips_unreadable_clock_fields():
    s = bench.ClockSampler(0)
    s.samples = [_row("[N/A]", "[N/A]"), _row(2000, 2032)]
    out = s.summary()
    assert out["sm_mhz"] == 2000.0 and out["sm_max_mhz"] == 2032.0


def test_clock_summary_without_samples_says_so():
    out = bench.ClockSampler(0).summary()
    assert out["sm_mhz"] is None and out["reasons"] == ["unsampled"]


def test_single_process_aggregation():
    # One rank: the whole-job rate is its own rate, the maximum its own value.
    assert bench.whole_job_rate(2.0e6, 0.5, 1, None) == 4.0e6
    assert bench.max_over_ranks(3.5, None) == 3.5
