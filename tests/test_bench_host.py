"""Host-side pieces of the benchmark that need no GPU: the clock record that
decides whether a run is kept (throttle reasons, median SM clock)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sampler(lines, skip=0):
    c = bench.ClockSampler(0)
    c.lines = list(lines)
    c.skip = skip
    return c.summary()


IDLE = "1965, 2070, 310.2, 0x0000000000000001, Not Active, Not Active, Not Active, Not Active"
BUSY = "2070, 2070, 1180.4, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
CAPPED = "1890, 2070, 1398.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
HOT = "1500, 2070, 1200.0, 0x0000000000000020, Not Active, Not Active, Active, Not Active"


def test_clean_run_has_no_reasons_and_the_median_clock():
    s = _sampler([BUSY, BUSY, BUSY.replace("2070, 2070", "2055, 2070", 1), BUSY])
    assert s["samples"] == 4 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == [] and s["sm_mhz"] == 2070.0


def test_reasons_are_collected_by_name():
    s = _sampler([BUSY, CAPPED, HOT, BUSY])
    assert s["reasons"] == ["sw_power_cap", "sw_thermal_slowdown"]
    assert s["sm_mhz"] == (2070.0 + 1890.0) / 2


def test_samples_before_the_timed_region_are_dropped():
    s = _sampler([IDLE, HOT, BUSY, BUSY, BUSY], skip=2)
    assert s["samples"] == 3 and s["reasons"] == [] and s["sm_mhz"] == 2070.0


def test_unreadable_lines_and_no_samples():
    s = _sampler(["", "[N/A], [N/A]", "garbage"])
    assert s["samples"] == 0 and s["reasons"] == ["unsampled"]
