"""Host logic of the benchmark: the clock-sample summary that accompanies every timed line."""
import datetime
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402

ROWS = [
    "2026/12/04 03:12:34.100, 0, 2070, 2070, 600.1, 0x0, Not Active, Not Active, Not Active, Not Active",
    "2026/12/04 03:12:34.150, 0, 2040, 2070, 900.2, 0x4, Not Active, Not Active, Not Active, Active",
    "2026/12/04 03:12:34.200, 0, 1980, 2070, 950.3, 0x4, Not Active, Not Active, Not Active, Active",
    "2026/12/04 03:12:34.250, 0, 2070, 2070, 610.4, 0x0, Not Active, Active, Not Active, Not Active",
    "garbage line",
]


def ts(s):
    return datetime.datetime.strptime(s, "%Y/%m/%d %H:%M:%S.%f")


def test_samples_inside_the_window_only():
    c = bench.parse_clock_samples(ROWS, ts("2026/12/04 03:12:34.120"), ts("2026/12/04 03:12:34.220"))
    assert c["samples"] == 2 and c["window"] == "timed region"
    assert c["sm_mhz"] == (2040 + 1980) / 2 and c["sm_max_mhz"] == 2070
    assert c["reasons"] == ["sw_power_cap"]           # the thermal sample lies outside the window


def test_no_window_takes_every_sample():
    c = bench.parse_clock_samples(ROWS)
    assert c["samples"] == 4
    assert c["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_window_shorter_than_the_interval_takes_the_nearest_sample():
    c = bench.parse_clock_samples(ROWS, ts("2026/12/04 03:12:34.101"), ts("2026/12/04 03:12:34.102"))
    assert c["samples"] == 1 and c["window"] == "nearest sample" and c["sm_mhz"] == 2070
    assert c["reasons"] == []


def test_empty_output():
    c = bench.parse_clock_samples([], ts("2026/12/04 03:12:34.1"), ts("2026/12/04 03:12:34.2"))
    assert c["samples"] == 0 and c["sm_mhz"] is None
