"""Host logic of bench.py that needs no GPU: the sweep count behind the headline metric and
the parsing of the clock log that decides whether a run was throttled."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_sweeps_count_every_smoothed_level_but_not_the_coarsest():
    # a V(1,1) cycle sweeps each level above the coarsest twice; the 3x3 level is solved
    assert bench.sweeps_per_cycle([7, 3]) == pytest.approx(2 * 49 / 1e6)
    sizes = [1023, 511, 255, 127, 63, 31, 15, 7, 3]
    assert bench.sweeps_per_cycle(sizes) == pytest.approx(2 * sum(n * n for n in sizes[:-1]) / 1e6)
    # nu1 + nu2 sweeps per level with multi-step smoothing
    assert bench.sweeps_per_cycle(sizes, 6, 6) == pytest.approx(6 * bench.sweeps_per_cycle(sizes))
    assert bench.sweeps_per_cycle([3]) == 0


def _summary(tmp_path, rows):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    return s.summary()


def test_clock_log_median_max_and_throttle_reasons(tmp_path):
    na, act = "Not Active", "Active"
    rows = [f"0, {mhz}, 2070, 900.0, 0x0, {na}, {na}, {na}, {cap}"
            for mhz, cap in ((2070, na), (1995, act), (2040, na))]
    rows.append("garbage line")
    s = _summary(tmp_path, rows)
    assert s["sm_mhz"] == 2040 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]  # kept and noted, not a rejection
    rows[0] = f"0, 1500, 2070, 900.0, 0x0, {na}, {act}, {na}, {na}"
    assert _summary(tmp_path, rows)["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert not os.path.exists(tmp_path / "clocks.csv")  # the log is removed after reading


def test_clock_log_missing_gives_no_samples(tmp_path):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "absent.csv")
    assert s.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
