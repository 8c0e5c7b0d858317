"""The bench's clock record and kernel-time summary (CPU only): nvidia-smi
lines parsed into the median SM clock, the maximum clock and the throttle
reasons seen, from the samples taken inside the timed region only; every
kernel's mean, median and best per-step duration."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def sampler(lines, first):
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.lines = list(lines)
    c.first = first
    return c


def line(sm, reasons=("Not Active",) * 4):
    return ", ".join([str(sm), "2070", "950.5", "0x0"] + list(reasons))


def test_samples_before_the_timed_region_are_left_out():
    lines = [line(1200), line(2070), line(2070), line(2055)]
    s = sampler(lines, 1).summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}


def test_throttle_reasons_are_reported():
    lines = [line(2070), line(1980, ("Not Active", "Not Active", "Not Active", "Active")),
             line(1500, ("Active", "Not Active", "Not Active", "Not Active"))]
    s = sampler(lines, 0).summary()
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert s["sm_mhz"] == 1980.0 and s["samples"] == 3


def test_malformed_and_unsupported_lines_are_skipped():
    lines = [line(2070), "[N/A], [N/A], 1.0, 0x0, a, b, c, d", "garbage", line(2040)]
    s = sampler(lines, 0).summary()
    assert s["samples"] == 2 and s["sm_mhz"] == 2055.0


def test_no_sample_inside_the_region_falls_back_to_all():
    s = sampler([line(2070)], 1).summary()
    assert s["samples"] == 1 and s["sm_mhz"] == 2070.0


def test_no_tool_gives_an_empty_record():
    s = sampler([], 0).summary()
    assert s == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_kernel_times_mean_median_best():
    sys.path.insert(0, ROOT)
    import bench
    mean, med, best = bench.kernel_times({"a": [3.0, 1.0, 2.0, 10.0], "b": [0.5]})
    assert mean == {"a": 4.0, "b": 0.5}
    assert med == {"a": 2.5, "b": 0.5}
    assert best == {"a": 1.0, "b": 0.5}
