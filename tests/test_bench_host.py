"""Host-side pieces of bench.py that decide what its JSON line reports: the
measured peak, the traffic record's validity, the dominant stage and the
clock / throttle-reason summary of the timed region."""
import json
import os

import pytest

import bench


def test_peak_is_the_measured_copy_bandwidth():
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    peak, src = bench.peak_hbm()
    if os.path.exists(path):
        assert src == "measured" and peak == pytest.approx(float(json.load(open(path))["hbm_gbs"]))
    else:
        assert (peak, src) == (bench.FALLBACK_HBM_GBS, "fallback")


def test_traffic_record_only_for_its_workload():
    t = bench.k1_traffic("dst-96^3-phi0.50-N882")
    # the record carries the kernel source's hash: a value means it is current
    assert t is None or 1e6 < t < 2 * 134479872
    assert bench.k1_traffic("some-other-workload") is None


def test_dominant_stage():
    d = bench.dominant_stage({"collide_stream": 48.0, "particles": 69.0, "links": 46.0})
    assert d["stage"] == "particles" and d["share"] == pytest.approx(69.0 / 163.0)
    assert "k_dem_step" in d["kernel"]


def test_clock_lines():
    ok = "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
    capped = "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active\n"
    hot = "0, 1500, 2070, 1400.0, 0x40, Not Active, Active, Not Active, Not Active\n"
    r = bench.parse_clock_lines([ok, ok, capped])
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    r = bench.parse_clock_lines([ok, hot, "garbage\n", "0, [N/A], 2070, 1, 0, a, b, c, d\n"])
    assert r["samples"] == 2 and r["reasons"] == ["hw_thermal_slowdown"]
    assert r["sm_mhz"] == pytest.approx(1785.0)
    assert bench.parse_clock_lines([]) is None
