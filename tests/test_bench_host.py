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


def test_traffic_record_only_for_its_workload_and_kernel():
    t = bench.k1_traffic("dst-96^3-phi0.50-N882", "k_collide_stream<fp32>")
    # the record carries the kernel source's hash: a value means it is current
    assert t is None or 1e6 < t < 2 * 134479872
    assert bench.k1_traffic("some-other-workload", "k_collide_stream<fp32>") is None
    assert bench.k1_traffic("dst-96^3-phi0.50-N882", "some-other-kernel<fp32>") is None
    tb = bench.k1_traffic("batch64-bf16", "k_collide_stream<bf16>", "k_collide_stream_bf16_batch64_traffic.txt")
    assert tb is None or 1e9 < tb < 2 * 2041593168
    assert bench.k1_traffic("batch64-bf16", "k_collide_stream<fp32>", "k_collide_stream_bf16_batch64_traffic.txt") is None
    assert bench.lb_kernel({"staged": True}, "fp16") == "k_collide_stream_tma<fp16>"
    assert bench.lb_kernel({"staged": False}, "fp32") == "k_collide_stream<fp32>"


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


def _clk(mhz, reasons=()):
    return {"sm_mhz": mhz, "sm_max_mhz": 2070.0, "reasons": list(reasons), "samples": 5}


def test_clock_records_that_void_a_number():
    assert not bench.clocks_rejected(None)
    assert not bench.clocks_rejected(_clk(2070.0))
    assert not bench.clocks_rejected(_clk(1500.0, ["sw_power_cap"]))      # kept and noted
    assert bench.clocks_rejected(_clk(2070.0, ["hw_slowdown"]))
    assert bench.clocks_rejected(_clk(1900.0, ["sw_thermal_slowdown", "sw_power_cap"]))
    assert bench.clocks_rejected(_clk(1200.0))                             # locked low, no reason
    assert not bench.clocks_rejected(_clk(1800.0))


class _FakeSampler:
    def __init__(self, rec):
        self.rec = rec

    def stop(self):
        return self.rec


def test_timed_region_is_retaken_once_on_a_void_clock_record():
    runs = []

    def run():
        runs.append(1)
        return 10.0 * len(runs)

    recs = iter([_clk(2070.0, ["hw_thermal_slowdown"]), _clk(2070.0)])
    res, clk, first = bench.timed_with_retake(run, lambda: _FakeSampler(next(recs)))
    assert (res, len(runs)) == (20.0, 2)
    assert clk["reasons"] == [] and first["reasons"] == ["hw_thermal_slowdown"]
    # a second void record is reported as it is, not retaken again
    runs.clear()
    recs = iter([_clk(1000.0), _clk(1000.0)])
    res, clk, first = bench.timed_with_retake(run, lambda: _FakeSampler(next(recs)))
    assert len(runs) == 2 and bench.clocks_rejected(clk) and first is not None
    # clean first try; ranks without a sampler follow rank 0's decision
    runs.clear()
    res, clk, first = bench.timed_with_retake(run, lambda: None)
    assert (len(runs), clk, first) == (1, None, None)
    runs.clear()
    res, clk, first = bench.timed_with_retake(run, lambda: None, agree=lambda f: len(runs) == 1)
    assert len(runs) == 2


def test_fixed_launch_shape():
    class Fake:
        def __init__(self):
            self.set = None

        def tune(self):
            return {"tile_rows": 8, "blocks_per_sm": 2, "staged": False, "us": 1.0}

        def set_launch_shape(self, rows, bps, staged):
            self.set = (rows, bps, staged)

        def set_overlap(self, on):
            self.ov = on

        def launch_shape(self):
            return {"tile_rows": self.set[0], "blocks_per_sm": self.set[1], "staged": self.set[2]}

    old = bench.LAUNCH_SHAPE
    try:
        bench.LAUNCH_SHAPE = None
        assert bench.shape_for(Fake())["us"] == 1.0
        bench.LAUNCH_SHAPE = (4, 1, True, False)
        f = Fake()
        got = bench.shape_for(f)
        assert f.set == (4, 1, True) and not f.ov and got["staged"] and got["fixed"] and got["us"] is None
    finally:
        bench.LAUNCH_SHAPE = old


def test_batched_launch_count():
    assert bench.batched_launches([(100, 1), (800, 1)]) == 5      # brute-force pair search everywhere
    assert bench.batched_launches([(100, 1), (5000, 0)]) == 9     # one box builds a cell list
    assert bench.batched_launches([(0, 1), (0, 1)]) == 2          # fluid only
