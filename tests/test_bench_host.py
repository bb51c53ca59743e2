"""The bench's host arithmetic (no GPU): the algorithmic bytes per launch of
each stage from its per-unit figures, and the roofline object built from
stage times -- the dominant stage is the one with the most time, achieved is
its bytes over its time per launch, frac is achieved over the peak, and
traffic is its recorded DRAM figure."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_stage_bytes_follow_the_per_unit_figures():
    n_s, n_n, nnzb, n_corr, n_pix, k = 1000, 20, 150, 300, 4800, 7
    b = bench.stage_bytes(n_s, n_n, nnzb, n_corr, n_pix, k)
    assert b["depth"] == 4800 * (4 + 32)
    assert b["reg_assembly"] == 150 * 144 + 20 * 80
    assert b["data_assembly"] == 1000 * 64 + 300 * 32 + 20 * 32 + 150 * 144 + 20 * 24 + 20 * 80
    b = bench.stage_bytes(n_s, n_n, nnzb, n_corr, n_pix, k, merged=False)
    assert b["data_assembly"] == 1000 * 64 + 300 * 32 + 20 * 32 + 150 * 144 + 20 * 24
    assert b["pcg"] == 7 * (150 * 144 + 20 * 192) + 20 * 252
    assert b["fusion"] == 1000 * (64 + 32 + 24) + 4800 * 160


def test_roofline_picks_the_stage_with_the_most_time():
    n_s, n_n, nnzb, n_corr, n_pix, k = 300000, 2048, 32000, 83000, 640 * 480, 20
    stage_ms = {"depth": 0.09, "reg_assembly": 1.0, "data_assembly": 3.5, "pcg": 16.0, "fusion": 0.5,
                "visibility": 0.0}
    stage_n = {"depth": 10, "reg_assembly": 100, "data_assembly": 100, "pcg": 100, "fusion": 10, "visibility": 0}
    r = bench.roofline(stage_ms, stage_n, n_s, n_n, nnzb, n_corr, n_pix, k)
    peak, _ = bench.measured_hbm_peak()
    d = r["dominant"]
    assert d["kernel"] == "pcg" and d["bound"] == "hbm" and d["unit"] == "GB/s"
    assert "visibility" not in r["stages"]          # a stage that never ran has no line
    want_bytes = k * (144.0 * nnzb + 192.0 * n_n) + 252.0 * n_n
    assert d["bytes_per_launch"] == want_bytes
    assert d["us_per_launch"] == pytest.approx(160.0)     # 16 ms over 100 launches
    assert d["achieved"] == pytest.approx(want_bytes / 160e-6 / 1e9)
    assert d["peak"] == peak and d["frac"] == pytest.approx(d["achieved"] / peak)
    assert d["traffic"] == bench.PROFILED_TRAFFIC["pcg"]
    # every stage that ran has its own line on the same arithmetic
    for name, line in r["stages"].items():
        per_launch_s = stage_ms[name] / stage_n[name] / 1000.0
        assert line["achieved"] == pytest.approx(line["bytes_per_launch"] / per_launch_s / 1e9)


def test_peak_is_the_measured_copy_bandwidth_or_the_fallback():
    peak, src = bench.measured_hbm_peak()
    assert src in ("measured", "fallback") and peak > 1000.0
    if src == "fallback":
        assert peak == 6800.0


def test_whole_job_throughput_counts_every_replica():
    assert bench.job_frames_per_s(2.0, 1) == pytest.approx(500.0)
    assert bench.job_frames_per_s(4.0, 8) == pytest.approx(2000.0)


def test_clock_summary_keeps_the_samples_inside_the_timed_region():
    import datetime

    def line(t, mhz, power_cap="Not Active", thermal="Not Active"):
        ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"{ts}, 0, {mhz}, 2070, 900.00, 0x0, Not Active, Not Active, {thermal}, {power_cap}"

    t0 = 1_800_000_000.0
    lines = [line(t0 - 0.05, 1200), line(t0 + 0.01, 2070), line(t0 + 0.02, 2055, power_cap="Active"),
             line(t0 + 0.03, 2070), line(t0 + 0.2, 1000, thermal="Active")]
    samples = bench.Clocks.parse(lines + ["garbage, line", ""])
    assert len(samples) == 5
    s = bench.Clocks.summarise(samples, t0, t0 + 0.04)
    assert s["samples"] == 3 and s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]   # the thermal sample lies after the region
    # a region between two samples: the nearest one on each side
    s = bench.Clocks.summarise(samples, t0 + 0.1, t0 + 0.15)
    assert s["samples"] == 0 and s["samples_used"] == 2 and s["reasons"] == ["sw_thermal_slowdown"]
    assert bench.Clocks.summarise([], t0, t0 + 1)["reasons"] == ["no samples"]
