"""Host logic of bench.py's measurement: parsing of the nvidia-smi clock
samples (median SM clock, throttle reasons), --set overrides, and the sweep
traffic record's link to the smoother's source (the committed ncu figures
apply to the current smoother; a changed smoother reports no traffic)."""
import json
import os
import sys

from conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_clock_samples_summary_flags_throttling():
    c = bench.Clocks(0)
    c.out = "\n".join([
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1010.4, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1800, 2070, 1390.0, 0x8, Active, Not Active, Not Active, Not Active",
        "garbage line",
    ])
    s = c.summary()
    assert s["sm_mhz"] == 2055 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    c.out = ""
    assert c.summary()["reasons"] == ["unavailable"]


def test_set_overrides_parse_numbers():
    class A:
        set = ["nu1=1", "lin_rtol=1e-3", "tile_assembly=0", "newton_predictor=0.5"]
    assert bench.config_overrides(A) == {"nu1": 1, "lin_rtol": 1e-3, "tile_assembly": 0, "newton_predictor": 0.5}


def test_sweep_traffic_record_matches_the_current_smoother():
    rec = json.load(open(os.path.join(ROOT, "profiles", "k_sweep_counters.json")))
    assert rec["f64"]["smoother_source_sha256"] == bench.smoother_source_sha256()
    t = bench.sweep_traffic(1.0e6, "f64")
    assert t is not None and 0.9e6 < t < 1.0e6          # traffic / algorithmic 0.975
    assert bench.sweep_traffic(1.0e6, "f16") is None


def test_workload_rejects_qoi_sets_other_than_the_standard_pair():
    import pytest
    import torch
    from paper_2302_07804_gb300 import henry
    with pytest.raises(ValueError) as e:
        bench.Workload(henry, torch, "cpu", [4], henry.HENRY_FP64, [], qoi_set=henry.HENRY_QOI_PAPER)
    assert "not 15 per sample" in str(e.value)


def test_roofline_from_profile_picks_the_dominant_kernel_and_its_bound():
    from paper_2302_07804_gb300 import henry
    prof = {k: [0.0, 0, 0.0, 0.0] for k in henry.KERNEL_CLASSES}
    prof["smooth"] = [30.0, 100, 150e9, 10e9]          # 30 ms over 100 launches
    prof["smooth_coarse"] = [10.0, 300, 10e9, 1e9]
    prof["spmv"] = [35.0, 50, 175e9, 12e9]             # more time than either smoother class alone
    roof, classes, launches = bench.roofline_from_profile(prof, "f64", 6000.0, "measured")
    assert launches == 450
    # the smoother's classes are one kernel: 40 ms, 400 launches, 160 GB -> 4000 GB/s
    assert roof["kernel"] == "k_sweep" and roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert abs(roof["achieved"] - 4000.0) < 1e-9 and abs(roof["frac"] - 4000.0 / 6000.0) < 1e-12
    assert abs(roof["avg_launch_us"] - 100.0) < 1e-9 and roof["alg_bytes_per_launch"] == 160e9 / 400
    assert abs(roof["alu"]["achieved"] - 11e9 / 0.04 / 1e12) < 1e-12
    assert abs(roof["by_grid"]["fine grids"]["GBps"] - 5000.0) < 1e-9
    assert abs(classes["spmv"]["share"] - 35.0 / 75.0) < 1e-12 and classes["qoi"]["GBps"] is None
    # a flop-heavy kernel is reported against the ALU peak
    prof["smooth"], prof["smooth_coarse"] = [1.0, 1, 1e9, 0.0], [0.0, 0, 0.0, 0.0]
    prof["spmv"] = [35.0, 50, 7e9, 40e12 * 0.035]      # 0.2 TB/s, 40 TFLOP/s
    roof, _, _ = bench.roofline_from_profile(prof, "f32", 6000.0, "fallback")
    assert roof["kernel"] == "spmv" and roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    assert roof["traffic"] is None and "by_grid" not in roof
    assert roof["hbm"]["peak_source"].startswith("fallback")
