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
