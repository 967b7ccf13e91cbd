"""The benchmark's roofline arithmetic on CPU: a made-up launch profile of the
shape the library returns (one record per kernel kind, launches counted per
level step) gives the achieved bandwidth, fraction, per-launch figures and
the whole-build figure by hand, and the recorded DRAM traffic is reported
only for the workload, size and sources it was captured on."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _stats():
    # Two steps of a build with 9 level steps each: 18 level steps timed in
    # 8.0 ms over 36.0 GB of the level-wise model; level 0's counts 0.8 ms
    # over 4.0 GB.
    return {
        "level_pass": {"launches": 18, "kernels": 90, "total_ms": 8.0, "alg_bytes": 36.0e9,
                       "variant_bytes": 30.0e9},
        "level0_count": {"launches": 4, "kernels": 8, "total_ms": 0.8, "alg_bytes": 4.0e9,
                         "variant_bytes": 4.5e9},
        "query_multi": {"launches": 2, "kernels": 2, "total_ms": 0.2, "alg_bytes": 2.0e6,
                        "variant_bytes": 2.0e6},
    }


def test_roofline_of_the_kernel_with_most_device_time(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: {"hbm_gbs": 6000.0})
    monkeypatch.setitem(bench.RUN, "workload", "other")
    roof, kernels, launches = bench.roofline_of(_stats(), 2)
    assert roof["kernel"] == "level_pass"
    assert roof["achieved"] == pytest.approx(36.0e9 / 8.0e-3 / 1e9)          # 4500 GB/s
    assert roof["frac"] == pytest.approx(4500.0 / 6000.0)
    assert roof["alg_bytes_per_launch"] == pytest.approx(2.0e9)               # per level step
    assert roof["avg_launch_ms"] == pytest.approx(8.0 / 18)
    assert roof["variant_bytes_frac"] == pytest.approx(30.0e9 / 8.0e-3 / 1e9 / 6000.0)
    # Whole build: level 0's counts and the level steps, bytes over time.
    assert roof["build"]["kernels"] == ["level0_count", "level_pass"]
    assert roof["build"]["achieved"] == pytest.approx(40.0e9 / 8.8e-3 / 1e9)
    assert roof["build"]["ms_per_step"] == pytest.approx(4.4)
    assert roof["peak_source"].startswith("measured")
    assert kernels["level_pass"]["ms_per_step"] == pytest.approx(4.0)
    assert kernels["query_multi"]["launches"] == 2
    assert launches == 100
    assert roof["traffic"] is None  # recorded for the default workload only


def test_fallback_peak_without_measured_peaks(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: {})
    roof, _, _ = bench.roofline_of(_stats(), 2)
    assert roof["peak"] == 6800.0 and roof["peak_source"].startswith("fallback")


def test_recorded_traffic_follows_workload_size_and_sources(monkeypatch):
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)["level_pass"]
    monkeypatch.setitem(bench.RUN, "workload", rec["workload"])
    monkeypatch.setitem(bench.RUN, "size_log2", None)
    monkeypatch.setitem(bench.RUN, "variant", 0)
    expect = rec["dram_bytes_per_launch"] if rec["source_hash"] == bench.source_hash() else None
    assert bench.ncu_traffic("level_pass") == expect
    # A smaller size, another workload or the two-level variant: no figure.
    monkeypatch.setitem(bench.RUN, "size_log2", 28)
    assert bench.ncu_traffic("level_pass") is None
    monkeypatch.setitem(bench.RUN, "size_log2", None)
    monkeypatch.setitem(bench.RUN, "variant", 3)
    assert bench.ncu_traffic("level_pass") is None
    monkeypatch.setitem(bench.RUN, "variant", 0)
    monkeypatch.setitem(bench.RUN, "workload", "words")
    assert bench.ncu_traffic("level_pass") is None
