"""Host-side logic of bench.py, without a GPU: the gate that attaches a
measured DRAM traffic figure only when the committed ncu summary was taken
on the current kernel source and workload, the peak fallback, the workload
description, and the CPU-baseline record (on a tiny sample)."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _profile(tmp_path, sha, kernel="leaf_tc2_kernel", n=16384, depth=2, traffic=123000000000):
    p = tmp_path / "traffic.md"
    p.write_text("# summary\n\n"
                 f"- kernel: {kernel}\n- n: {n}\n- depth: {depth}\n"
                 f"- traffic_bytes_per_launch: {traffic}\n- kernel_source_sha256: `{sha}`\n")
    return str(p)


def test_traffic_attached_only_for_the_captured_source(tmp_path, monkeypatch):
    sha = bench.leaf_source_hash()
    # an absolute profile path (os.path.join keeps it; the sources stay under ROOT)
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", _profile(tmp_path, sha))
    assert bench.measured_traffic(16384, 2, bench.PAIR_KERNEL) == 123e9
    # another workload, another kernel, or a changed source: no figure
    assert bench.measured_traffic(8192, 2, bench.PAIR_KERNEL) is None
    assert bench.measured_traffic(16384, 3, bench.PAIR_KERNEL) is None
    assert bench.measured_traffic(16384, 2, "leaf_tc_kernel") is None
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", _profile(tmp_path, "0" * 64))
    assert bench.measured_traffic(16384, 2, bench.PAIR_KERNEL) is None


def test_leaf_source_hash_covers_the_leaf_kernel_files():
    for rel in bench.LEAF_SOURCES:
        assert os.path.exists(os.path.join(ROOT, rel)), rel
    assert len(bench.leaf_source_hash()) == 64


def test_peaks_fall_back_without_measurements(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    pk = bench.peaks()
    assert pk["source"] == "fallback" and pk["hbm_gbs"] > 0 and pk["bf16_sustained"] > 0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps(
        {"hbm_gbs": 7000.0, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1800.0}))
    pk = bench.peaks()
    assert pk == {"hbm_gbs": 7000.0, "bf16": 2000.0, "bf16_sustained": 1800.0, "source": "measured"}


def test_workload_names_sizes():
    class A:
        n, dtype = 16384, "bf16"
    cfg = bench.workload_config(A, 2)
    assert cfg["n"] == 16384 and cfg["depth"] == 2 and "16384" in cfg["workload"]


def test_cpu_baseline_record_on_a_tiny_sample():
    pytest.importorskip("oracle")
    rec = bench.cpu_baseline(64, 7, budget_s=0.01, rows_cap=16)
    assert rec["kind"] == "oracle" and rec["unit"] == "TFLOP/s" and rec["value"] > 0 and rec["cores"] >= 1
    assert "of 64 rows" in rec["sample"]
