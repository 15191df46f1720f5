"""Host-side logic of bench.py, without a GPU: the gate that attaches a
measured DRAM traffic figure only when the committed ncu summary was taken
on the current kernel source and workload, the peak fallback, the workload
description, the CPU-baseline record (on a tiny sample), and the reference
arm's line (the CPU oracle) alone and under torchrun."""
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
                 f"- traffic_bytes_per_launch.combine0: {traffic}\n"
                 f"- traffic_bytes_per_launch.combine2: {traffic // 2}\n"
                 f"- kernel_source_sha256: `{sha}`\n")
    return str(p)


def test_traffic_attached_only_for_the_captured_source(tmp_path, monkeypatch):
    sha = bench.leaf_source_hash()
    # an absolute profile path (os.path.join keeps it; the sources stay under ROOT)
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", _profile(tmp_path, sha))
    assert bench.measured_traffic(16384, 2, bench.PAIR_KERNEL) == 123e9
    assert bench.measured_traffic(16384, 2, bench.PAIR_KERNEL, combine=2) == 61.5e9
    assert bench.measured_traffic(16384, 2, bench.PAIR_KERNEL, combine=3) is None  # not captured
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


def _run_reference(cmd, env_extra=None):
    import subprocess
    env = dict(os.environ, **(env_extra or {}))
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    return [json.loads(ln) for ln in lines]


def test_reference_arm_line():
    pytest.importorskip("oracle")
    (out,) = _run_reference([sys.executable, "bench.py", "--impl", "reference", "--n", "256", "--steps", "2",
                             "--warmup", "3"], {"OMP_NUM_THREADS": "3"})
    assert out["impl"] == "reference" and out["n_gpus"] == 1 and out["steps"] == 2 and out["warmup"] == 3
    assert out["value"] > 0 and out["e2e"]["value"] == out["value"]
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["e2e"]["d2h_bytes_per_step"] == 0
    # one row of C per OpenMP thread, and the record says how many threads worked
    assert out["cpu_baseline"]["cores"] == 3 and "3 of 256 rows" in out["cpu_baseline"]["sample"]


def test_reference_arm_under_torchrun_prints_once_on_all_cores():
    pytest.importorskip("oracle")
    outs = _run_reference([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                           "--master-addr", "127.0.0.1", "--master-port", "29561", "bench.py", "--impl",
                           "reference", "--gpus", "2", "--steps", "2", "--warmup", "3"])  # (torchrun reads --n as its own)
    assert len(outs) == 1 and outs[0]["n_gpus"] == 2  # rank 0 alone
    # the launcher's one thread per rank does not bind the one rank that works
    assert outs[0]["cpu_baseline"]["cores"] == len(os.sched_getaffinity(0))


def test_error_record_normwise_rms_and_componentwise():
    import numpy as np
    want = np.array([[1.0, -2.0], [0.0, 4.0]])
    got = np.array([[1.5, -2.0], [0.0, 4.0]], np.float32)
    abs_prod = np.array([[4.0, 8.0], [0.0, 5.0]])  # a zero row of |A||B|: C is exactly zero there
    e = bench.error_vs_fp64(got, want, abs_prod, 2.0, 3.0)
    assert e["max_abs_over_normA_normB"] == 0.5 / 6.0
    assert abs(e["rel_rms"] - np.sqrt(0.25 / 4) / np.sqrt(21.0 / 4)) < 1e-15
    assert e["componentwise_max"] == 0.5 / 4.0
    exact = bench.error_vs_fp64(want, want, abs_prod, 2.0, 3.0)
    assert exact["max_abs_over_normA_normB"] == 0.0 and exact["componentwise_max"] == 0.0
