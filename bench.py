"""Benchmark: Strassen C = A.B at n = 16384, FP32 inputs N(0,1), 3xBF16 split
leaves on the tcgen05 tensor cores, through libstark.so.

One step = one full product (divide A and B into every leaf operand, one
leaf-product launch, and the combine of Alg. 5: fused into that launch's
epilogue, or stored by it and summed by an ordered pass; the plan measures
which is fastest, stark_plan_set_combine(-1)) on inputs already resident in
HBM.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--n 16384] [--depth 2] [--dtype bf16|tf32]

Multi-GPU (torchrun, one rank per GPU): every rank multiplies its own
independent pair of matrices (the units of this workload are independent
products), no collective on the data path; value = all ranks' flops / the
slowest rank's time ("scaling": "weak").

--impl reference times the CPU oracle (plain C, the classical FP64 triple
loop that defines the result) on the host cores, on a bounded sample of rows
of the same product per step, reported in the same unit.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# Hardware work queues for the process's streams (read when CUDA starts):
# with the default 8, streams share queues, and a copy that waits on a later
# event holds back the copies queued behind it; the host pipeline's copy-in,
# product and copy-out streams overlap only on queues of their own.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "effective TFLOP/s (2n³/t) at n=16384, stated error vs FP64; p50/p99 serve latency"
_T0 = time.perf_counter()


def progress(what):
    """One line on stderr per finished leg (the JSON line stays on stdout)."""
    _LINE["last"] = what
    print(f"[bench {time.perf_counter() - _T0:7.1f} s] {what}", file=sys.stderr, flush=True)


# The JSON line: assembled as soon as the timed product's figures exist and
# completed leg by leg; printed once, at the end, or by the watchdog when the
# run overstays its deadline (then with "incomplete" naming where it was).
_LINE = {"out": None, "printed": False, "last": "start", "lock": threading.Lock()}


def print_line(extra=None):
    with _LINE["lock"]:
        if _LINE["printed"] or _LINE["out"] is None:
            return False
        out = dict(_LINE["out"], **(extra or {}))
        print(json.dumps(out), flush=True)
        _LINE["printed"] = True
        return True


def start_watchdog(deadline_s):
    def run():
        time.sleep(max(1.0, deadline_s - (time.perf_counter() - _T0)))
        if print_line({"incomplete": f"deadline of {deadline_s:.0f} s passed after: {_LINE['last']}"}):
            progress("deadline passed: printed the line gathered so far")
            os._exit(0)
    threading.Thread(target=run, daemon=True).start()


LEAF_SOURCES = ["paper_1811_07325_gb300/csrc/leaf_tc2.cu", "paper_1811_07325_gb300/csrc/leaf_common.cuh",
                "paper_1811_07325_gb300/csrc/ptx.cuh", "paper_1811_07325_gb300/csrc/stark_internal.h"]
TRAFFIC_PROFILE = "profiles/leaf_tc2_traffic_n16384_d2_bf16.md"
PAIR_KERNEL = "leaf_tc2_kernel"


def leaf_source_hash():
    import hashlib
    h = hashlib.sha256()
    for rel in LEAF_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic(n, depth, kernel, combine=0):
    """DRAM bytes per leaf launch from the committed ncu summary, if it was
    taken on this exact kernel source, kernel, combine mode and workload;
    else None."""
    if kernel != PAIR_KERNEL:
        return None
    try:
        kv = {}
        with open(os.path.join(ROOT, TRAFFIC_PROFILE)) as f:
            for line in f:
                if ":" in line and line.startswith("- "):
                    k, v = line[2:].split(":", 1)
                    kv[k.strip()] = v.strip().strip("`")
        if kv.get("kernel_source_sha256") != leaf_source_hash():
            return None
        if int(kv.get("n", -1)) != n or int(kv.get("depth", -1)) != depth:
            return None
        key = f"traffic_bytes_per_launch.combine{combine}"
        return float(kv[key]) if key in kv else None
    except Exception:
        return None


def split_dtype(stark, name):
    return {"bf16": stark.DType.F32_SPLIT_BF16, "tf32": stark.DType.F32_SPLIT_TF32,
            "fp16": stark.DType.F32_SPLIT_FP16}[name]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "bf16": d["bf16_tflops"], "bf16_sustained": d["bf16_tflops_sustained"],
                "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(n, seed, budget_s=12.0, rows_cap=4096):
    """The oracle's classical FP64 row product on the host cores, on a bounded
    row sample of the n x n workload; eff TFLOP/s = 2 n^2 rows / t."""
    import oracle
    from paper_1811_07325_gb300 import synth
    A = synth.normal(n, seed, 0)
    B = synth.normal(n, seed, 1)
    oracle.gemm_rows(A, B, np.arange(min(4, n)))  # warm (page-in, thread pool)
    t0 = time.perf_counter()
    oracle.gemm_rows(A, B, np.arange(min(16, n)))
    per_row = (time.perf_counter() - t0) / min(16, n)
    rows = int(max(16, min(rows_cap, budget_s / max(per_row, 1e-9))))
    idx = synth.sample_rows(n, rows, seed + 1)
    t0 = time.perf_counter()
    oracle.gemm_rows(A, B, idx)
    t = time.perf_counter() - t0
    threads = min(int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)), rows)  # one row per thread at most
    return {"value": 2.0 * n * n * rows / t / 1e12, "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
            "sample": f"classical FP64 row products (C rows = A rows . B), {rows} of {n} rows, "
                      f"{t:.1f} s on {threads} OpenMP threads"}


def error_vs_fp64(got, want, abs_prod, norm_a, norm_b):
    """Error of sampled rows of C against the FP64 oracle's rows: the
    normwise max|dC| / (||A||_F ||B||_F) that the bound applies to, the
    relative RMS, and, as a diagnostic only, the componentwise
    max |dC_ij| / (|A||B|)_ij (abs_prod: the oracle's rows of |A||B|; entries
    where it is 0 are exact zeros of C and count as 0)."""
    diff = np.asarray(got, np.float64) - np.asarray(want, np.float64)
    denom = np.asarray(abs_prod, np.float64)
    comp = np.divide(np.abs(diff), denom, out=np.zeros_like(diff), where=denom > 0)
    return {"max_abs_over_normA_normB": float(np.abs(diff).max() / (norm_a * norm_b)),
            "rel_rms": float(np.sqrt(np.mean(diff ** 2)) / np.sqrt(np.mean(np.asarray(want) ** 2))),
            "componentwise_max": float(comp.max())}


def oracle_timings(seed):
    """The oracle's own times at the smaller configurations, beside the GPU:
    the classical FP64 product on all host cores (n = 1024, 4096) and on one
    core (n = 1024), and the serial FP64 Strassen recursion (Alg. 1) on one
    core (n = 1024 at depth 3, n = 2048 at depth 3), the latter scaled to
    n = 16384 at depth 6 (the same leaf side, 256) by 7^3 and labelled as
    extrapolated."""
    import oracle
    from paper_1811_07325_gb300 import synth
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"classical_cores": threads, "strassen_cores": 1}

    def timed(f):
        t0 = time.perf_counter()
        f()
        return time.perf_counter() - t0
    for n in (1024, 4096):
        A, B = synth.uniform(n, seed, 0), synth.uniform(n, seed, 1)
        t = timed(lambda: oracle.gemm_classical(A, B))
        out[f"classical_n{n}_s"] = t
        out[f"classical_n{n}_tflops"] = 2.0 * n ** 3 / t / 1e12
    # one core: a child process, so that OpenMP starts with a single thread
    code = ("import time, oracle\nfrom paper_1811_07325_gb300 import synth\n"
            f"A, B = synth.uniform(1024, {int(seed)}, 0), synth.uniform(1024, {int(seed)}, 1)\n"
            "t0 = time.perf_counter()\noracle.gemm_classical(A, B)\nprint(time.perf_counter() - t0)\n")
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=dict(os.environ, OMP_NUM_THREADS="1"),
                           capture_output=True, text=True, timeout=900)
        if r.returncode == 0:
            t = float(r.stdout.split()[-1])
            out["classical_n1024_1core_s"] = t
            out["classical_n1024_1core_tflops"] = 2.0 * 1024 ** 3 / t / 1e12
    except (subprocess.SubprocessError, OSError, ValueError, IndexError):
        pass  # the bench line stands without this figure
    for n in (1024, 2048):
        A, B = synth.uniform(n, seed, 0), synth.uniform(n, seed, 1)
        t = timed(lambda: oracle.strassen(A, B, 3))
        out[f"strassen_n{n}_d3_s"] = t
        out[f"strassen_n{n}_d3_effective_tflops"] = 2.0 * n ** 3 / t / 1e12
    out["strassen_n16384_d6_s_extrapolated"] = out["strassen_n2048_d3_s"] * 7 ** 3
    return out


def link_bandwidth(torch, A_h, B_h, A, B, C, C_h, e2e_s):
    """Host link measured in the same process as the end-to-end leg: plain
    pinned copies of one step's inputs (host->device, 2 n^2 floats) and of
    its result (device->host, n^2 floats), each timed alone with CUDA events
    (best of 3).  The end-to-end step cannot beat the link: at best the two
    directions overlap each other and the product (bound = the larger copy
    time), at worst they take turns (bound = their sum)."""
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def best(f):
        ts = []
        for _ in range(3):
            torch.cuda.synchronize()
            e0.record(s)
            f()
            e1.record(s)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e-3)
        return min(ts)
    t_in = best(lambda: (A.copy_(A_h, non_blocking=True), B.copy_(B_h, non_blocking=True)))
    t_out = best(lambda: C_h.copy_(C, non_blocking=True))
    b_in = A_h.numel() * A_h.element_size() + B_h.numel() * B_h.element_size()
    b_out = C.numel() * C.element_size()
    overlap, serial = max(t_in, t_out), t_in + t_out
    return {"link_h2d_gbs": b_in / t_in / 1e9, "link_d2h_gbs": b_out / t_out / 1e9,
            "link_bound_ms_overlapped": overlap * 1e3, "link_bound_ms_serial": serial * 1e3,
            "frac_of_link_bound_overlapped": overlap / e2e_s, "frac_of_link_bound_serial": serial / e2e_s}


def run_depth_sweep(args, stark, synth, torch, A, B):
    """The bench product at depths 0 (one classical 3xBF16 product through
    the same leaf kernel) to 3 with the default combine, with the
    deterministic combine at depths 2 and 3 and with the sibling-folded
    combine at depths 1 to 3: ms per product, effective TFLOP/s and the
    phases."""
    n = args.n
    C = torch.empty_like(A)
    out = {"n": n, "dtype": args.dtype}
    runs = [(d, 0) for d in range(4)] + [(2, 2), (3, 2), (1, 3), (2, 3), (3, 3)]
    for d, combine in runs:
        key = f"d{d}" + ("" if combine == 0 else f"_combine{combine}")
        try:
            with stark.Plan(n, d, stark.DType.F32_SPLIT_BF16) as p:
                if combine:
                    p.set_combine(combine)
                for _ in range(2):
                    p.mul(A, B, C)
                p.check()
                p.set_timing(5)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(5):
                    p.mul(A, B, C)
                e1.record()
                torch.cuda.synchronize()
                p.check()
                ms = e0.elapsed_time(e1) / 5
                out[key] = {"ms": ms, "tflops": 2.0 * n ** 3 / (ms * 1e-3) / 1e12, "phases_ms": p.phase_ms(),
                            "leaf": p.leaf, "leaves": p.leaves, "workspace_bytes": p.workspace_bytes}
        except stark.StarkError as e:
            out[key] = {"error": str(e)}
        torch.cuda.empty_cache()
    del C
    torch.cuda.empty_cache()
    return out


def run_batch(args, stark, synth, torch):
    """Batched form: 64 products, n drawn from {512, ..., 4096}, FP32 U[-1,1],
    3xBF16, autotuned depth; one grouped graph-replayed launch per step,
    compared with the same products issued one by one."""
    sizes = synth.batch_sizes(args.batch_count, args.seed + 11)
    As = [torch.from_numpy(synth.uniform(n, args.seed + 100 + i, 0, dtype=np.float32)).cuda()
          for i, n in enumerate(sizes)]
    Bs = [torch.from_numpy(synth.uniform(n, args.seed + 100 + i, 1, dtype=np.float32)).cuda()
          for i, n in enumerate(sizes)]
    Cs = [torch.empty((n, n), device="cuda") for n in sizes]
    flops = sum(2.0 * n ** 3 for n in sizes)
    t_create = time.perf_counter()
    bt = stark.Batch(sizes, -1, stark.DType.F32_SPLIT_BF16)
    t_create = time.perf_counter() - t_create
    progress(f"batch created and tuned in {t_create:.1f} s")
    for _ in range(3):
        bt.mul(As, Bs, Cs)
    bt.check()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    e0.record()
    for _ in range(reps):
        bt.mul(As, Bs, Cs)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    info = bt.info()
    depths = bt.depths()
    bt.close()
    # the same products one plan at a time (no grouping, no graph)
    plans = {}
    for n, d in zip(sizes, depths):
        if n not in plans:
            plans[n] = stark.Plan(n, d, stark.DType.F32_SPLIT_BF16)
    for i, n in enumerate(sizes):
        plans[n].mul(As[i], Bs[i], Cs[i])
    torch.cuda.synchronize()
    e0.record()
    for _ in range(3):
        for i, n in enumerate(sizes):
            plans[n].mul(As[i], Bs[i], Cs[i])
    e1.record()
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1) / 3
    for p in plans.values():
        p.close()
    return {"workload": f"{len(sizes)} products, n in {{512..4096}} (seeded), fp32 U[-1,1], 3xbf16, autotuned depth",
            "value": flops / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_batch": ms,
            "one_by_one_tflops": flops / (ms_seq * 1e-3) / 1e12, "depths": depths, "tile_n": info["tile_n"],
            "work_items": info["work_items"], "create_and_autotune_s": t_create,
            "graph_replays": info["graph_replays"]}


def run_peel(args, stark, synth, torch):
    """Sizes just above a multiple of the tile granularity: padding to the next
    multiple against peeling the edge (STARK_PLAN_PEEL), depth 2, 3xBF16."""
    out = {"depth": 2}
    for n in (4097, 16385):
        A = torch.from_numpy(synth.normal(n, args.seed + 5, 0)).cuda()
        B = torch.from_numpy(synth.normal(n, args.seed + 5, 1)).cuda()
        C = torch.empty_like(A)
        row = {}
        for label, peel in (("pad", False), ("peel", True)):
            with stark.Plan(n, 2, stark.DType.F32_SPLIT_BF16, peel=peel) as p:
                for _ in range(2):
                    p.mul(A, B, C)
                p.check()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(5):
                    p.mul(A, B, C)
                e1.record()
                torch.cuda.synchronize()
                p.check()
                ms = e0.elapsed_time(e1) / 5
                row[label] = {"ms": ms, "tflops": 2.0 * n ** 3 / (ms * 1e-3) / 1e12, "recursion_side": p.n_pad,
                              "edge": p.peel}
        out[f"n{n}"] = row
        del A, B, C
        torch.cuda.empty_cache()
    return out


def run_traversal(args, stark, synth, torch, A, B):
    """The bench product depth first over the top 1 and 2 levels (smaller
    workspace, one subtree's operands at a time) beside breadth first."""
    out = {"n": args.n, "depth": args.depth}
    C = torch.empty_like(A)
    for levels in (0, 1, 2):
        with stark.Plan(args.n, args.depth, stark.DType.F32_SPLIT_BF16) as p:
            try:
                p.set_traversal(levels)
            except stark.StarkError as e:
                out[f"levels{levels}"] = {"unsupported": str(e)}
                continue
            for _ in range(2):
                p.mul(A, B, C)
            p.check()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(5):
                p.mul(A, B, C)
            e1.record()
            torch.cuda.synchronize()
            p.check()
            ms = e0.elapsed_time(e1) / 5
            out[f"levels{levels}"] = {"ms": ms, "tflops": 2.0 * args.n ** 3 / (ms * 1e-3) / 1e12,
                                      "workspace_bytes": p.workspace_bytes}
    del C
    torch.cuda.empty_cache()
    return out


def run_serve(args, stark, synth, torch):
    """Served form: Poisson arrivals at 200 req/s (the workload) and, as a
    rate sweep toward capacity, at 2000 and 8000 req/s; n log-uniform in
    [256, 8192], FP32 N(0,1), 3xBF16, device budget 150 GB, 4 stream slots.
    Latency of a request runs from its scheduled arrival to the dispatcher's
    observation of its completion: the host's delay from the scheduled time
    to the return of the submit call plus the server's own submit-to-
    completion time (an over-estimate by the length of the call).  Output
    buffers are allocated before any clock starts; a first pass at 200 req/s
    warms the workspace cache (not measured)."""
    count = args.serve_requests
    sizes = synth.loguniform_sizes(count, args.seed + 21, 256, 8192)
    nmax = max(sizes)
    poolA = torch.from_numpy(synth.normal(nmax, args.seed + 22, 0)).cuda().reshape(-1)
    poolB = torch.from_numpy(synth.normal(nmax, args.seed + 22, 1)).cuda().reshape(-1)
    As = [poolA[:n * n].view(n, n) for n in sizes]
    Bs = [poolB[:n * n].view(n, n) for n in sizes]
    Cs = [torch.empty((n, n), device="cuda") for n in sizes]
    flops = sum(2.0 * n ** 3 for n in sizes)
    srv = stark.Server(150 * 10 ** 9, slots=4)

    def one_pass(gaps):
        ids, late = [], []
        torch.cuda.synchronize()
        start = time.perf_counter()
        t = start
        for i, g in enumerate(gaps):
            t += g
            while True:
                now = time.perf_counter()
                if now >= t:
                    break
                if t - now > 0.0003:
                    time.sleep(t - now - 0.0002)
            ids.append(srv.submit(As[i], Bs[i], Cs[i]))
            late.append(time.perf_counter() - t)  # scheduled arrival -> submit returned
        srv.drain()
        wall = time.perf_counter() - start
        lat = []
        for rid, lt in zip(ids, late):
            done, st = srv.poll(rid)
            assert done and st == stark.Status.OK, st
            lat.append(srv.latency(rid) + lt)
        return np.array(lat), wall

    one_pass(synth.exponential_gaps(count, args.seed + 23, 200.0))  # warm the workspace cache
    progress("serve warm-up pass done")
    sweep = []
    for k, rate in enumerate((200.0, 2000.0, 8000.0)):
        before = srv.load()
        lat, wall = one_pass(synth.exponential_gaps(count, args.seed + 24 + k, rate))
        progress(f"serve pass at {rate:.0f} req/s done")
        after = srv.load()
        sweep.append({"rate_per_s": rate, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                      "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
                      "aggregate_tflops": flops / wall / 1e12, "offered_tflops": flops / (count / rate) / 1e12,
                      "wall_s": wall, "max_queued": after["max_queued"],
                      "deferred_admissions": after["deferred"] - before["deferred"]})
    stats = srv.stats()
    srv.close()
    base = sweep[0]
    return {"workload": f"Poisson 200 req/s, {count} requests, n log-uniform [256, 8192], fp32 N(0,1), 3xbf16, "
                        f"budget 150 GB, 4 slots; latency from scheduled arrival",
            "p50_ms": base["p50_ms"], "p99_ms": base["p99_ms"], "mean_ms": base["mean_ms"],
            "aggregate_tflops": base["aggregate_tflops"], "offered_tflops": base["offered_tflops"],
            "wall_s": base["wall_s"], "rate_sweep": sweep,
            "cached_workspaces": stats["cached_workspaces"], "workspace_bytes": stats["owned_bytes"]}


def run_sharded(args, stark, synth, torch, dist, rank, world, local):
    """--shard: ONE n x n product split over the ranks (the paper's setting,
    Sec. III-C / V-F): every rank holds A and B, a plan restricted to its
    balanced leaf range (its own subtrees' divide and workspace), computes
    its partial C, and one NCCL sum reduce-scatter leaves it its block of
    rows of C.  A step is the whole product (local leaves + the exchange);
    value = 2 n^3 / the slowest rank's time ("scaling": "strong")."""
    from paper_1811_07325_gb300 import shard
    n, d = args.n, args.depth
    dt = split_dtype(stark, args.dtype)
    A = torch.from_numpy(synth.normal(n, args.seed, 0)).cuda()
    B = torch.from_numpy(synth.normal(n, args.seed, 1)).cuda()
    plan = shard.shard_plan(n, d, dt, world, rank)
    b, e = getattr(plan, "shard", None) or (0, plan.leaves)

    def step():
        if dist is None:
            return 0, n, plan.mul_leaves(A, B, b, e)
        return shard.mul_sharded_rows(plan, A, B)

    def barrier():
        if dist is not None:
            dist.barrier()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    plan.check()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        r0, r1, rows = step()
    e1.record()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    plan.check()
    ms = e0.elapsed_time(e1) / args.steps
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    error = None
    if rank == 0 and not args.no_check and r1 > r0:
        import oracle
        idx = np.unique(synth.sample_rows(r1 - r0, min(64, r1 - r0), args.seed + 5))
        Ah, Bh = A.cpu().numpy(), B.cpu().numpy()
        want = oracle.gemm_rows(Ah, Bh, idx + r0)
        absprod = oracle.gemm_rows(np.abs(Ah), np.abs(Bh), idx + r0)
        got = rows[torch.from_numpy(idx).cuda()].double().cpu().numpy()
        an = float(torch.linalg.vector_norm(A.double()).item())
        bn = float(torch.linalg.vector_norm(B.double()).item())
        error = dict(error_vs_fp64(got, want, absprod, an, bn), rows_checked=int(idx.size))
    flops = 2.0 * n ** 3
    return {"metric": METRIC, "value": flops / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": f"strassen n={n} depth={d} fp32 N(0,1) split-{args.dtype}, one product "
                                   f"sharded over {world} ranks (leaf ranges, NCCL reduce-scatter of C rows)",
                       "n": n, "depth": d, "leaves": plan.leaves, "rank0_leaves": [b, e],
                       "rank0_workspace_bytes": plan.workspace_bytes, "collective": "reduce_scatter" if world > 1
                       else "none (one rank)"},
            "clocks": clocks, "error_vs_fp64": error, "e2e": None,
            "note": "strong scaling of one product; the default bench line runs independent products per rank"}


def workload_config(args, depth):
    n = args.n
    promo = f", accumulator promotion every {args.promotion} of K" if getattr(args, "promotion", 0) else ""
    return {"workload": f"strassen n={n} depth={depth} fp32 N(0,1) split-{args.dtype}{promo}", "n": n, "depth": depth,
            "per_rank": "one independent product per rank",
            "l2": "inputs (2 x 1 GiB) and workspace larger than L2; no flush needed"}


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle, timed on the host cores, rank 0 only."""
    if rank != 0:
        return None
    if world > 1:
        # the launcher gives every rank one OpenMP thread; rank 0 alone works
        # here, so it takes the host's cores (set before the oracle's OpenMP
        # runtime loads)
        os.environ["OMP_NUM_THREADS"] = str(len(os.sched_getaffinity(0)))
    import oracle
    from paper_1811_07325_gb300 import synth
    n = args.n
    A = synth.normal(n, args.seed, 0)
    B = synth.normal(n, args.seed, 1)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    # the oracle spreads rows over its OpenMP threads: one row per thread by default
    rows_per_step = max(1, min(n, args.ref_rows if args.ref_rows > 0 else threads))
    cores = min(threads, rows_per_step)
    for w in range(args.warmup):
        oracle.gemm_rows(A, B, (np.arange(rows_per_step) + w * rows_per_step) % n)
    times = []
    for k in range(args.steps):
        idx = (np.arange(rows_per_step) + k * rows_per_step) % n
        t0 = time.perf_counter()
        oracle.gemm_rows(A, B, idx)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    value = 2.0 * n * n * rows_per_step / t / 1e12
    sample = f"classical FP64 oracle, {rows_per_step} of {n} rows of C per step on {cores} OpenMP threads"
    return {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(args, args.depth), reference_arm="CPU oracle (classical FP64), "
                           "row-sampled: each step computes a bounded sample of rows of this product"),
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--depth", type=int, default=2)
    ap.add_argument("--dtype", default="bf16", choices=["bf16", "tf32", "fp16"])
    ap.add_argument("--seed", type=int, default=2024)
    ap.add_argument("--e2e-steps", type=int, default=36)
    ap.add_argument("--ref-rows", type=int, default=0,
                    help="--impl reference: rows of C per step (0: one per OpenMP thread)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-comparators", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-tf32", action="store_true")
    ap.add_argument("--pairing", type=int, default=-1,
                    help="leaf schedule: 0 single CTAs, 2 cta_group::2 pairs")
    ap.add_argument("--combine", type=int, default=-1,
                    help="combine mode: 0 fused, 2 deterministic, 3 sibling fold, -1 the fastest, measured")
    ap.add_argument("--deep-pipeline", type=int, default=-1)
    ap.add_argument("--raster", type=int, default=-1, help="leaf tile raster band (0: row-major)")
    ap.add_argument("--traversal", type=int, default=0, help="k > 0: depth first over the top k levels")
    ap.add_argument("--promotion", type=int, default=0,
                    help="accumulator promotion of the main plan every K of the leaf side (0: off)")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--deadline", type=float, default=900.0,
                    help="seconds after which the line gathered so far is printed and the run ends")
    ap.add_argument("--shard", action="store_true",
                    help="one product sharded over the ranks: leaf ranges + NCCL reduce-scatter (strong scaling)")
    ap.add_argument("--no-oracle-timings", action="store_true")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--serve-requests", type=int, default=600)
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return

    if rank == 0:
        start_watchdog(args.deadline)
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1811_07325_gb300 import stark, synth

    n, d = args.n, args.depth
    dt = split_dtype(stark, args.dtype)
    if args.shard:
        out = run_sharded(args, stark, synth, torch, dist, rank, world, local)
        if rank == 0:
            print(json.dumps(out), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return
    seed = args.seed + 7919 * rank  # independent product per rank
    A_h = torch.from_numpy(synth.normal(n, seed, 0)).pin_memory()
    B_h = torch.from_numpy(synth.normal(n, seed, 1)).pin_memory()
    A = A_h.cuda()
    B = B_h.cuda()
    C = torch.empty_like(A)
    plan = stark.Plan(n, d, dt)
    if args.pairing >= 0:
        plan.set_pairing(args.pairing)
    if args.combine:
        plan.set_combine(args.combine)
    if args.deep_pipeline >= 0:
        plan.set_pipeline(bool(args.deep_pipeline))
    if args.raster >= 0:
        plan.set_raster(args.raster)
    if args.traversal:
        plan.set_traversal(args.traversal)
    if args.promotion:
        plan.set_promotion(args.promotion)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        plan.mul(A, B, C)
    plan.check()

    progress(f"plan ready (combine mode {plan.combine}), warm-up done")
    # ---------------------------------------------------------------- timed region
    plan.set_timing(args.steps)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    launches0 = stark.launch_count()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        plan.mul(A, B, C)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    launches = stark.launch_count() - launches0
    plan.check()
    ms = ev0.elapsed_time(ev1) / args.steps
    phases = plan.phase_ms()
    plan.set_timing(0)
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    flops = 2.0 * n ** 3
    value = world * flops / (ms * 1e-3) / 1e12

    progress("timed region done")
    # ---------------------------------------------------------------- error vs FP64
    error = None
    abs_prod = None  # the oracle's sampled rows of |A||B|, shared by the error checks
    if not args.no_check and rank == 0:
        import oracle
        rows = synth.sample_rows(n, 256, args.seed + 5)
        want = oracle.gemm_rows(A_h.numpy(), B_h.numpy(), rows)
        abs_prod = oracle.gemm_rows(np.abs(A_h.numpy()), np.abs(B_h.numpy()), rows)
        # the FP64 reductions on the GPU (stark_error_norms): norms of A, B
        # and the error of the sampled rows against the oracle's
        rep = stark.error_norms(A, B, C, rows, want, abs_prod)
        error = {"max_abs_over_normA_normB": rep["max_abs_over_normA_normB"], "rel_rms": rep["rel_rms"],
                 "componentwise_max": rep["max_componentwise"], "rows_checked": int(rows.size),
                 "reference": "oracle classical FP64 rows", "bound": 1e-6,
                 "reduced_by": "stark_error_norms (FP64 on the GPU)"}
        # anchor for "FP32-level": one classical FP32 product (cuBLAS SGEMM,
        # TF32 off) judged the same way on the same rows
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
        c32 = torch.matmul(A, B)
        torch.backends.cuda.matmul.allow_tf32 = prev
        r32 = stark.error_norms(A, B, c32, rows, want, abs_prod)
        error["fp32_classical"] = {"max_abs_over_normA_normB": r32["max_abs_over_normA_normB"],
                                   "rel_rms": r32["rel_rms"], "componentwise_max": r32["max_componentwise"]}
        del c32
        torch.cuda.empty_cache()

    progress("error vs FP64 done")
    # ---------------------------------------------------------------- end to end (host buffers)
    # every step copies its inputs host->device and its result device->host
    # (pinned buffers); the asynchronous entry point overlaps one step's
    # copies with the neighbouring steps' products.  The host link sometimes
    # runs a round's first copies at 15-25 GB/s for 50-140 ms before every
    # copy returns to ~200 GB/s; rounds of 36 products keep that start from
    # dominating the per-product time
    C_hs = [torch.empty((n, n), dtype=torch.float32).pin_memory() for _ in range(2)]
    plan.mul_host(A_h, B_h, C_hs[0])
    rounds = []
    for _ in range(3):  # three rounds of e2e_steps products; the median round is reported
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            plan.mul_host_enqueue(A_h, B_h, C_hs[k % 2])
        plan.host_wait()
        torch.cuda.synchronize()
        rounds.append((time.perf_counter() - t0) / args.e2e_steps)
    plan.check()
    e2e_s = statistics.median(rounds)
    if dist is not None:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": world * flops / e2e_s / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": 2 * n * n * 4,
           "d2h_bytes_per_step": n * n * 4, "ms_per_step": e2e_s * 1e3, "steps": args.e2e_steps,
           "rounds_ms_per_step": [r * 1e3 for r in rounds],
           "cuda_device_max_connections": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS"),
           "api": "stark_mul_host_enqueue + stark_plan_host_wait (pinned host buffers, copies overlapped with the neighbouring products)"}
    e2e.update(link_bandwidth(torch, A_h, B_h, A, B, C, C_hs[0], e2e_s))

    progress("end to end done")
    # ---------------------------------------------------------------- roofline of the leaf kernel
    pk = peaks()
    leaf_flops = 3 * 2.0 * plan.leaves * plan.leaf ** 3  # three bf16 products per leaf
    achieved = leaf_flops / (phases["leaf_kernel"] * 1e-3) / 1e12
    pair_mode = args.pairing if args.pairing >= 0 else 2
    kernel = PAIR_KERNEL if (pair_mode == 2 and plan.leaf % 256 == 0 and args.deep_pipeline != 1) \
        else "leaf_tc_kernel"
    # the leaf launch lasts ~10-20 ms inside a timed region of well under a
    # second at full clocks: the burst peak is its denominator; the sustained
    # (power-capped, seconds-long) figure is kept beside it
    epilogue = {0: "fused combine", 1: "fused combine (atomics)", 2: "stores each M_l; an ordered pass combines",
                3: "folds siblings into parent planes; an ordered pass combines one level up"}[plan.combine]
    roofline = {"kernel": f"{kernel} (3xBF16 leaf GEMMs; epilogue {epilogue})", "bound": "tensor",
                "achieved": achieved, "peak": pk["bf16"], "unit": "TFLOP/s",
                "frac": achieved / pk["bf16"], "traffic": measured_traffic(n, plan.depth, kernel, plan.combine),
                "peak_source": f"{pk['source']} bf16 burst",
                "peak_sustained": pk["bf16_sustained"], "frac_of_sustained": achieved / pk["bf16_sustained"],
                "algorithmic_flops_per_launch": leaf_flops,
                "launch_ms": phases["leaf_kernel"]}
    esz = 8 if args.dtype == "tf32" else 4  # bytes per leaf element per operand (hi + lo)
    operand_bytes = 2 * plan.leaves * plan.leaf ** 2 * esz
    divide_bytes = 2 * (n * n * 4) + operand_bytes  # read A, B; write every leaf operand (hi+lo)
    # the combine's HBM bytes: fused, C cleared and written once (the L2
    # reductions in between are not algorithmic); stored, the planes written
    # by the leaf kernel and read by the pass, C written once
    planes = {2: plan.leaves * plan.leaf ** 2 * 4, 3: plan.leaves // 7 * (2 * plan.leaf) ** 2 * 4}.get(plan.combine, 0)
    combine_bytes = (2 * planes + n * n * 4) if planes else 2 * n * n * 4
    combine_pass = None
    if planes:
        combine_pass = {"kernel": "combine_kernel (ordered pass)", "bound": "hbm", "ms": phases["after_leaf"],
                        "algorithmic_bytes": planes + n * n * 4,
                        "achieved_gbs": (planes + n * n * 4) / (phases["after_leaf"] * 1e-3) / 1e9,
                        "peak_gbs": pk["hbm_gbs"]}
        combine_pass["frac"] = combine_pass["achieved_gbs"] / pk["hbm_gbs"]
    # the whole path's roofline (phases serialize): leaf flops at the tensor
    # peak + divide and combine bytes at HBM bandwidth
    t_roof = leaf_flops / (pk["bf16"] * 1e12) + (divide_bytes + combine_bytes) / (pk["hbm_gbs"] * 1e9)
    path_roofline = {"t_roof_ms": t_roof * 1e3, "t_ms": ms, "frac": t_roof * 1e3 / ms,
                     "effective_tflops_at_roof": flops / t_roof / 1e12,
                     "effective_over_bf16_peak": value / world / pk["bf16"],
                     "model": "leaf 3*2*L^3*7^d flops / bf16 burst + (divide bytes + combine bytes) / HBM; "
                              "combine bytes: C cleared and written (fused) or planes written, read and C written"}

    if rank == 0:
        _LINE["out"] = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype,
            "dtype_detail": f"fp32 in/out; 3x{args.dtype} split tensor-core leaf products, fp32 accumulate; "
                            "fp32 divide sums and combine",
            "data": "synthetic",
            "config": dict(workload_config(args, plan.depth), leaves=plan.leaves, leaf=plan.leaf,
                           tile=list(plan.tile), combine=plan.combine,
                           combine_choice="measured per plan" if args.combine == -1 else "given"),
            "gpu_launches": launches, "clocks": clocks, "e2e": e2e, "roofline": roofline,
            "phases_ms": phases, "divide_algorithmic_bytes": divide_bytes,
            "divide_gbs": divide_bytes / (phases["divide"] * 1e-3) / 1e9, "path_roofline": path_roofline,
            "error_vs_fp64": error, "combine_pass": combine_pass}
    line = _LINE["out"] if rank == 0 else {}

    comparators = None
    if not args.no_comparators and rank == 0:
        comparators = {}
        for name, tdt in (("torch_matmul_bf16", torch.bfloat16), ("torch_matmul_fp32", torch.float32)):
            prev = torch.backends.cuda.matmul.allow_tf32
            torch.backends.cuda.matmul.allow_tf32 = False
            a, b = A.to(tdt), B.to(tdt)
            torch.matmul(a, b)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            reps = 3
            for _ in range(reps):
                torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            comparators[name] = flops / (e0.elapsed_time(e1) / reps * 1e-3) / 1e12
            torch.backends.cuda.matmul.allow_tf32 = prev
            del a, b
        torch.cuda.empty_cache()
        try:
            a64, b64 = A.double(), B.double()
            p64 = stark.Plan(n, 3, stark.DType.F64)
            c64 = torch.empty_like(a64)
            p64.mul(a64, b64, c64)
            p64.check()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            p64.mul(a64, b64, c64)
            e1.record()
            torch.cuda.synchronize()
            comparators["strassen_fp64_d3"] = flops / (e0.elapsed_time(e1) * 1e-3) / 1e12
            p64.close()
            e0.record()
            torch.matmul(a64, b64)
            e1.record()
            torch.cuda.synchronize()
            comparators["torch_matmul_fp64"] = flops / (e0.elapsed_time(e1) * 1e-3) / 1e12
            del a64, b64, c64
        except Exception as ex:  # report, do not hide
            comparators["fp64_error"] = str(ex)
        comparators["unit"] = "effective TFLOP/s (2n^3/t), same GPU"

    line["comparators"] = comparators
    progress("comparators done")
    tf32 = fp16 = None
    if rank == 0 and not args.no_tf32 and args.dtype == "bf16":
        # the same product with 3xTF32 and with 3xFP16 leaves, each also with
        # accumulator promotion every 256 of K (one tensor-core accumulation
        # then spans 256 instead of the leaf side)
        del C
        torch.cuda.empty_cache()
        C32 = torch.empty_like(A)
        if not args.no_check:
            import oracle
            rows = synth.sample_rows(n, 256, args.seed + 5)
            want = oracle.gemm_rows(A_h.numpy(), B_h.numpy(), rows)
            if abs_prod is None:
                abs_prod = oracle.gemm_rows(np.abs(A_h.numpy()), np.abs(B_h.numpy()), rows)

        def split_leg(p32, promotion):
            p32.set_promotion(promotion)
            for _ in range(2):
                p32.mul(A, B, C32)
            p32.check()
            p32.set_timing(5)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(5):
                p32.mul(A, B, C32)
            e1.record()
            torch.cuda.synchronize()
            p32.check()
            ms32 = e0.elapsed_time(e1) / 5
            leg = {"value": flops / (ms32 * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms32,
                   "phases_ms": p32.phase_ms(), "combine": p32.combine}
            p32.set_timing(0)
            if not args.no_check:
                r = stark.error_norms(A, B, C32, rows, want, abs_prod)
                leg["error_vs_fp64"] = {"max_abs_over_normA_normB": r["max_abs_over_normA_normB"],
                                        "rel_rms": r["rel_rms"], "componentwise_max": r["max_componentwise"]}
            return leg

        legs = {}
        for name in ("tf32", "fp16"):
            p32 = stark.Plan(n, d, split_dtype(stark, name))
            try:
                p32.set_combine(plan.combine)  # the main line's combine mode
                legs[name] = split_leg(p32, 0)
                for kc in ((256, 512) if name == "fp16" else (256,)):
                    try:
                        legs[name][f"promoted_k{kc}"] = split_leg(p32, kc)
                    except stark.StarkError as ex:  # report, do not hide
                        legs[name][f"promoted_k{kc}"] = str(ex)
            except stark.StarkError as ex:
                legs[name] = str(ex)
            p32.close()
            torch.cuda.empty_cache()
        tf32, fp16 = legs["tf32"], legs["fp16"]
        del C32
        torch.cuda.empty_cache()

    line["tf32"] = tf32
    line["fp16"] = fp16
    progress("tf32 leg done")
    int64 = None
    if rank == 0 and not args.no_batch:
        # integer form (n = 4096, entries in [-16, 16]): exact int64 Strassen on
        # the bf16 tensor cores (declared bound) and on the CUDA cores
        ni = 4096
        Ai = torch.from_numpy(synth.integers(ni, args.seed + 31, 0, -16, 16)).cuda()
        Bi = torch.from_numpy(synth.integers(ni, args.seed + 31, 1, -16, 16)).cuda()
        Ci = torch.empty_like(Ai)
        int64 = {"workload": "n=4096 int64 U{-16..16}, exact (bit-identical to the oracle in the tests)"}
        for label, d, bound, reps in (("tensor_core_d1", 1, 16, 10), ("tensor_core_d2", 2, 16, 10),
                                      ("cuda_core_d2", 2, 0, 2)):
            pi = stark.Plan(ni, d, stark.DType.I64)
            if bound:
                pi.set_input_bound(bound)
            pi.mul(Ai, Bi, Ci)
            pi.check()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                pi.mul(Ai, Bi, Ci)
            e1.record()
            torch.cuda.synchronize()
            pi.check()
            msi = e0.elapsed_time(e1) / reps
            int64[label] = {"ms": msi, "effective_tops": 2.0 * ni ** 3 / (msi * 1e-3) / 1e12}
            pi.close()
        del Ai, Bi, Ci
        torch.cuda.empty_cache()

    batch = serve = None
    if rank == 0 and not args.no_batch:
        line["int64"] = int64
        progress("int64 leg done")
        batch = line["batch"] = run_batch(args, stark, synth, torch)
        progress("batch leg done")
    if rank == 0 and not args.no_serve:
        serve = line["serve"] = run_serve(args, stark, synth, torch)
        progress("serve leg done")
    peel = None
    traversal = None
    depth_sweep = None
    if rank == 0 and not args.no_batch:
        peel = line["peel"] = run_peel(args, stark, synth, torch)
        progress("peel leg done")
        if args.dtype == "bf16" and args.depth <= 3:
            traversal = line["traversal"] = run_traversal(args, stark, synth, torch, A, B)
            progress("traversal leg done")
        if args.dtype == "bf16":
            depth_sweep = line["depth_sweep"] = run_depth_sweep(args, stark, synth, torch, A, B)
            progress("depth sweep done")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = line["cpu_baseline"] = cpu_baseline(n, args.seed)
        progress("cpu baseline done")
        if not args.no_oracle_timings:
            cpu["oracle_timings"] = oracle_timings(args.seed)
            progress("oracle timings done")

    if rank == 0:
        print_line()
    plan.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
