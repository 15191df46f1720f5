"""Seeded sweep of random plan configurations against the CPU oracle.

Each case draws a size, depth, dtype and a combination of plan options
(combine mode, leaf schedule, raster, traversal, edge peeling, tf32 B
layout), runs one product through the C ABI and compares every element with
the oracle: bit-exact for int64, the split-precision bound for fp32, the
Higham bound for fp64.  Options that do not apply to a draw (e.g. a tf32
layout on a bf16 plan) are left at their defaults.
"""
import random

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bounds  # noqa: E402
import oracle  # noqa: E402
from paper_1811_07325_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu



def draw(rng):
    dtype = rng.choice(["F32_SPLIT_BF16", "F32_SPLIT_BF16", "F32_SPLIT_TF32", "F64", "I64"])
    n = rng.choice([1, 17, 64, 130, 257, 300, 513, 700, 777, 1024, 1100, 1300, 1500])
    d = rng.randint(0, 3)
    opts = {
        "peel": rng.random() < 0.3,
        "combine": rng.choice([0, 3, 1, 2]) if dtype.startswith("F32") else 0,
        "pairing": rng.choice([0, 0, 2, 2]) if dtype.startswith("F32") else 2,
        "raster": rng.choice([0, 0, 2, 4]),
        "dfs": rng.random() < 0.3 and d >= 1,
        "tf32_mn": rng.random() < 0.7,
        "bound": dtype == "I64" and rng.random() < 0.5,
    }
    return dtype, n, d, opts


def draw_fp16(rng):
    # 3xFP16 leaves, with accumulator promotion where the draw allows it
    dtype, n, d, opts = draw(rng)
    opts["promotion"] = rng.choice([0, 256, 512])
    opts["tf32_mn"] = True
    return "F32_SPLIT_FP16", n, d, dict(opts, bound=False, combine=rng.choice([0, 3, 1, 2]),
                                        pairing=rng.choice([0, 2, 2]))


CASES = [draw(random.Random(1000 + k)) for k in range(120)] + \
        [draw_fp16(random.Random(3000 + k)) for k in range(40)]


@pytest.mark.parametrize("k", range(len(CASES)))
def test_random_configuration(stark_lib, k):
    S = stark_lib
    dtype, n, d, o = CASES[k]
    if dtype == "I64":
        A = synth.integers(n, 500 + k, 0, -16, 16)
        B = synth.integers(n, 500 + k, 1, -16, 16)
    elif dtype == "F64":
        A = synth.uniform(n, 500 + k, 0)
        B = synth.uniform(n, 500 + k, 1)
    else:
        A = synth.normal(n, 500 + k, 0)
        B = synth.normal(n, 500 + k, 1)
    want = oracle.gemm_classical(A, B) if dtype == "I64" else \
        oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    with S.Plan(n, d, S.DType[dtype], peel=o["peel"]) as p:
        if o["bound"] and (p.leaf % 128 == 0):
            try:
                p.set_input_bound(16)
            except S.StarkError:
                pass  # bound outside the exact range at this depth: CUDA-core path
        if o["combine"] and p.depth <= 3:
            try:
                p.set_combine(o["combine"])
            except S.StarkError as e:
                # the sibling fold needs depth >= 1 and a leaf side that is a
                # multiple of 256 (and, for 3xTF32, the MN-major layout)
                assert o["combine"] == 3 and e.status == S.Status.EUNSUPPORTED, e
        p.set_pairing(o["pairing"])
        p.set_raster(o["raster"])
        if dtype == "F32_SPLIT_TF32":
            p.set_tf32_layout(o["tf32_mn"])
        if o["dfs"] and o["combine"] < 2:
            p.set_traversal(True)
        kc = 0
        if o.get("promotion") and o["pairing"] == 2:
            try:
                p.set_promotion(o["promotion"])
                kc = o["promotion"]
            except S.StarkError as e:
                # promotion runs on the CTA-pair kernel: leaf side a multiple
                # of 256, and not with the sibling fold
                assert e.status == S.Status.EUNSUPPORTED, e
        C = p.mul(dA, dB).cpu().numpy()
        p.check()
        L = p.leaf
        d_used, peeled = p.depth, p.peel > 0
    if dtype == "I64":
        assert np.array_equal(C, want), (dtype, n, d, o)
        return
    diff = C.astype(np.float64) - want
    if dtype == "F64":
        u = 2.0 ** -53
        Lc = -(-n // 2 ** d)
        bound = 2 * ((12 ** d * (Lc * Lc + 5 * Lc) - 5 * n) + n) * u * np.abs(A).max() * np.abs(B).max()
        assert np.abs(diff).max() <= bound, (n, d, o)
        return
    an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
    if not peeled:
        # componentwise against the oracle's error majorant (tests/bounds.py);
        # a peeled edge is a classical fp32 product with a bound of its own
        S = bounds.majorant(oracle, A.astype(np.float64), B.astype(np.float64), d_used, L)
        bound = bounds.componentwise_c(dtype, L, d_used, kc) * S
        if dtype in bounds.FLOOR:
            bound = bound + bounds.FLOOR[dtype] * bounds.floor_majorant(
                oracle, A.astype(np.float64), B.astype(np.float64), d_used, L)
        assert np.all(np.abs(diff) <= bound), (dtype, n, d, o, float((np.abs(diff) / (bound + 1e-300)).max()))
    if n >= 64:
        assert np.abs(diff).max() / (an * bn) <= 1e-6, (dtype, n, d, o)
        rel = np.sqrt(np.mean(diff ** 2)) / np.sqrt(np.mean(want ** 2))
        assert rel <= bounds.rms_bound(dtype, L, d_used, kc), (dtype, n, d, o, rel)
