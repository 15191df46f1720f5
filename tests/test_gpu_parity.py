"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bars (written here, derived in the comments):
  * int64: bit-exact (wrapping mod 2^64 on both sides).
  * divide phase: bit-exact operand sums and splits (every sum is a two-term
    fp32 addition per level, so the order cannot matter; the splits are
    round-to-nearest-even on both sides).
  * fp64: max|dC| <= Higham's first-order Strassen bound (Thm. 23.2,
    "Accuracy and Stability of Numerical Algorithms", 2nd ed.), and the
    normwise ratio max|dC| / (||A||_F ||B||_F) <= 1e-12.
  * split fp32 (3xBF16, 3xTF32): normwise ratio <= 1e-6, and a bug-signal
    bound on the relative RMS error, rms(dC) / rms(C) <= s + 3 (L / k) 2^-24:
      s: the split.  3xBF16 operands carry 16 significant bits (8 + 8), each
      product is off by ~2^-16 relative, a dropped cross term would leave
      ~2^-8: s = 2^-12.  3xTF32 carries 22 bits: s = 2^-16 (a dropped term
      leaves ~2^-11).
      3 (L / k) 2^-24: the tensor-core accumulation, up to one fp32 ulp per
      accumulating MMA (k = 16 bf16 / 8 tf32 per MMA, 3 MMAs per K step,
      L = leaf side): at L = 4096 this term, not the split, dominates, which
      is why 3xTF32 is measured no more accurate than 3xBF16 there.  With
      accumulator promotion every kc of K the term covers kc instead of L
      (plus the fp32 additions of the chunks; tests/bounds.py).
"""
import time

import numpy as np
import pytest

import bounds
import oracle
from paper_1811_07325_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S(stark_lib):
    return stark_lib


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def higham_bound(n, d, A, B):
    u = 2.0 ** -53
    L = -(-n // 2 ** d)
    return 2 * ((12 ** d * (L * L + 5 * L) - 5 * n) + n) * u * np.abs(A).max() * np.abs(B).max()


# ----------------------------------------------------------------- self test
def test_bounded_wait_reports_timeout_and_context_survives(S):
    assert S.selftest_bounded_wait(20_000_000) == S.Status.ETIMEOUT
    with S.Plan(64, 1, S.DType.I64) as p:
        A = synth.integers(64, 1, 0, -5, 5)
        B = synth.integers(64, 1, 1, -5, 5)
        C = p.mul(dev(A), dev(B))
        p.check()
        assert np.array_equal(C.cpu().numpy(), oracle.gemm_classical(A, B))


# ----------------------------------------------------------------- int64
@pytest.mark.parametrize("n,depths", [(1, [0, 1]), (63, [0, 1, 2]), (200, [1, 2, 3]), (512, [0, 1, 2, 3]),
                                      (1000, [2, 3, 4])])
def test_int64_bit_exact(S, n, depths):
    A = synth.integers(n, 100 + n, 0, -16, 16)
    B = synth.integers(n, 100 + n, 1, -16, 16)
    want = oracle.gemm_classical(A, B)
    dA, dB = dev(A), dev(B)
    for d in depths:
        with S.Plan(n, d, S.DType.I64) as p:
            C = p.mul(dA, dB)
            p.check()
            assert np.array_equal(C.cpu().numpy(), want), d


@pytest.mark.parametrize("n,depths", [(1000, [1, 2, 3]), (512, [0, 1, 2]), (2048, [1, 2, 3, 4])])
def test_int64_tensor_core_exact(S, n, depths):
    # bounded integers on the bf16 tensor cores: bit-identical to the oracle
    A = synth.integers(n, 200 + n, 0, -16, 16)
    B = synth.integers(n, 200 + n, 1, -16, 16)
    want = oracle.gemm_classical(A, B)
    dA, dB = dev(A), dev(B)
    for d in depths:
        with S.Plan(n, d, S.DType.I64) as p:
            p.set_input_bound(16)
            C = p.mul(dA, dB)
            p.check()
            assert np.array_equal(C.cpu().numpy(), want), d


def test_int64_tensor_core_bound_checks(S):
    n = 512
    with S.Plan(n, 2, S.DType.I64) as p:
        with pytest.raises(S.StarkError) as e:
            p.set_input_bound(200)  # 200 * 4 > 256: not exact at depth 2
        assert e.value.status == S.Status.EUNSUPPORTED
        p.set_input_bound(16)
        # an input beyond the declared bound is reported, not silently wrong
        A = synth.integers(n, 9, 0, -16, 16)
        A[3, 5] = 1000
        B = synth.integers(n, 9, 1, -16, 16)
        p.mul(dev(A), dev(B))
        with pytest.raises(S.StarkError) as e:
            p.check()
        assert e.value.status == S.Status.EINVAL
        # within the bound again: exact
        A[3, 5] = 7
        C = p.mul(dev(A), dev(B))
        p.check()
        assert np.array_equal(C.cpu().numpy(), oracle.gemm_classical(A, B))
        p.set_input_bound(0)  # back to the CUDA-core path
        C = p.mul(dev(A), dev(B))
        p.check()
        assert np.array_equal(C.cpu().numpy(), oracle.gemm_classical(A, B))


def test_int64_wraps_modulo_2_64(S):
    n = 130
    A = synth.integers(n, 5, 0, -2**63, 2**63 - 1)
    B = synth.integers(n, 5, 1, -2**63, 2**63 - 1)
    want = oracle.gemm_classical(A, B)
    for d in (1, 2):
        with S.Plan(n, d, S.DType.I64) as p:
            assert np.array_equal(p.mul(dev(A), dev(B)).cpu().numpy(), want)


def test_int64_equals_oracle_strassen(S):
    n = 256
    A = synth.integers(n, 6, 0, -16, 16)
    B = synth.integers(n, 6, 1, -16, 16)
    with S.Plan(n, 3, S.DType.I64) as p:
        assert np.array_equal(p.mul(dev(A), dev(B)).cpu().numpy(), oracle.strassen(A, B, 3))


# ----------------------------------------------------------------- divide phase
@pytest.mark.parametrize("dtype", ["F32_SPLIT_BF16", "F32_SPLIT_TF32", "F32_SPLIT_FP16"])
@pytest.mark.parametrize("n,d", [(256, 0), (300, 1), (500, 2), (1000, 3), (1001, 4),
                                 # depth 3 with L a multiple of 256: the staged one-pass divide
                                 # (aligned rows; ragged rows and columns; unaligned row stride)
                                 (2048, 3), (2044, 3), (2001, 3)])
def test_divide_split_bit_exact(S, dtype, n, d):
    dt = S.DType[dtype]
    A = synth.normal(n, 7 + d, 0)
    B = synth.normal(n, 7 + d, 1)
    split = {S.DType.F32_SPLIT_BF16: oracle.split_bf16, S.DType.F32_SPLIT_TF32: oracle.split_tf32,
             S.DType.F32_SPLIT_FP16: oracle.split_fp16}[dt]
    with S.Plan(n, d, dt) as p:
        xa = oracle.strassen_operands(A, p.n_pad, d, "A")
        yb = oracle.strassen_operands(B, p.n_pad, d, "B")
        xh, xl = split(xa)
        yh, yl = split(yb)
        P = p.leaves
        # TF32: row-major Y planes (MN-major operand, the default), then the
        # transposed planes of the K-major layout
        for kmajor in ((False, True) if dt == S.DType.F32_SPLIT_TF32 else (False,)):
            if kmajor:
                p.set_tf32_layout(False)
            X, Y = p.operands(dev(A), dev(B))
            torch.cuda.synchronize()
            X = X.float().cpu().numpy()
            Y = Y.float().cpu().numpy()
            assert np.array_equal(X[:P], xh) and np.array_equal(X[P:], xl)
            if kmajor:  # stored N x K
                Y = Y.transpose(0, 2, 1)
            assert np.array_equal(Y[:P], yh) and np.array_equal(Y[P:], yl)


@pytest.mark.parametrize("n,d", [(200, 1), (300, 2), (513, 3), (999, 4)])
def test_divide_plain_f64_matches_oracle_sums(S, n, d):
    # integer-valued doubles: the oracle's fp32 sums are exact, so they must equal the fp64 planes
    A = synth.integers(n, 3, 0, -1000, 1000).astype(np.float64)
    B = synth.integers(n, 3, 1, -1000, 1000).astype(np.float64)
    with S.Plan(n, d, S.DType.F64) as p:
        X, Y = p.operands(dev(A), dev(B))
        torch.cuda.synchronize()
        xa = oracle.strassen_operands(A.astype(np.float32), p.n_pad, d, "A")
        yb = oracle.strassen_operands(B.astype(np.float32), p.n_pad, d, "B")
        assert np.array_equal(X.cpu().numpy(), xa.astype(np.float64))
        assert np.array_equal(Y.cpu().numpy(), yb.astype(np.float64))


# ----------------------------------------------------------------- n = 4096 depth sweep (fp64, int64)
@pytest.mark.slow
def test_n4096_depth_sweep_int64_and_f64(S):
    n = 4096
    Ai = synth.integers(n, 4096, 0, -16, 16)
    Bi = synth.integers(n, 4096, 1, -16, 16)
    want_i = oracle.gemm_classical(Ai, Bi)
    dA, dB = dev(Ai), dev(Bi)
    for d in (1, 2, 3, 4):
        with S.Plan(n, d, S.DType.I64) as p:
            C = p.mul(dA, dB)
            p.check()
            assert np.array_equal(C.cpu().numpy(), want_i), d
    del dA, dB
    Af = synth.uniform(n, 4096, 2)
    Bf = synth.uniform(n, 4096, 3)
    rows = synth.sample_rows(n, 64, 4096)
    want_f = oracle.gemm_rows(Af, Bf, rows)
    dA, dB = dev(Af), dev(Bf)
    for d in (1, 2, 3, 4):
        with S.Plan(n, d, S.DType.F64) as p:
            C = p.mul(dA, dB)
            p.check()
            got = C[torch.from_numpy(rows).cuda()].cpu().numpy()
        err = np.abs(got - want_f).max()
        assert err <= higham_bound(n, d, Af, Bf), (d, err)
        assert err / (np.linalg.norm(Af) * np.linalg.norm(Bf)) <= 1e-12


# ----------------------------------------------------------------- fp64
@pytest.mark.parametrize("n,depths", [(129, [0, 1]), (640, [1, 2, 3]), (1024, [3])])
def test_f64_within_bound(S, n, depths):
    A = synth.uniform(n, 11, 0)
    B = synth.uniform(n, 11, 1)
    want = oracle.gemm_classical(A, B)
    dA, dB = dev(A), dev(B)
    for d in depths:
        with S.Plan(n, d, S.DType.F64) as p:
            C = p.mul(dA, dB).cpu().numpy()
            p.check()
        err = np.abs(C - want).max()
        assert err <= higham_bound(n, d, A, B), (d, err)
        assert err / (np.linalg.norm(A) * np.linalg.norm(B)) <= 1e-12


# ----------------------------------------------------------------- split fp32
def check_split(C, want, A64norm, B64norm, dtype, A=None, B=None, d=None, L=None, kc=None):
    """The split-precision bars (tests/bounds.py): with the inputs given and
    every row of C compared, the componentwise bound |dC_ij| <= c S_ij
    against the oracle's error majorant, at every n; for n >= 64 the
    normwise ratio <= 1e-6 (the configs' bound) and the relative RMS model
    bound.  (Below n = 64 the 16/22-bit split cannot average down to 1e-6 of
    ||A|| ||B||; the componentwise bound is the bar there.)  kc: the K of
    one tensor-core accumulation under accumulator promotion."""
    diff = C.astype(np.float64) - want
    ratio = np.abs(diff).max() / (A64norm * B64norm)
    rel_rms = np.sqrt(np.mean(diff ** 2)) / max(np.sqrt(np.mean(want ** 2)), 1e-300)
    n = want.shape[1]
    L = n if L is None else L
    d = bounds.infer_depth(n, L) if d is None else d
    if A is not None and want.shape[0] == n and n <= 2048:
        S = bounds.majorant(oracle, A.astype(np.float64), B.astype(np.float64), d, L)
        c = bounds.componentwise_c(dtype, L, d, kc)
        bound = c * S
        if dtype in bounds.FLOOR:
            bound = bound + bounds.FLOOR[dtype] * bounds.floor_majorant(
                oracle, A.astype(np.float64), B.astype(np.float64), d, L)
        excess = np.abs(diff) / np.maximum(bound, 1e-300)
        assert np.all(np.abs(diff) <= bound), excess.max()
    else:
        assert n >= 64, "small products need the inputs for the componentwise bound"
    if n >= 64:
        assert ratio <= 1e-6, ratio
        assert rel_rms <= bounds.rms_bound(dtype, L, d, kc), rel_rms
    return ratio, rel_rms


@pytest.mark.parametrize("dtype", ["F32_SPLIT_BF16", "F32_SPLIT_TF32", "F32_SPLIT_FP16"])
@pytest.mark.parametrize("n,depths", [(1, [0, 1]), (37, [0, 1]), (100, [0, 1]), (384, [0, 1]), (1000, [1, 2, 3]),
                                      (2048, [0, 2, 3])])
def test_split_within_bound(S, dtype, n, depths):
    dt = S.DType[dtype]
    A = synth.normal(n, 21, 0)
    B = synth.normal(n, 21, 1)
    want = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
    an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
    dA, dB = dev(A), dev(B)
    for d in depths:
        with S.Plan(n, d, dt) as p:
            C = p.mul(dA, dB)
            p.check()
            check_split(C.cpu().numpy(), want, an, bn, dtype, A, B, d, L=p.leaf)


def test_split_repeatable_and_stream_ordered(S):
    n = 1024
    A = synth.normal(n, 31, 0)
    B = synth.normal(n, 31, 1)
    with S.Plan(n, 2, S.DType.F32_SPLIT_BF16) as p:
        s = torch.cuda.Stream()
        dA, dB = dev(A), dev(B)
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            C1 = p.mul(dA, dB, stream=s)
            C2 = p.mul(dA, dB, stream=s)
        s.synchronize()
        want = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
        an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
        check_split(C1.cpu().numpy(), want, an, bn, "F32_SPLIT_BF16", A, B, L=p.leaf)
        check_split(C2.cpu().numpy(), want, an, bn, "F32_SPLIT_BF16", A, B, L=p.leaf)


@pytest.mark.parametrize("n,d", [(1024, 2), (1000, 3), (1004, 1), (1001, 2), (777, 1)])
def test_split_combine_modes_agree(S, n, d):
    # TMA bulk reductions and the vector-atomic fallback give the same product
    A = synth.normal(n, 61, 0)
    B = synth.normal(n, 61, 1)
    want = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
    an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
    out = []
    for mode in (0, 1):
        with S.Plan(n, d, S.DType.F32_SPLIT_BF16) as p:
            p.set_combine(mode)
            C = p.mul(dev(A), dev(B))
            p.check()
            out.append(C.cpu().numpy())
            check_split(out[-1], want, an, bn, "F32_SPLIT_BF16", A, B, L=p.leaf)
    # same products, different addition order into C: fp32-level agreement
    assert np.abs(out[0] - out[1]).max() <= 1e-5 * np.abs(want).max()


@pytest.mark.parametrize("n,d,dtype", [(1024, 2, "F32_SPLIT_BF16"), (1001, 3, "F32_SPLIT_BF16"),
                                       (777, 1, "F32_SPLIT_TF32"), (2048, 0, "F32_SPLIT_BF16")])
def test_deterministic_combine_is_bitwise_reproducible(S, n, d, dtype):
    A = synth.normal(n, 63, 0)
    B = synth.normal(n, 63, 1)
    want = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
    an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
    with S.Plan(n, d, S.DType[dtype]) as p:
        p.set_combine(2)
        dA, dB = dev(A), dev(B)
        C1 = p.mul(dA, dB).cpu().numpy()
        C2 = p.mul(dA, dB).cpu().numpy()
        p.check()
        L = p.leaf
        p.set_combine(0)
        Cf = p.mul(dA, dB).cpu().numpy()
    assert np.array_equal(C1.view(np.uint32), C2.view(np.uint32))  # bit for bit
    check_split(C1, want, an, bn, dtype, A, B, L=L)
    assert np.abs(C1 - Cf).max() <= 1e-5 * np.abs(want).max()  # same products, other order


@pytest.mark.parametrize("n,d", [(2048, 1), (4096, 2), (1536, 0)])
def test_leaf_schedules_agree(S, n, d):
    # one CTA per tile, the four-stage 64-byte-row pipeline and CTA pairs on
    # one cta_group::2 MMA (row-major and banded rasters): same products
    A = synth.normal(n, 62, 0)
    B = synth.normal(n, 62, 1)
    rows = synth.sample_rows(n, 64, 62)
    want = oracle.gemm_rows(A, B, rows)
    an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
    out = []
    for pair, deep, band in ((0, False, 0), (0, True, 0), (2, False, 0), (2, False, 2), (0, False, 2)):
        with S.Plan(n, d, S.DType.F32_SPLIT_BF16) as p:
            p.set_pairing(pair)
            p.set_pipeline(deep)
            p.set_raster(band)
            C = p.mul(dev(A), dev(B))
            p.check()
            got = C[torch.from_numpy(rows).cuda()].cpu().numpy()
            out.append(got)
            diff = got.astype(np.float64) - want
            assert np.abs(diff).max() / (an * bn) <= 1e-6
            rel = np.sqrt(np.mean(diff ** 2)) / np.sqrt(np.mean(want ** 2))
            assert rel <= bounds.rms_bound("F32_SPLIT_BF16", p.leaf, d)
    for k in (1, 2, 3, 4):
        assert np.abs(out[k] - out[0]).max() <= 1e-5 * np.abs(want).max()


def test_multicast_pairing_is_refused(S):
    # no leaf schedule shares tiles between the CTAs of a cluster by
    # multicast loads: mode 1 is refused and the plan keeps its schedule
    n = 512
    A = synth.normal(n, 63, 0)
    B = synth.normal(n, 63, 1)
    with S.Plan(n, 1, S.DType.F32_SPLIT_BF16) as p:
        with pytest.raises(S.StarkError) as e:
            p.set_pairing(1)
        assert e.value.status == S.Status.EUNSUPPORTED
        C = p.mul(dev(A), dev(B)).cpu().numpy()
        p.check()
    want = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
    an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
    assert np.abs(C - want).max() / (an * bn) <= 1e-6


@pytest.mark.parametrize("dtype,n,d,combine,dfs", [
    ("F32_SPLIT_BF16", 1024, 1, 0, False), ("F32_SPLIT_BF16", 1001, 1, 0, False),
    ("F32_SPLIT_BF16", 2048, 2, 2, False), ("F32_SPLIT_BF16", 2048, 2, 0, True),
    ("F32_SPLIT_BF16", 1900, 2, 1, False), ("F32_SPLIT_BF16", 777, 0, 0, False),
    ("F32_SPLIT_TF32", 1024, 1, 0, False), ("F32_SPLIT_TF32", 1001, 1, 2, False),
    ("F32_SPLIT_TF32", 2048, 2, 0, True)])
def test_pair_mma_matches_oracle(S, dtype, n, d, combine, dfs):
    # CTA pairs on one 256 x 256 cta_group::2 MMA, every element against the
    # FP64 oracle; leaf sides that are not a multiple of 256 (n=777, d=0) take
    # the single-CTA kernel
    A = synth.normal(n, 65, 0)
    B = synth.normal(n, 65, 1)
    want = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
    an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
    dA, dB = dev(A), dev(B)
    with S.Plan(n, d, S.DType[dtype]) as p:
        p.set_pairing(2)
        p.set_combine(combine)
        if dfs:
            p.set_traversal(True)
        C1 = p.mul(dA, dB).cpu().numpy()
        C2 = p.mul(dA, dB).cpu().numpy()
        p.check()
        check_split(C1, want, an, bn, dtype, A, B, L=p.leaf)
        p.set_pairing(0)
        C0 = p.mul(dA, dB).cpu().numpy()
    assert np.abs(C1 - C0).max() <= 1e-5 * np.abs(want).max()
    if combine == 2:
        assert np.array_equal(C1.view(np.uint32), C2.view(np.uint32))
    else:
        assert np.abs(C1 - C2).max() <= 1e-5 * np.abs(want).max()


@pytest.mark.parametrize("n,d,dtype,levels", [(2048, 2, "F32_SPLIT_BF16", 1), (1001, 3, "F32_SPLIT_BF16", 1),
                                              (777, 1, "F32_SPLIT_TF32", 1), (2048, 2, "F32_SPLIT_BF16", 2),
                                              (1001, 3, "F32_SPLIT_BF16", 2), (1300, 3, "F32_SPLIT_TF32", 2),
                                              (900, 2, "F32_SPLIT_TF32", 2)])
def test_depth_first_traversal_matches(S, n, d, dtype, levels):
    # depth first over the top 1 or 2 levels: the divide reads A and B
    # through the prefix sums of each subtree; same products as breadth first
    A = synth.normal(n, 64, 0)
    B = synth.normal(n, 64, 1)
    want = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
    an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
    dA, dB = dev(A), dev(B)
    with S.Plan(n, d, S.DType[dtype]) as p:
        ws_bfs = p.workspace_bytes
        Cb = p.mul(dA, dB).cpu().numpy()
        p.set_traversal(levels)
        # the leaf operands shrink to one subtree's (the tables and a staging
        # copy of C, if any, stay)
        operands = 2 * p.leaves * p.leaf ** 2 * (4 if dtype == "F32_SPLIT_BF16" else 8)
        assert ws_bfs - p.workspace_bytes == operands - operands // 7 ** levels
        Cd = p.mul(dA, dB).cpu().numpy()
        p.check()
        check_split(Cd, want, an, bn, dtype, A, B, L=p.leaf)
        p.set_traversal(0)
        assert p.workspace_bytes == ws_bfs
    assert np.abs(Cd - Cb).max() <= 1e-5 * np.abs(want).max()


def test_depth_first_levels_rejected_where_unsupported(S):
    with S.Plan(500, 1, S.DType.F32_SPLIT_BF16) as p:
        with pytest.raises(S.StarkError):
            p.set_traversal(2)  # more levels than the depth
        with pytest.raises(S.StarkError):
            p.set_traversal(3)
    with S.Plan(500, 2, S.DType.I64) as p:
        with pytest.raises(S.StarkError):
            p.set_traversal(2)  # the two-level loader serves the split dtypes


@pytest.mark.parametrize("bound", [0, 16])
def test_depth_first_int64_exact_and_leaf_ranges(S, bound):
    n, d = 1000, 2
    A = synth.integers(n, 65, 0, -16, 16)
    B = synth.integers(n, 65, 1, -16, 16)
    want = oracle.gemm_classical(A, B)
    dA, dB = dev(A), dev(B)
    with S.Plan(n, d, S.DType.I64) as p:
        p.set_traversal(True)
        if bound:
            p.set_input_bound(bound)
        C = p.mul(dA, dB)
        p.check()
        assert np.array_equal(C.cpu().numpy(), want)
        total = torch.zeros((n, n), dtype=torch.int64, device="cuda")
        for a, b in ((0, 10), (10, 30), (30, 49)):  # ranges across subtree boundaries
            total += p.mul_leaves(dA, dB, a, b)
        p.check()
        assert np.array_equal(total.cpu().numpy(), want)


# ----------------------------------------------------------------- API paths
def test_leaf_partition_sums_to_product(S):
    n, d = 300, 2
    A = synth.integers(n, 41, 0, -16, 16)
    B = synth.integers(n, 41, 1, -16, 16)
    dA, dB = dev(A), dev(B)
    with S.Plan(n, d, S.DType.I64) as p:
        cuts = [0, 5, 20, 21, 49]
        total = torch.zeros((n, n), dtype=torch.int64, device="cuda")
        for a, b in zip(cuts[:-1], cuts[1:]):
            total += p.mul_leaves(dA, dB, a, b)
        assert np.array_equal(total.cpu().numpy(), oracle.gemm_classical(A, B))


@pytest.mark.parametrize("n,d,dfs,combine", [(1000, 1, False, 0), (2048, 2, False, 0), (777, 1, False, 2),
                                             (1536, 0, False, 0), (2048, 2, True, 0), (1300, 2, False, 1)])
def test_tf32_mn_major_layout_matches(S, n, d, dfs, combine):
    # 3xTF32 with the Y planes read MN-major (32-byte-atom swizzle, no
    # transpose pass; the default) and K-major (transposed planes): both
    # against the FP64 oracle and each other; pair kernel (L a multiple of
    # 256) and single-CTA kernel (otherwise)
    A = synth.normal(n, 66, 0)
    B = synth.normal(n, 66, 1)
    want = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
    an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
    dA, dB = dev(A), dev(B)
    with S.Plan(n, d, S.DType.F32_SPLIT_TF32) as p:
        p.set_combine(combine)
        if dfs:
            p.set_traversal(True)
        Cm = p.mul(dA, dB).cpu().numpy()  # default: MN-major
        p.set_tf32_layout(False)
        Ck = p.mul(dA, dB).cpu().numpy()
        check_split(Ck, want, an, bn, "F32_SPLIT_TF32", A, B, L=p.leaf)
        p.set_tf32_layout(True)
        assert np.array_equal(p.mul(dA, dB).cpu().numpy(), Cm) or combine != 2
        p.check()
        check_split(Cm, want, an, bn, "F32_SPLIT_TF32", A, B, L=p.leaf)
    assert np.abs(Cm - Ck).max() <= 1e-5 * np.abs(want).max()
    with S.Plan(64, 0, S.DType.F32_SPLIT_BF16) as q:
        with pytest.raises(S.StarkError):
            q.set_tf32_layout(True)


# ----------------------------------------------------------------- peeling
@pytest.mark.parametrize("dtype,n,d,combine,dfs,peel", [
    ("F32_SPLIT_BF16", 1025, 1, 0, False, 1),    # n % 4 != 0: staged C
    ("F32_SPLIT_BF16", 2049, 2, 0, False, 1),
    ("F32_SPLIT_BF16", 1300, 1, 0, False, 20),
    ("F32_SPLIT_BF16", 777, 0, 0, False, 9),
    ("F32_SPLIT_BF16", 2050, 2, 2, False, 2),    # deterministic combine
    ("F32_SPLIT_BF16", 2060, 2, 0, True, 12),    # depth-first traversal
    ("F32_SPLIT_BF16", 1100, 1, 1, False, 76),   # vector-atomic combine
    ("F32_SPLIT_TF32", 1030, 1, 0, False, 6),
    ("F64", 1000, 2, 0, False, 232),
    ("F64", 130, 1, 0, False, 2)])
def test_peeled_edge_matches_oracle(S, dtype, n, d, combine, dfs, peel):
    # recursion on the m x m core, classical products for the r-wide edge:
    # every element against the FP64 oracle, as the padded plan
    A = synth.normal(n, 95, 0) if dtype != "F64" else synth.uniform(n, 95, 0)
    B = synth.normal(n, 95, 1) if dtype != "F64" else synth.uniform(n, 95, 1)
    want = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
    dA, dB = dev(A), dev(B)
    with S.Plan(n, d, S.DType[dtype], peel=True) as p:
        assert p.peel == peel and p.n_pad == n - peel
        p.set_combine(combine)
        if dfs:
            p.set_traversal(True)
        C = p.mul(dA, dB).cpu().numpy()
        if combine == 2:  # deterministic: the edge is computed without atomics too
            assert np.array_equal(p.mul(dA, dB).cpu().numpy().view(np.uint32), C.view(np.uint32))
        p.check()
        L = p.leaf
    with S.Plan(n, d, S.DType[dtype]) as q:
        assert q.peel == 0 and q.n_pad > n
        Cpad = q.mul(dA, dB).cpu().numpy()
        Lpad = q.leaf
    if dtype == "F64":
        err = np.abs(C - want).max()
        assert err <= higham_bound(n, d, A, B), err
        assert err / (np.linalg.norm(A) * np.linalg.norm(B)) <= 1e-12
    else:
        an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
        check_split(C, want, an, bn, dtype, L=L)
        # the edge itself is a plain fp32 product: far inside the split bound
        edge = np.abs(C[:, n - peel:] - want[:, n - peel:]).max() / (an * bn)
        assert edge <= 1e-8, edge
        # the padded plan splits differently (other leaf side): same bound
        check_split(Cpad, want, an, bn, dtype, L=Lpad)


@pytest.mark.parametrize("n,d,bound", [(1029, 2, 0), (300, 1, 0), (1100, 2, 16)])
def test_peeled_int64_exact_and_leaf_ranges(S, n, d, bound):
    # int64 (CUDA cores, or bf16 tensor cores with a declared bound): exact;
    # partial products over a leaf partition still sum to A B (the edge is
    # added once, with the range that holds leaf 0)
    A = synth.integers(n, 97, 0, -16, 16)
    B = synth.integers(n, 97, 1, -16, 16)
    want = oracle.gemm_classical(A, B)
    dA, dB = dev(A), dev(B)
    with S.Plan(n, d, S.DType.I64, peel=True) as p:
        assert p.peel > 0
        if bound:
            p.set_input_bound(bound)
        assert np.array_equal(p.mul(dA, dB).cpu().numpy(), want)
        cuts = [0, 3, p.leaves // 2, p.leaves]
        total = torch.zeros((n, n), dtype=torch.int64, device="cuda")
        for a, b in zip(cuts[:-1], cuts[1:]):
            total += p.mul_leaves(dA, dB, a, b)
        p.check()
        assert np.array_equal(total.cpu().numpy(), want)


def test_peel_is_a_no_op_where_nothing_is_left(S):
    for n, d in ((1024, 1), (100, 1)):  # g divides n; n below one granule
        with S.Plan(n, d, S.DType.F32_SPLIT_BF16, peel=True) as p:
            assert p.peel == 0
    import ctypes
    h = ctypes.c_void_p()
    assert S._lib.stark_plan_ex(64, 1, int(S.DType.F64), 0x80, ctypes.byref(h)) == S.Status.EINVAL  # unknown flag


def test_mul_host_matches_device(S):
    n = 777
    A = synth.normal(n, 51, 0)
    B = synth.normal(n, 51, 1)
    with S.Plan(n, 2, S.DType.F32_SPLIT_BF16) as p:
        Ch = p.mul_host(A, B)
        Cd = p.mul(dev(A), dev(B)).cpu().numpy()
        L = p.leaf
    want = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
    an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
    check_split(Ch, want, an, bn, "F32_SPLIT_BF16", A, B, L=L)
    check_split(Cd, want, an, bn, "F32_SPLIT_BF16", A, B, L=L)


def test_mul_host_async_pipeline(S):
    # consecutive asynchronous host products with different inputs, results
    # read after one synchronisation: each equals its own product
    n = 640
    pairs = [(synth.normal(n, 80 + k, 0), synth.normal(n, 80 + k, 1)) for k in range(4)]
    As = [torch.from_numpy(a).pin_memory() for a, _ in pairs]
    Bs = [torch.from_numpy(b).pin_memory() for _, b in pairs]
    Cs = [torch.empty((n, n), dtype=torch.float32).pin_memory() for _ in pairs]
    with S.Plan(n, 1, S.DType.F32_SPLIT_BF16) as p:
        for k in range(4):
            p.mul_host(As[k], Bs[k], Cs[k], asynchronous=True)
        torch.cuda.synchronize()
        p.check()
    for k, (a, b) in enumerate(pairs):
        want = oracle.gemm_classical(a.astype(np.float64), b.astype(np.float64))
        an, bn = np.linalg.norm(a.astype(np.float64)), np.linalg.norm(b.astype(np.float64))
        check_split(Cs[k].numpy(), want, an, bn, "F32_SPLIT_BF16", a, b, L=p.leaf)


def test_mul_host_enqueue_and_wait(S):
    # the host pipeline without a stream wait: five products through two
    # staging sets, collected by one host_wait; then a second round on the
    # same plan reusing the first C buffers
    n = 1000
    pairs = [(synth.normal(n, 80 + k, 0), synth.normal(n, 80 + k, 1)) for k in range(5)]
    As = [torch.from_numpy(a).pin_memory() for a, _ in pairs]
    Bs = [torch.from_numpy(b).pin_memory() for _, b in pairs]
    Cs = [torch.full((n, n), float("nan"), dtype=torch.float32).pin_memory() for _ in pairs]
    with S.Plan(n, 2, S.DType.F32_SPLIT_BF16) as p:
        p.host_wait()  # nothing pending yet
        for k in range(5):
            p.mul_host_enqueue(As[k], Bs[k], Cs[k])
        p.host_wait()
        first = [c.clone() for c in Cs]
        for k in range(2):
            p.mul_host_enqueue(As[4 - k], Bs[4 - k], Cs[k])
        p.host_wait()
        with pytest.raises(ValueError):
            p.mul_host_enqueue(As[0].cuda(), Bs[0], Cs[0])
    for k, (a, b) in enumerate(pairs):
        want = oracle.gemm_classical(a.astype(np.float64), b.astype(np.float64))
        an, bn = np.linalg.norm(a.astype(np.float64)), np.linalg.norm(b.astype(np.float64))
        check_split(first[k].numpy(), want, an, bn, "F32_SPLIT_BF16", a, b, L=p.leaf)
    for k in range(2):
        assert np.abs(Cs[k].numpy() - first[4 - k].numpy()).max() <= 1e-5 * np.abs(first[4 - k].numpy()).max()


def test_empty_and_bad_arguments(S):
    with S.Plan(0, 1, S.DType.F32_SPLIT_BF16) as p:
        e = torch.empty((0, 0), dtype=torch.float32, device="cuda")
        p.mul(e, e, e)
    with pytest.raises(S.StarkError):
        S.Plan(-1, 1, S.DType.F64)
    with pytest.raises(S.StarkError):
        S.Plan(64, 5, S.DType.F64)
    with S.Plan(64, 1, S.DType.F64) as p:
        with pytest.raises(TypeError):
            p.mul(torch.zeros(64, 64, device="cuda"), torch.zeros(64, 64, device="cuda"))


def test_auto_depth(S):
    # depth -1: measured autotuner (tensor-core dtypes), cached per size class
    with S.Plan(16384, -1, S.DType.F32_SPLIT_BF16) as p:
        assert 1 <= p.depth <= 3
        d16 = p.depth
    with S.Plan(16384, -1, S.DType.F32_SPLIT_BF16) as p:
        assert p.depth == d16  # cached decision
    with S.Plan(300, -1, S.DType.F32_SPLIT_BF16) as p:
        assert p.depth in (0, 1)  # leaves of side >= 128 only
    with S.Plan(1000, -1, S.DType.I64) as p:  # cost model for the CUDA-core dtypes
        assert 0 <= p.depth <= 4


# ----------------------------------------------------------------- sibling-folded combine
@pytest.mark.parametrize("dtype,n,d", [("F32_SPLIT_BF16", 1024, 1), ("F32_SPLIT_BF16", 2048, 2),
                                       ("F32_SPLIT_BF16", 1001, 1), ("F32_SPLIT_BF16", 2048, 3),
                                       ("F32_SPLIT_BF16", 4096, 4), ("F32_SPLIT_TF32", 2048, 2),
                                       ("F32_SPLIT_TF32", 2001, 2)])
def test_sibling_fold_matches_oracle(S, dtype, n, d):
    # combine mode 3: the seven children of each parent fold into its
    # quadrants (store, then add-reductions in sibling order), one ordered
    # pass one level up writes C.  Every element against the FP64 oracle
    # (sampled rows above n = 2048), bitwise equal across runs, and within
    # fp32 reordering of the fused combine
    A = synth.normal(n, 66 + d, 0)
    B = synth.normal(n, 66 + d, 1)
    rows = np.arange(n) if n <= 2048 else synth.sample_rows(n, 128, 66)
    want = oracle.gemm_rows(A, B, rows)
    an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
    dA, dB = dev(A), dev(B)
    r = torch.from_numpy(rows).cuda()
    with S.Plan(n, d, S.DType[dtype]) as p:
        p.set_combine(3)
        C1 = p.mul(dA, dB)[r].cpu().numpy()
        C2 = p.mul(dA, dB)[r].cpu().numpy()
        p.check()
        check_split(C1, want, an, bn, dtype, A, B, L=p.leaf)
        p.set_combine(0)
        Cf = p.mul(dA, dB)[r].cpu().numpy()
        p.check()
    assert np.array_equal(C1.view(np.uint32), C2.view(np.uint32))
    assert np.abs(C1 - Cf).max() <= 1e-5 * np.abs(want).max()


@pytest.mark.parametrize("dtype,n,d", [("F32_SPLIT_BF16", 2048, 2), ("F32_SPLIT_BF16", 777, 1), ("F64", 512, 2)])
def test_measured_combine_choice(S, dtype, n, d):
    # mode -1 keeps the fastest applicable mode (fp64: the fused one), and
    # the product stays within its bounds; the phase split is consistent
    A = synth.normal(n, 68, 0) if dtype != "F64" else synth.uniform(n, 68, 0)
    B = synth.normal(n, 68, 1) if dtype != "F64" else synth.uniform(n, 68, 1)
    want = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
    an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
    with S.Plan(n, d, S.DType[dtype]) as p:
        ws0 = p.workspace_bytes
        p.set_combine(-1)
        assert p.combine in ((0, 2, 3) if dtype != "F64" else (0,))
        if p.combine == 0:
            assert p.workspace_bytes == ws0  # the losers' product planes were released
        p.set_timing(2)
        C = p.mul(dev(A), dev(B)).cpu().numpy()
        C = p.mul(dev(A), dev(B)).cpu().numpy()
        p.check()
        ph = p.phase_ms()
        assert ph["leaf_kernel"] > 0 and ph["after_leaf"] >= 0
        assert abs(ph["leaf_combine"] - ph["leaf_kernel"] - ph["after_leaf"]) < 1e-3
    if dtype == "F64":
        assert np.abs(C - want).max() / (an * bn) <= 1e-12
    else:
        check_split(C, want, an, bn, dtype, A, B, L=p.leaf)


def test_sibling_fold_conditions_and_fallbacks(S):
    n = 1024
    A = synth.normal(n, 67, 0)
    B = synth.normal(n, 67, 1)
    want = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
    an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
    dA, dB = dev(A), dev(B)
    for d, m in ((0, 1024), (1, 640)):  # depth 0; a leaf side (384) that is not a multiple of 256
        with S.Plan(m, d, S.DType.F32_SPLIT_BF16) as p:
            with pytest.raises(S.StarkError) as e:
                p.set_combine(3)
            assert e.value.status == S.Status.EUNSUPPORTED
    with S.Plan(n, 2, S.DType.F32_SPLIT_BF16) as p:
        p.set_combine(3)
        with pytest.raises(S.StarkError):
            p.set_traversal(1)  # depth first keeps one subtree: no parent planes
        # products mode 3 cannot serve run the fused path: single CTAs, and a
        # partition of the leaves whose partial products sum to A B
        p.set_pairing(0)
        check_split(p.mul(dA, dB).cpu().numpy(), want, an, bn, "F32_SPLIT_BF16", A, B, L=p.leaf)
        p.set_pairing(2)
        parts = []
        for lb, le in ((0, 20), (20, 49)):
            parts.append(p.mul_leaves(dA, dB, lb, le))
        p.check()
        check_split((parts[0] + parts[1]).cpu().numpy(), want, an, bn, "F32_SPLIT_BF16", A, B, L=p.leaf)


# ----------------------------------------------------------------- accumulator promotion
@pytest.mark.parametrize("dtype,n,d,k,combine", [
    ("F32_SPLIT_BF16", 512, 1, 256, 2),    # L = 256: one chunk, promotion changes nothing
    ("F32_SPLIT_BF16", 1024, 1, 256, 0),   # L = 512: two chunks, the second added at read-out
    ("F32_SPLIT_BF16", 2048, 1, 256, 2),   # L = 1024: four chunks, two drains in TMEM
    ("F32_SPLIT_BF16", 1536, 1, 512, 1),   # L = 768: chunks of 512 and 256; vector atomics
    ("F32_SPLIT_BF16", 1001, 2, 256, 0),   # ragged n: the staging copy of C
    ("F32_SPLIT_BF16", 2048, 2, 256, 2),
    ("F32_SPLIT_TF32", 1024, 1, 256, 0),
    ("F32_SPLIT_TF32", 2048, 1, 256, 2),
    ("F32_SPLIT_TF32", 1536, 1, 512, 0),
    ("F32_SPLIT_FP16", 2048, 1, 256, 2),
    ("F32_SPLIT_FP16", 1001, 2, 256, 0),
])
def test_promotion_matches_oracle(S, dtype, n, d, k, combine):
    # every K chunk's tensor-core partial sum joins an fp32 running sum; the
    # product stays within the split bounds against the FP64 oracle, a second
    # product on the same plan agrees (the barrier phases carry over), and it
    # differs from the unpromoted product only by rounding
    A = synth.normal(n, 71 + d, 0)
    B = synth.normal(n, 71 + d, 1)
    want = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
    an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
    dA, dB = dev(A), dev(B)
    with S.Plan(n, d, S.DType[dtype]) as p:
        p.set_combine(combine)
        p.set_promotion(k)
        assert p.info().promotion_k == k
        C1 = p.mul(dA, dB).cpu().numpy()
        C2 = p.mul(dA, dB).cpu().numpy()
        p.check()
        check_split(C1, want, an, bn, dtype, A, B, L=p.leaf, kc=k)
        p.set_promotion(0)
        Cn = p.mul(dA, dB).cpu().numpy()
        p.check()
        single_chunk = k >= p.leaf
    if combine == 2:
        assert np.array_equal(C1.view(np.uint32), C2.view(np.uint32))
        if single_chunk:
            assert np.array_equal(C1.view(np.uint32), Cn.view(np.uint32))
    else:
        assert np.abs(C1 - C2).max() <= 1e-5 * np.abs(want).max()
    assert np.abs(C1 - Cn).max() <= 1e-5 * np.abs(want).max()


@pytest.mark.parametrize("dtype,gain", [("F32_SPLIT_TF32", 4.0), ("F32_SPLIT_BF16", 1.0), ("F32_SPLIT_FP16", 2.0)])
def test_promotion_cuts_accumulation_error(S, dtype, gain):
    # one leaf of side 4096 (depth 0): the tensor core's accumulation over K
    # = 4096 dominates the 3xTF32 error, and it grows in proportion to the K
    # it spans, so promotion every 512 should cut it ~8x (required: 4x);
    # 3xBF16's 16-bit split dominates its own error, so there promotion
    # must only not hurt.  Both within the promoted bounds.
    n = 4096
    A = synth.normal(n, 75, 0)
    B = synth.normal(n, 75, 1)
    rows = synth.sample_rows(n, 64, 75)
    want = oracle.gemm_rows(A, B, rows)
    an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
    dA, dB = dev(A), dev(B)
    r = torch.from_numpy(rows).cuda()
    rms = {}
    with S.Plan(n, 0, S.DType[dtype]) as p:
        for k in (0, 512):
            p.set_promotion(k)
            C = p.mul(dA, dB)[r].cpu().numpy()
            p.check()
            _, rms[k] = check_split(C, want, an, bn, dtype, L=p.leaf, kc=k)
    assert rms[512] * gain <= rms[0], rms


def test_promotion_conditions(S):
    n = 1024
    A = synth.normal(n, 73, 0)
    B = synth.normal(n, 73, 1)
    dA, dB = dev(A), dev(B)
    with S.Plan(n, 1, S.DType.F32_SPLIT_BF16) as p:
        for bad in (-256, 300):
            with pytest.raises(S.StarkError) as e:
                p.set_promotion(bad)
            assert e.value.status == S.Status.EINVAL
        p.set_promotion(512)
        with pytest.raises(S.StarkError) as e:
            p.set_combine(3)  # the sibling fold keeps its own accumulators
        assert e.value.status == S.Status.EUNSUPPORTED
        p.set_pairing(0)  # single CTAs: promotion has no kernel there
        with pytest.raises(S.StarkError) as e:
            p.mul(dA, dB)
        assert e.value.status == S.Status.EUNSUPPORTED
        p.set_pairing(2)
        p.mul(dA, dB)
        p.check()
    with S.Plan(n, 1, S.DType.F32_SPLIT_BF16) as p:
        p.set_combine(3)
        with pytest.raises(S.StarkError) as e:
            p.set_promotion(256)
        assert e.value.status == S.Status.EUNSUPPORTED
    with S.Plan(640, 1, S.DType.F32_SPLIT_BF16) as p:  # leaf side 384
        with pytest.raises(S.StarkError) as e:
            p.set_promotion(256)
        assert e.value.status == S.Status.EUNSUPPORTED
    with S.Plan(512, 1, S.DType.F64) as p:
        with pytest.raises(S.StarkError) as e:
            p.set_promotion(256)
        assert e.value.status == S.Status.EUNSUPPORTED
    with S.Plan(n, 1, S.DType.F32_SPLIT_TF32) as p:
        p.set_tf32_layout(False)
        with pytest.raises(S.StarkError) as e:
            p.set_promotion(256)
        assert e.value.status == S.Status.EUNSUPPORTED


# ----------------------------------------------------------------- 3xFP16 range
def test_fp16_split_range_flag(S):
    # an operand sum beyond fp16's largest finite value (65504) raises the
    # plan's device range flag: stark_plan_check reports EINVAL once and the
    # flag is cleared; inputs inside the range then multiply normally
    n, d = 512, 1
    A = synth.normal(n, 77, 0)
    B = synth.normal(n, 77, 1)
    big = A.copy()
    big[3, 5] = 40000.0  # A11 + A22 sums stay below 65520 only if A22 is small there
    big[3 + n // 2, 5 + n // 2] = 30000.0
    with S.Plan(n, d, S.DType.F32_SPLIT_FP16) as p:
        p.mul(dev(big), dev(B))
        with pytest.raises(S.StarkError) as e:
            p.check()
        assert e.value.status == S.Status.EINVAL
        C = p.mul(dev(A), dev(B)).cpu().numpy()
        p.check()
    want = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
    an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
    check_split(C, want, an, bn, "F32_SPLIT_FP16", A, B, d)


@pytest.mark.parametrize("n,d", [(512, 1), (1000, 2)])
def test_fp16_split_small_values(S, n, d):
    # a quarter of A's rows scaled into fp16's subnormal range: their leaf
    # operands keep only the fixed spacing 2^-24, and the product must still
    # meet the bound with its absolute floor term (the tensor cores take
    # fp16 subnormal inputs as they are)
    A = synth.normal(n, 79 + d, 0)
    B = synth.normal(n, 79 + d, 1)
    A[: n // 4] *= 2.0 ** -18
    want = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
    an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
    with S.Plan(n, d, S.DType.F32_SPLIT_FP16) as p:
        C = p.mul(dev(A), dev(B)).cpu().numpy()
        p.check()
        L = p.leaf
    check_split(C, want, an, bn, "F32_SPLIT_FP16", A, B, d, L)


def test_fp16_split_in_batches_and_the_server(S):
    # the grouped launches carry the fp16 format too: a batch and served
    # requests of 3xFP16 agree with the oracle within the split bounds
    sizes = [512, 1024, 777]
    As = [synth.normal(m, 78 + i, 0) for i, m in enumerate(sizes)]
    Bs = [synth.normal(m, 78 + i, 1) for i, m in enumerate(sizes)]
    dAs, dBs = [dev(a) for a in As], [dev(b) for b in Bs]
    Cs = [torch.empty_like(a) for a in dAs]
    with S.Batch(sizes, 1, S.DType.F32_SPLIT_FP16) as b:
        b.mul(dAs, dBs, Cs)
        b.mul(dAs, dBs, Cs)  # a graph replay
        b.check()
    with S.Server(1 << 32) as srv:
        Cr = [torch.empty_like(a) for a in dAs]
        pending = {srv.submit(a, b, c, S.DType.F32_SPLIT_FP16) for a, b, c in zip(dAs, dBs, Cr)}
        t0 = time.time()
        while pending:
            for rid in list(pending):
                done, st = srv.poll(rid)
                if done:
                    assert st == S.Status.OK
                    pending.discard(rid)
            assert time.time() - t0 < 120, "server did not finish"
            time.sleep(0.0005)
    for A, B, C, Cs_ in zip(As, Bs, Cs, Cr):
        want = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
        an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
        m = A.shape[0]
        L = -(-m // 2 // 128) * 128
        check_split(C.cpu().numpy(), want, an, bn, "F32_SPLIT_FP16", A, B, 1, L)
        check_split(Cs_.cpu().numpy(), want, an, bn, "F32_SPLIT_FP16")


# ----------------------------------------------------------------- full size, sampled rows
@pytest.mark.slow
@pytest.mark.parametrize("dtype,d,combine", [("F32_SPLIT_BF16", 2, 0), ("F32_SPLIT_BF16", 3, 0),
                                             ("F32_SPLIT_TF32", 2, 0), ("F32_SPLIT_TF32", 3, 0),
                                             ("F32_SPLIT_BF16", 2, 2), ("F32_SPLIT_BF16", 3, 2),
                                             ("F32_SPLIT_BF16", 2, 3), ("F32_SPLIT_BF16", 3, 3),
                                             ("F32_SPLIT_TF32", 3, 3), ("F32_SPLIT_FP16", 2, 2),
                                             ("F32_SPLIT_FP16", 3, 0)])
def test_full_size_sampled_rows(S, dtype, d, combine):
    # the bench workload in the bench's launch configuration (CTA pairs;
    # fused combine, or the deterministic one of its second leg)
    n = 16384
    A = synth.normal(n, 2024, 0)
    B = synth.normal(n, 2024, 1)
    rows = synth.sample_rows(n, 256, 2024)
    want = oracle.gemm_rows(A, B, rows)
    an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
    dA, dB = dev(A), dev(B)
    with S.Plan(n, d, S.DType[dtype]) as p:
        p.set_combine(combine)
        C = p.mul(dA, dB)
        p.check()
        got = C[torch.from_numpy(rows).cuda()].cpu().numpy()
        L = p.leaf
    del C, dA, dB
    torch.cuda.empty_cache()
    check_split(got, want, an, bn, dtype, L=L)


@pytest.mark.slow
def test_full_size_host_pipeline(S):
    # the bench's end-to-end leg: pinned host buffers through the enqueue
    # pipeline, two products in flight, sampled rows of both results
    n = 16384
    rows = synth.sample_rows(n, 64, 2025)
    with S.Plan(n, 2, S.DType.F32_SPLIT_BF16) as p:
        outs = []
        for seed in (2025, 2026):
            A = torch.from_numpy(synth.normal(n, seed, 0)).pin_memory()
            B = torch.from_numpy(synth.normal(n, seed, 1)).pin_memory()
            C = torch.empty((n, n), dtype=torch.float32).pin_memory()
            p.mul_host_enqueue(A, B, C)
            outs.append((A, B, C))
        p.host_wait()
    for A, B, C in outs:
        a, b = A.numpy(), B.numpy()
        want = oracle.gemm_rows(a, b, rows)
        an, bn = np.linalg.norm(a.astype(np.float64)), np.linalg.norm(b.astype(np.float64))
        check_split(C.numpy()[rows], want, an, bn, "F32_SPLIT_BF16", L=4096)


def test_mul_sharded_single_rank_nccl(S, tmp_path):
    # the sharding path end to end on one GPU: local leaves + NCCL all-reduce
    import datetime
    import socket
    import torch.distributed as dist
    from paper_1811_07325_gb300 import shard
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1,
                            timeout=datetime.timedelta(seconds=60))
    try:
        n = 500
        A = synth.integers(n, 91, 0, -16, 16)
        B = synth.integers(n, 91, 1, -16, 16)
        with S.Plan(n, 2, S.DType.I64) as p:
            C = torch.empty((n, n), dtype=torch.int64, device="cuda")
            shard.mul_sharded(p, dev(A), dev(B), C)
            r0, r1, rows = shard.mul_sharded_rows(p, dev(A), dev(B))
            torch.cuda.synchronize()
        want = oracle.gemm_classical(A, B)
        assert np.array_equal(C.cpu().numpy(), want)
        assert (r0, r1) == (0, n) and np.array_equal(rows[:n].cpu().numpy(), want)
    finally:
        dist.destroy_process_group()


# ----------------------------------------------------------------- sharding one product (rank-local shards)
@pytest.mark.parametrize("dtype,n,d,world", [("F32_SPLIT_BF16", 1024, 2, 3), ("F32_SPLIT_BF16", 2048, 3, 8),
                                             ("F32_SPLIT_TF32", 1001, 2, 2), ("I64", 512, 3, 4),
                                             ("F64", 640, 2, 3)])
def test_shards_partition_the_product(S, dtype, n, d, world):
    # each "rank" (run one after another on this GPU) holds a plan restricted
    # to its leaf range: a smaller workspace, a divide of its own subtrees
    # only; the partial products sum to A.B (int64 bit-exact)
    from paper_1811_07325_gb300 import shard
    if dtype == "I64":
        A, B = synth.integers(n, 69, 0, -16, 16), synth.integers(n, 69, 1, -16, 16)
        want = oracle.gemm_classical(A, B)
    else:
        A, B = synth.normal(n, 69, 0), synth.normal(n, 69, 1)
        if dtype == "F64":
            A, B = A.astype(np.float64), B.astype(np.float64)
        want = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
    dA, dB = dev(A), dev(B)
    with S.Plan(n, d, S.DType[dtype]) as full:
        full_ws, leaves = full.workspace_bytes, full.leaves
    total = None
    for r in range(world):
        with shard.shard_plan(n, d, S.DType[dtype], world, r) as p:
            b, e = shard.leaf_range(leaves, world, r)
            assert p.shard == (b, e) and p.workspace_bytes < full_ws
            with pytest.raises(S.StarkError) as ex:
                p.mul(dA, dB)  # not the whole product
            assert ex.value.status == S.Status.EINVAL
            part = p.mul_leaves(dA, dB, b, e)
            p.check()
            total = part if total is None else total + part
    got = total.cpu().numpy()
    if dtype == "I64":
        assert np.array_equal(got, want)
    elif dtype == "F64":
        an, bn = np.linalg.norm(A), np.linalg.norm(B)
        assert np.abs(got - want).max() / (an * bn) <= 1e-12
    else:
        an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
        L = (n + (128 << d) - 1) // (128 << d) * 128
        check_split(got, want, an, bn, dtype, L=L)


def test_shard_divides_only_its_subtrees(S):
    # the shard's workspace holds exactly the operands of the subtrees that
    # contain its leaves (bit-identical to the oracle's divide for them)
    n, d = 1024, 3
    A = synth.normal(n, 70, 0)
    B = synth.normal(n, 70, 1)
    with S.Plan(n, d, S.DType.F32_SPLIT_BF16) as p:
        p.set_shard(100, 150)
        assert p.shard_levels == 2 and p.shard_first == 98  # groups of 7 leaves: 98 .. 153
        planes = 154 - 98
        L = p.leaf
        X, Y = p.operands(dev(A), dev(B))
        torch.cuda.synchronize()
        for side, got, M in (("A", X, A), ("B", Y, B)):
            ops = oracle.strassen_operands(M, p.n_pad, d, side)[98:154]
            hi, lo = oracle.split_bf16(ops)
            g = got.view(2, planes, L, L).float().cpu().numpy()
            assert np.array_equal(g[0], hi) and np.array_equal(g[1], lo), side
        p.set_shard(0, p.leaves)  # the whole product again
        C = p.mul(dev(A), dev(B)).cpu().numpy()
        p.check()
    want = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
    an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
    check_split(C, want, an, bn, "F32_SPLIT_BF16", A, B, L=L)
