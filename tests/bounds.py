"""Accuracy bounds of the split-precision path, derived from its arithmetic.

Shared by the CPU tests that show what the bounds catch and by the GPU
parity tests.  Notation: u = the relative residual of one operand split
x = hi + lo + r (|r| <= u |x|: two roundings to 8 significant bits for
bf16, u = 2^-16; to 11 bits for tf32, u = 2^-22), L = leaf side, k = inputs
per tensor-core MMA step (16 bf16, 8 tf32), d = recursion depth.

* componentwise_c: |dC_ij| <= c S_ij, S = oracle.strassen_abs (Alg. 1 on
  |A|, |B| with every sign +).  Per leaf product term x y the three kept
  products miss lo_x lo_y and the two residual terms (<= 3u |x y|); the
  fp32 accumulation takes 3 L / k MMA steps, each off by at most 2 ulp
  (2^-22, the tensor cores' rounding is not specified as round-to-nearest)
  of the running sum of |terms|; the divide forms each operand with one
  fp32 addition per level (2^-24 per level and operand, 2d); the combine
  adds 3^d contributions per element in fp32 (2^-24 each).  Every one of
  these is at most its coefficient times the matching term of S.
* rms_bound: rms(dC) / rms(C) for i.i.d. inputs.  The split's error per
  product has RMS below u; Strassen's operand sums grow it by 2^d (per
  level an output quadrant sums 8 quadrant products on average, against 2
  for the classical product, over half the inner dimension: sqrt(8/2) = 2);
  the accumulation adds at most 3 (L / k) ulp of 2^-23 (no cancellation
  assumed).
* With accumulator promotion every kc of K (stark_plan_set_promotion) one
  tensor-core accumulation spans min(L, kc) instead of L, and the chunks'
  partial sums are added on the CUDA cores with round to nearest:
  ceil(L / kc) - 1 additions of at most 2^-24 of the running sum of |terms|
  each.  Measured on GB300, the accumulation error of the tensor core grows
  in proportion to the K it spans (3xTF32 at n = 16384, d = 2: relative RMS
  2.96e-5 over 4096, 1.5e-5 over 2048, 4.0e-6 over 512, 2.2e-6 over 256),
  the signature of a biased rounding of the running sum.
"""
import math

import numpy as np

U_SPLIT = {"F32_SPLIT_BF16": 2.0 ** -16, "F32_SPLIT_TF32": 2.0 ** -22, "F32_SPLIT_FP16": 2.0 ** -22}
MMA_K = {"F32_SPLIT_BF16": 16, "F32_SPLIT_TF32": 8, "F32_SPLIT_FP16": 16}
# fp16 halves: below fp16's normal range (2^-14) values are kept to the
# fixed spacing 2^-24, so a split's residual is max(2^-22 |x|, 2^-25)
FLOOR = {"F32_SPLIT_FP16": 2.0 ** -25}


def _span(L, kc):
    """K of one tensor-core accumulation and the fp32 additions of the
    chunks (promotion every kc of K; kc = None or 0: none)."""
    if not kc or kc >= L:
        return L, 0
    return kc, -(-L // kc) - 1


def componentwise_c(dtype, L, d, kc=None):
    span, adds = _span(L, kc)
    return (3 * U_SPLIT[dtype] + (3 * span / MMA_K[dtype]) * 2.0 ** -22 + adds * 2.0 ** -24
            + (2 * d + 3 ** d) * 2.0 ** -24)


def rms_bound(dtype, L, d, kc=None):
    span, adds = _span(L, kc)
    return 2 ** d * U_SPLIT[dtype] + 3 * (span / MMA_K[dtype]) * 2.0 ** -23 + adds * 2.0 ** -24


def floor_majorant(oracle, A, B, d, L):
    """The absolute part of the split residual: an operand element off by up
    to f absolutely moves C_ij by at most f times this majorant (Alg. 1 on
    |A| with the all-ones matrix, and on the all-ones matrix with |B|; the
    ones cover the n x n inputs, the zero padding splits exactly)."""
    J = np.ones(A.shape)
    return majorant(oracle, A, J, d, L) + majorant(oracle, J, B, d, L)


def infer_depth(n, L):
    """Recursion depth of a product of side n whose leaves have side L
    (n_pad = L 2^d with n <= n_pad < 2 n, or L >= n at depth 0)."""
    return max(0, math.ceil(math.log2(n / L) - 1e-9)) if L < n else 0


def majorant(oracle, A, B, d, L):
    """S of the zero-padded L 2^d square product (the padding the recursion
    uses), cut to n x n."""
    n = A.shape[0]
    m = L << d
    Ap = np.zeros((m, m)); Ap[:n, :n] = A
    Bp = np.zeros((m, m)); Bp[:n, :n] = B
    return oracle.strassen_abs(Ap, Bp, d)[:n, :n]
