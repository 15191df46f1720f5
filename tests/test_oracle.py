"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself: brute force on tiny
inputs, the paper's formulas restated as a coefficient table and checked
against the Brent equations, closed forms (identity, permutation, rank-1),
the exact integer ring identity, a worked example derived by hand, library
rounding, and floating-point error bounds.  Each test is chosen so that a
plausible slip inside the oracle (a dropped term, a wrong sign, a swapped
index or operand) fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_1811_07325_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# ---------------------------------------------------------------------------
# Alg. 1 (Sec. III-A) restated as a 2x2 coefficient table: rows M1..M7,
# columns the quadrants 11, 12, 21, 22.
U = np.array([[1, 0, 0, 1], [0, 0, 1, 1], [1, 0, 0, 0], [0, 0, 0, 1],
              [1, 1, 0, 0], [-1, 0, 1, 0], [0, 1, 0, -1]])
V = np.array([[1, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, -1], [-1, 0, 1, 0],
              [0, 0, 0, 1], [1, 1, 0, 0], [0, 0, 1, 1]])
# W[c, m]: C quadrant c from M_m.  C22 row with +M3 (corrected) ...
W = np.array([[1, 0, 0, 1, -1, 0, 1], [0, 0, 1, 0, 1, 0, 0],
              [0, 1, 0, 1, 0, 0, 0], [1, -1, 1, 0, 0, 1, 0]])
# ... and exactly as printed, with -M3.
W_PRINTED = W.copy()
W_PRINTED[3, 2] = -1


def brent_residual(U, V, W):
    """max |sum_m W[c,m] U[m,a] V[m,b] - [a,b,c form a classical product term]|.

    For 2x2 blocks, C_{ik} = sum_j A_{ij} B_{jk}; quadrant index = 2*row + col."""
    worst = 0
    for a, b, c in itertools.product(range(4), repeat=3):
        ai, aj = divmod(a, 2)
        bj, bk = divmod(b, 2)
        ci, ck = divmod(c, 2)
        want = 1 if (aj == bj and ai == ci and bk == ck) else 0
        got = sum(W[c, m] * U[m, a] * V[m, b] for m in range(7))
        worst = max(worst, abs(got - want))
    return worst


def test_table_corrected_satisfies_brent_equations():
    assert brent_residual(U, V, W) == 0


def test_table_as_printed_fails_brent_equations():
    # The printed C22 = M1 - M2 - M3 + M6 is not A.B.
    assert brent_residual(U, V, W_PRINTED) > 0


def test_table_replication_counts():
    # Sec. III-C: A11 and A22 are used four times, A12 and A21 twice, 12 in all.
    assert list(np.count_nonzero(U, axis=0)) == [4, 2, 2, 4]
    assert np.count_nonzero(U) == 12 and np.count_nonzero(V) == 12
    assert list(np.count_nonzero(V, axis=0)) == [4, 2, 2, 4]
    # 7 products and 18 additions (Sec. III-A): sums inside the operands plus combine terms.
    adds = sum(max(0, k - 1) for k in np.count_nonzero(U, axis=1)) \
        + sum(max(0, k - 1) for k in np.count_nonzero(V, axis=1)) \
        + sum(max(0, k - 1) for k in np.count_nonzero(W, axis=1))
    assert adds == 18


def _read_golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            rows[key] = vals
    return rows


def test_worked_2x2_example():
    g = _read_golden("strassen_2x2_worked.txt")
    A = np.array([int(v) for v in g["A"]], dtype=np.int64).reshape(2, 2)
    B = np.array([int(v) for v in g["B"]], dtype=np.int64).reshape(2, 2)
    C = np.array([int(v) for v in g["C"]], dtype=np.int64).reshape(2, 2)
    assert np.array_equal(oracle.strassen(A, B, 1), C)
    assert np.array_equal(oracle.strassen(A.astype(float), B.astype(float), 1), C.astype(float))
    # the divide oracle forms the operands of each M_i
    Xa = oracle.strassen_operands(A.astype(np.float32), 2, 1, "A").reshape(7)
    Yb = oracle.strassen_operands(B.astype(np.float32), 2, 1, "B").reshape(7)
    M = Xa.astype(np.int64) * Yb.astype(np.int64)
    assert [int(v) for v in M] == [int(g[f"M{i}"][0]) for i in range(1, 8)]
    assert int(W_PRINTED[3] @ M) == int(g["C22_as_printed"][0])
    assert int(W[3] @ M) == int(g["C"][3])


def test_strassen_depth1_all_basis_pairs():
    # Bilinearity: agreeing on every pair of basis matrices E_ij, E_kl is the
    # full identity for 2x2 blocks.  E_ij E_kl = delta_jk E_il.
    for i, j, k, l in itertools.product(range(2), repeat=4):
        A = np.zeros((2, 2), np.int64); A[i, j] = 1
        B = np.zeros((2, 2), np.int64); B[k, l] = 1
        want = np.zeros((2, 2), np.int64)
        if j == k:
            want[i, l] = 1
        assert np.array_equal(oracle.strassen(A, B, 1), want), (i, j, k, l)


def brute_force(A, B):
    n = len(A)
    return [[sum(A[i][k] * B[k][j] for k in range(n)) for j in range(n)] for i in range(n)]


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_classical_int_vs_brute_force(n):
    for seed in range(5):
        A = synth.integers(n, seed, 0, -50, 50)
        B = synth.integers(n, seed, 1, -50, 50)
        want = np.array(brute_force(A.tolist(), B.tolist()), dtype=np.int64)
        assert np.array_equal(oracle.gemm_classical(A, B), want)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 8])
def test_classical_f64_vs_python_loop(n):
    # Same k order in Python floats (IEEE double, no fused multiply-add).
    A = synth.uniform(n, 7, 0)
    B = synth.uniform(n, 7, 1)
    want = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            s = 0.0
            for k in range(n):
                s = s + float(A[i, k]) * float(B[k, j])
            want[i, j] = s
    assert np.array_equal(oracle.gemm_classical(A, B), want)


def test_classical_int_wraps_like_numpy():
    # numpy's int64 matmul wraps modulo 2^64 as well: an independent library routine.
    n = 48
    A = synth.integers(n, 3, 0, -2**62, 2**62)
    B = synth.integers(n, 3, 1, -2**62, 2**62)
    with np.errstate(over="ignore"):
        want = A @ B
    assert np.array_equal(oracle.gemm_classical(A, B), want)


def test_wrapping_matches_big_integers():
    n = 4
    A = synth.integers(n, 11, 0, -2**63, 2**63 - 1)
    B = synth.integers(n, 11, 1, -2**63, 2**63 - 1)
    big = brute_force([[int(v) for v in r] for r in A], [[int(v) for v in r] for r in B])
    want = np.array([[((v + 2**63) % 2**64) - 2**63 for v in r] for r in big], dtype=np.int64)
    assert np.array_equal(oracle.gemm_classical(A, B), want)
    for d in (1, 2):
        assert np.array_equal(oracle.strassen(A, B, d), want)


@pytest.mark.parametrize("n,depths", [(2, [1]), (4, [1, 2]), (8, [1, 2, 3]), (16, [1, 2, 3, 4]),
                                      (64, [1, 3, 6]), (256, [1, 2, 4]), (6, [1]), (12, [2]),
                                      (20, [2, 3]), (33, [1, 2]), (100, [3])])
def test_strassen_int_equals_classical(n, depths):
    A = synth.integers(n, n, 0, -16, 16)
    B = synth.integers(n, n, 1, -16, 16)
    C = oracle.gemm_classical(A, B)
    for d in depths:
        assert np.array_equal(oracle.strassen(A, B, d), C), d


def test_strassen_int_equals_classical_every_size_to_256():
    """Every n <= 256 at every depth the GPU path supports (0..4, while 2^d
    does not exceed the padded side); for n <= 32 also every deeper depth,
    down to 1 x 1 leaves.  Exact integers leave one correct answer."""
    for n in range(1, 257):
        A = synth.integers(n, 900 + n, 0, -16, 16)
        B = synth.integers(n, 900 + n, 1, -16, 16)
        C = oracle.gemm_classical(A, B)
        top = max(1, math.ceil(math.log2(max(n, 2))))
        for d in range(0, (top if n <= 32 else min(4, top)) + 1):
            assert np.array_equal(oracle.strassen(A, B, d), C), (n, d)


def test_strassen_int_depth0_is_classical():
    A = synth.integers(10, 1, 0, -5, 5)
    B = synth.integers(10, 1, 1, -5, 5)
    assert np.array_equal(oracle.strassen(A, B, 0), oracle.gemm_classical(A, B))


@pytest.mark.parametrize("d", [1, 2, 3])
def test_identity_and_permutation(d):
    n = 16
    B = synth.integers(n, 5, 1, -1000, 1000)
    I = np.eye(n, dtype=np.int64)
    assert np.array_equal(oracle.strassen(I, B, d), B)
    assert np.array_equal(oracle.strassen(B, I, d), B)
    perm = np.roll(np.arange(n), 5)[::-1].copy()
    P = np.zeros((n, n), np.int64)
    P[np.arange(n), perm] = 1
    # (P B)[i, :] = B[perm[i], :] and (B P^T)[:, i] = B[:, perm[i]]
    assert np.array_equal(oracle.strassen(P, B, d), B[perm, :])
    assert np.array_equal(oracle.strassen(B, P.T.copy(), d), B[:, perm])
    # float path: integer-valued doubles stay exact
    assert np.array_equal(oracle.strassen(P.astype(float), B.astype(float), d), B[perm, :].astype(float))


@pytest.mark.parametrize("d", [1, 2, 3])
def test_rank1_closed_form_int(d):
    # (u v^T)(w z^T) = (v . w) u z^T
    n = 32
    u, v, w, z = (synth.integers(1, 40 + k, 0, -9, 9, m=n)[0] for k in range(4))
    A, B = np.outer(u, v), np.outer(w, z)
    want = int(v @ w) * np.outer(u, z)
    assert np.array_equal(oracle.strassen(A, B, d), want)
    assert np.array_equal(oracle.gemm_classical(A, B), want)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_rank1_closed_form_f64(d):
    n = 64
    u, v, w, z = (synth.uniform(1, 50 + k, 0, m=n)[0] for k in range(4))
    A, B = np.outer(u, v), np.outer(w, z)
    want = math.fsum(v * w) * np.outer(u, z)
    got = oracle.strassen(A, B, d)
    # normwise bound: Strassen's error grows by at most ~12^d over classical's n*eps
    scale = np.linalg.norm(A) * np.linalg.norm(B)
    assert np.max(np.abs(got - want)) <= (n + 12 ** d) * 2.0 ** -52 * scale * 4


@pytest.mark.parametrize("n,d", [(100, 2), (128, 3), (256, 4)])
def test_strassen_f64_error_bound(n, d):
    A = synth.uniform(n, 2, 0)
    B = synth.uniform(n, 2, 1)
    classical = oracle.gemm_classical(A, B)
    got = oracle.strassen(A, B, d)
    # Higham, "Accuracy and Stability of Numerical Algorithms" (2nd ed.), Thm. 23.2:
    # max-norm error of Strassen with d levels over classical leaves of side L is
    # at most [12^d (L^2 + 5L) - 5n] u ||A|| ||B|| to first order; the classical
    # reference itself is within n u ||A|| ||B||.
    u = 2.0 ** -53
    L = -(-n // 2 ** d)
    bound = 2 * ((12 ** d * (L * L + 5 * L) - 5 * n) + n) * u * np.abs(A).max() * np.abs(B).max()
    err = np.max(np.abs(got - classical))
    assert err <= bound
    assert err > 0  # floats do round: the check is not vacuous
    # computing any level in fp32 instead would blow the bound
    assert 2.0 ** -24 * np.abs(classical).max() > bound


def test_padding_keeps_top_left_block():
    n = 37
    A = synth.integers(n, 9, 0, -16, 16)
    B = synth.integers(n, 9, 1, -16, 16)
    C = oracle.gemm_classical(A, B)
    for d in (1, 2, 3, 5):
        assert np.array_equal(oracle.strassen(A, B, d), C)


def test_empty_matrix():
    A = np.zeros((0, 0), np.int64)
    assert oracle.strassen(A, A, 2).shape == (0, 0)


def test_rows_match_full_product():
    n = 40
    A = synth.normal(n, 1, 0)
    B = synth.normal(n, 1, 1)
    rows = synth.sample_rows(n, 7, 3)
    full = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
    assert np.array_equal(oracle.gemm_rows(A, B, rows), full[rows])
    assert np.array_equal(oracle.gemm_rows(A.astype(np.float64), B.astype(np.float64), rows), full[rows])


# ---------------------------------------------------------------------------
# Divide phase: leaf operand sums


def kron_table(T, d):
    out = np.ones((1, 1), dtype=np.int64)
    for _ in range(d):
        out = np.kron(out, T)
    return out


def quadrant_blocks(X, d):
    """Sub-blocks of X by base-4 quadrant path, top level most significant."""
    n = X.shape[0]
    L = n >> d
    blocks = []
    for q in range(4 ** d):
        r = c = 0
        for k in range(d):
            digit = (q // 4 ** (d - 1 - k)) % 4
            r += (digit >> 1) * (n >> (k + 1))
            c += (digit & 1) * (n >> (k + 1))
        blocks.append(X[r:r + L, c:c + L])
    return blocks


@pytest.mark.parametrize("n,npad,d", [(8, 8, 1), (16, 16, 2), (12, 16, 2), (32, 32, 3), (24, 32, 3)])
def test_operands_reproduce_product(n, npad, d):
    # Small integers: every sum and product is exact in fp32/fp64, so
    # sum_l W_d[q, l] X_l Y_l must reproduce A.B exactly (zero padded).
    A = synth.integers(n, d, 0, -8, 8)
    B = synth.integers(n, d, 1, -8, 8)
    X = oracle.strassen_operands(A.astype(np.float32), npad, d, "A").astype(np.int64)
    Y = oracle.strassen_operands(B.astype(np.float32), npad, d, "B").astype(np.int64)
    Wd = kron_table(W, d)
    L = npad >> d
    C = np.zeros((npad, npad), np.int64)
    Cq = quadrant_blocks(C, d)
    for l in range(7 ** d):
        M = X[l] @ Y[l]
        for q in range(4 ** d):
            if Wd[q, l]:
                Cq[q] += Wd[q, l] * M
    Ap = np.zeros((npad, npad), np.int64); Ap[:n, :n] = A
    Bp = np.zeros((npad, npad), np.int64); Bp[:n, :n] = B
    assert np.array_equal(C, Ap @ Bp)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_operands_are_kronecker_sums(d):
    # X_l = sum_q U_d[l, q] A_q with U_d the d-fold Kronecker power of the 2x2 table.
    n = 8 << d
    A = synth.integers(n, 21, 0, -100, 100).astype(np.float32)
    B = synth.integers(n, 21, 1, -100, 100).astype(np.float32)
    for side, T, X in (("A", U, A), ("B", V, B)):
        got = oracle.strassen_operands(X, n, d, side)
        Td = kron_table(T, d)
        blocks = quadrant_blocks(X.astype(np.int64), d)
        for l in range(7 ** d):
            want = sum(int(Td[l, q]) * blocks[q] for q in range(4 ** d) if Td[l, q])
            assert np.array_equal(got[l].astype(np.int64), want), (side, l)


def test_operands_fp32_rounding_is_per_level():
    # The divide adds two fp32 values per level; with values that round, the
    # result must equal level-by-level fp32 addition, not an exact sum.
    n = 4
    A = np.array([[1.0, 2**-30, 3.0, 2**-25], [5.0, 6.0, 7.0, 8.0],
                  [2**24, 1.0, 1.5, 2**-24], [1.0, 2.0, 3.0, 4.0]], dtype=np.float32)
    got = oracle.strassen_operands(A, 4, 2, "A")
    f = np.float32
    q = [A[:2, :2], A[:2, 2:], A[2:, :2], A[2:, 2:]]
    lvl1 = [f(q[0] + q[3]), f(q[2] + q[3]), q[0], q[3], f(q[0] + q[1]), f(q[2] - q[0]), f(q[1] - q[3])]
    for i1 in range(7):
        s = lvl1[i1]
        a11, a12, a21, a22 = s[0, 0], s[0, 1], s[1, 0], s[1, 1]
        lvl2 = [f(a11 + a22), f(a21 + a22), a11, a22, f(a11 + a12), f(a21 - a11), f(a12 - a22)]
        for i2 in range(7):
            assert got[i1 * 7 + i2, 0, 0] == lvl2[i2], (i1, i2)


# ---------------------------------------------------------------------------
# Rounding to tensor-core formats


def test_round_ties_golden():
    with open(os.path.join(GOLDEN, "round_ties.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            bits, x, want = line.split()
            got = oracle.round_sig(float.fromhex(x), int(bits))
            assert got == float.fromhex(want), line


def test_bf16_split_matches_library_rounding():
    torch = pytest.importorskip("torch")
    x = np.concatenate([synth.normal(256, 4, 0).reshape(-1),
                        synth.uniform(64, 4, 1, dtype=np.float32).reshape(-1) * 1e-38,
                        np.array([0.0, -0.0, 1.0 + 2**-8, 3.0e38, 1e-45], np.float32)]).astype(np.float32)
    hi, lo = oracle.split_bf16(x)
    t = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(hi, t)
    r = (x - hi).astype(np.float32)
    t2 = torch.from_numpy(r).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(lo, t2)


def _tf32_bits_reference(x):
    # Bit-level RN-even to 10 stored mantissa bits on the float32 pattern.
    u = x.view(np.uint32).astype(np.uint64)
    low = u & 0x1FFF
    base = u & ~np.uint64(0x1FFF) & 0xFFFFFFFF
    keep_odd = (u >> 13) & 1
    up = (low > 0x1000) | ((low == 0x1000) & (keep_odd == 1))
    out = (base + np.where(up, 0x2000, 0)).astype(np.uint32)
    return out.view(np.float32)


def test_tf32_split_matches_bit_reference():
    x = np.concatenate([synth.normal(128, 6, 0).reshape(-1),
                        np.array([1.0 + 2**-11, 1.0 + 3 * 2**-11, -(1.0 + 3 * 2**-11), 0.0], np.float32)])
    x = x.astype(np.float32)
    hi, lo = oracle.split_tf32(x)
    assert np.array_equal(hi, _tf32_bits_reference(x))
    assert np.array_equal(lo, _tf32_bits_reference((x - hi).astype(np.float32)))


def _fp16_cases():
    # normals over the whole binary16 range, the subnormal range, exact
    # halfway points (ties) at several exponents, the overflow threshold
    x = [synth.normal(128, 9, 0).reshape(-1),
         synth.normal(64, 9, 1).reshape(-1) * 1e4,
         synth.normal(64, 9, 2).reshape(-1) * 3e-5,   # around the normal/subnormal edge
         synth.normal(64, 9, 3).reshape(-1) * 1e-7]   # subnormal, some below half the spacing
    ties = []
    for e in (-20, -14, -3, 0, 7, 14):
        ulp = 2.0 ** (e - 10) if e >= -14 else 2.0 ** -24
        for k in (1025, 1026, 2047, 1500):
            ties.append((k + 0.5) * ulp * (1 if k % 2 else -1))
    ties += [65504.0, 65519.0, 65520.0, 65536.0, -65520.0, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26, 0.0, -0.0]
    return np.concatenate(x + [np.array(ties)]).astype(np.float32)


def test_fp16_rounding_matches_library_conversion():
    # binary16 round to nearest even, subnormals and overflow included, equals
    # numpy's float32 -> float16 conversion element for element
    x = _fp16_cases()
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).astype(np.float32)
    got = np.array([oracle.round_fp16(float(v)) for v in x], dtype=np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    hi, lo = oracle.split_fp16(x)
    assert np.array_equal(hi.view(np.uint32), ref.view(np.uint32))
    fin = np.isfinite(hi)
    r = (x[fin] - hi[fin]).astype(np.float32)
    assert np.array_equal(lo[fin].view(np.uint32), r.astype(np.float16).astype(np.float32).view(np.uint32))
    assert not np.all(fin)  # the overflow cases are there


def test_fp16_split_reconstruction_error():
    # hi and lo carry 11 bits each where lo stays normal: the remainder is
    # below 2^-22 relative; below that, lo rounds to the fixed subnormal
    # spacing 2^-24, an absolute error of at most 2^-25
    x = np.concatenate([synth.normal(512, 10, 0).reshape(-1),
                        synth.normal(64, 10, 1).reshape(-1) * 1e-5]).astype(np.float32)
    hi, lo = oracle.split_fp16(x)
    x64 = x.astype(np.float64)
    err = np.abs(x64 - (hi.astype(np.float64) + lo.astype(np.float64)))
    assert np.all(err <= np.maximum(2.0 ** -22 * np.abs(x64), 2.0 ** -25))
    big = np.abs(x64) >= 2.0 ** -3  # lo normal: the relative bound alone
    assert np.all(err[big] <= 2.0 ** -22 * np.abs(x64[big]))
    assert (err[big] / np.abs(x64[big])).max() > 2.0 ** -30  # and lo is really rounded


@pytest.mark.parametrize("split,bits", [(oracle.split_bf16, 8), (oracle.split_tf32, 11)])
def test_split_reconstruction_error(split, bits):
    x = synth.normal(512, 8, 0).reshape(-1)
    hi, lo = split(x)
    x64 = x.astype(np.float64)
    rel = np.abs(x64 - (hi.astype(np.float64) + lo.astype(np.float64))) / np.abs(x64)
    # hi carries `bits` bits, lo the next `bits`: the remainder is below 2^-(2 bits) relative
    assert rel.max() <= 2.0 ** (-2 * bits)
    assert rel.max() > 2.0 ** (-2 * bits - 8)  # and lo is really truncated


# ---------------------------------------------------------------------------
# The error majorant (oracle.strassen_abs): Alg. 1 on |A|, |B| with every
# sign +.  Pinned by the classical product at depth 0, by its closed form on
# the all-ones matrix, by the literal 2x2 formulas and by dominance over
# |A||B|; then used to show what the split-precision bounds catch.
T_ABS = (12, 4, 4, 12)  # quadrant products (all signs +) in C11, C12, C21, C22 of one level


@pytest.mark.parametrize("d", [0, 1, 2, 3])
def test_strassen_abs_depth0_and_dominance(d):
    # exact small integers (every sum exact in fp64); at depth 0 the
    # majorant is the classical |A||B|, at every depth it dominates it
    n = 24
    A = synth.integers(n, 40 + d, 0, -9, 9)
    B = synth.integers(n, 40 + d, 1, -9, 9)
    S = oracle.strassen_abs(A.astype(np.float64), B.astype(np.float64), d)
    absAB = (np.abs(A) @ np.abs(B)).astype(np.float64)
    if d == 0:
        assert np.array_equal(S, absAB)
    else:
        assert np.all(S >= absAB) and np.any(S > absAB)
    assert np.array_equal(oracle.strassen_abs(-A.astype(np.float64), B.astype(np.float64), d), S)  # |.| of the inputs


@pytest.mark.parametrize("d", [1, 2, 3])
def test_strassen_abs_closed_form_on_ones(d):
    # all-ones n x n: every quadrant product of side h is h, so
    # S_ij = L * prod over levels of the count of quadrant products in the
    # C quadrant that (i, j) falls in: 12 (C11, C22) or 4 (C12, C21)
    n = 8 << d
    S = oracle.strassen_abs(np.ones((n, n)), np.ones((n, n)), d)
    L = n >> d
    want = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            v = L
            for k in range(1, d + 1):
                q = 2 * ((i >> (int(math.log2(n)) - k)) & 1) + ((j >> (int(math.log2(n)) - k)) & 1)
                v *= T_ABS[q]
            want[i, j] = v
    assert np.array_equal(S, want)


def test_strassen_abs_2x2_literal():
    # depth 1 on 2x2 scalars, the seven products with absolute values written out
    a11, a12, a21, a22 = 3.0, -1.0, 2.0, -5.0
    b11, b12, b21, b22 = -2.0, 4.0, 1.0, 6.0
    A = np.array([[a11, a12], [a21, a22]])
    B = np.array([[b11, b12], [b21, b22]])
    x = lambda v: abs(v)  # noqa: E731
    m1 = (x(a11) + x(a22)) * (x(b11) + x(b22))
    m2 = (x(a21) + x(a22)) * x(b11)
    m3 = x(a11) * (x(b12) + x(b22))
    m4 = x(a22) * (x(b21) + x(b11))
    m5 = (x(a11) + x(a12)) * x(b22)
    m6 = (x(a21) + x(a11)) * (x(b11) + x(b12))
    m7 = (x(a12) + x(a22)) * (x(b21) + x(b22))
    want = np.array([[m1 + m4 + m5 + m7, m3 + m5], [m2 + m4, m1 + m2 + m3 + m6]])
    assert np.array_equal(oracle.strassen_abs(A, B, 1), want)


def emulated_split_product(A, B, d, drop=None, split=None):
    """The 3xBF16 Strassen product emulated on the CPU from the oracle's
    pieces: fp32 leaf operands (the divide), their bf16 hi/lo split, the
    three kept products per leaf in fp64, combined by W_d.  drop = (leaf,
    row0, col0, size): that tile of that leaf's product is left out, the
    way a lost output tile of the leaf kernel would be.  split: another
    split of the oracle (the fp16 one)."""
    split = split or oracle.split_bf16
    n = A.shape[0]
    L = n >> d
    X = oracle.strassen_operands(A, n, d, "A")
    Y = oracle.strassen_operands(B, n, d, "B")
    xh, xl = split(X)
    yh, yl = split(Y)
    Wd = kron_table(W, d)
    C = np.zeros((n, n))
    Cq = quadrant_blocks(C, d)
    for l in range(7 ** d):
        M = xh[l].astype(np.float64) @ yh[l] + xh[l].astype(np.float64) @ yl[l] + xl[l].astype(np.float64) @ yh[l]
        if drop is not None and drop[0] == l:
            _, r0, c0, s = drop
            M[r0:r0 + s, c0:c0 + s] = 0.0
        for q in range(4 ** d):
            if Wd[q, l]:
                Cq[q] += Wd[q, l] * M
    return C, L


@pytest.mark.parametrize("kc", [None, 128])
@pytest.mark.parametrize("d", [1, 2])
def test_split_bounds_pass_correct_and_catch_a_dropped_tile(d, kc):
    # the bars of the GPU parity tests (tests/bounds.py): the emulated split
    # product meets them, and the same product with one 128 x 128 output
    # tile of one leaf left out fails both the componentwise bound and the
    # relative RMS bound -- also with the tighter bars of accumulator
    # promotion every kc of K
    import bounds
    n = 512
    A = synth.normal(n, 50 + d, 0)
    B = synth.normal(n, 50 + d, 1)
    want = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
    S = oracle.strassen_abs(A.astype(np.float64), B.astype(np.float64), d)
    C, L = emulated_split_product(A, B, d)
    c = bounds.componentwise_c("F32_SPLIT_BF16", L, d, kc)
    rms = bounds.rms_bound("F32_SPLIT_BF16", L, d, kc)
    rel = lambda X: np.sqrt(np.mean((X - want) ** 2)) / np.sqrt(np.mean(want ** 2))  # noqa: E731
    assert np.all(np.abs(C - want) <= c * S)
    assert rel(C) <= rms
    leaf = 7 ** d - 3  # a leaf with targets in several quadrants
    Cbad, _ = emulated_split_product(A, B, d, drop=(leaf, L - 128, 0, 128))
    assert not np.all(np.abs(Cbad - want) <= c * S)
    assert rel(Cbad) > rms


@pytest.mark.parametrize("d", [1, 2])
def test_fp16_bound_needs_and_holds_with_its_floor_term(d):
    # fp16 halves keep values below 2^-14 only to the spacing 2^-24: rows of A
    # scaled into that range lose relative accuracy, which the relative term
    # c S alone does not cover; with the absolute floor 2^-25 F (F: the
    # majorant of |A| with the all-ones matrix and of it with |B|) the bound
    # holds for the emulated 3xFP16 product, and it still catches a dropped
    # 128 x 128 output tile
    import bounds
    n = 512
    A = synth.normal(n, 60 + d, 0)
    B = synth.normal(n, 60 + d, 1)
    A[: n // 4] *= 2.0 ** -18  # a quarter of the rows far below fp16's normal range
    want = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    S = oracle.strassen_abs(A64, B64, d)
    L = n >> d
    F = bounds.floor_majorant(oracle, A64, B64, d, L)
    c = bounds.componentwise_c("F32_SPLIT_FP16", L, d)
    C, _ = emulated_split_product(A, B, d, split=oracle.split_fp16)
    err = np.abs(C - want)
    assert not np.all(err <= c * S)  # the relative term alone is not enough
    bound = c * S + bounds.FLOOR["F32_SPLIT_FP16"] * F
    assert np.all(err <= bound), float((err / bound).max())
    leaf = 7 ** d - 3
    Cbad, _ = emulated_split_product(A, B, d, drop=(leaf, L - 128, 0, 128), split=oracle.split_fp16)
    assert not np.all(np.abs(Cbad - want) <= bound)


def test_promoted_bounds_shrink_the_accumulation_term():
    # promotion every kc of K: one tensor-core accumulation spans kc instead
    # of L (3 kc / k MMA steps of at most 2 ulp) plus ceil(L / kc) - 1
    # round-to-nearest fp32 additions; kc >= L or 0 leaves the bound as is
    import bounds
    for dt in ("F32_SPLIT_BF16", "F32_SPLIT_TF32"):
        for L, d in ((4096, 2), (2048, 3), (768, 1)):
            base_c, base_r = bounds.componentwise_c(dt, L, d), bounds.rms_bound(dt, L, d)
            assert bounds.componentwise_c(dt, L, d, 0) == base_c
            assert bounds.componentwise_c(dt, L, d, L) == base_c
            assert bounds.rms_bound(dt, L, d, 2 * L) == base_r
            prev = base_c
            for kc in (512, 256):
                if kc >= L:
                    continue
                cc = bounds.componentwise_c(dt, L, d, kc)
                assert cc < prev
                acc_full = 3 * L / bounds.MMA_K[dt] * 2.0 ** -22
                acc_kc = 3 * kc / bounds.MMA_K[dt] * 2.0 ** -22 + (-(-L // kc) - 1) * 2.0 ** -24
                assert cc == pytest.approx(base_c - acc_full + acc_kc)
                assert bounds.rms_bound(dt, L, d, kc) < base_r
                prev = cc
