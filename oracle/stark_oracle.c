/*
 * stark_oracle.c -- plain, slow, obviously-correct CPU reference for the
 * Strassen path of "Stark: Fast and Scalable Strassen's Matrix Multiplication
 * using Apache Spark" (arXiv 1811.07325).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or helper with the CUDA
 * path.
 *
 * What it computes, and the passage each function follows:
 *   oracle_gemm_classical_{f64,i64}   C_ij = sum_k A_ik B_kj, k ascending: the
 *                                     "naive approach" used at the leaves of
 *                                     Alg. 1 (Sec. III-A) and the definition
 *                                     the Strassen result must equal.
 *   oracle_gemm_rows_f64              the same definition evaluated for a list
 *                                     of rows only (large-n sampling).
 *   oracle_strassen_{f64,i64}         Alg. 1 (Sec. III-A): 2x2 split, the seven
 *                                     products M1..M7, then C11..C22, recursing
 *                                     `depth` times and multiplying classically
 *                                     at the leaves.  C22 uses +M3 (the printed
 *                                     -M3 is a sign typo: only +M3 makes the
 *                                     identity equal A*B).
 *   oracle_strassen_abs_f64           Alg. 1 with every input entry and every
 *                                     +-1 coefficient of its sums and of its
 *                                     combine replaced by its absolute value:
 *                                     the majorant S of the recursion's
 *                                     rounding errors (each leaf term
 *                                     a_ik b_kj enters S_ij with weight 1), so
 *                                     a relative error e per leaf product or
 *                                     addition bounds |dC_ij| by about e S_ij.
 *   oracle_strassen_operands_f32      the divide phase of Alg. 1 / Alg. 3
 *                                     (Sec. III-C): the leaf operand sums of
 *                                     all 7^depth leaves, each level forming
 *                                     the two-term sums of Alg. 1 in fp32.
 *   oracle_round_bf16 / _tf32         round-to-nearest-even of an fp32 value
 *                                     to bfloat16 (8 significant bits) or
 *                                     TF32 (11 significant bits), written from
 *                                     the definition (nearest representable,
 *                                     ties to even significand).
 *   oracle_round_fp16                 the same to IEEE binary16 (11
 *                                     significant bits, exponent range
 *                                     2^-14 .. 2^15, subnormal spacing 2^-24,
 *                                     overflow to infinity); the split of the
 *                                     3xFP16 leaves.
 *
 * Integer arithmetic is done in uint64_t so that it wraps modulo 2^64 (two's
 * complement); Strassen's identities hold in any commutative ring, so the
 * wrapped Strassen result equals the wrapped classical result bit for bit.
 *
 * Leaf numbering: a leaf is identified by its path of M-indices (i_1..i_d),
 * i_k in 0..6 meaning M_{i_k+1} at recursion level k, packed as the base-7
 * number i_1*7^(d-1) + ... + i_d (top level most significant), so that the
 * parent of a leaf is its index divided by 7 (Alg. 5, Sec. III-C).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------ */
/* Classical product (the definition)                                  */
/* ------------------------------------------------------------------ */

/* C = A*B for row-major n x n matrices; every C_ij accumulates k = 0..n-1 in
 * order, in double.  (Alg. 1's leaf, "naive approach".) */
void oracle_gemm_classical_f64(int64_t n, const double *A, const double *B, double *C)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double *crow = C + i * n;
        for (int64_t j = 0; j < n; ++j) crow[j] = 0.0;
        for (int64_t k = 0; k < n; ++k) {
            const double a = A[i * n + k];
            const double *brow = B + k * n;
            for (int64_t j = 0; j < n; ++j) crow[j] += a * brow[j];
        }
    }
}

/* Integer version, modulo 2^64. */
void oracle_gemm_classical_i64(int64_t n, const int64_t *A, const int64_t *B, int64_t *C)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        uint64_t *crow = (uint64_t *)(C + i * n);
        for (int64_t j = 0; j < n; ++j) crow[j] = 0;
        for (int64_t k = 0; k < n; ++k) {
            const uint64_t a = (uint64_t)A[i * n + k];
            const uint64_t *brow = (const uint64_t *)(B + k * n);
            for (int64_t j = 0; j < n; ++j) crow[j] += a * brow[j];
        }
    }
}

/* Rows rows[0..nrows) of C = A*B (n x n, row-major), written densely to
 * Crows[r*n + j].  Same k-ascending order as the full product. */
void oracle_gemm_rows_f64(int64_t n, const int64_t *rows, int64_t nrows,
                          const double *A, const double *B, double *Crows)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t i = rows[r];
        double *crow = Crows + r * n;
        for (int64_t j = 0; j < n; ++j) crow[j] = 0.0;
        for (int64_t k = 0; k < n; ++k) {
            const double a = A[i * n + k];
            const double *brow = B + k * n;
            for (int64_t j = 0; j < n; ++j) crow[j] += a * brow[j];
        }
    }
}

/* Same rows for fp32 inputs, widened to double before use. */
void oracle_gemm_rows_f32in(int64_t n, const int64_t *rows, int64_t nrows,
                            const float *A, const float *B, double *Crows)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t i = rows[r];
        double *crow = Crows + r * n;
        for (int64_t j = 0; j < n; ++j) crow[j] = 0.0;
        for (int64_t k = 0; k < n; ++k) {
            const double a = (double)A[i * n + k];
            const float *brow = B + k * n;
            for (int64_t j = 0; j < n; ++j) crow[j] += a * (double)brow[j];
        }
    }
}

/* ------------------------------------------------------------------ */
/* Strassen recursion, Alg. 1                                          */
/* ------------------------------------------------------------------ */

/* Views of square sub-blocks inside a larger row-major array. */
typedef struct { double *p; int64_t ld; } dview;
typedef struct { uint64_t *p; int64_t ld; } uview;

static dview dsub(dview v, int64_t m, int r, int c)
{ dview s = { v.p + (int64_t)r * m * v.ld + (int64_t)c * m, v.ld }; return s; }
static uview usub(uview v, int64_t m, int r, int c)
{ uview s = { v.p + (int64_t)r * m * v.ld + (int64_t)c * m, v.ld }; return s; }

static dview dalloc(int64_t m)
{ dview v = { (double *)calloc((size_t)(m * m), sizeof(double)), m }; return v; }
static uview ualloc(int64_t m)
{ uview v = { (uint64_t *)calloc((size_t)(m * m), sizeof(uint64_t)), m }; return v; }

/* out = x + s*y, s in {+1,-1}; s == 0 means out = x. */
static void dadd(int64_t m, dview x, dview y, int s, dview out)
{
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < m; ++j) {
            double a = x.p[i * x.ld + j];
            if (s > 0) a = a + y.p[i * y.ld + j];
            else if (s < 0) a = a - y.p[i * y.ld + j];
            out.p[i * out.ld + j] = a;
        }
}
static void uadd(int64_t m, uview x, uview y, int s, uview out)
{
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < m; ++j) {
            uint64_t a = x.p[i * x.ld + j];
            if (s > 0) a = a + y.p[i * y.ld + j];
            else if (s < 0) a = a - y.p[i * y.ld + j];
            out.p[i * out.ld + j] = a;
        }
}

/* Leaf products, rows spread over OpenMP threads (each row of C is one
 * thread's, k ascending: the same arithmetic as one thread). */
static void dclassical(int64_t m, dview A, dview B, dview C)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < m; ++j) C.p[i * C.ld + j] = 0.0;
        for (int64_t k = 0; k < m; ++k) {
            const double a = A.p[i * A.ld + k];
            for (int64_t j = 0; j < m; ++j) C.p[i * C.ld + j] += a * B.p[k * B.ld + j];
        }
    }
}
static void uclassical(int64_t m, uview A, uview B, uview C)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < m; ++j) C.p[i * C.ld + j] = 0;
        for (int64_t k = 0; k < m; ++k) {
            const uint64_t a = A.p[i * A.ld + k];
            for (int64_t j = 0; j < m; ++j) C.p[i * C.ld + j] += a * B.p[k * B.ld + j];
        }
    }
}

/* Alg. 1 on an m x m problem with `level` more splits to go. */
static void dstrassen(int64_t m, int level, dview A, dview B, dview C)
{
    if (level == 0) { dclassical(m, A, B, C); return; }
    const int64_t h = m / 2;
    dview A11 = dsub(A, h, 0, 0), A12 = dsub(A, h, 0, 1), A21 = dsub(A, h, 1, 0), A22 = dsub(A, h, 1, 1);
    dview B11 = dsub(B, h, 0, 0), B12 = dsub(B, h, 0, 1), B21 = dsub(B, h, 1, 0), B22 = dsub(B, h, 1, 1);
    dview S = dalloc(h), T = dalloc(h);
    dview M[7];
    for (int i = 0; i < 7; ++i) M[i] = dalloc(h);
    /* M1 = (A11 + A22)(B11 + B22) */
    dadd(h, A11, A22, +1, S); dadd(h, B11, B22, +1, T); dstrassen(h, level - 1, S, T, M[0]);
    /* M2 = (A21 + A22) B11 */
    dadd(h, A21, A22, +1, S); dstrassen(h, level - 1, S, B11, M[1]);
    /* M3 = A11 (B12 - B22) */
    dadd(h, B12, B22, -1, T); dstrassen(h, level - 1, A11, T, M[2]);
    /* M4 = A22 (B21 - B11) */
    dadd(h, B21, B11, -1, T); dstrassen(h, level - 1, A22, T, M[3]);
    /* M5 = (A11 + A12) B22 */
    dadd(h, A11, A12, +1, S); dstrassen(h, level - 1, S, B22, M[4]);
    /* M6 = (A21 - A11)(B11 + B12) */
    dadd(h, A21, A11, -1, S); dadd(h, B11, B12, +1, T); dstrassen(h, level - 1, S, T, M[5]);
    /* M7 = (A12 - A22)(B21 + B22) */
    dadd(h, A12, A22, -1, S); dadd(h, B21, B22, +1, T); dstrassen(h, level - 1, S, T, M[6]);
    /* Combine, left to right as printed:
     * C11 = M1 + M4 - M5 + M7, C12 = M3 + M5, C21 = M2 + M4,
     * C22 = M1 - M2 + M3 + M6  (sign of M3 corrected). */
    dview C11 = dsub(C, h, 0, 0), C12 = dsub(C, h, 0, 1), C21 = dsub(C, h, 1, 0), C22 = dsub(C, h, 1, 1);
    dadd(h, M[0], M[3], +1, C11); dadd(h, C11, M[4], -1, C11); dadd(h, C11, M[6], +1, C11);
    dadd(h, M[2], M[4], +1, C12);
    dadd(h, M[1], M[3], +1, C21);
    dadd(h, M[0], M[1], -1, C22); dadd(h, C22, M[2], +1, C22); dadd(h, C22, M[5], +1, C22);
    for (int i = 0; i < 7; ++i) free(M[i].p);
    free(S.p); free(T.p);
}

static void ustrassen(int64_t m, int level, uview A, uview B, uview C)
{
    if (level == 0) { uclassical(m, A, B, C); return; }
    const int64_t h = m / 2;
    uview A11 = usub(A, h, 0, 0), A12 = usub(A, h, 0, 1), A21 = usub(A, h, 1, 0), A22 = usub(A, h, 1, 1);
    uview B11 = usub(B, h, 0, 0), B12 = usub(B, h, 0, 1), B21 = usub(B, h, 1, 0), B22 = usub(B, h, 1, 1);
    uview S = ualloc(h), T = ualloc(h);
    uview M[7];
    for (int i = 0; i < 7; ++i) M[i] = ualloc(h);
    uadd(h, A11, A22, +1, S); uadd(h, B11, B22, +1, T); ustrassen(h, level - 1, S, T, M[0]);
    uadd(h, A21, A22, +1, S); ustrassen(h, level - 1, S, B11, M[1]);
    uadd(h, B12, B22, -1, T); ustrassen(h, level - 1, A11, T, M[2]);
    uadd(h, B21, B11, -1, T); ustrassen(h, level - 1, A22, T, M[3]);
    uadd(h, A11, A12, +1, S); ustrassen(h, level - 1, S, B22, M[4]);
    uadd(h, A21, A11, -1, S); uadd(h, B11, B12, +1, T); ustrassen(h, level - 1, S, T, M[5]);
    uadd(h, A12, A22, -1, S); uadd(h, B21, B22, +1, T); ustrassen(h, level - 1, S, T, M[6]);
    uview C11 = usub(C, h, 0, 0), C12 = usub(C, h, 0, 1), C21 = usub(C, h, 1, 0), C22 = usub(C, h, 1, 1);
    uadd(h, M[0], M[3], +1, C11); uadd(h, C11, M[4], -1, C11); uadd(h, C11, M[6], +1, C11);
    uadd(h, M[2], M[4], +1, C12);
    uadd(h, M[1], M[3], +1, C21);
    uadd(h, M[0], M[1], -1, C22); uadd(h, C22, M[2], +1, C22); uadd(h, C22, M[5], +1, C22);
    for (int i = 0; i < 7; ++i) free(M[i].p);
    free(S.p); free(T.p);
}

/* The error majorant: Alg. 1's recursion on |A| and |B| with all signs +
 * (the operand sums of M1..M7 and the four combines add absolute values).
 * A and B are already nonnegative here. */
static void dstrassen_abs(int64_t m, int level, dview A, dview B, dview C)
{
    if (level == 0) { dclassical(m, A, B, C); return; }
    const int64_t h = m / 2;
    dview A11 = dsub(A, h, 0, 0), A12 = dsub(A, h, 0, 1), A21 = dsub(A, h, 1, 0), A22 = dsub(A, h, 1, 1);
    dview B11 = dsub(B, h, 0, 0), B12 = dsub(B, h, 0, 1), B21 = dsub(B, h, 1, 0), B22 = dsub(B, h, 1, 1);
    dview S = dalloc(h), T = dalloc(h);
    dview M[7];
    for (int i = 0; i < 7; ++i) M[i] = dalloc(h);
    /* |M1| <= (|A11| + |A22|)(|B11| + |B22|) */
    dadd(h, A11, A22, +1, S); dadd(h, B11, B22, +1, T); dstrassen_abs(h, level - 1, S, T, M[0]);
    /* |M2| <= (|A21| + |A22|) |B11| */
    dadd(h, A21, A22, +1, S); dstrassen_abs(h, level - 1, S, B11, M[1]);
    /* |M3| <= |A11| (|B12| + |B22|) */
    dadd(h, B12, B22, +1, T); dstrassen_abs(h, level - 1, A11, T, M[2]);
    /* |M4| <= |A22| (|B21| + |B11|) */
    dadd(h, B21, B11, +1, T); dstrassen_abs(h, level - 1, A22, T, M[3]);
    /* |M5| <= (|A11| + |A12|) |B22| */
    dadd(h, A11, A12, +1, S); dstrassen_abs(h, level - 1, S, B22, M[4]);
    /* |M6| <= (|A21| + |A11|)(|B11| + |B12|) */
    dadd(h, A21, A11, +1, S); dadd(h, B11, B12, +1, T); dstrassen_abs(h, level - 1, S, T, M[5]);
    /* |M7| <= (|A12| + |A22|)(|B21| + |B22|) */
    dadd(h, A12, A22, +1, S); dadd(h, B21, B22, +1, T); dstrassen_abs(h, level - 1, S, T, M[6]);
    /* C11: M1 M4 M5 M7, C12: M3 M5, C21: M2 M4, C22: M1 M2 M3 M6, all added */
    dview C11 = dsub(C, h, 0, 0), C12 = dsub(C, h, 0, 1), C21 = dsub(C, h, 1, 0), C22 = dsub(C, h, 1, 1);
    dadd(h, M[0], M[3], +1, C11); dadd(h, C11, M[4], +1, C11); dadd(h, C11, M[6], +1, C11);
    dadd(h, M[2], M[4], +1, C12);
    dadd(h, M[1], M[3], +1, C21);
    dadd(h, M[0], M[1], +1, C22); dadd(h, C22, M[2], +1, C22); dadd(h, C22, M[5], +1, C22);
    for (int i = 0; i < 7; ++i) free(M[i].p);
    free(S.p); free(T.p);
}

/* Pad an n x n matrix with zeros to m x m (m >= n).  Alg. 1 is stated for
 * n = 2^p; other sizes are embedded in a zero-padded square whose side is a
 * multiple of 2^depth, and the top-left n x n block of the product is kept. */
static void *pad_copy(int64_t n, int64_t m, const void *src, size_t esz)
{
    char *dst = (char *)calloc((size_t)(m * m), esz);
    for (int64_t i = 0; i < n; ++i) memcpy(dst + (size_t)(i * m) * esz, (const char *)src + (size_t)(i * n) * esz, (size_t)n * esz);
    return dst;
}

static int64_t padded_side(int64_t n, int depth)
{
    const int64_t g = (int64_t)1 << depth;
    return (n + g - 1) / g * g;
}

/* C = A*B by Alg. 1 with `depth` levels of recursion; n need not be a power
 * of two (zero padding to a multiple of 2^depth).  Returns 0, or -1 on bad
 * arguments / allocation failure. */
int oracle_strassen_f64(int64_t n, int depth, const double *A, const double *B, double *C)
{
    if (n < 0 || depth < 0 || depth > 12) return -1;
    if (n == 0) return 0;
    const int64_t m = padded_side(n, depth);
    double *Ap = (double *)pad_copy(n, m, A, sizeof(double));
    double *Bp = (double *)pad_copy(n, m, B, sizeof(double));
    double *Cp = (double *)calloc((size_t)(m * m), sizeof(double));
    if (!Ap || !Bp || !Cp) { free(Ap); free(Bp); free(Cp); return -1; }
    dview a = { Ap, m }, b = { Bp, m }, c = { Cp, m };
    dstrassen(m, depth, a, b, c);
    for (int64_t i = 0; i < n; ++i) memcpy(C + i * n, Cp + i * m, (size_t)n * sizeof(double));
    free(Ap); free(Bp); free(Cp);
    return 0;
}

/* S = the error majorant of Alg. 1 with `depth` levels on |A|, |B| (zero
 * padding as oracle_strassen_f64).  Returns 0, or -1 on bad arguments. */
int oracle_strassen_abs_f64(int64_t n, int depth, const double *A, const double *B, double *S)
{
    if (n < 0 || depth < 0 || depth > 12) return -1;
    if (n == 0) return 0;
    const int64_t m = padded_side(n, depth);
    double *Ap = (double *)pad_copy(n, m, A, sizeof(double));
    double *Bp = (double *)pad_copy(n, m, B, sizeof(double));
    double *Sp = (double *)calloc((size_t)(m * m), sizeof(double));
    if (!Ap || !Bp || !Sp) { free(Ap); free(Bp); free(Sp); return -1; }
    for (int64_t i = 0; i < m * m; ++i) { Ap[i] = fabs(Ap[i]); Bp[i] = fabs(Bp[i]); }
    dview a = { Ap, m }, b = { Bp, m }, c = { Sp, m };
    dstrassen_abs(m, depth, a, b, c);
    for (int64_t i = 0; i < n; ++i) memcpy(S + i * n, Sp + i * m, (size_t)n * sizeof(double));
    free(Ap); free(Bp); free(Sp);
    return 0;
}

int oracle_strassen_i64(int64_t n, int depth, const int64_t *A, const int64_t *B, int64_t *C)
{
    if (n < 0 || depth < 0 || depth > 12) return -1;
    if (n == 0) return 0;
    const int64_t m = padded_side(n, depth);
    uint64_t *Ap = (uint64_t *)pad_copy(n, m, A, sizeof(uint64_t));
    uint64_t *Bp = (uint64_t *)pad_copy(n, m, B, sizeof(uint64_t));
    uint64_t *Cp = (uint64_t *)calloc((size_t)(m * m), sizeof(uint64_t));
    if (!Ap || !Bp || !Cp) { free(Ap); free(Bp); free(Cp); return -1; }
    uview a = { Ap, m }, b = { Bp, m }, c = { Cp, m };
    ustrassen(m, depth, a, b, c);
    for (int64_t i = 0; i < n; ++i) memcpy(C + i * n, Cp + i * m, (size_t)n * sizeof(uint64_t));
    free(Ap); free(Bp); free(Cp);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Divide phase: leaf operand sums (Alg. 1 / Alg. 3)                   */
/* ------------------------------------------------------------------ */

/* One level of the divide for the A side or the B side: from the four
 * quadrants of an m x m block X (row-major, leading dimension ldx), form the
 * seven h x h operands of M1..M7 of Alg. 1 into out[0..6] (each h x h,
 * contiguous).  All sums are single fp32 additions/subtractions. */
static void divide_level_f32(int64_t m, const float *X, int64_t ldx, int side, float *out[7])
{
    const int64_t h = m / 2;
    for (int64_t i = 0; i < h; ++i)
        for (int64_t j = 0; j < h; ++j) {
            const float x11 = X[i * ldx + j], x12 = X[i * ldx + j + h];
            const float x21 = X[(i + h) * ldx + j], x22 = X[(i + h) * ldx + j + h];
            const int64_t o = i * h + j;
            if (side == 0) {            /* A side */
                out[0][o] = x11 + x22;  /* M1: A11 + A22 */
                out[1][o] = x21 + x22;  /* M2: A21 + A22 */
                out[2][o] = x11;        /* M3: A11       */
                out[3][o] = x22;        /* M4: A22       */
                out[4][o] = x11 + x12;  /* M5: A11 + A12 */
                out[5][o] = x21 - x11;  /* M6: A21 - A11 */
                out[6][o] = x12 - x22;  /* M7: A12 - A22 */
            } else {                    /* B side */
                out[0][o] = x11 + x22;  /* M1: B11 + B22 */
                out[1][o] = x11;        /* M2: B11       */
                out[2][o] = x12 - x22;  /* M3: B12 - B22 */
                out[3][o] = x21 - x11;  /* M4: B21 - B11 */
                out[4][o] = x22;        /* M5: B22       */
                out[5][o] = x11 + x12;  /* M6: B11 + B12 */
                out[6][o] = x21 + x22;  /* M7: B21 + B22 */
            }
        }
}

static void divide_rec_f32(int64_t m, int level, const float *X, int64_t ldx, int side,
                           float *planes, int64_t leaf_base, int64_t nleaves)
{
    /* nleaves = 7^level leaves lie under this node, numbered from leaf_base */
    if (level == 0) {
        float *dst = planes + leaf_base * m * m;
        for (int64_t i = 0; i < m; ++i) memcpy(dst + i * m, X + i * ldx, (size_t)m * sizeof(float));
        return;
    }
    const int64_t h = m / 2;
    const int64_t per_child = nleaves / 7;
    float *child[7];
    for (int c = 0; c < 7; ++c) child[c] = (float *)malloc((size_t)(h * h) * sizeof(float));
    divide_level_f32(m, X, ldx, side, child);
    for (int c = 0; c < 7; ++c) {
        divide_rec_f32(h, level - 1, child[c], h, side, planes, leaf_base + c * per_child, per_child);
        free(child[c]);
    }
}

/* planes[leaf][L][L], L = npad / 2^depth, leaf = base-7 path (top level most
 * significant).  X is n x n row-major; it is read as the zero-padded npad x npad
 * matrix (npad must be a multiple of 2^depth and >= n).  side: 0 = A, 1 = B.
 * Returns 0 or -1. */
int oracle_strassen_operands_f32(int64_t n, int64_t npad, int depth, const float *X, int side, float *planes)
{
    if (n < 0 || npad < n || depth < 0 || depth > 8 || (npad % ((int64_t)1 << depth)) != 0) return -1;
    if (side != 0 && side != 1) return -1;
    float *Xp = (float *)pad_copy(n, npad, X, sizeof(float));
    if (!Xp) return -1;
    int64_t leaves = 1;
    for (int k = 0; k < depth; ++k) leaves *= 7;
    divide_rec_f32(npad, depth, Xp, npad, side, planes, 0, leaves);
    free(Xp);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Rounding to the tensor-core input formats                           */
/* ------------------------------------------------------------------ */

/* Round a finite fp32 value to the nearest value with `bits` significant bits
 * (including the leading one), ties to the candidate whose last kept bit is
 * 0.  Works in double, where both candidates and the midpoint are exact. */
static float round_sig(float xf, int bits)
{
    const double x = (double)xf;
    if (x == 0.0 || !isfinite(x)) return xf;
    int e;
    frexp(fabs(x), &e);                 /* |x| = f * 2^e, f in [0.5, 1) */
    double ulp = ldexp(1.0, e - bits);  /* spacing of `bits`-bit values near |x| */
    /* The format keeps fp32's exponent range, so below 2^-126 it is subnormal
     * with the fixed spacing 2^(-126-(bits-1)). */
    const double min_ulp = ldexp(1.0, -125 - bits);
    if (ulp < min_ulp) ulp = min_ulp;
    const double ax = fabs(x);
    const double lo = floor(ax / ulp) * ulp;
    const double hi = lo + ulp;
    double r;
    if (ax - lo < hi - ax) r = lo;
    else if (ax - lo > hi - ax) r = hi;
    else r = (fmod(lo / ulp, 2.0) == 0.0) ? lo : hi;
    return (float)(x < 0 ? -r : r);
}

/* hi = RN_bf16(x) (8 significant bits), lo = RN_bf16(x - hi).  Outputs are the
 * rounded values held in fp32 (the bf16 value widened exactly). */
void oracle_split_bf16(int64_t count, const float *x, float *hi, float *lo)
{
    for (int64_t i = 0; i < count; ++i) {
        const float h = round_sig(x[i], 8);
        const float r = x[i] - h;   /* exact in fp32 */
        hi[i] = h;
        lo[i] = round_sig(r, 8);
    }
}

/* hi = RN_tf32(x) (11 significant bits), lo = RN_tf32(x - hi). */
void oracle_split_tf32(int64_t count, const float *x, float *hi, float *lo)
{
    for (int64_t i = 0; i < count; ++i) {
        const float h = round_sig(x[i], 11);
        const float r = x[i] - h;
        hi[i] = h;
        lo[i] = round_sig(r, 11);
    }
}

/* Round a finite fp32 value to IEEE binary16: 11 significant bits where the
 * exponent is normal (|x| >= 2^-14), the fixed spacing 2^-24 below that, ties
 * to the candidate whose last kept bit is 0; a result beyond the largest
 * finite value 65504 is infinity (so |x| >= 65520 overflows). */
static float round_fp16(float xf)
{
    const double x = (double)xf;
    if (x == 0.0 || !isfinite(x)) return xf;
    const double ax = fabs(x);
    int e;
    frexp(ax, &e);
    double ulp = ldexp(1.0, e - 11);
    const double min_ulp = ldexp(1.0, -24);
    if (ulp < min_ulp) ulp = min_ulp;
    const double lo = floor(ax / ulp) * ulp;
    const double hi = lo + ulp;
    double r;
    if (ax - lo < hi - ax) r = lo;
    else if (ax - lo > hi - ax) r = hi;
    else r = (fmod(lo / ulp, 2.0) == 0.0) ? lo : hi;
    if (r > 65504.0) r = INFINITY;
    return (float)(x < 0 ? -r : r);
}

/* hi = RN_fp16(x), lo = RN_fp16(x - hi) (x - hi is exact in fp32). */
void oracle_split_fp16(int64_t count, const float *x, float *hi, float *lo)
{
    for (int64_t i = 0; i < count; ++i) {
        const float h = round_fp16(x[i]);
        const float r = x[i] - h;
        hi[i] = h;
        lo[i] = round_fp16(r);
    }
}

/* Single rounding, exposed for the pins. */
float oracle_round_sig_f32(float x, int bits) { return round_sig(x, bits); }
float oracle_round_fp16_f32(float x) { return round_fp16(x); }
