// stark_internal.h -- shared declarations between the host side (plans,
// batches, server) and the kernels of libstark.so.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <vector>

#include "../../include/stark.h"

namespace stark {

// ------------------------------------------------------------------ tables
// Alg. 1 coefficients per recursion level.  Quadrant q: 0 = X11, 1 = X12,
// 2 = X21, 3 = X22.  Product m: 0..6 = M1..M7.
//   A side: M1 A11+A22, M2 A21+A22, M3 A11, M4 A22, M5 A11+A12,
//           M6 A21-A11, M7 A12-A22
//   B side: M1 B11+B22, M2 B11, M3 B12-B22, M4 B21-B11, M5 B22,
//           M6 B11+B12, M7 B21+B22
//   C side: C11 = M1+M4-M5+M7, C12 = M3+M5, C21 = M2+M4, C22 = M1-M2+M3+M6
__host__ __device__ constexpr int coef_a(int m, int q) {
  constexpr signed char t[7][4] = {{1, 0, 0, 1}, {0, 0, 1, 1}, {1, 0, 0, 0}, {0, 0, 0, 1},
                                   {1, 1, 0, 0}, {-1, 0, 1, 0}, {0, 1, 0, -1}};
  return t[m][q];
}
__host__ __device__ constexpr int coef_b(int m, int q) {
  constexpr signed char t[7][4] = {{1, 0, 0, 1}, {1, 0, 0, 0}, {0, 1, 0, -1}, {-1, 0, 1, 0},
                                   {0, 0, 0, 1}, {1, 1, 0, 0}, {0, 0, 1, 1}};
  return t[m][q];
}
// coefficient of M_m in C quadrant q
__host__ __device__ constexpr int coef_c(int m, int q) {
  constexpr signed char t[4][7] = {{1, 0, 0, 1, -1, 0, 1}, {0, 0, 1, 0, 1, 0, 0},
                                   {0, 1, 0, 1, 0, 0, 0}, {1, -1, 1, 0, 0, 1, 0}};
  return t[q][m];
}

// One entry of the device quadrant-index table: where a leaf's product
// lands in C and with which sign.
struct CTarget {
  int32_t row_off;  // element row offset of the target quadrant in C
  int32_t col_off;  // element column offset
  int32_t sign;     // +1 or -1
  int32_t pad;
};

// Host construction of the per-leaf term lists (side 0 A, 1 B, 2 C).
void build_quadrant_table(int depth, int side, std::vector<int32_t>& count, std::vector<int32_t>& quad,
                          std::vector<int8_t>& sign);
// Row/column element offsets of base-4 quadrant path q for side npad.
void quadrant_offsets(int depth, int64_t npad, int32_t q, int64_t* row, int64_t* col);

// The fp32 dtypes with split-precision tensor-core leaves, and among them
// those whose halves are 16-bit (bf16 or fp16: kind::f16 MMAs, 2-byte planes).
inline bool is_split(stark_dtype dt) {
  return dt == STARK_F32_SPLIT_BF16 || dt == STARK_F32_SPLIT_TF32 || dt == STARK_F32_SPLIT_FP16;
}
inline bool half_split(stark_dtype dt) { return dt == STARK_F32_SPLIT_BF16 || dt == STARK_F32_SPLIT_FP16; }

// ------------------------------------------------------------------ launches
enum OutMode { kOutSplitBf16 = 0, kOutSplitTf32 = 1, kOutPlain = 2, kOutBf16Exact = 3, kOutSplitFp16 = 4 };
enum InType { kInF32 = 0, kInF64 = 1, kInI64 = 2 };

struct DivideArgs {
  const void* X;      // n x n row-major input (row stride ld)
  int64_t n;          // input side read (the core of a peeled product)
  int64_t npad;       // padded side (zeros beyond n)
  int64_t L;          // leaf side = npad >> depth
  void* out_hi;       // planes [P][L][L] (split: hi part; plain: the value)
  void* out_lo;       // planes [P][L][L] (split: lo part; plain: unused)
  int* range_flag;    // bf16-exact output: set to kDevIntRange when |value| > 256
  int top;            // >= 0: depth-first subtree; the input is read through the
                      // operand sums of the top `top_levels` levels along the
                      // M-index path `top` (base 7, top level most significant;
                      // M1..M7 = 0..6) and npad is the subproblem's side (the
                      // full padded side >> top_levels)
  int64_t ld;         // row stride of X in elements (>= n)
  int top_levels;     // levels above the subtree (1, or 2 for the split dtypes) when top >= 0
};

// Divide phase for one operand: writes the 7^depth leaf operand sums as
// row-major L x L planes.  side 0 = A (M x K planes), side 1 = B (K x N).
cudaError_t launch_divide(const DivideArgs& a, int depth, int side, InType in, OutMode out, cudaStream_t s);
// The same for a depth-first subtree (a.top >= 0); launch_divide forwards.
cudaError_t launch_divide_top(const DivideArgs& a, int depth, int side, InType in, OutMode out, cudaStream_t s);
// Depth 3, split-fp32 outputs, breadth first (a.top < 0): one pass per
// operand with the input tile staged in shared memory (divide_staged.cu);
// needs L % 128 == 0 (divide_staged_fits).  Same planes as launch_divide.
bool divide_staged_fits(int64_t L);
cudaError_t launch_divide_staged(const DivideArgs& a, int side, OutMode out, cudaStream_t s);
// C (+)= A B on sub-blocks (M x K times K x N, row strides lda, ldb, ldc in
// elements) on the CUDA cores: the edges of a peeled product.  Element type
// float (fp32 accumulate), double or int64 (wrapping); accumulate = 0
// overwrites C (then K is not split).  kc is set by the launcher.
struct BorderArgs {
  const void* A;
  int64_t lda;
  const void* B;
  int64_t ldb;
  void* C;
  int64_t ldc;
  int64_t M, N, K;
  int accumulate;
  int split;   // 1: K may be split across blocks (atomic adds; fp32 order varies)
  int64_t kc;  // K per block (grid z splits K), set by the launcher
};
cudaError_t launch_border(const BorderArgs& a, InType t, int num_sms, cudaStream_t s);

// Deterministic combine of stored leaf products: C_q = sum over leaves l
// (ascending) of W_d[q, l] * M_l, every element written once.  M planes are
// [leaves][L][L] fp32 for leaves [0, P); depth <= 3.
cudaError_t launch_combine(const float* M, int depth, int64_t L, int64_t npad, int64_t n, float* C, int64_t ldc,
                           cudaStream_t s);
bool make_tmap_mplanes(CUtensorMap* m, void* base, int64_t L, int64_t planes);
// In-place transpose of `count` square L x L fp32 planes.
cudaError_t launch_transpose_planes(float* planes, int64_t L, int64_t count, cudaStream_t s);

// One member of a grouped leaf launch (a batch): its operand and C tensor
// maps, where its work items start, and its combine table.  Lives in device
// memory; 128-byte aligned for the tensor maps.
struct alignas(128) GroupDesc {
  CUtensorMap tmA, tmB, tmC;
  int32_t item_base;   // first work item of this member
  int32_t P, L;        // leaves, leaf side
  int32_t use_tma_c;
  const CTarget* ctab;
  const int32_t* ccount;
  int32_t maxT, pad;
  float* C;     // combine target (the caller's C, or a staging copy)
  int64_t n;    // problem side (rows and columns of C)
  int64_t ldc;  // row pitch of the combine target in elements
};

struct LeafTcArgs {
  int32_t P;           // leaves per operand side (planes 0..P-1 hi, P..2P-1 lo)
  int32_t L;           // leaf side
  int32_t leaf_begin;  // leaves [leaf_begin, leaf_end) are computed
  int32_t leaf_end;
  const CTarget* ctab; // [P][maxT]
  const int32_t* ccount;
  int32_t maxT;
  float* C;
  int64_t ldc;
  int64_t n;
  int* err;
  uint64_t timeout_ns;
  int32_t use_tma_c;   // 1: combine by TMA bulk add-reductions through tmC
  int32_t pair;        // 2: cta_group::2 pair MMA where the tiling allows; 0: single CTAs
  int32_t row_bytes;   // swizzled smem row of the operand tiles: 128 or 64 (tensor maps must match)
  int32_t store_m;     // 1: store each leaf tile to the M planes (tmC = their map) instead of combining
  int32_t plane_base;  // leaf stored in workspace plane 0 (depth-first traversal); P = planes per half
  int32_t b_mn;        // tf32: 1 = Y planes row-major (K x N) read MN-major with 32-byte-atom
                       // swizzle; 0 = Y planes transposed to N x K, read K-major
  int32_t band;        // > 0: a leaf's tiles run in bands of `band` tile columns (row-major inside a
                       // band); 0 or not dividing the tile columns: row-major over the whole leaf
  int32_t sib;         // 1: sibling-folded combine (CTA-pair kernel): the 7 children of one parent
                       // run back to back at one tile position and their tiles are stored or added
                       // into the parent's quadrants (tmC = parent planes [P/7][2L][2L]); leaf
                       // range of whole parents
  int32_t fp16;        // 1: the 16-bit planes hold fp16 halves (kind::f16 A and B format fp16
                       // instead of bf16); 0 for every other dtype and for grouped launches
  int32_t promo_kb;    // > 0 (CTA-pair kernel): accumulator promotion -- every promo_kb K blocks
                       // the tensor-core partial sum is added into a running fp32 sum in the
                       // epilogue warps' registers (round to nearest); 0: one tensor-core
                       // accumulation over K
  // grouped launch (batch): when groups != nullptr the fields above that
  // describe one problem are ignored and every item is looked up here
  const GroupDesc* groups;
  int32_t ngroups;
  int32_t total_items;
};

// 3xBF16 / 3xTF32 leaf GEMMs with the combine fused in the epilogue.
cudaError_t launch_leaf_tc(const LeafTcArgs& a, const CUtensorMap* tmA, const CUtensorMap* tmB,
                           const CUtensorMap* tmC, bool tf32, int bn, int num_sms, cudaStream_t s);
// Exact integer leaves: one bf16 product per K step over [P][L][L] bf16
// planes holding integers, combined into an int64 C (a.C reinterpreted).
cudaError_t launch_leaf_tc_int(const LeafTcArgs& a, const CUtensorMap* tmA, const CUtensorMap* tmB, int bn,
                               int num_sms, cudaStream_t s);
// Grouped single-CTA launch over a.groups (tensor maps taken from the
// descriptors), 128 x 128 tiles (bn == 128 only).
cudaError_t launch_leaf_tc_grouped(const LeafTcArgs& a, bool tf32, int bn, int num_sms, cudaStream_t s);
// 3xBF16 / 3xTF32 leaves on CTA pairs sharing one cta_group::2 MMA of
// 256 x 256 (requires L a multiple of 256).  The tf32 Y map's box is 128
// rows (each CTA stages half of the 256 columns).
bool leaf_tc2_fits(const LeafTcArgs& a);
cudaError_t launch_leaf_tc2(const LeafTcArgs& a, const CUtensorMap* tmA, const CUtensorMap* tmB,
                            const CUtensorMap* tmC, bool tf32, int num_sms, cudaStream_t s);
// Grouped CTA-pair launch over a.groups: every member's L a multiple of 256,
// items numbered per member as leaf * (L/256)^2 + row * (L/256) + column of
// 256 x 256 pair tiles; tf32 members' Y maps with 128-row boxes.
cudaError_t launch_leaf_tc2_grouped(const LeafTcArgs& a, bool tf32, int num_sms, cudaStream_t s);

struct LeafCcArgs {
  int32_t P, L, leaf_begin, leaf_end;
  int32_t plane_base;  // leaf stored in workspace plane 0
  const void* X;  // planes [P][L][L]
  const void* Y;  // planes [P][L][L] (K x N, row-major)
  const CTarget* ctab;
  const int32_t* ccount;
  int32_t maxT;
  void* C;
  int64_t ldc, n;
};
cudaError_t launch_leaf_f64(const LeafCcArgs& a, cudaStream_t s);
cudaError_t launch_leaf_i64(const LeafCcArgs& a, cudaStream_t s);

cudaError_t launch_wait_selftest(int* err, uint64_t timeout_ns, cudaStream_t s);

// ------------------------------------------------------------------ misc
void count_launch(int k = 1);
int device_sm_count();
bool device_is_sm100_family();
// [planes][L][L] operand planes, boxes of row_bytes x box_rows with the
// matching swizzle; atom32: the 128-byte swizzle with 32-byte atoms (tf32
// planes read MN-major).
bool make_tmap_planes(CUtensorMap* m, void* base, bool tf32, int64_t L, int64_t planes, int box_rows,
                      int row_bytes = 128, bool atom32 = false);
// n x n fp32 row-major C with row pitch ld elements, 32 x 32 boxes,
// 128-byte swizzle (reduction target).  Needs ld % 4 == 0 and a 16-byte
// aligned base.
bool make_tmap_c(CUtensorMap* m, void* C, int64_t n, int64_t ld);
// Row pitch of the staging copy of C used when C itself cannot be a TMA
// target (n not a multiple of 4): n rounded up to a multiple of 4.
inline int64_t staged_ld(int64_t n) { return (n + 3) / 4 * 4; }
// True when the caller's C can take the TMA bulk reductions directly.
inline bool c_is_tma_target(const void* C, int64_t n) {
  return n > 0 && (n % 4) == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0;
}

}  // namespace stark
