// plan.h -- the plan object behind stark_plan_t and the helpers shared by
// plans, batches and the server.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "stark_internal.h"

namespace stark {

constexpr int kMaxDepth = 4;
constexpr int kTimingEvents = 5;  // per timed product (see stark_plan_s::ev)
constexpr uint64_t kDefaultTimeoutNs = 4000000000ull;  // 4 s per bounded device wait

int64_t pow7i(int d);
int tile_granularity(stark_dtype dt);
int64_t padded_side(int64_t n, int depth, stark_dtype dt);
size_t element_size(stark_dtype dt);
int64_t operand_bytes(int64_t n, int depth, stark_dtype dt);
double model_seconds(int64_t n, int depth, stark_dtype dt);
int choose_depth(int64_t n, stark_dtype dt);
// Measured depth choice: times the candidate depths on the current device for
// the size class of n (n rounded up to 64 / 128 / 256 for n up to 1024 /
// 2048 / beyond) and caches the winner per (class, dtype) for the process.
// Tensor-core dtypes.
int autotune_depth(int64_t n, stark_dtype dt);
// The same search over (depth, leaf tile): tile 256 = CTA pairs on 256 x 256
// tiles (leaf sides that are multiples of 256), 128 = single CTAs on 128 x 128.
void autotune(int64_t n, stark_dtype dt, int* depth, int* tile);

}  // namespace stark

struct stark_plan_s {
  int64_t n = 0, npad = 0, L = 0, P = 1;
  int64_t P_ws = 1;   // leaves whose operands the workspace holds (P, or P / 7 depth-first)
  int dfs = 0;        // depth-first over this many top recursion levels (0: breadth first)
  int depth = 0;
  stark_dtype dt = STARK_F64;
  bool is_tc = false;  // tensor-core (split) path
  int bn = 128;        // leaf GEMM tile width (tensor-core path)
  size_t esz = 8;      // element size of A, B, C
  int device = 0;
  int num_sms = 1;
  // workspace: leaf operand planes; split paths hold [2P][L][L] (hi planes
  // then lo planes), plain paths [P][L][L]
  void* X = nullptr;
  void* Y = nullptr;
  int64_t ws_bytes = 0;
  // quadrant-index table: C targets per leaf
  stark::CTarget* d_ctab = nullptr;
  int32_t* d_ccount = nullptr;
  int32_t maxT = 1;
  int* d_err = nullptr;
  uint64_t timeout_ns = stark::kDefaultTimeoutNs;
  int combine_mode = 0;  // 0: TMA bulk reductions where C allows, 1: always vector atomics,
                         // 2: deterministic (store M planes, ordered combine pass),
                         // 3: sibling fold (parent planes in L2, ordered pass at depth - 1)
  void* m_planes = nullptr;  // [P][L][L] fp32 leaf products (combine mode 2)
  CUtensorMap tmM;
  void* q_planes = nullptr;  // [P/7][2L][2L] fp32 parent products (combine mode 3, sibling fold)
  CUtensorMap tmQ;
  int pair_mode = 2;     // leaf schedule where the tiling allows (L % 256 == 0): 2 CTA pairs on one
                         // cta_group::2 MMA, 0 single CTAs
  CUtensorMap tmBp;      // tf32 Y map with 128-row boxes for the pair MMA
  int tf32_mn = 1;       // tf32 Y planes row-major, read MN-major (0: transposed, K-major)
  bool has_mapbp = false;
  int deep_pipeline = 0; // 1: 3xBF16 with 64-byte rows, 4 stages of 48 KB (256-wide tiles)
  int raster_band = 0;   // tile columns per raster band of a leaf (0: row-major)
  int promo_k = 0;       // accumulator promotion every promo_k of K (CTA-pair leaves), 0: off
  CUtensorMap tmA64, tmB64;  // operand maps for the 64-byte-row schedule
  bool has_maps64 = false;
  // I64 with a declared input bound: exact bf16 tensor-core leaves
  int64_t int_bound = 0;
  bool int_tc = false;
  int int_bn = 128;
  CUtensorMap tmAi, tmBi;
  CUtensorMap tmA;
  CUtensorMap tmB;
  // end-to-end staging (stark_mul_host / _async), allocated on first use:
  // two buffer sets so consecutive products overlap copies with compute
  void* stage_A = nullptr;
  void* stage_B = nullptr;
  void* stage_C = nullptr;
  void* stage2[3] = {nullptr, nullptr, nullptr};
  cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
  int host_calls = 0;
  int64_t peel = 0;           // edge rows/columns done classically (n = core + peel)
  // leaf-range shard (stark_plan_set_shard): the workspace holds the operands
  // of the subtrees below shard_levels top levels that cover leaves
  // [shard_lb, shard_le); workspace plane 0 is leaf shard_first
  int shard_levels = 0;  // 0: no shard (every leaf's operands, or depth first)
  int64_t shard_lb = 0, shard_le = 0, shard_first = 0;
  int pend_set = -1;          // staging set whose copy out is not yet enqueued
  void* pend_C = nullptr;     // its host destination
  // staging copy of C (row pitch staged_ld(n)) for the tensor-core combine
  // when C cannot be a TMA target (n not a multiple of 4)
  void* cstage = nullptr;
  // optional phase timing: event sets for up to timing_cap products
  int timing_cap = 0;
  int timing_used = 0;
  bool timing_active = false;  // the current product records events
  bool timing_leaf_marked = false;  // the current product recorded the end of its leaf kernel
  std::vector<cudaEvent_t> ev;  // kTimingEvents per recorded product: start, after zeroing C,
                                // after the divide, after the leaf kernel, end
};

namespace stark {
// peel: run the recursion on the largest m <= n that the tiling divides and
// finish the r = n - m edge rows/columns with classical products (when n is
// already a multiple, or smaller than one tile granule, nothing is peeled).
// dfs: allocate the workspace for the depth-first traversal over that many
// top levels (one subtree's operands) from the start; traversal_supported
// must hold for it.
stark_status plan_init(stark_plan_s* p, int64_t n, int depth, stark_dtype dt, bool peel = false, int dfs = 0);
// Whether the depth-first traversal over `levels` top levels exists for this
// depth and dtype (subtree loaders cover depth <= 3; two levels only for the
// split dtypes).  0 (breadth first) always does.
bool traversal_supported(int depth, stark_dtype dt, int levels);
// Tensor maps of the split dtypes' operand planes (for `planes` leaves per half).
stark_status plan_operand_maps(stark_plan_s* p, int64_t planes);
// Side of the product the recursion covers (n minus the peeled edge).
inline int64_t core_side(const stark_plan_s* p) { return p->n - p->peel; }
void plan_release(stark_plan_s* p);
// Enqueue C = sum over leaves [lb, le) of their combine contributions.
stark_status plan_run(stark_plan_s* p, const void* A, const void* B, void* C, int64_t lb, int64_t le,
                      cudaStream_t s);
// Staging copy of C for the combine (allocated once; see stark_plan_s::cstage).
stark_status plan_ensure_cstage(stark_plan_s* p);
bool plan_uses_cstage(const stark_plan_s* p, const void* C);
stark_status plan_copy_cstage(const stark_plan_s* p, void* C, cudaStream_t s);
// Divide phase only: all leaf operands of A and B into the workspace.
stark_status plan_divide(stark_plan_s* p, const void* A, const void* B, cudaStream_t s);
// The same without zeroing C first (C accumulates).
stark_status plan_run_accumulate(stark_plan_s* p, const void* A, const void* B, void* C, int64_t lb, int64_t le,
                                 cudaStream_t s);
}  // namespace stark
