// batch.cu -- many independent products in one grouped, graph-captured pass.
//
// Each member keeps its own plan (operand planes, C-target table, operand
// tensor maps).  One stark_batch_mul enqueues, for every member, the zeroing
// of C and the divide of A and B, then ONE persistent grouped leaf launch
// whose work items are all (member, leaf, tile) triples: the 7^d leaf
// products of every member share the GPU in a single launch, and each
// item's epilogue combines into its own member's C.  The whole sequence is
// captured once in a CUDA graph and replayed while the pointers are
// unchanged.
//
// Depth per member: given, or chosen by the autotuner, which times the
// candidate (depth, leaf tile) pairs on the device (one warm-up and three
// timed products per candidate on scratch inputs) and caches the winner per
// size class and dtype for the process.  The tile candidates are CTA pairs
// on 256 x 256 tiles (cta_group::2; leaf sides that are multiples of 256)
// and single CTAs on 128 x 128 tiles.  Members whose tile is 256 share one
// grouped launch of CTA pairs, the others a second one of single CTAs.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "plan.h"
#include "stark_internal.h"

namespace stark {
namespace {

std::mutex g_tune_mu;
std::map<std::pair<int64_t, int>, std::pair<int, int>> g_tuned;  // (n class, dtype) -> (depth, tile)

// Device time (ms) of one product of side n at `depth` with leaf tiles of
// width `tile` (256: CTA pairs; 128: single CTAs), averaged over 3.
float time_depth(int64_t n, int depth, stark_dtype dt, int tile, void* A, void* B, void* C, cudaStream_t s) {
  stark_plan_s p;
  if (plan_init(&p, n, depth, dt) != STARK_OK) {
    plan_release(&p);
    return -1.f;
  }
  if (tile == 128 && p.bn == 256) {  // single CTAs on 128-wide tiles (operand maps do not depend on it)
    p.bn = 128;
    p.pair_mode = 0;
  } else if (tile != p.bn) {
    plan_release(&p);
    return -1.f;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = -1.f;
  if (plan_run(&p, A, B, C, 0, p.P, s) == STARK_OK) {
    cudaEventRecord(e0, s);
    bool ok = true;
    for (int r = 0; r < 3 && ok; ++r) ok = plan_run(&p, A, B, C, 0, p.P, s) == STARK_OK;
    cudaEventRecord(e1, s);
    if (ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) ms /= 3;
  }
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  plan_release(&p);
  cudaGetLastError();
  return ms;
}

}  // namespace

// Measured depth choice for n x n products (cached per process).
void autotune(int64_t n_req, stark_dtype dt, int* depth_out, int* tile_out) {
  // size class: n rounded up to 64 (n <= 1024), 128 (n <= 2048), else 256
  const int64_t q = n_req <= 1024 ? 64 : n_req <= 2048 ? 128 : 256;
  const int64_t n = (n_req + q - 1) / q * q;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find({n, (int)dt});
    if (it != g_tuned.end()) {
      *depth_out = it->second.first;
      *tile_out = it->second.second;
      return;
    }
  }
  int best = choose_depth(n, dt);
  int best_tile = (padded_side(n, best, dt) >> best) % 256 == 0 ? 256 : 128;
  const size_t bytes = (size_t)n * n * element_size(dt);
  void *A = nullptr, *B = nullptr, *C = nullptr;
  cudaStream_t s = nullptr;
  if (n > 0 && cudaMalloc(&A, bytes) == cudaSuccess && cudaMalloc(&B, bytes) == cudaSuccess &&
      cudaMalloc(&C, bytes) == cudaSuccess && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess) {
    cudaMemsetAsync(A, 0x3c, bytes, s);  // bounded, nonzero values
    cudaMemsetAsync(B, 0x3c, bytes, s);
    float best_ms = 1e30f;
    for (int d = 0; d <= 3; ++d) {
      if ((padded_side(n, d, dt) >> d) < tile_granularity(dt)) continue;
      if (d > 0 && (n >> d) < 128) break;
      const bool wide = (padded_side(n, d, dt) >> d) % 256 == 0;
      for (int tile : {256, 128}) {
        if (tile == 256 && !wide) continue;
        const float ms = time_depth(n, d, dt, tile, A, B, C, s);
        if (ms > 0 && ms < best_ms) {
          best_ms = ms;
          best = d;
          best_tile = tile;
        }
      }
    }
  }
  if (s) cudaStreamDestroy(s);
  cudaFree(A);
  cudaFree(B);
  cudaFree(C);
  cudaGetLastError();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[{n, (int)dt}] = {best, best_tile};
  *depth_out = best;
  *tile_out = best_tile;
}

int autotune_depth(int64_t n, stark_dtype dt) {
  int d = 0, tile = 128;
  autotune(n, dt, &d, &tile);
  return d;
}

}  // namespace stark

struct stark_batch_s {
  stark_dtype dt = STARK_F32_SPLIT_BF16;
  int bn = 128;     // 256 when any member runs 256-wide tiles
  int split = 0;    // members [0, split) run 256-wide tiles, the rest 128-wide
  int items_wide = 0;
  std::vector<stark_plan_s*> plans;
  std::vector<stark::GroupDesc> host_desc;
  stark::GroupDesc* d_desc = nullptr;
  int total_items = 0;
  int* d_err = nullptr;
  cudaStream_t cap = nullptr;  // private capture stream
  // the members' clears and divides are captured on kForks side streams
  // forked from `cap`, so the graph runs them concurrently (small members'
  // kernels are launch- and latency-bound one after another)
  static constexpr int kForks = 8;
  cudaStream_t side[kForks] = {};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[kForks] = {};
  cudaGraphExec_t exec = nullptr;
  std::vector<int> caller_index;  // caller's index of each (size-sorted) member
  std::vector<int> tiles;         // leaf tile width of each member (caller's order)
  std::vector<const void*> last;  // pointers the graph was captured with
  int64_t replays = 0;
};

using namespace stark;

static void batch_free(stark_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto* p : b->plans) {
    plan_release(p);
    delete p;
  }
  cudaFree(b->d_desc);
  cudaFree(b->d_err);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (int i = 0; i < stark_batch_s::kForks; ++i) {
    if (b->side[i]) cudaStreamDestroy(b->side[i]);
    if (b->join_ev[i]) cudaEventDestroy(b->join_ev[i]);
  }
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  cudaGetLastError();
  delete b;
}

extern "C" {

stark_status stark_batch_create(int32_t count, const int64_t* n, int depth, stark_dtype dt, stark_batch_t* out) {
  if (!out || !n || count <= 0 || count > 4096 || depth < -1 || depth > kMaxDepth) return STARK_EINVAL;
  *out = nullptr;
  if (!is_split(dt)) return STARK_EUNSUPPORTED;
  for (int i = 0; i < count; ++i)
    if (n[i] <= 0 || n[i] > (int64_t)1 << 20) return STARK_EINVAL;
  if (!device_is_sm100_family()) return STARK_EUNSUPPORTED;
  auto* b = new (std::nothrow) stark_batch_s();
  if (!b) return STARK_ENOMEM;
  b->dt = dt;
  stark_status st = STARK_OK;
  // members in order of decreasing size so the big tiles start first
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  b->plans.assign(count, nullptr);
  b->tiles.assign(count, 128);
  for (int i = 0; i < count && st == STARK_OK; ++i) {
    int d = depth, tile = 0;
    if (depth < 0) autotune(n[i], dt, &d, &tile);
    auto* p = new (std::nothrow) stark_plan_s();
    if (!p) {
      st = STARK_ENOMEM;
      break;
    }
    b->plans[i] = p;
    st = plan_init(p, n[i], d, dt);
    // the tuned tile, or 256-wide wherever the leaf side allows it
    if (st == STARK_OK) b->tiles[i] = (p->L % 256 == 0 && tile != 128) ? 256 : 128;
  }
  if (st != STARK_OK) {
    batch_free(b);
    return st;
  }
  // two grouped launches: members on 256-wide tiles (CTA pairs) first, then
  // the rest on 128-wide tiles; largest products first in each
  const std::vector<int> tiles = b->tiles;
  auto wide = [&](int i) { return tiles[i] == 256; };
  std::sort(order.begin(), order.end(), [&](int x, int y) {
    if (wide(x) != wide(y)) return wide(x);
    return b->plans[x]->n > b->plans[y]->n;
  });
  b->split = 0;
  while (b->split < count && wide(order[b->split])) ++b->split;
  b->bn = b->split > 0 ? 256 : 128;
  b->host_desc.resize(count);
  int64_t items = 0, items_wide = 0;
  for (int k = 0; k < count; ++k) {
    if (k == b->split) {
      items_wide = items;
      items = 0;  // the second launch numbers its own items
    }
    stark_plan_s* p = b->plans[order[k]];
    const int bn = k < b->split ? 256 : 128;
    GroupDesc& g = b->host_desc[k];
    std::memset(&g, 0, sizeof(g));
    g.tmA = p->tmA;
    if (dt == STARK_F32_SPLIT_TF32 && !p->tf32_mn) {
      // K-major tf32 Y; 256-wide members run CTA pairs: each CTA loads 128 Y rows
      if (!make_tmap_planes(&g.tmB, p->Y, true, p->L, 2 * p->P, bn == 256 ? 128 : bn)) st = STARK_EUNSUPPORTED;
    } else {
      g.tmB = p->tmB;
    }
    g.item_base = (int32_t)items;
    g.P = (int32_t)p->P;
    g.L = (int32_t)p->L;
    g.ctab = p->d_ctab;
    g.ccount = p->d_ccount;
    g.maxT = p->maxT;
    g.n = p->n;
    // 256-wide members: 256 x 256 pair tiles (CTA pairs); others 128 x 128
    items += bn == 256 ? p->P * (p->L / 256) * (p->L / 256) : p->P * (p->L / 128) * (p->L / 128);
  }
  if (b->split == count) {
    items_wide = items;
    items = 0;
  }
  if (items_wide > 0x7FFFFFFF) st = STARK_EINVAL;
  b->items_wide = (int)items_wide;
  if (items > 0x7FFFFFFF) st = STARK_EINVAL;
  b->total_items = (int)items;  // items of the 128-wide launch
  // keep the member order used by the descriptors
  std::vector<stark_plan_s*> sorted(count);
  for (int k = 0; k < count; ++k) sorted[k] = b->plans[order[k]];
  b->last.clear();
  if (st == STARK_OK && (cudaMalloc(&b->d_desc, sizeof(GroupDesc) * count) != cudaSuccess ||
                         cudaMalloc(&b->d_err, sizeof(int)) != cudaSuccess ||
                         cudaMemset(b->d_err, 0, sizeof(int)) != cudaSuccess ||
                         cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
                         cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) != cudaSuccess))
    st = STARK_ENOMEM;
  for (int i = 0; i < stark_batch_s::kForks && st == STARK_OK; ++i)
    if (cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join_ev[i], cudaEventDisableTiming) != cudaSuccess)
      st = STARK_ENOMEM;
  if (st != STARK_OK) {
    batch_free(b);
    return st;
  }
  // members are kept in the descriptor order; remember the caller's index
  b->plans = sorted;
  b->caller_index = order;
  *out = b;
  return STARK_OK;
}

stark_status stark_batch_destroy(stark_batch_t b) {
  if (!b) return STARK_OK;
  cudaDeviceSynchronize();
  batch_free(b);
  return STARK_OK;
}

stark_status stark_batch_tile(stark_batch_t b, int32_t index, int32_t* tile_n) {
  if (!b || !tile_n || index < 0 || index >= (int32_t)b->tiles.size()) return STARK_EINVAL;
  *tile_n = b->tiles[index];
  return STARK_OK;
}

stark_status stark_batch_depth(stark_batch_t b, int32_t index, int32_t* depth) {
  if (!b || !depth || index < 0 || index >= (int32_t)b->plans.size()) return STARK_EINVAL;
  for (size_t k = 0; k < b->plans.size(); ++k)
    if (b->caller_index[k] == index) {
      *depth = b->plans[k]->depth;
      return STARK_OK;
    }
  return STARK_EINVAL;
}

stark_status stark_batch_info(stark_batch_t b, int32_t* tile_n, int64_t* work_items, int64_t* workspace_bytes,
                              int64_t* graph_replays) {
  if (!b) return STARK_EINVAL;
  if (tile_n) *tile_n = b->bn;
  if (work_items) *work_items = (int64_t)b->total_items + b->items_wide;
  if (workspace_bytes) {
    int64_t w = 0;
    for (auto* p : b->plans) w += p->ws_bytes;
    *workspace_bytes = w;
  }
  if (graph_replays) *graph_replays = b->replays;
  return STARK_OK;
}

stark_status stark_batch_mul(stark_batch_t b, const void* const* A, const void* const* B, void* const* C,
                             void* stream) {
  if (!b || !A || !B || !C) return STARK_EINVAL;
  const int count = (int)b->plans.size();
  std::vector<const void*> ptrs((size_t)count * 3);
  for (int k = 0; k < count; ++k) {
    const int i = b->caller_index[k];
    if (!A[i] || !B[i] || !C[i]) return STARK_EINVAL;
    ptrs[3 * k] = A[i];
    ptrs[3 * k + 1] = B[i];
    ptrs[3 * k + 2] = C[i];
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (ptrs != b->last || !b->exec) {
    // new pointers: refresh the C maps and re-record the graph (the device
    // descriptors may be read by a replay still in flight, so wait first)
    if (cudaDeviceSynchronize() != cudaSuccess) return STARK_ECUDA;
    for (int k = 0; k < count; ++k) {
      GroupDesc& g = b->host_desc[k];
      void* Cuser = const_cast<void*>(ptrs[3 * k + 2]);
      const bool staged = plan_uses_cstage(b->plans[k], Cuser);
      g.C = static_cast<float*>(staged ? b->plans[k]->cstage : Cuser);
      g.ldc = staged ? staged_ld(g.n) : g.n;
      g.use_tma_c = make_tmap_c(&g.tmC, g.C, g.n, g.ldc) ? 1 : 0;
    }
    if (cudaMemcpy(b->d_desc, b->host_desc.data(), sizeof(GroupDesc) * count, cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return STARK_ECUDA;
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return STARK_ECUDA;
    stark_status st = STARK_OK;
    // fork: members' clears and divides on the side streams, joined before
    // the grouped leaf launches
    constexpr int F = stark_batch_s::kForks;
    if (cudaEventRecord(b->fork_ev, b->cap) != cudaSuccess) st = STARK_ECUDA;
    for (int i = 0; i < F && st == STARK_OK; ++i)
      if (cudaStreamWaitEvent(b->side[i], b->fork_ev, 0) != cudaSuccess) st = STARK_ECUDA;
    for (int k = 0; k < count && st == STARK_OK; ++k) {
      stark_plan_s* p = b->plans[k];
      const GroupDesc& g = b->host_desc[k];
      cudaStream_t sk = b->side[k % F];
      if (cudaMemsetAsync(g.C, 0, (size_t)p->n * g.ldc * sizeof(float), sk) != cudaSuccess)
        st = STARK_ECUDA;
      else
        st = plan_divide(p, ptrs[3 * k], ptrs[3 * k + 1], sk);
    }
    for (int i = 0; i < F; ++i)  // join (also after an error, so the capture can end)
      if (cudaEventRecord(b->join_ev[i], b->side[i]) != cudaSuccess ||
          cudaStreamWaitEvent(b->cap, b->join_ev[i], 0) != cudaSuccess)
        st = STARK_ECUDA;
    if (st == STARK_OK) {
      LeafTcArgs a{};
      a.err = b->d_err;
      a.timeout_ns = kDefaultTimeoutNs;
      const bool tf32 = b->dt == STARK_F32_SPLIT_TF32;
      a.b_mn = tf32 && b->plans[0]->tf32_mn;  // every member has the plan default
      a.fp16 = b->dt == STARK_F32_SPLIT_FP16 ? 1 : 0;
      // the two grouped launches on two branches of the graph: the second
      // takes SMs as the first one's tail frees them
      const bool both = b->split > 0 && b->split < count;
      cudaStream_t s_wide = both ? b->side[0] : b->cap, s_narrow = both ? b->side[1] : b->cap;
      if (both && (cudaEventRecord(b->fork_ev, b->cap) != cudaSuccess ||
                   cudaStreamWaitEvent(s_wide, b->fork_ev, 0) != cudaSuccess ||
                   cudaStreamWaitEvent(s_narrow, b->fork_ev, 0) != cudaSuccess))
        st = STARK_ECUDA;
      if (st == STARK_OK && b->split > 0) {  // 256-wide members
        a.groups = b->d_desc;
        a.ngroups = b->split;
        a.total_items = b->items_wide;
        if (launch_leaf_tc2_grouped(a, tf32, device_sm_count(), s_wide) != cudaSuccess) st = STARK_ECUDA;
      }
      if (st == STARK_OK && b->split < count) {  // 128-wide members
        a.groups = b->d_desc + b->split;
        a.ngroups = count - b->split;
        a.total_items = b->total_items;
        if (launch_leaf_tc_grouped(a, tf32, 128, device_sm_count(), s_narrow) != cudaSuccess) st = STARK_ECUDA;
      }
      if (both)
        for (int i = 0; i < 2; ++i)
          if (cudaEventRecord(b->join_ev[i], b->side[i]) != cudaSuccess ||
              cudaStreamWaitEvent(b->cap, b->join_ev[i], 0) != cudaSuccess)
            st = STARK_ECUDA;
      // members combined into a staging copy: move the result into C
      for (int k = 0; k < count && st == STARK_OK; ++k)
        if (b->host_desc[k].C != ptrs[3 * k + 2])
          st = plan_copy_cstage(b->plans[k], const_cast<void*>(ptrs[3 * k + 2]), b->cap);
    }
    const cudaError_t ec = cudaStreamEndCapture(b->cap, &graph);
    if (st != STARK_OK || ec != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return st != STARK_OK ? st : STARK_ECUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      b->exec = nullptr;
      cudaGetLastError();
      return STARK_ECUDA;
    }
    b->last = ptrs;
  }
  if (cudaGraphLaunch(b->exec, s) != cudaSuccess) {
    cudaGetLastError();
    return STARK_ECUDA;
  }
  ++b->replays;
  return STARK_OK;
}

stark_status stark_batch_check(stark_batch_t b, void* stream) {
  if (!b) return STARK_EINVAL;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return STARK_ECUDA;
  int e = 0;
  if (cudaMemcpy(&e, b->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return STARK_ECUDA;
  if (e != 0) {
    cudaMemset(b->d_err, 0, sizeof(int));
    return STARK_ETIMEOUT;
  }
  return STARK_OK;
}

}  // extern "C"
