// plan.cu -- plans (stark_plan_*), the product entry points (stark_mul*),
// the quadrant-index table and small utilities of the C ABI.
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>

#include "plan.h"
#include "ptx.cuh"
#include "stark_internal.h"

namespace stark {

static std::atomic<int64_t> g_launches{0};
void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int device_sm_count() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  return v > 0 ? v : 1;
}

bool device_is_sm100_family() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3;  // the library carries sm_103a code only
}

// ------------------------------------------------------------------ tables

void build_quadrant_table(int depth, int side, std::vector<int32_t>& count, std::vector<int32_t>& quad,
                          std::vector<int8_t>& sign) {
  int64_t P = 1;
  for (int k = 0; k < depth; ++k) P *= 7;
  const int maxT = 1 << depth;
  count.assign((size_t)P, 0);
  quad.assign((size_t)(P * maxT), 0);
  sign.assign((size_t)(P * maxT), 0);
  for (int64_t l = 0; l < P; ++l) {
    // digits, top level first
    int dig[8] = {0};
    int64_t x = l;
    for (int k = depth - 1; k >= 0; --k) {
      dig[k] = (int)(x % 7);
      x /= 7;
    }
    // enumerate the product of the per-level term lists
    std::vector<std::pair<int32_t, int>> cur{{0, 1}};
    for (int k = 0; k < depth; ++k) {
      std::vector<std::pair<int32_t, int>> nxt;
      for (auto& e : cur)
        for (int q = 0; q < 4; ++q) {
          const int c = side == 0 ? coef_a(dig[k], q) : side == 1 ? coef_b(dig[k], q) : coef_c(dig[k], q);
          if (c != 0) nxt.push_back({e.first * 4 + q, e.second * c});
        }
      cur.swap(nxt);
    }
    count[(size_t)l] = (int32_t)cur.size();
    for (size_t t = 0; t < cur.size(); ++t) {
      quad[(size_t)(l * maxT) + t] = cur[t].first;
      sign[(size_t)(l * maxT) + t] = (int8_t)cur[t].second;
    }
  }
}

void quadrant_offsets(int depth, int64_t npad, int32_t q, int64_t* row, int64_t* col) {
  int64_t r = 0, c = 0;
  for (int k = 1; k <= depth; ++k) {
    const int digit = (q >> (2 * (depth - k))) & 3;
    r += (int64_t)(digit >> 1) * (npad >> k);
    c += (int64_t)(digit & 1) * (npad >> k);
  }
  *row = r;
  *col = c;
}

// ------------------------------------------------------------------ TMA maps

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// planes [planes][L][L] of bf16 (or fp32 holding tf32), row-major; box =
// row_bytes of a row x box_rows rows of one plane, with the matching
// swizzle (128- or 64-byte; atom32: 128-byte with 32-byte atoms).  For the
// K-major X planes a box is a K slice of box_rows M rows; for the MN-major
// Y planes it is an N chunk of box_rows K rows.
bool make_tmap_planes(CUtensorMap* m, void* base, bool tf32, int64_t L, int64_t planes, int box_rows,
                      int row_bytes, bool atom32) {
  auto fn = encode_fn();
  if (!fn || (row_bytes != 128 && row_bytes != 64) || (atom32 && row_bytes != 128)) return false;
  const int esz = tf32 ? 4 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)L, (cuuint64_t)L, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)(L * esz), (cuuint64_t)(L * L * esz)};
  cuuint32_t box[3] = {(cuuint32_t)(row_bytes / esz), (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  atom32 ? CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B
                         : row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool make_tmap_mplanes(CUtensorMap* m, void* base, int64_t L, int64_t planes) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)L, (cuuint64_t)L, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)(L * 4), (cuuint64_t)(L * L * 4)};
  cuuint32_t box[3] = {32, 32, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool make_tmap_c(CUtensorMap* m, void* C, int64_t n, int64_t ld) {
  auto fn = encode_fn();
  if (!fn || n <= 0 || ld < n || (ld % 4) != 0 || (reinterpret_cast<uintptr_t>(C) & 15) != 0) return false;
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, C, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// ------------------------------------------------------------------ self test

__global__ void wait_selftest_kernel(const int* flag, int* err, uint64_t timeout_ns) {
  const uint64_t t0 = globaltimer_ns();
  while (*(volatile const int*)flag == 0) {
    if (globaltimer_ns() - t0 > timeout_ns) {
      record_error(err, kDevTimeoutTest);
      return;
    }
  }
}

cudaError_t launch_wait_selftest(int* buf, uint64_t timeout_ns, cudaStream_t s) {
  wait_selftest_kernel<<<1, 1, 0, s>>>(buf, buf + 1, timeout_ns);
  count_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ planning

int64_t pow7i(int d) {
  int64_t p = 1;
  for (int k = 0; k < d; ++k) p *= 7;
  return p;
}

int tile_granularity(stark_dtype dt) { return is_split(dt) ? 128 : 64; }

int64_t padded_side(int64_t n, int depth, stark_dtype dt) {
  const int64_t g = ((int64_t)1 << depth) * tile_granularity(dt);
  return std::max<int64_t>(g, (n + g - 1) / g * g);
}

size_t element_size(stark_dtype dt) { return is_split(dt) ? 4 : 8; }

// Device bytes of the leaf operand planes of one product.
int64_t operand_bytes(int64_t n, int depth, stark_dtype dt) {
  const int64_t npad = padded_side(n, depth, dt);
  const int64_t L = npad >> depth;
  const int64_t P = pow7i(depth);
  const int64_t per = half_split(dt) ? 4 : 8;  // hi+lo bf16 or fp16, hi+lo tf32, or one 8-byte value
  return 2 * P * L * L * per;
}

// Cost model for the depth choice (Sec. IV's per-stage cost with GB300
// rates in place of Spark's): the leaf launch's work at the kernel's
// measured rate, stretched by the quantisation of its tiles over the SMs,
// plus the divide's and C's bytes at HBM bandwidth and a fixed cost per
// launch.  Constants measured on GB300 (152 SMs): fp64 CUDA-core leaves
// 1.25 TFLOP/s, int64 6.85 TOP/s (64 x 64 tiles, one tile per SM at a time
// reaches the per-SM rate), 3xBF16 pair leaves 1.76 PFLOP/s and 3xTF32 0.93
// (three products per leaf term), HBM 6.7 TB/s, 22 us per divide launch
// (the depth-3 divide is one launch per top-level product and side, 14, and
// reads its input three times over).  The SM count is the device's (152
// when the host has no device).
double model_seconds(int64_t n, int depth, stark_dtype dt) {
  const int64_t npad = padded_side(n, depth, dt);
  const double L = (double)(npad >> depth);
  const double P = (double)pow7i(depth);
  // the device's SM count; host-only callers without a device get GB300's
  int dev = 0, v = 0;
  const bool have = cudaGetDevice(&dev) == cudaSuccess &&
                    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0;
  cudaGetLastError();
  const double sms = have ? (double)v : 152.0;
  double flops = 2.0 * P * L * L * L, rate, items, slots;
  switch (dt) {
    case STARK_F32_SPLIT_BF16:
    case STARK_F32_SPLIT_FP16:
    case STARK_F32_SPLIT_TF32: {
      flops *= 3;
      rate = half_split(dt) ? 1.76e15 : 0.93e15;
      const bool pair = (npad >> depth) % 256 == 0;  // 256 x 256 tiles on CTA pairs, else 128 x 128 on one CTA
      const double t = pair ? 256.0 : 128.0;
      items = P * (L / t) * (L / t);
      slots = pair ? sms / 2 : sms;
      if (!pair) rate *= 0.85;
      break;
    }
    default:
      rate = dt == STARK_F64 ? 1.25e12 : 6.85e12;
      items = P * (L / 64.0) * (L / 64.0);
      slots = sms;
      break;
  }
  const double waves = std::ceil(items / slots) / std::max(items / slots, 1e-9);
  const double esz = (double)element_size(dt);
  // depth 3: the split dtypes divide in one staged pass per operand (leaf
  // side a multiple of 128); otherwise one launch per top-level product,
  // reading the input three times
  const bool staged = depth == 3 && is_split(dt) && divide_staged_fits(npad >> depth);
  const bool per_top = depth == 3 && !staged;
  const double in_bytes = 2.0 * (double)n * n * esz * (per_top ? 3.0 : 1.0);
  const double ws = (double)operand_bytes(n, depth, dt);
  const double c_bytes = (double)n * n * esz;  // clearing C; the combine's adds stay in L2 / under the leaf work
  const double launches = (per_top ? 14.0 : 2.0);
  return flops / rate * waves + (in_bytes + ws + c_bytes) / 6.7e12 + launches * 22e-6 + 5e-6;
}

int choose_depth(int64_t n, stark_dtype dt) {
  int best = 0;
  double best_t = 1e300;
  // depths 0..3: the range the constants were measured over (depth 4 stays
  // available when asked for)
  for (int d = 0; d <= 3; ++d) {
    if ((padded_side(n, d, dt) >> d) < tile_granularity(dt)) continue;
    const double t = model_seconds(n, d, dt);
    if (t < best_t) {
      best_t = t;
      best = d;
    }
  }
  return best;
}

}  // namespace stark

using namespace stark;

// ====================================================================== C ABI
extern "C" {

const char* stark_strerror(stark_status s) {
  switch (s) {
    case STARK_OK: return "ok";
    case STARK_EINVAL: return "invalid argument";
    case STARK_ENOMEM: return "out of memory or over the memory budget";
    case STARK_EUNSUPPORTED: return "unsupported on this device or build";
    case STARK_ETIMEOUT: return "a bounded device-side wait expired";
    case STARK_EBUSY: return "request still pending";
    case STARK_ENOTFOUND: return "unknown request id";
    case STARK_ECUDA: return "CUDA runtime error";
  }
  return "unknown status";
}

int64_t stark_launch_count(void) { return g_launches.load(); }

stark_status stark_quadrant_table(int depth, int side, int32_t* count, int32_t* quad, int8_t* sign) {
  if (depth < 0 || depth > kMaxDepth || side < 0 || side > 2 || !count || !quad || !sign) return STARK_EINVAL;
  std::vector<int32_t> c, q;
  std::vector<int8_t> s;
  build_quadrant_table(depth, side, c, q, s);
  std::memcpy(count, c.data(), c.size() * sizeof(int32_t));
  std::memcpy(quad, q.data(), q.size() * sizeof(int32_t));
  std::memcpy(sign, s.data(), s.size());
  return STARK_OK;
}

stark_status stark_plan(int64_t n, int depth, stark_dtype dt, stark_plan_t* out) {
  return stark_plan_ex(n, depth, dt, 0u, out);
}

stark_status stark_plan_ex(int64_t n, int depth, stark_dtype dt, unsigned flags, stark_plan_t* out) {
  if (!out) return STARK_EINVAL;
  if (flags & ~(unsigned)STARK_PLAN_PEEL) return STARK_EINVAL;
  *out = nullptr;
  if (n < 0 || depth < -1 || depth > kMaxDepth) return STARK_EINVAL;
  if (dt != STARK_F64 && dt != STARK_I64 && !is_split(dt)) return STARK_EINVAL;
  if (n > (int64_t)1 << 20) return STARK_EINVAL;
  if (!device_is_sm100_family()) return STARK_EUNSUPPORTED;
  if (depth < 0) depth = is_split(dt) ? autotune_depth(n, dt) : choose_depth(n, dt);
  auto* p = new (std::nothrow) stark_plan_s();
  if (!p) return STARK_ENOMEM;
  stark_status st = plan_init(p, n, depth, dt, (flags & STARK_PLAN_PEEL) != 0);
  if (st != STARK_OK) {
    plan_release(p);
    delete p;
    return st;
  }
  *out = p;
  return STARK_OK;
}

static bool flush_copy_out(stark_plan_t p);

stark_status stark_plan_destroy(stark_plan_t p) {
  if (!p) return STARK_OK;
  if (p->s_out) flush_copy_out(p);  // a product still owed to host memory
  cudaDeviceSynchronize();
  plan_release(p);
  delete p;
  return STARK_OK;
}

stark_status stark_plan_get_info(stark_plan_t p, stark_plan_info* info) {
  if (!p || !info) return STARK_EINVAL;
  std::memset(info, 0, sizeof(*info));
  info->n = p->n;
  info->n_pad = p->npad;
  info->peel = (int32_t)p->peel;
  info->leaf = p->L;
  info->depth = p->depth;
  info->dtype = p->dt;
  info->leaves = p->P;
  info->workspace_bytes = p->ws_bytes;
  info->tile_m = p->is_tc ? 128 : 64;
  info->tile_n = p->is_tc ? p->bn : 64;
  info->combine = p->combine_mode;
  info->shard_levels = p->shard_levels;
  info->shard_first = (int32_t)p->shard_first;
  info->workspace_leaves = (int32_t)p->P_ws;
  info->promotion_k = p->promo_k;
  return STARK_OK;
}

stark_status stark_mul(stark_plan_t p, const void* A, const void* B, void* C, void* stream) {
  if (!p) return STARK_EINVAL;
  return plan_run(p, A, B, C, 0, p->P, (cudaStream_t)stream);
}

stark_status stark_mul_leaves(stark_plan_t p, const void* A, const void* B, void* C, int64_t leaf_begin,
                              int64_t leaf_end, void* stream) {
  if (!p || leaf_begin < 0 || leaf_end > p->P || leaf_begin > leaf_end) return STARK_EINVAL;
  return plan_run(p, A, B, C, leaf_begin, leaf_end, (cudaStream_t)stream);
}

// Staging buffers and pipeline streams for the host entry points.
static stark_status ensure_host_pipeline(stark_plan_t p) {
  if (p->ev_out[1]) return STARK_OK;  // created last: the whole pipeline exists
  // all or nothing: on any failure release what this call created
  const size_t bytes = (size_t)p->n * p->n * p->esz;
  void** bufs[6] = {&p->stage_A, &p->stage_B, &p->stage_C, &p->stage2[0], &p->stage2[1], &p->stage2[2]};
  cudaStream_t* streams[3] = {&p->s_in, &p->s_comp, &p->s_out};
  cudaEvent_t* events[6] = {&p->ev_in[0], &p->ev_comp[0], &p->ev_out[0], &p->ev_in[1], &p->ev_comp[1], &p->ev_out[1]};
  stark_status st = STARK_OK;
  for (void** b : bufs)
    if (st == STARK_OK && cudaMalloc(b, bytes) != cudaSuccess) st = STARK_ENOMEM;
  for (cudaStream_t* x : streams)
    if (st == STARK_OK && cudaStreamCreateWithFlags(x, cudaStreamNonBlocking) != cudaSuccess) st = STARK_ECUDA;
  for (cudaEvent_t* e : events)
    if (st == STARK_OK && cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) st = STARK_ECUDA;
  if (st != STARK_OK) {
    cudaGetLastError();
    for (void** b : bufs) {
      cudaFree(*b);
      *b = nullptr;
    }
    for (cudaStream_t* x : streams) {
      if (*x) cudaStreamDestroy(*x);
      *x = nullptr;
    }
    for (cudaEvent_t* e : events) {
      if (*e) cudaEventDestroy(*e);
      *e = nullptr;
    }
  }
  return st;
}

// The host pipeline: copies in on s_in, products on s_comp, copies out on
// s_out, two staging sets used alternately.  CUDA feeds streams to the GPU
// through a few hardware queues, and two streams may share one; an operation
// that waits on a later event then holds back everything queued behind it.
// So operations are enqueued in the order they become ready on the GPU: the
// copy out of product k (ready when product k ends) goes in after the copy
// in of product k+1 (ready when product k-1 ends), i.e. during the next call
// or at the wait that collects the results.
static bool flush_copy_out(stark_plan_t p) {
  if (p->pend_set < 0) return true;
  const int k = p->pend_set;
  const size_t bytes = (size_t)p->n * p->n * p->esz;
  void* dC = k ? p->stage2[2] : p->stage_C;
  bool ok = cudaStreamWaitEvent(p->s_out, p->ev_comp[k], 0) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(p->pend_C, dC, bytes, cudaMemcpyDeviceToHost, p->s_out) == cudaSuccess;
  ok = ok && cudaEventRecord(p->ev_out[k], p->s_out) == cudaSuccess;
  p->pend_set = -1;
  p->pend_C = nullptr;
  return ok;
}

// Enqueues copy in and product of one call; its copy out stays pending.
static stark_status host_enqueue(stark_plan_t p, const void* A, const void* B, void* C) {
  if (stark_status st = ensure_host_pipeline(p); st != STARK_OK) return st;
  const size_t bytes = (size_t)p->n * p->n * p->esz;
  const int k = p->host_calls++ & 1;  // buffer set of this call
  void* dA = k ? p->stage2[0] : p->stage_A;
  void* dB = k ? p->stage2[1] : p->stage_B;
  void* dC = k ? p->stage2[2] : p->stage_C;
  bool ok = true;
  // inputs of this set may be overwritten once the product two calls ago has
  // read them
  ok = ok && cudaStreamWaitEvent(p->s_in, p->ev_comp[k], 0) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(dA, A, bytes, cudaMemcpyHostToDevice, p->s_in) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(dB, B, bytes, cudaMemcpyHostToDevice, p->s_in) == cudaSuccess;
  ok = ok && cudaEventRecord(p->ev_in[k], p->s_in) == cudaSuccess;
  ok = ok && flush_copy_out(p);  // the previous call's result
  // this set's C may be overwritten once it has been copied out
  ok = ok && cudaStreamWaitEvent(p->s_comp, p->ev_in[k], 0) == cudaSuccess;
  ok = ok && cudaStreamWaitEvent(p->s_comp, p->ev_out[k], 0) == cudaSuccess;
  if (!ok) return STARK_ECUDA;
  stark_status st = plan_run(p, dA, dB, dC, 0, p->P, p->s_comp);
  if (st != STARK_OK) return st;
  if (cudaEventRecord(p->ev_comp[k], p->s_comp) != cudaSuccess) return STARK_ECUDA;
  p->pend_set = k;
  p->pend_C = C;
  return STARK_OK;
}

stark_status stark_mul_host_async(stark_plan_t p, const void* A, const void* B, void* C, void* stream) {
  if (!p || (p->n > 0 && (!A || !B || !C))) return STARK_EINVAL;
  if (p->n == 0) return STARK_OK;
  if (stark_status st = host_enqueue(p, A, B, C); st != STARK_OK) return st;
  const int k = p->pend_set;
  if (!flush_copy_out(p)) return STARK_ECUDA;
  // the caller's stream observes completion of this product
  if (cudaStreamWaitEvent((cudaStream_t)stream, p->ev_out[k], 0) != cudaSuccess) return STARK_ECUDA;
  return STARK_OK;
}

stark_status stark_mul_host_enqueue(stark_plan_t p, const void* A, const void* B, void* C) {
  if (!p || (p->n > 0 && (!A || !B || !C))) return STARK_EINVAL;
  if (p->n == 0) return STARK_OK;
  return host_enqueue(p, A, B, C);
}

stark_status stark_plan_host_wait(stark_plan_t p) {
  if (!p) return STARK_EINVAL;
  if (!p->s_out) return STARK_OK;  // nothing was ever enqueued
  if (!flush_copy_out(p)) return STARK_ECUDA;
  // s_out carries every copy out in call order: its completion covers all
  return stark_plan_check(p, p->s_out);
}

stark_status stark_mul_host(stark_plan_t p, const void* A, const void* B, void* C, void* stream) {
  stark_status st = stark_mul_host_async(p, A, B, C, stream);
  if (st != STARK_OK) return st;
  if (p->n == 0) return STARK_OK;
  return stark_plan_check(p, stream);
}

static stark_status plan_tune_combine(stark_plan_t p);

stark_status stark_plan_set_combine(stark_plan_t p, int mode) {
  if (!p || mode < -1 || mode > 3) return STARK_EINVAL;
  if (mode == -1) return plan_tune_combine(p);
  if (mode == 3) {
    // sibling fold on the CTA-pair kernel: 256-wide tiles, breadth first;
    // not with accumulator promotion
    if (!p->is_tc || p->depth < 1 || p->dfs || p->L % 256 != 0 || (p->dt == STARK_F32_SPLIT_TF32 && !p->tf32_mn) ||
        p->promo_k)
      return STARK_EUNSUPPORTED;
    if (!p->q_planes && p->n > 0) {
      const int64_t parents = p->P / 7, side = 2 * p->L;
      const size_t bytes = (size_t)parents * side * side * sizeof(float);
      if (cudaMalloc(&p->q_planes, bytes) != cudaSuccess) {
        cudaGetLastError();
        p->q_planes = nullptr;
        return STARK_ENOMEM;
      }
      p->ws_bytes += (int64_t)bytes;
      if (!make_tmap_mplanes(&p->tmQ, p->q_planes, side, parents)) return STARK_EUNSUPPORTED;
    }
  }
  if (mode == 2) {
    if (!p->is_tc || p->depth > 3 || p->dfs) return STARK_EUNSUPPORTED;
    if (!p->m_planes && p->n > 0) {
      const size_t bytes = (size_t)p->P * p->L * p->L * sizeof(float);
      if (cudaMalloc(&p->m_planes, bytes) != cudaSuccess) {
        cudaGetLastError();
        p->m_planes = nullptr;
        return STARK_ENOMEM;
      }
      p->ws_bytes += (int64_t)bytes;
      if (!make_tmap_mplanes(&p->tmM, p->m_planes, p->L, p->P)) return STARK_EUNSUPPORTED;
    }
  }
  p->combine_mode = mode;
  return STARK_OK;
}

// Measured choice of the combine mode for a tensor-core plan: every mode that
// applies (0 fused; 2 deterministic at depth <= 3; 3 sibling fold) runs one
// warm-up and three timed products on scratch inputs, and the fastest stays;
// the product buffers of the others are released.  Other plans keep mode 0.
static stark_status plan_tune_combine(stark_plan_t p) {
  if (!p->is_tc || p->n == 0 || p->dfs) return stark_plan_set_combine(p, 0);
  const size_t bytes = (size_t)p->n * p->n * p->esz;
  void *A = nullptr, *B = nullptr, *C = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  stark_status st = STARK_OK;
  if (cudaMalloc(&A, bytes) != cudaSuccess || cudaMalloc(&B, bytes) != cudaSuccess ||
      cudaMalloc(&C, bytes) != cudaSuccess) {
    st = STARK_ENOMEM;
  } else if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
             cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = STARK_ECUDA;
  }
  int best = 0;
  if (st == STARK_OK) {
    cudaMemsetAsync(A, 0x3c, bytes, s);  // bounded, nonzero values
    cudaMemsetAsync(B, 0x3c, bytes, s);
    float best_ms = 1e30f;
    for (int mode : {0, 2, 3}) {
      if (stark_plan_set_combine(p, mode) != STARK_OK) continue;
      bool ok = plan_run(p, A, B, C, 0, p->P, s) == STARK_OK;
      ok = ok && cudaEventRecord(e0, s) == cudaSuccess;
      for (int k = 0; k < 3 && ok; ++k) ok = plan_run(p, A, B, C, 0, p->P, s) == STARK_OK;
      ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
      float ms = 0;
      if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms) {
        best_ms = ms;
        best = mode;
      }
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) st = STARK_ECUDA;
    int e = 0;  // a device error during the trials is reported, not kept
    if (cudaMemcpy(&e, p->d_err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && e) {
      cudaMemset(p->d_err, 0, sizeof(int));
      st = STARK_ETIMEOUT;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(A);
  cudaFree(B);
  cudaFree(C);
  cudaGetLastError();
  // keep the winner's buffers only
  if (best != 2 && p->m_planes) {
    cudaFree(p->m_planes);
    p->m_planes = nullptr;
    p->ws_bytes -= (int64_t)((size_t)p->P * p->L * p->L * sizeof(float));
  }
  if (best != 3 && p->q_planes) {
    cudaFree(p->q_planes);
    p->q_planes = nullptr;
    p->ws_bytes -= (int64_t)((size_t)(p->P / 7) * (2 * p->L) * (2 * p->L) * sizeof(float));
  }
  p->combine_mode = best;
  return st;
}

// Workspace for `planes_per_half` leaves per operand side, with its maps.
static stark_status plan_alloc_operands(stark_plan_s* p, int64_t planes) {
  const int64_t per = half_split(p->dt) ? 4 : 8;  // bytes per leaf element per operand
  const int64_t bytes = planes * p->L * p->L * per;
  if (cudaDeviceSynchronize() != cudaSuccess) return STARK_ECUDA;
  const int64_t old = p->P_ws * p->L * p->L * per;
  // the new workspace first, so that on failure the plan keeps the old one;
  // when shrinking on a nearly full device, release the old one first
  void* X = nullptr;
  void* Y = nullptr;
  bool ok = cudaMalloc(&X, (size_t)bytes) == cudaSuccess && cudaMalloc(&Y, (size_t)bytes) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    cudaFree(X);
    cudaFree(Y);
    X = Y = nullptr;
    if (bytes > old) return STARK_ENOMEM;  // the plan keeps its workspace and traversal
    cudaFree(p->X);
    cudaFree(p->Y);
    p->X = p->Y = nullptr;
    p->ws_bytes -= 2 * old;
    p->P_ws = 0;
    if (cudaMalloc(&X, (size_t)bytes) != cudaSuccess || cudaMalloc(&Y, (size_t)bytes) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(X);
      cudaFree(Y);
      return STARK_ENOMEM;  // no workspace: products report ENOMEM until a traversal change succeeds
    }
  } else {
    cudaFree(p->X);
    cudaFree(p->Y);
    p->ws_bytes -= 2 * old;
  }
  p->X = X;
  p->Y = Y;
  p->ws_bytes += 2 * bytes;
  p->P_ws = planes;
  if (stark_status st = plan_operand_maps(p, planes); st != STARK_OK) return st;
  if (p->int_tc && (!make_tmap_planes(&p->tmAi, p->X, false, p->L, planes, 128) ||
                    !make_tmap_planes(&p->tmBi, p->Y, false, p->L, planes, 64)))
    return STARK_EUNSUPPORTED;
  return STARK_OK;
}

stark_status stark_plan_set_traversal(stark_plan_t p, int levels) {
  if (!p || levels < 0 || levels > 2) return STARK_EINVAL;
  if (levels && p->shard_levels) return STARK_EUNSUPPORTED;  // a shard keeps its own workspace
  if (!traversal_supported(p->depth, p->dt, levels) || (levels && p->combine_mode >= 2)) return STARK_EUNSUPPORTED;
  if (levels == p->dfs || p->n == 0) {
    p->dfs = levels;
    return STARK_OK;
  }
  const int prev = p->dfs;
  const stark_status st = plan_alloc_operands(p, p->P / pow7i(levels));
  // the traversal follows the workspace that exists (on a failed growth the
  // plan keeps its previous one)
  p->dfs = p->P_ws == p->P / pow7i(levels) ? levels : prev;
  return st;
}

stark_status stark_plan_set_shard(stark_plan_t p, int64_t lb, int64_t le) {
  if (!p || lb < 0 || le > p->P || lb >= le) return STARK_EINVAL;
  if (p->dfs) return STARK_EUNSUPPORTED;
  if (lb == 0 && le == p->P) {  // the whole product: breadth first, full workspace
    const stark_status st = p->shard_levels && p->n > 0 ? plan_alloc_operands(p, p->P) : STARK_OK;
    if (st == STARK_OK) {
      p->shard_levels = 0;
      p->shard_lb = 0;
      p->shard_le = p->P;
      p->shard_first = 0;
    }
    return st;
  }
  // subtrees below two top levels where the loaders have them, else one
  const int k = traversal_supported(p->depth, p->dt, 2) ? 2 : traversal_supported(p->depth, p->dt, 1) ? 1 : 0;
  if (k == 0 || (p->dt == STARK_F32_SPLIT_TF32 && !p->tf32_mn)) return STARK_EUNSUPPORTED;
  const int64_t gs = pow7i(p->depth - k);
  const int64_t g0 = lb / gs, g1 = (le + gs - 1) / gs;
  if (p->n > 0) {
    const stark_status st = plan_alloc_operands(p, (g1 - g0) * gs);
    if (st != STARK_OK) return st;
  }
  p->shard_levels = k;
  p->shard_lb = lb;
  p->shard_le = le;
  p->shard_first = g0 * gs;
  return STARK_OK;
}

stark_status stark_plan_set_input_bound(stark_plan_t p, int64_t max_abs) {
  if (!p || p->dt != STARK_I64 || max_abs < 0) return STARK_EINVAL;
  if (max_abs == 0) {
    p->int_tc = false;
    p->int_bound = 0;
    return STARK_OK;
  }
  // leaf operands are sums of 2^depth inputs: exact in bf16 up to 256, and
  // every fp32 partial sum of a leaf product exact up to 2^24
  const double xb = (double)max_abs * (double)((int64_t)1 << p->depth);
  if (xb > 256.0 || (double)p->L * xb * xb > 16777216.0 || p->L % 128 != 0 || !device_is_sm100_family())
    return STARK_EUNSUPPORTED;
  p->int_bn = (p->L % 256 == 0) ? 256 : 128;
  if (!make_tmap_planes(&p->tmAi, p->X, false, p->L, p->P_ws, 128) ||
      !make_tmap_planes(&p->tmBi, p->Y, false, p->L, p->P_ws, 64))
    return STARK_EUNSUPPORTED;
  p->int_bound = max_abs;
  p->int_tc = true;
  return STARK_OK;
}

stark_status stark_plan_set_pairing(stark_plan_t p, int enable) {
  if (!p || enable < 0 || enable > 2) return STARK_EINVAL;
  if (enable == 1) return STARK_EUNSUPPORTED;  // no schedule shares tiles between CTAs by multicast
  p->pair_mode = enable;
  return STARK_OK;
}

stark_status stark_plan_set_promotion(stark_plan_t p, int k_chunk) {
  if (!p || k_chunk < 0 || k_chunk % 256 != 0) return STARK_EINVAL;
  if (k_chunk == 0) {
    p->promo_k = 0;
    return STARK_OK;
  }
  // CTA-pair leaves (256-wide tiles, L % 256 == 0), bf16 or MN-major tf32,
  // not with the sibling fold
  if (!p->is_tc || p->L % 256 != 0 || p->bn != 256 || p->combine_mode == 3 ||
      (p->dt == STARK_F32_SPLIT_TF32 && !p->tf32_mn))
    return STARK_EUNSUPPORTED;
  p->promo_k = k_chunk;
  return STARK_OK;
}

stark_status stark_plan_set_raster(stark_plan_t p, int band) {
  if (!p || band < 0 || band > 4096) return STARK_EINVAL;
  p->raster_band = band;
  return STARK_OK;
}

stark_status stark_plan_set_pipeline(stark_plan_t p, int deep) {
  if (!p || deep < 0 || deep > 1) return STARK_EINVAL;
  p->deep_pipeline = deep;
  return STARK_OK;
}

stark_status stark_plan_check(stark_plan_t p, void* stream) {
  if (!p) return STARK_EINVAL;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return STARK_ECUDA;
  int e = 0;
  if (cudaMemcpy(&e, p->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return STARK_ECUDA;
  if (e != 0) {
    cudaMemset(p->d_err, 0, sizeof(int));
    return (e == kDevIntRange || e == kDevFp16Range) ? STARK_EINVAL : STARK_ETIMEOUT;
  }
  return STARK_OK;
}

stark_status stark_plan_set_timing(stark_plan_t p, int records) {
  if (!p || records < 0 || records > 100000) return STARK_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return STARK_ECUDA;
  for (auto e : p->ev) cudaEventDestroy(e);
  p->ev.clear();
  p->timing_cap = 0;
  p->timing_used = 0;
  p->ev.resize((size_t)records * kTimingEvents, nullptr);
  for (auto& e : p->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return STARK_ECUDA;
  p->timing_cap = records;
  return STARK_OK;
}

stark_status stark_plan_phase_ms(stark_plan_t p, float out_ms[3]) {
  float four[4];
  const stark_status st = stark_plan_phases(p, four, 4);
  if (st != STARK_OK) return st;
  out_ms[0] = four[0];
  out_ms[1] = four[1];
  out_ms[2] = four[2] + four[3];  // leaf products with the combine
  return STARK_OK;
}

stark_status stark_plan_phases(stark_plan_t p, float* out_ms, int count) {
  if (!p || !out_ms || count < 1 || count > 4 || p->timing_used == 0) return STARK_EINVAL;
  const size_t E = kTimingEvents;
  if (cudaEventSynchronize(p->ev[(size_t)(p->timing_used - 1) * E + E - 1]) != cudaSuccess) return STARK_ECUDA;
  double sum[4] = {0, 0, 0, 0};
  for (int r = 0; r < p->timing_used; ++r)
    for (int i = 0; i < 4; ++i) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, p->ev[(size_t)r * E + i], p->ev[(size_t)r * E + i + 1]) != cudaSuccess)
        return STARK_ECUDA;
      sum[i] += ms;
    }
  for (int i = 0; i < count; ++i) out_ms[i] = (float)(sum[i] / p->timing_used);
  return STARK_OK;
}

stark_status stark_selftest_bounded_wait(uint64_t timeout_ns) {
  int* buf = nullptr;
  if (cudaMalloc(&buf, 2 * sizeof(int)) != cudaSuccess) return STARK_ENOMEM;
  cudaMemset(buf, 0, 2 * sizeof(int));
  stark_status st = STARK_OK;
  if (launch_wait_selftest(buf, timeout_ns, 0) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    st = STARK_ECUDA;
  } else {
    int h[2] = {0, 0};
    cudaMemcpy(h, buf, sizeof(h), cudaMemcpyDeviceToHost);
    st = h[1] == kDevTimeoutTest ? STARK_ETIMEOUT : STARK_OK;
  }
  cudaFree(buf);
  return st;
}

}  // extern "C"

// ====================================================================== plan internals
namespace stark {

bool traversal_supported(int depth, stark_dtype dt, int levels) {
  if (levels == 0) return true;
  // the subtree below `levels` is at most 2 (one level) or 1 (two levels) deep
  if (levels < 0 || levels > 2 || depth < levels || depth > 3) return false;
  return levels == 1 || is_split(dt);
}

stark_status plan_init(stark_plan_s* p, int64_t n, int depth, stark_dtype dt, bool peel, int dfs) {
  if (!traversal_supported(depth, dt, dfs)) return STARK_EUNSUPPORTED;
  p->n = n;
  p->depth = depth;
  p->dt = dt;
  p->is_tc = is_split(dt);
  p->esz = element_size(dt);
  const int64_t g = ((int64_t)1 << depth) * tile_granularity(dt);
  p->peel = (peel && n >= g) ? n % g : 0;
  const int64_t core = n - p->peel;  // the recursion's side; a multiple of g when peeled
  p->npad = padded_side(core, depth, dt);
  p->L = p->npad >> depth;
  p->P = pow7i(depth);
  p->P_ws = p->P / pow7i(dfs);
  p->dfs = dfs;
  p->bn = (p->L % 256 == 0) ? 256 : 128;
  cudaGetDevice(&p->device);
  p->num_sms = device_sm_count();
  if (p->L > 0x7FFFFFFF / 2) return STARK_EINVAL;

  const int64_t ws = operand_bytes(core, depth, dt) / pow7i(dfs);
  if (cudaMalloc(&p->X, (size_t)(ws / 2)) != cudaSuccess || cudaMalloc(&p->Y, (size_t)(ws / 2)) != cudaSuccess) {
    cudaGetLastError();
    return STARK_ENOMEM;
  }
  p->ws_bytes = ws;

  // C targets of every leaf (side 2 of the quadrant-index table)
  std::vector<int32_t> cnt, quad;
  std::vector<int8_t> sign;
  build_quadrant_table(depth, 2, cnt, quad, sign);
  p->maxT = 1 << depth;
  std::vector<CTarget> tab((size_t)(p->P * p->maxT));
  for (int64_t l = 0; l < p->P; ++l)
    for (int t = 0; t < cnt[(size_t)l]; ++t) {
      int64_t r = 0, c = 0;
      quadrant_offsets(depth, p->npad, quad[(size_t)(l * p->maxT + t)], &r, &c);
      CTarget& e = tab[(size_t)(l * p->maxT + t)];
      e.row_off = (int32_t)r;
      e.col_off = (int32_t)c;
      e.sign = sign[(size_t)(l * p->maxT + t)];
      e.pad = 0;
    }
  const size_t tab_bytes = tab.size() * sizeof(CTarget);
  if (cudaMalloc(&p->d_ctab, tab_bytes) != cudaSuccess || cudaMalloc(&p->d_ccount, cnt.size() * 4) != cudaSuccess ||
      cudaMalloc(&p->d_err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return STARK_ENOMEM;
  }
  p->ws_bytes += (int64_t)(tab_bytes + cnt.size() * 4 + sizeof(int));
  if (cudaMemcpy(p->d_ctab, tab.data(), tab_bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->d_ccount, cnt.data(), cnt.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(p->d_err, 0, sizeof(int)) != cudaSuccess)
    return STARK_ECUDA;

  if (p->is_tc && n > 0 && n % 4 != 0) {
    // C cannot be a TMA target: combine into a staging copy with an aligned pitch
    if (stark_status e = plan_ensure_cstage(p); e != STARK_OK) return e;
  }
  return plan_operand_maps(p, p->P_ws);
}

stark_status plan_operand_maps(stark_plan_s* p, int64_t planes) {
  p->has_maps64 = false;
  p->has_mapbp = false;
  if (!p->is_tc) return STARK_OK;
  const bool tf32 = p->dt == STARK_F32_SPLIT_TF32;
  // (16-bit planes -- bf16 or fp16 halves -- use bf16 maps: a tiled load
  // copies the 2-byte elements bit for bit and fills out-of-range with 0)
  // X: K-major 128-byte rows.  Y: bf16 MN-major 64 x 64 boxes; tf32 either
  // MN-major 32 x 32 boxes with the 32-byte-atom swizzle, or (transposed
  // planes) K-major boxes of a whole tile's rows
  bool ok = make_tmap_planes(&p->tmA, p->X, tf32, p->L, 2 * planes, 128);
  if (!tf32)
    ok = ok && make_tmap_planes(&p->tmB, p->Y, false, p->L, 2 * planes, 64);
  else if (p->tf32_mn)
    ok = ok && make_tmap_planes(&p->tmB, p->Y, true, p->L, 2 * planes, 32, 128, true);
  else
    ok = ok && make_tmap_planes(&p->tmB, p->Y, true, p->L, 2 * planes, p->bn);
  return ok ? STARK_OK : STARK_EUNSUPPORTED;
}

void plan_release(stark_plan_s* p) {
  cudaFree(p->X);
  cudaFree(p->Y);
  cudaFree(p->d_ctab);
  cudaFree(p->d_ccount);
  cudaFree(p->d_err);
  cudaFree(p->stage_A);
  cudaFree(p->stage_B);
  cudaFree(p->stage_C);
  for (void* b : p->stage2) cudaFree(b);
  for (cudaStream_t st : {p->s_in, p->s_comp, p->s_out})
    if (st) cudaStreamDestroy(st);
  for (int i = 0; i < 2; ++i)
    for (cudaEvent_t e : {p->ev_in[i], p->ev_comp[i], p->ev_out[i]})
      if (e) cudaEventDestroy(e);
  cudaFree(p->cstage);
  cudaFree(p->m_planes);
  cudaFree(p->q_planes);
  for (auto e : p->ev)
    if (e) cudaEventDestroy(e);
  p->ev.clear();
  cudaGetLastError();
}

static stark_status to_status(cudaError_t e) {
  if (e == cudaSuccess) return STARK_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? STARK_ENOMEM : STARK_ECUDA;
}

// Divide phase into the workspace.  top < 0: every leaf operand (breadth
// first); top = i1: only the subtree below top-level product M_{i1+1}
// (depth-first traversal), its leaves in planes 0..7^(d-1)-1.
stark_status plan_divide_top(stark_plan_s* p, const void* A, const void* B, cudaStream_t s, int top, int levels,
                             int64_t plane_off) {
  if (!p->X || !p->Y) return STARK_ENOMEM;  // no workspace (failed reallocation)
  // depth first: the subtree below `levels` top levels along the M-index path `top`
  const int lv = top >= 0 ? levels : 0;
  const int64_t npad = p->npad >> lv;
  const int depth = p->depth - lv;
  // bytes per element of a (hi) plane: bf16 for 3xBF16 and for bounded
  // integers, tf32 in fp32 containers, else the input type
  const size_t ehi = (half_split(p->dt) || p->int_tc) ? 2 : p->dt == STARK_F32_SPLIT_TF32 ? 4 : 8;
  const size_t off = (size_t)plane_off * (size_t)p->L * p->L * ehi;  // first output plane
  // the core of A and B (all of them unless an edge is peeled), row stride n
  DivideArgs da{A, core_side(p), npad, p->L, static_cast<char*>(p->X) + off, nullptr, p->d_err, top, p->n};
  DivideArgs db{B, core_side(p), npad, p->L, static_cast<char*>(p->Y) + off, nullptr, p->d_err, top, p->n};
  da.top_levels = db.top_levels = lv;
  InType in = p->dt == STARK_F64 ? kInF64 : p->dt == STARK_I64 ? kInI64 : kInF32;
  OutMode om = p->dt == STARK_F32_SPLIT_BF16   ? kOutSplitBf16
              : p->dt == STARK_F32_SPLIT_FP16 ? kOutSplitFp16
              : p->dt == STARK_F32_SPLIT_TF32 ? kOutSplitTf32
                                              : kOutPlain;
  if (p->int_tc) om = kOutBf16Exact;  // bounded integers: exact bf16 operands, range checked
  if (p->is_tc) {
    const int64_t half = p->P_ws * p->L * p->L * (half_split(p->dt) ? 2 : 4);
    da.out_lo = static_cast<char*>(p->X) + half + off;
    db.out_lo = static_cast<char*>(p->Y) + half + off;
  }
  stark_status st = STARK_OK;
  if (top < 0 && depth == 3 && (om == kOutSplitBf16 || om == kOutSplitTf32 || om == kOutSplitFp16) &&
      divide_staged_fits(p->L)) {
    // breadth first at depth 3, split fp32: one pass per operand, the
    // input tile staged in shared memory
    st = to_status(launch_divide_staged(da, 0, om, s));
    if (st == STARK_OK) st = to_status(launch_divide_staged(db, 1, om, s));
  } else if (top < 0 && depth == 3) {
    // breadth first at depth 3: one launch per top-level product, each a
    // depth-2 subtree read through that product's level-1 sum and written
    // to its block of 7^(d-1) planes (the outer-prefix form of the deep
    // kernel keeps too few loads in flight to stream at HBM bandwidth)
    const int64_t sub = pow7i(depth - 1);
    const size_t plane = (size_t)p->L * p->L * ehi;
    for (int t = 0; t < 7 && st == STARK_OK; ++t) {
      for (int side = 0; side < 2 && st == STARK_OK; ++side) {
        DivideArgs a = side ? db : da;
        a.top = t;
        a.top_levels = 1;
        a.npad = p->npad / 2;
        a.out_hi = static_cast<char*>(a.out_hi) + (size_t)t * sub * plane;
        if (a.out_lo) a.out_lo = static_cast<char*>(a.out_lo) + (size_t)t * sub * plane;
        st = to_status(launch_divide(a, depth - 1, side, in, om, s));
      }
    }
  } else {
    st = to_status(launch_divide(da, depth, 0, in, om, s));
    if (st == STARK_OK) st = to_status(launch_divide(db, depth, 1, in, om, s));
  }
  if (st != STARK_OK) return st;
  if (p->dt == STARK_F32_SPLIT_TF32 && !p->tf32_mn)  // K-major tf32 B: N x K planes
    st = to_status(launch_transpose_planes(static_cast<float*>(p->Y), p->L, 2 * p->P_ws, s));
  return st;
}

// Divide of a shard's subtrees that hold leaves [lb, le) (stark_plan_set_shard).
static stark_status plan_divide_shard(stark_plan_s* p, const void* A, const void* B, cudaStream_t s, int64_t lb,
                                      int64_t le) {
  const int k = p->shard_levels;
  const int64_t gs = pow7i(p->depth - k);
  stark_status st = STARK_OK;
  for (int64_t g = lb / gs; g * gs < le && st == STARK_OK; ++g)
    st = plan_divide_top(p, A, B, s, (int)g, k, g * gs - p->shard_first);
  return st;
}

stark_status plan_divide(stark_plan_s* p, const void* A, const void* B, cudaStream_t s) {
  if (p->dfs) return STARK_EUNSUPPORTED;  // the workspace holds one subtree only
  if (p->shard_levels) return plan_divide_shard(p, A, B, s, p->shard_lb, p->shard_le);
  return plan_divide_top(p, A, B, s, -1, 0, 0);
}

// The event set of the product being timed (stark_plan_set_timing), or null.
static cudaEvent_t* plan_timing_events(stark_plan_s* p) {
  return (p->timing_used > 0 && p->timing_used <= p->timing_cap && p->timing_active)
             ? &p->ev[(size_t)(p->timing_used - 1) * kTimingEvents]
             : nullptr;
}

// Whether leaves [lb, le) use the deterministic combine (stored M planes and
// an ordered pass) rather than the fused epilogue.
static bool plan_deterministic(const stark_plan_s* p, int64_t lb, int64_t le) {
  return p->is_tc && p->combine_mode == 2 && p->m_planes && lb == 0 && le == p->P;
}

// Whether leaves [lb, le) use the sibling-folded combine (combine mode 3): the
// whole product, breadth first, on the CTA-pair kernel (256-wide tiles).
static bool plan_sib(const stark_plan_s* p, int64_t lb, int64_t le) {
  return p->is_tc && p->combine_mode == 3 && p->q_planes && lb == 0 && le == p->P && p->pair_mode == 2 &&
         p->bn == 256 && p->L % 256 == 0 && !p->dfs && !p->deep_pipeline && p->depth >= 1 &&
         (half_split(p->dt) || p->tf32_mn);
}

// Whether a separate pass writes every element of C (combine modes 2 and 3):
// then C is not cleared first and no staging copy is used.
static bool plan_stored(const stark_plan_s* p, int64_t lb, int64_t le) {
  return plan_deterministic(p, lb, le) || plan_sib(p, lb, le);
}

// Leaf products of leaves [lb, le) with the combine, operands in workspace
// planes numbered from plane_base.  With a staging copy of C the products
// land there; plan_run_accumulate moves them into C.
static stark_status plan_leaves(stark_plan_s* p, void* C, int64_t lb, int64_t le, int64_t plane_base,
                                cudaStream_t s) {
  stark_status st = STARK_OK;
  if (p->is_tc) {
    LeafTcArgs a{};
    a.P = (int32_t)p->P_ws;
    a.plane_base = (int32_t)plane_base;
    a.L = (int32_t)p->L;
    a.leaf_begin = (int32_t)lb;
    a.leaf_end = (int32_t)le;
    a.ctab = p->d_ctab;
    a.ccount = p->d_ccount;
    a.maxT = p->maxT;
    const bool deterministic = plan_deterministic(p, lb, le);
    const bool sib = plan_sib(p, lb, le);
    const bool staged = !deterministic && !sib && plan_uses_cstage(p, C);
    a.C = static_cast<float*>(staged ? p->cstage : C);
    a.ldc = staged ? staged_ld(p->n) : p->n;
    a.n = core_side(p);  // C rows/columns the combine covers
    a.err = p->d_err;
    a.timeout_ns = p->timeout_ns;
    CUtensorMap tmC;
    std::memset(&tmC, 0, sizeof(tmC));
    a.use_tma_c = (p->combine_mode == 0 && make_tmap_c(&tmC, a.C, core_side(p), a.ldc)) ? 1 : 0;
    if (deterministic) {
      a.store_m = 1;
      a.use_tma_c = 0;
      tmC = p->tmM;
    } else if (sib) {
      a.sib = 1;
      a.use_tma_c = 0;
      tmC = p->tmQ;
    }
    a.pair = p->pair_mode;
    a.fp16 = p->dt == STARK_F32_SPLIT_FP16 ? 1 : 0;
    a.band = p->raster_band;
    a.b_mn = p->tf32_mn;
    a.row_bytes = 128;
    if (p->deep_pipeline && p->dt == STARK_F32_SPLIT_BF16 && p->bn == 256) {
      a.pair = 0;  // the 64-byte-row schedule runs single CTAs
      a.row_bytes = 64;
      if (!p->has_maps64) {
        if (!make_tmap_planes(&p->tmA64, p->X, false, p->L, 2 * p->P_ws, 128, 64) ||
            !make_tmap_planes(&p->tmB64, p->Y, false, p->L, 2 * p->P_ws, 32, 64))
          return STARK_EUNSUPPORTED;
        p->has_maps64 = true;
      }
    }
    const bool tf32 = p->dt == STARK_F32_SPLIT_TF32;
    if (p->promo_k) {
      // accumulator promotion runs on the CTA-pair kernel only
      if (a.pair != 2 || p->bn != 256 || !leaf_tc2_fits(a) || sib || (tf32 && !p->tf32_mn))
        return STARK_EUNSUPPORTED;
      a.promo_kb = p->promo_k / (tf32 ? 32 : 64);
    }
    if (a.pair == 2 && p->bn == 256 && leaf_tc2_fits(a)) {
      // CTA pairs on one 256 x 256 MMA; K-major tf32 needs Y boxes of 128 rows
      if (tf32 && !p->tf32_mn && !p->has_mapbp) {
        if (!make_tmap_planes(&p->tmBp, p->Y, true, p->L, 2 * p->P_ws, 128)) return STARK_EUNSUPPORTED;
        p->has_mapbp = true;
      }
      st = to_status(launch_leaf_tc2(a, &p->tmA, (tf32 && !p->tf32_mn) ? &p->tmBp : &p->tmB, &tmC, tf32, p->num_sms, s));
    } else {
      st = to_status(launch_leaf_tc(a, a.row_bytes == 64 ? &p->tmA64 : &p->tmA,
                                    a.row_bytes == 64 ? &p->tmB64 : &p->tmB, &tmC, tf32, p->bn, p->num_sms, s));
    }
    if (st == STARK_OK && (deterministic || sib)) {
      if (cudaEvent_t* ev = plan_timing_events(p)) {
        cudaEventRecord(ev[3], s);  // the leaf products end, the combine pass starts
        p->timing_leaf_marked = true;
      }
    }
    if (st == STARK_OK && deterministic)
      st = to_status(launch_combine(static_cast<const float*>(p->m_planes), p->depth, p->L, p->npad, core_side(p),
                                    static_cast<float*>(C), p->n, s));
    // sibling fold: the parent planes are the leaf products of the depth-1
    // recursion; one ordered pass combines them into C
    if (st == STARK_OK && sib)
      st = to_status(launch_combine(static_cast<const float*>(p->q_planes), p->depth - 1, 2 * p->L, p->npad,
                                    core_side(p), static_cast<float*>(C), p->n, s));
  } else if (p->int_tc) {
    LeafTcArgs a{};
    a.P = (int32_t)p->P_ws;
    a.plane_base = (int32_t)plane_base;
    a.L = (int32_t)p->L;
    a.leaf_begin = (int32_t)lb;
    a.leaf_end = (int32_t)le;
    a.ctab = p->d_ctab;
    a.ccount = p->d_ccount;
    a.maxT = p->maxT;
    a.C = static_cast<float*>(C);  // int64 C, reinterpreted by the integer epilogue
    a.ldc = p->n;
    a.n = core_side(p);
    a.err = p->d_err;
    a.timeout_ns = p->timeout_ns;
    st = to_status(launch_leaf_tc_int(a, &p->tmAi, &p->tmBi, p->int_bn, p->num_sms, s));
  } else {
    LeafCcArgs a{};
    a.P = (int32_t)p->P_ws;
    a.plane_base = (int32_t)plane_base;
    a.L = (int32_t)p->L;
    a.leaf_begin = (int32_t)lb;
    a.leaf_end = (int32_t)le;
    a.X = p->X;
    a.Y = p->Y;
    a.ctab = p->d_ctab;
    a.ccount = p->d_ccount;
    a.maxT = p->maxT;
    a.C = C;
    a.ldc = p->n;
    a.n = core_side(p);
    st = to_status(p->dt == STARK_F64 ? launch_leaf_f64(a, s) : launch_leaf_i64(a, s));
  }
  return st;
}

// The peeled edge of a product with n = m + r (Ct: C or its staging copy,
// row stride ldc): the rank-r update of the core and the two edge strips,
//   C[:m, :m] += A[:m, m:] B[m:, :m],  C[:m, m:] = A[:m, :] B[:, m:],
//   C[m:, :] = A[m:, :] B,
// so that with the recursion's C[:m, :m] = A[:m, :m] B[:m, :m] every
// element of C is the classical product's (block form of A B).
static stark_status plan_border(stark_plan_s* p, const void* A, const void* B, void* Ct, int64_t ldc,
                                bool deterministic, cudaStream_t s) {
  const int64_t n = p->n, m = core_side(p), r = p->peel;
  const InType t = p->dt == STARK_F64 ? kInF64 : p->dt == STARK_I64 ? kInI64 : kInF32;
  const int64_t e = (int64_t)p->esz;
  auto in = [&](const void* base, int64_t row, int64_t col) {
    return static_cast<const void*>(static_cast<const char*>(base) + (row * n + col) * e);
  };
  auto out = [&](int64_t row, int64_t col) { return static_cast<void*>(static_cast<char*>(Ct) + (row * ldc + col) * e); };
  // the strips are added into zeros (the deterministic combine does not
  // clear C), so their K can be split across blocks, except where results
  // must be bitwise reproducible
  const int split = deterministic ? 0 : 1;
  if (cudaMemset2DAsync(out(0, m), (size_t)(ldc * e), 0, (size_t)(r * e), (size_t)m, s) != cudaSuccess ||
      cudaMemset2DAsync(out(m, 0), (size_t)(ldc * e), 0, (size_t)(n * e), (size_t)r, s) != cudaSuccess)
    return to_status(cudaGetLastError());
  const BorderArgs parts[3] = {
      {in(A, 0, m), n, in(B, m, 0), n, out(0, 0), ldc, m, m, r, 1, split, 0},  // core update
      {A, n, in(B, 0, m), n, out(0, m), ldc, m, r, n, 1, split, 0},            // right strip
      {in(A, m, 0), n, B, n, out(m, 0), ldc, r, n, n, 1, split, 0},            // bottom strip
  };
  for (const BorderArgs& a : parts)
    if (stark_status st = to_status(launch_border(a, t, p->num_sms, s)); st != STARK_OK) return st;
  return STARK_OK;
}

stark_status plan_run_accumulate(stark_plan_s* p, const void* A, const void* B, void* C, int64_t lb, int64_t le,
                                 cudaStream_t s) {
  if (p->n == 0) return STARK_OK;
  if (!A || !B || !C) return STARK_EINVAL;
  if (!p->X || !p->Y) return STARK_ENOMEM;  // a failed workspace reallocation left none
  cudaEvent_t* ev = plan_timing_events(p);
  if (ev) cudaEventRecord(ev[1], s);
  stark_status st = STARK_OK;
  if (lb == le) {
    // no leaves: C keeps what the caller put there (the peeled edge below
    // still belongs to the range that starts at leaf 0)
    if (ev) cudaEventRecord(ev[2], s);
  } else if (p->shard_levels) {
    // a shard: divide only the subtrees holding leaves [lb, le), whose
    // operands fill the workspace from leaf shard_first on
    if (lb < p->shard_lb || le > p->shard_le) return STARK_EINVAL;
    st = plan_divide_shard(p, A, B, s, lb, le);
    if (st != STARK_OK) return st;
    if (ev) cudaEventRecord(ev[2], s);
    st = plan_leaves(p, C, lb, le, p->shard_first, s);
    if (ev && !p->timing_leaf_marked) {
      cudaEventRecord(ev[3], s);
      p->timing_leaf_marked = true;
    }
  } else if (!p->dfs) {
    st = plan_divide_top(p, A, B, s, -1, 0, 0);
    if (st != STARK_OK) return st;
    if (ev) cudaEventRecord(ev[2], s);
    st = plan_leaves(p, C, lb, le, 0, s);
    if (ev && !p->timing_leaf_marked) {  // fused: the leaf kernel ends here
      cudaEventRecord(ev[3], s);
      p->timing_leaf_marked = true;
    }
  } else {
    // depth-first over the top p->dfs levels: one subtree's operands at a
    // time (divide and leaves interleave; the phase timer reports them
    // together)
    if (ev) cudaEventRecord(ev[2], s);
    const int tops = (int)pow7i(p->dfs);
    int last = -1;
    for (int top = 0; top < tops; ++top)
      if (std::max<int64_t>(lb, top * p->P_ws) < std::min<int64_t>(le, (top + 1) * p->P_ws)) last = top;
    for (int top = 0; top <= last && st == STARK_OK; ++top) {
      const int64_t b0 = top * p->P_ws, b1 = b0 + p->P_ws;
      const int64_t lo = lb > b0 ? lb : b0, hi = le < b1 ? le : b1;
      if (lo >= hi) continue;
      st = plan_divide_top(p, A, B, s, top, p->dfs, 0);
      if (st == STARK_OK) st = plan_leaves(p, C, lo, hi, b0, s);
    }
  }
  // the peeled edge, once per product (with the range that holds leaf 0, so
  // the partial products of a leaf partition still sum to A B), then the
  // staging copy into C
  const bool staged = p->is_tc && !plan_stored(p, lb, le) && plan_uses_cstage(p, C);
  if (st == STARK_OK && p->peel > 0 && lb == 0)
    st = plan_border(p, A, B, staged ? p->cstage : C, staged ? staged_ld(p->n) : p->n, plan_stored(p, lb, le), s);
  if (st == STARK_OK && staged) st = plan_copy_cstage(p, C, s);
  if (ev && !p->timing_leaf_marked) cudaEventRecord(ev[3], s);  // depth first: one interleaved phase
  if (ev) cudaEventRecord(ev[4], s);
  p->timing_active = false;
  p->timing_leaf_marked = false;
  return st;
}

stark_status plan_run(stark_plan_s* p, const void* A, const void* B, void* C, int64_t lb, int64_t le,
                      cudaStream_t s) {
  if (p->n == 0) return STARK_OK;
  if (!A || !B || !C) return STARK_EINVAL;
  if (p->timing_used < p->timing_cap) {
    cudaEventRecord(p->ev[(size_t)p->timing_used * kTimingEvents], s);
    ++p->timing_used;
    p->timing_active = true;
  }
  if (plan_stored(p, lb, le)) {
    // a separate combine pass writes every element of C: nothing to clear
  } else if (p->is_tc && plan_uses_cstage(p, C)) {
    if (cudaMemsetAsync(p->cstage, 0, (size_t)p->n * staged_ld(p->n) * 4, s) != cudaSuccess)
      return to_status(cudaGetLastError());
  } else if (cudaMemsetAsync(C, 0, (size_t)p->n * p->n * p->esz, s) != cudaSuccess) {
    return to_status(cudaGetLastError());
  }
  return plan_run_accumulate(p, A, B, C, lb, le, s);
}

stark_status plan_ensure_cstage(stark_plan_s* p) {
  if (p->cstage) return STARK_OK;
  const size_t bytes = (size_t)p->n * staged_ld(p->n) * 4;
  if (cudaMalloc(&p->cstage, bytes) != cudaSuccess) {
    cudaGetLastError();
    p->cstage = nullptr;
    return STARK_ENOMEM;
  }
  p->ws_bytes += (int64_t)bytes;
  return STARK_OK;
}

bool plan_uses_cstage(const stark_plan_s* p, const void* C) {
  return p->is_tc && p->combine_mode != 1 && p->cstage != nullptr && !c_is_tma_target(C, p->n);
}

stark_status plan_copy_cstage(const stark_plan_s* p, void* C, cudaStream_t s) {
  const size_t w = (size_t)p->n * 4;
  return to_status(cudaMemcpy2DAsync(C, w, p->cstage, (size_t)staged_ld(p->n) * 4, w, (size_t)p->n,
                                     cudaMemcpyDeviceToDevice, s));
}

}  // namespace stark

extern "C" stark_status stark_plan_set_tf32_layout(stark_plan_t p, int mn) {
  if (!p || mn < 0 || mn > 1) return STARK_EINVAL;
  if (p->dt != STARK_F32_SPLIT_TF32) return mn ? STARK_EUNSUPPORTED : STARK_OK;
  if (!mn && p->shard_levels) return STARK_EUNSUPPORTED;  // a shard's planes are transposed by group
  if (cudaDeviceSynchronize() != cudaSuccess) return STARK_ECUDA;
  p->tf32_mn = mn;
  return plan_operand_maps(p, p->P_ws);
}

extern "C" stark_status stark_plan_operands(stark_plan_t p, const void* A, const void* B, void* stream,
                                            const void** X, const void** Y) {
  if (!p || !X || !Y) return STARK_EINVAL;
  *X = p->X;
  *Y = p->Y;
  if (p->n == 0) return STARK_OK;
  if (!A || !B) return STARK_EINVAL;
  return stark::plan_divide(p, A, B, (cudaStream_t)stream);
}
