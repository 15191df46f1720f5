// noalloc.cu -- stark_mul_noalloc: the 3xBF16 product without any device
// allocation, for callers that cannot call cudaMalloc (for example code that
// runs where a memory allocator must not be entered, or a host that hands
// this library a fixed device-memory budget it may not grow).
//
// The workspace (leaf operand planes, the C-target table, the error word)
// lives in one file-scope __device__ array of fixed size, kNoallocScratch
// bytes.  Every device that loads this file's module holds that array until
// the process exits (with CUDA's lazy module loading the module, and so the
// array, is loaded by the first call of this entry point on the device).
//
// In host code `g_scratch` names a host-side stand-in, not device memory: a
// kernel given that name would fault or, where the GPU can reach host memory,
// silently use the wrong memory.  So the first call on each device (with
// that device current) asks the runtime for the array's device address with
// cudaGetSymbolAddress, checks the result and caches it per device; every
// kernel receives that address.  Do that first call before any stream
// capture.  All calls share the one array and it keeps the contents of the
// last call: the error word is cleared on every call, and calls that overlap
// on the GPU (different streams, or different host threads) race on the
// array, so callers must order them.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "plan.h"
#include "stark_internal.h"

namespace stark {
namespace {

constexpr size_t kNoallocScratch = STARK_NOALLOC_SCRATCH_BYTES;
constexpr int kNoallocMaxDepth = 3;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kNoallocScratch];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once).
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// C targets of every leaf (Alg. 5 with the C22 = M1 - M2 + M3 + M6 sign),
// written into fixed host arrays (no heap use on this path).
void c_targets(int depth, int64_t npad, CTarget* tab, int32_t* count) {
  int64_t P = 1;
  for (int k = 0; k < depth; ++k) P *= 7;
  const int maxT = 1 << depth;
  for (int64_t l = 0; l < P; ++l) {
    int dig[kNoallocMaxDepth + 1] = {0};
    int64_t x = l;
    for (int k = depth - 1; k >= 0; --k) {
      dig[k] = (int)(x % 7);
      x /= 7;
    }
    int q[16] = {0}, s[16] = {1};
    int cnt = 1;
    for (int k = 0; k < depth; ++k) {
      int q2[16], s2[16], c2 = 0;
      for (int e = 0; e < cnt; ++e)
        for (int cq = 0; cq < 4; ++cq) {
          const int c = coef_c(dig[k], cq);
          if (c != 0) {
            q2[c2] = q[e] * 4 + cq;
            s2[c2] = s[e] * c;
            ++c2;
          }
        }
      cnt = c2;
      std::memcpy(q, q2, sizeof(int) * (size_t)c2);
      std::memcpy(s, s2, sizeof(int) * (size_t)c2);
    }
    count[l] = cnt;
    for (int t = 0; t < cnt; ++t) {
      int64_t r = 0, c = 0;
      quadrant_offsets(depth, npad, q[t], &r, &c);
      tab[l * maxT + t] = CTarget{(int32_t)r, (int32_t)c, (int32_t)s[t], 0};
    }
  }
}

}  // namespace
}  // namespace stark

using namespace stark;

extern "C" stark_status stark_mul_noalloc(int64_t n, int depth, const void* A, const void* B, void* C,
                                          void* stream) {
  if (n < 0 || depth < 0 || depth > kNoallocMaxDepth || n > (int64_t)1 << 20) return STARK_EINVAL;
  if (n == 0) return STARK_OK;
  if (!A || !B || !C) return STARK_EINVAL;
  if (!device_is_sm100_family()) return STARK_EUNSUPPORTED;
  const stark_dtype dt = STARK_F32_SPLIT_BF16;

  // scratch layout: X planes | Y planes | C-target table | counts | error word
  const int64_t ws = operand_bytes(n, depth, dt);
  const int64_t P = pow7i(depth);
  const int maxT = 1 << depth;
  const size_t off_tab = align_up((size_t)ws, 256);
  const size_t off_cnt = align_up(off_tab + (size_t)(P * maxT) * sizeof(CTarget), 256);
  const size_t off_err = align_up(off_cnt + (size_t)P * sizeof(int32_t), 256);
  if (off_err + 256 > kNoallocScratch) return STARK_ENOMEM;  // over the fixed scratch size

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return STARK_ECUDA;
  void* base = nullptr;
  if (scratch_address(dev, &base) != cudaSuccess) {
    cudaGetLastError();
    return STARK_ECUDA;
  }
  unsigned char* sb = static_cast<unsigned char*>(base);
  cudaStream_t s = (cudaStream_t)stream;

  // a plan object on the stack pointing into the scratch array
  stark_plan_s p;
  p.n = n;
  p.depth = depth;
  p.dt = dt;
  p.is_tc = true;
  p.esz = element_size(dt);
  p.npad = padded_side(n, depth, dt);
  p.L = p.npad >> depth;
  p.P = P;
  p.P_ws = P;
  p.bn = (p.L % 256 == 0) ? 256 : 128;
  p.device = dev;
  p.num_sms = device_sm_count();
  p.X = sb;
  p.Y = sb + ws / 2;
  p.ws_bytes = 0;
  p.d_ctab = reinterpret_cast<CTarget*>(sb + off_tab);
  p.d_ccount = reinterpret_cast<int32_t*>(sb + off_cnt);
  p.d_err = reinterpret_cast<int*>(sb + off_err);
  p.maxT = maxT;

  // the table of this (n_pad, depth), and a cleared error word
  CTarget tab[343 * 8];
  int32_t cnt[343];
  c_targets(depth, p.npad, tab, cnt);
  if (cudaMemcpyAsync(p.d_ctab, tab, (size_t)(P * maxT) * sizeof(CTarget), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(p.d_ccount, cnt, (size_t)P * sizeof(int32_t), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(p.d_err, 0, sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    return STARK_ECUDA;
  }
  if (!make_tmap_planes(&p.tmA, p.X, false, p.L, 2 * p.P, 128) ||
      !make_tmap_planes(&p.tmB, p.Y, false, p.L, 2 * p.P, 64))
    return STARK_EUNSUPPORTED;
  return plan_run(&p, A, B, C, 0, p.P, s);
}
