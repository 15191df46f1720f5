// noalloc.cu -- stark_mul_noalloc: the 3xBF16 product without any device
// allocation, for callers that cannot call cudaMalloc (for example code that
// runs where a memory allocator must not be entered, or a host that hands
// this library a fixed device-memory budget it may not grow).
//
// The workspace (error word, C-target table, leaf operand planes) lives in
// one file-scope __device__ array of fixed size, kNoallocScratch bytes.
// Every device that loads this file's module holds that array until the
// process exits (with CUDA's lazy module loading the module, and so the
// array, is loaded by the first call of this entry point on the device).
//
// In host code `g_scratch` names a host-side stand-in, not device memory: a
// kernel given that name would fault or, where the GPU can reach host memory,
// silently use the wrong memory.  So the first call on each device (with
// that device current) asks the runtime for the array's device address with
// cudaGetSymbolAddress, checks the result and caches it per device; every
// kernel receives that address.  Do that first call before any stream
// capture.  Each call rebuilds the C-target table in the array with a small
// kernel on the caller's stream (no host-to-device copy), so nothing a call
// enqueues refers to host memory.  All calls share the one array and it
// keeps the contents of the last call; calls that overlap on the GPU
// (different streams, or different host threads) race on the array, so
// callers must order them.  The error word at the start of the array keeps a
// device-side timeout until stark_noalloc_check reads and clears it.
#include <cuda_runtime.h>

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

// Offsets of the quadrant path q (base 4, top level most significant) in a
// padded side npad: each level halves the block (device form of the plan's
// quadrant_offsets).
__device__ void quadrant_offset(int depth, int64_t npad, int q, int64_t* row, int64_t* col) {
  int64_t r = 0, c = 0;
  for (int k = 1; k <= depth; ++k) {
    const int digit = (q >> (2 * (depth - k))) & 3;
    r += (int64_t)(digit >> 1) * (npad >> k);
    c += (int64_t)(digit & 1) * (npad >> k);
  }
  *row = r;
  *col = c;
}

// C targets of every leaf (Alg. 5 with the C22 = M1 - M2 + M3 + M6 sign):
// one thread per leaf l (base-7 M-index path, top level most significant)
// expands the product over levels of the C coefficients of its digits.
__global__ void noalloc_table_kernel(int depth, int64_t npad, CTarget* tab, int32_t* count) {
  int64_t P = 1;
  for (int k = 0; k < depth; ++k) P *= 7;
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= P) return;
  const int maxT = 1 << depth;
  int dig[kNoallocMaxDepth + 1] = {0};
  int64_t x = l;
  for (int k = depth - 1; k >= 0; --k) {
    dig[k] = (int)(x % 7);
    x /= 7;
  }
  int q[8] = {0}, sg[8] = {1};
  int cnt = 1;
  for (int k = 0; k < depth; ++k) {
    int q2[8], s2[8], c2 = 0;
    for (int e = 0; e < cnt; ++e)
      for (int cq = 0; cq < 4; ++cq) {
        const int c = coef_c(dig[k], cq);
        if (c != 0 && c2 < 8) {
          q2[c2] = q[e] * 4 + cq;
          s2[c2] = sg[e] * c;
          ++c2;
        }
      }
    cnt = c2;
    for (int e = 0; e < c2; ++e) {
      q[e] = q2[e];
      sg[e] = s2[e];
    }
  }
  count[l] = cnt;
  for (int t = 0; t < cnt; ++t) {
    int64_t r = 0, c = 0;
    quadrant_offset(depth, npad, q[t], &r, &c);
    tab[l * maxT + t] = CTarget{(int32_t)r, (int32_t)c, (int32_t)sg[t], 0};
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

  // scratch layout: error word | C-target table | counts | X planes | Y planes
  const int64_t ws = operand_bytes(n, depth, dt);
  const int64_t P = pow7i(depth);
  const int maxT = 1 << depth;
  const size_t off_tab = 256;
  const size_t off_cnt = align_up(off_tab + (size_t)(P * maxT) * sizeof(CTarget), 256);
  const size_t off_x = align_up(off_cnt + (size_t)P * sizeof(int32_t), 4096);
  if (off_x + (size_t)ws > kNoallocScratch) return STARK_ENOMEM;  // over the fixed scratch size

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
  p.X = sb + off_x;
  p.Y = sb + off_x + ws / 2;
  p.ws_bytes = 0;
  p.d_ctab = reinterpret_cast<CTarget*>(sb + off_tab);
  p.d_ccount = reinterpret_cast<int32_t*>(sb + off_cnt);
  p.d_err = reinterpret_cast<int*>(sb);
  p.maxT = maxT;

  // the C-target table of this (n_pad, depth), built on the device
  noalloc_table_kernel<<<(unsigned)((P + 127) / 128), 128, 0, s>>>(depth, p.npad, p.d_ctab, p.d_ccount);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return STARK_ECUDA;
  if (!make_tmap_planes(&p.tmA, p.X, false, p.L, 2 * p.P, 128) ||
      !make_tmap_planes(&p.tmB, p.Y, false, p.L, 2 * p.P, 64))
    return STARK_EUNSUPPORTED;
  return plan_run(&p, A, B, C, 0, p.P, s);
}

extern "C" stark_status stark_noalloc_check(void* stream) {
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return STARK_ECUDA;
  int e = 0;
  if (cudaMemcpyFromSymbol(&e, g_scratch, sizeof(int), 0, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return STARK_ECUDA;
  }
  if (e == 0) return STARK_OK;
  const int zero = 0;
  if (cudaMemcpyToSymbol(g_scratch, &zero, sizeof(int), 0, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return STARK_ECUDA;
  }
  return STARK_ETIMEOUT;
}
