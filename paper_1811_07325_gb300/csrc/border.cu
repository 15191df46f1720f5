// border.cu -- the peeled edges of a product whose side n = m + r is not a
// multiple of the Strassen tile granularity (peeling instead of padding):
// the recursion runs on the m x m core, and three thin classical products
// complete C = A B,
//   C[:m, :m] += A[:m, m:] B[m:, :m]     (rank-r update of the core)
//   C[:m, m:]  = A[:m, :]  B[:, m:]      (right edge)
//   C[m:, :]   = A[m:, :]  B             (bottom edge)
// on the CUDA cores: fp32 FMA with fp32 accumulation for the split-fp32
// dtypes (a K-term fp32 dot product, more accurate than the 3-term split
// leaves), fp64 for F64, wrapping 64-bit integer arithmetic for I64.
//
// Edges of at most 16 rows/columns (the case peeling is for) use three
// bandwidth-shaped kernels; wider ones a generic sub-block product C (+)= A B
// with strides: a 256-thread block computes a 64 x 64 tile, each thread 4 x 4
// elements (rows ty + 16 i, columns tx + 16 j), K in steps of 16 through
// shared memory.  A product that yields too few blocks to fill the GPU
// splits K across the grid (when the caller allows it: atomic adds make the
// fp32 rounding order vary), adding partial results with atomics into a C
// the caller has zeroed or that holds the core's result.
#include "stark_internal.h"

namespace stark {
namespace {

constexpr int BKb = 16;

template <typename T>
struct BorderAcc;
template <>
struct BorderAcc<float> {
  using Acc = float;
};
template <>
struct BorderAcc<double> {
  using Acc = double;
};
template <>
struct BorderAcc<int64_t> {
  using Acc = unsigned long long;  // wraps modulo 2^64 like the int64 path
};

__device__ __forceinline__ void atomic_add(float* p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add(double* p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add(int64_t* p, unsigned long long v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(p), v);
}

template <typename T, int TM, int TN>
__global__ void __launch_bounds__(256) border_kernel(BorderArgs a) {
  using Acc = typename BorderAcc<T>::Acc;
  constexpr int RM = TM / 16, RN = TN / 16;
  __shared__ Acc As[BKb][TM + 1];  // +1: the k-major stores below hit distinct banks
  __shared__ Acc Bs[BKb][TN];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t m0 = (int64_t)blockIdx.y * TM, n0 = (int64_t)blockIdx.x * TN;
  const T* __restrict__ A = static_cast<const T*>(a.A);
  const T* __restrict__ B = static_cast<const T*>(a.B);

  Acc acc[RM][RN];
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < RN; ++j) acc[i][j] = Acc(0);

  // this block's K range (grid z splits K in chunks of kc, a multiple of 16)
  const int64_t kbeg = (int64_t)blockIdx.z * a.kc;
  const int64_t kend = kbeg + a.kc < a.K ? kbeg + a.kc : a.K;
  for (int64_t k0 = kbeg; k0 < kend; k0 += BKb) {
    // A tile TM x 16 (read along k), B tile 16 x TN (read along n); zeros
    // outside the sub-blocks
    for (int idx = threadIdx.x; idx < TM * BKb; idx += 256) {
      const int am = idx / BKb, ak = idx % BKb;
      const int64_t row = m0 + am, k = k0 + ak;
      As[ak][am] = (row < a.M && k < kend) ? (Acc)A[row * a.lda + k] : Acc(0);
    }
    for (int idx = threadIdx.x; idx < TN * BKb; idx += 256) {
      const int bk = idx / TN, bn = idx % TN;
      const int64_t k = k0 + bk, col = n0 + bn;
      Bs[bk][bn] = (k < kend && col < a.N) ? (Acc)B[k * a.ldb + col] : Acc(0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BKb; ++k) {
      Acc av[RM], bv[RN];
#pragma unroll
      for (int i = 0; i < RM; ++i) av[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < RN; ++j) bv[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RN; ++j) acc[i][j] += av[i] * bv[j];
    }
    __syncthreads();
  }

  T* C = static_cast<T*>(a.C);
#pragma unroll
  for (int i = 0; i < RM; ++i) {
    const int64_t row = m0 + ty + 16 * i;
    if (row >= a.M) continue;
#pragma unroll
    for (int j = 0; j < RN; ++j) {
      const int64_t col = n0 + tx + 16 * j;
      if (col >= a.N) continue;
      T* dst = C + row * a.ldc + col;
      if (gridDim.z > 1)
        atomic_add(dst, acc[i][j]);
      else if (a.accumulate)
        *dst = (T)((Acc)*dst + acc[i][j]);
      else
        *dst = (T)acc[i][j];
    }
  }
}

template <typename T, int TM, int TN>
cudaError_t launch_tiles(BorderArgs a, int num_sms, cudaStream_t st) {
  const int64_t gx = (a.N + TN - 1) / TN, gy = (a.M + TM - 1) / TM;
  if (gx > 0x7FFFFFFF || gy > 65535) return cudaErrorInvalidValue;
  // split K (when accumulating and allowed) until there are about four
  // blocks per SM, keeping at least 256 K per block
  int64_t gz = 1;
  if (a.accumulate && a.split && a.K > 256) {
    const int64_t want = 4 * (int64_t)num_sms;
    if (gx * gy < want) gz = (want + gx * gy - 1) / (gx * gy);
    const int64_t most = (a.K + 255) / 256;
    if (gz > most) gz = most;
    if (gz > 65535) gz = 65535;
  }
  a.kc = a.K > 0 ? ((a.K + gz - 1) / gz + BKb - 1) / BKb * BKb : BKb;
  gz = a.K > 0 ? (a.K + a.kc - 1) / a.kc : 1;
  border_kernel<T, TM, TN><<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), 256, 0, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------- narrow edges
// For an edge of r <= kNarrow rows/columns the three products are
// bandwidth-shaped instead of tiled (a tile would compute mostly zeros).  R
// is r rounded up to a power of two (the extra terms are zeros); loops over
// rows and k are unrolled so each thread keeps many loads in flight.
constexpr int kNarrow = 16;

// Core update C[i, j] += sum_{k<r} A'[i, k] B'[k, j] (A' = A[:m, m:], B' =
// B[m:, :m]): a block covers 256 columns x 16 rows; each thread keeps its
// column's r values of B' in registers and updates 16 rows at once.
template <typename T, int R>
__global__ void __launch_bounds__(256) rank_update_kernel(BorderArgs a) {
  using Acc = typename BorderAcc<T>::Acc;
  constexpr int ROWS = 16;
  __shared__ Acc As[ROWS][R];
  const int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.y * ROWS;
  const int r = (int)a.K;
  const T* A = static_cast<const T*>(a.A);
  const T* B = static_cast<const T*>(a.B);
  for (int idx = threadIdx.x; idx < ROWS * R; idx += 256) {
    const int ii = idx / R, k = idx % R;
    As[ii][k] = (i0 + ii < a.M && k < r) ? (Acc)A[(i0 + ii) * a.lda + k] : Acc(0);
  }
  __syncthreads();
  if (j >= a.N) return;
  Acc b[R];
#pragma unroll
  for (int k = 0; k < R; ++k) b[k] = k < r ? (Acc)B[k * a.ldb + j] : Acc(0);
  T* C = static_cast<T*>(a.C);
  Acc c[ROWS];
#pragma unroll
  for (int ii = 0; ii < ROWS; ++ii) c[ii] = i0 + ii < a.M ? (Acc)C[(i0 + ii) * a.ldc + j] : Acc(0);
#pragma unroll
  for (int ii = 0; ii < ROWS; ++ii) {
#pragma unroll
    for (int k = 0; k < R; ++k) c[ii] += As[ii][k] * b[k];
  }
#pragma unroll
  for (int ii = 0; ii < ROWS; ++ii)
    if (i0 + ii < a.M) C[(i0 + ii) * a.ldc + j] = (T)c[ii];
}

// Right strip C[i, j] (+)= sum_k A[i, k] B[k, j], j < r: one warp per row i,
// lanes stride over k (coalesced A, eight loads in flight per lane), the
// strip of B staged in shared memory chunk by chunk, a warp reduction per
// column at the end (no atomics).
template <typename T, int R>
__global__ void __launch_bounds__(256) right_strip_kernel(BorderArgs a) {
  using Acc = typename BorderAcc<T>::Acc;
  constexpr int KCH = 256;
  __shared__ Acc Bs[KCH][R + 1];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t i = (int64_t)blockIdx.x * 8 + warp;
  const int r = (int)a.N;
  const T* A = static_cast<const T*>(a.A);
  const T* B = static_cast<const T*>(a.B);
  Acc acc[R];
#pragma unroll
  for (int j = 0; j < R; ++j) acc[j] = Acc(0);
  for (int64_t k0 = 0; k0 < a.K; k0 += KCH) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < KCH * R; idx += 256) {
      const int kk = idx / R, j = idx % R;
      const int64_t k = k0 + kk;
      Bs[kk][j] = (k < a.K && j < r) ? (Acc)B[k * a.ldb + j] : Acc(0);
    }
    __syncthreads();
    if (i < a.M) {
      Acc x[KCH / 32];
#pragma unroll
      for (int t = 0; t < KCH / 32; ++t) {
        const int64_t k = k0 + lane + 32 * t;
        x[t] = k < a.K ? (Acc)A[i * a.lda + k] : Acc(0);
      }
#pragma unroll
      for (int t = 0; t < KCH / 32; ++t)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[j] += x[t] * Bs[lane + 32 * t][j];
    }
  }
  if (i >= a.M) return;
#pragma unroll
  for (int j = 0; j < R; ++j) {
    Acc v = acc[j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    acc[j] = v;
  }
  if (lane == 0) {
    T* C = static_cast<T*>(a.C);
#pragma unroll
    for (int j = 0; j < R; ++j) {
      if (j >= r) break;
      T* dst = C + i * a.ldc + j;
      *dst = a.accumulate ? (T)((Acc)*dst + acc[j]) : (T)acc[j];
    }
  }
}

// Bottom strip C[i, j] (+)= sum_k A[i, k] B[k, j], i < r: one thread per
// column j (coalesced B, eight loads in flight), the r rows of A staged in
// shared memory chunk by chunk; grid y splits K (atomic adds) when the
// caller allows it.
template <typename T, int R>
__global__ void __launch_bounds__(256) bottom_strip_kernel(BorderArgs a) {
  using Acc = typename BorderAcc<T>::Acc;
  constexpr int KCH = 256, U = 8;
  __shared__ Acc As[KCH][R];
  const int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x;
  const int r = (int)a.M;
  const T* A = static_cast<const T*>(a.A);
  const T* B = static_cast<const T*>(a.B);
  const int64_t kbeg = (int64_t)blockIdx.y * a.kc;
  const int64_t kend = kbeg + a.kc < a.K ? kbeg + a.kc : a.K;
  Acc acc[R];
#pragma unroll
  for (int ii = 0; ii < R; ++ii) acc[ii] = Acc(0);
  for (int64_t k0 = kbeg; k0 < kend; k0 += KCH) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < KCH * R; idx += 256) {
      const int kk = idx / R, ii = idx % R;
      const int64_t k = k0 + kk;
      As[kk][ii] = (ii < r && k < kend) ? (Acc)A[ii * a.lda + k] : Acc(0);
    }
    __syncthreads();
    if (j < a.N) {
      for (int kb = 0; kb < KCH; kb += U) {
        if (k0 + kb >= kend) break;
        Acc b[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t k = k0 + kb + u;
          b[u] = k < kend ? (Acc)B[k * a.ldb + j] : Acc(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int ii = 0; ii < R; ++ii) acc[ii] += As[kb + u][ii] * b[u];
      }
    }
  }
  if (j >= a.N) return;
  T* C = static_cast<T*>(a.C);
#pragma unroll
  for (int ii = 0; ii < R; ++ii) {
    if (ii >= r) break;
    T* dst = C + ii * a.ldc + j;
    if (gridDim.y > 1)
      atomic_add(dst, acc[ii]);
    else
      *dst = a.accumulate ? (T)((Acc)*dst + acc[ii]) : (T)acc[ii];
  }
}

template <typename T, int R>
cudaError_t launch_narrow_r(BorderArgs a, int num_sms, cudaStream_t st) {
  if (a.K <= kNarrow && a.M > kNarrow && a.N > kNarrow) {  // core update, K = r
    const int64_t gx = (a.N + 255) / 256, gy = (a.M + 15) / 16;
    if (gy > 65535) return cudaErrorInvalidValue;
    rank_update_kernel<T, R><<<dim3((unsigned)gx, (unsigned)gy), 256, 0, st>>>(a);
  } else if (a.N <= kNarrow) {  // right strip
    const int64_t gx = (a.M + 7) / 8;
    right_strip_kernel<T, R><<<(unsigned)gx, 256, 0, st>>>(a);
  } else {  // bottom strip, M <= kNarrow
    const int64_t gx = (a.N + 255) / 256;
    int64_t gy = 1;
    if (a.accumulate && a.split && a.K > 256) {
      gy = (4 * (int64_t)num_sms + gx - 1) / gx;
      const int64_t most = (a.K + 255) / 256;
      if (gy > most) gy = most;
      if (gy > 65535) gy = 65535;
    }
    a.kc = (a.K + gy - 1) / gy;
    gy = (a.K + a.kc - 1) / a.kc;
    if (gy < 1) gy = 1;
    bottom_strip_kernel<T, R><<<dim3((unsigned)gx, (unsigned)gy), 256, 0, st>>>(a);
  }
  count_launch();
  return cudaGetLastError();
}

// r (the edge width: K of the core update, N of the right strip, M of the
// bottom strip) rounded up to a power of two
template <typename T>
cudaError_t launch_narrow(const BorderArgs& a, int num_sms, cudaStream_t st) {
  const int64_t r = (a.K <= kNarrow && a.M > kNarrow && a.N > kNarrow) ? a.K : a.N <= kNarrow ? a.N : a.M;
  if (r <= 1) return launch_narrow_r<T, 1>(a, num_sms, st);
  if (r <= 2) return launch_narrow_r<T, 2>(a, num_sms, st);
  if (r <= 4) return launch_narrow_r<T, 4>(a, num_sms, st);
  if (r <= 8) return launch_narrow_r<T, 8>(a, num_sms, st);
  return launch_narrow_r<T, 16>(a, num_sms, st);
}

template <typename T>
cudaError_t launch_typed(const BorderArgs& a, int num_sms, cudaStream_t st) {
  if (a.K > 0 && (a.K <= kNarrow || a.N <= kNarrow || a.M <= kNarrow)) return launch_narrow<T>(a, num_sms, st);
  return launch_tiles<T, 64, 64>(a, num_sms, st);
}

}  // namespace

cudaError_t launch_border(const BorderArgs& a, InType t, int num_sms, cudaStream_t st) {
  if (a.M < 0 || a.N < 0 || a.K < 0) return cudaErrorInvalidValue;
  if (a.M == 0 || a.N == 0) return cudaSuccess;
  if (a.lda < a.K || a.ldb < a.N || a.ldc < a.N) return cudaErrorInvalidValue;
  switch (t) {
    case kInF32: return launch_typed<float>(a, num_sms, st);
    case kInF64: return launch_typed<double>(a, num_sms, st);
    case kInI64: return launch_typed<int64_t>(a, num_sms, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace stark
