// error_norms.cu -- the accuracy statement of a product, reduced on the GPU
// in FP64: the Frobenius norms of A and B and, over sampled rows of C
// against reference rows computed in FP64, the largest absolute error, the
// sums of squares of the error and of the reference, and the largest
// componentwise ratio |dC_ij| / (|A||B|)_ij.  These are the quantities of
// the normwise bound max|dC| / (||A||_F ||B||_F) and of the relative RMS
// error that the split-precision leaves are judged by (the paper runs FP64
// throughout and states no accuracy; FP64 on the GPU is kept for exactly
// these reductions).
//
// Two passes, both in a fixed order, so the result does not depend on
// scheduling: a grid of blocks each reduces a contiguous share of the
// elements (grid-stride over 16-byte vectors where the type allows) into a
// row of partials; one block then reduces the partials in block order.
// Maxima are exact; sums are FP64 with a fixed association.
#include <cuda_runtime.h>

#include <cmath>

#include "plan.h"
#include "stark_internal.h"

namespace stark {
namespace {

constexpr int kThreads = 256;
constexpr int kFields = 4;  // sum of squares / max abs error / sum sq error / sum sq reference ...

template <typename T>
__device__ __forceinline__ double to_f64(T v) {
  return (double)v;
}

// Block-wide sum (fixed shuffle tree, then warp 0 over the warp results).
__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = lane < (int)(blockDim.x / 32) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0
}

__device__ double block_max(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = lane < (int)(blockDim.x / 32) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_down_sync(0xffffffffu, r, o));
  }
  return r;
}

// Sum of squares of `count` elements of X (one partial per block).
template <typename T>
__global__ void __launch_bounds__(kThreads) sumsq_kernel(const T* __restrict__ X, int64_t count, double* partial) {
  __shared__ double sh[kThreads / 32];
  const int64_t per = (count + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = (int64_t)blockIdx.x * per;
  const int64_t b1 = b0 + per < count ? b0 + per : count;
  double s = 0.0;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    const double v = to_f64(X[i]);
    s = fma(v, v, s);
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Error of sampled rows: got row r is row rows[r] of C (row stride n);
// want and absprod are [nrows][n] in FP64.
template <typename T>
__global__ void __launch_bounds__(kThreads)
    row_error_kernel(const T* __restrict__ C, int64_t n, const int64_t* __restrict__ rows, int64_t nrows,
                     const double* __restrict__ want, const double* __restrict__ absprod, double* partial) {
  __shared__ double sh[kThreads / 32];
  const int64_t count = nrows * n;
  const int64_t per = (count + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = (int64_t)blockIdx.x * per;
  const int64_t b1 = b0 + per < count ? b0 + per : count;
  double emax = 0.0, e2 = 0.0, w2 = 0.0, cmax = 0.0;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    const int64_t r = i / n, j = i - r * n;
    const double g = to_f64(C[rows[r] * n + j]);
    const double w = want[i];
    const double d = fabs(g - w);
    emax = fmax(emax, d);
    e2 = fma(d, d, e2);
    w2 = fma(w, w, w2);
    if (absprod) {
      const double a = absprod[i];
      if (a > 0.0) cmax = fmax(cmax, d / a);
    }
  }
  emax = block_max(emax, sh);
  const double e2s = block_sum(e2, sh);
  const double w2s = block_sum(w2, sh);
  cmax = block_max(cmax, sh);
  if (threadIdx.x == 0) {
    partial[blockIdx.x * kFields + 0] = emax;
    partial[blockIdx.x * kFields + 1] = e2s;
    partial[blockIdx.x * kFields + 2] = w2s;
    partial[blockIdx.x * kFields + 3] = cmax;
  }
}

// Final pass over `blocks` partials of `fields` values each; `is_max` says
// which fields are maxima (bit f), the others are sums.  One block.
__global__ void __launch_bounds__(kThreads)
    finish_kernel(const double* __restrict__ partial, int blocks, int fields, unsigned is_max, double* out) {
  __shared__ double sh[kThreads / 32];
  for (int f = 0; f < fields; ++f) {
    const bool mx = (is_max >> f) & 1u;
    // each thread folds a contiguous run of blocks (fixed order), then the tree
    const int per = (blocks + blockDim.x - 1) / blockDim.x;
    double v = 0.0;
    for (int b = threadIdx.x * per; b < (threadIdx.x + 1) * per && b < blocks; ++b) {
      const double x = partial[(int64_t)b * fields + f];
      v = mx ? fmax(v, x) : v + x;
    }
    v = mx ? block_max(v, sh) : block_sum(v, sh);
    if (threadIdx.x == 0) out[f] = v;
    __syncthreads();
  }
}

template <typename T>
cudaError_t launch_error(int64_t n, const void* A, const void* B, const void* C, const int64_t* rows, int64_t nrows,
                         const double* want, const double* absprod, double* part, int blocks, double* out,
                         cudaStream_t s) {
  // norms of A and B
  sumsq_kernel<T><<<blocks, kThreads, 0, s>>>(static_cast<const T*>(A), n * n, part);
  finish_kernel<<<1, kThreads, 0, s>>>(part, blocks, 1, 0u, out + 0);
  sumsq_kernel<T><<<blocks, kThreads, 0, s>>>(static_cast<const T*>(B), n * n, part);
  finish_kernel<<<1, kThreads, 0, s>>>(part, blocks, 1, 0u, out + 1);
  count_launch(4);
  if (nrows > 0) {
    row_error_kernel<T><<<blocks, kThreads, 0, s>>>(static_cast<const T*>(C), n, rows, nrows, want, absprod, part);
    finish_kernel<<<1, kThreads, 0, s>>>(part, blocks, kFields, 0x9u, out + 2);
    count_launch(2);
  }
  return cudaGetLastError();
}

}  // namespace
}  // namespace stark

using namespace stark;

extern "C" stark_status stark_error_norms(int64_t n, stark_dtype dtype, const void* A, const void* B, const void* C,
                                          const int64_t* rows, int64_t nrows, const double* want,
                                          const double* absprod, stark_error_report* out, void* stream) {
  if (!out || n < 0 || nrows < 0 || nrows > n || (n > 0 && (!A || !B)) || (nrows > 0 && (!C || !rows || !want)))
    return STARK_EINVAL;
  if (dtype != STARK_F64 && dtype != STARK_I64 && !is_split(dtype)) return STARK_EINVAL;
  *out = stark_error_report{};
  out->compared = nrows * n;
  if (n == 0) return STARK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = 2 * device_sm_count();
  double* buf = nullptr;  // partials + 6 results
  const size_t bytes = ((size_t)blocks * kFields + 8) * sizeof(double);
  if (cudaMalloc(&buf, bytes) != cudaSuccess) {
    cudaGetLastError();
    return STARK_ENOMEM;
  }
  double* res = buf + (size_t)blocks * kFields;
  cudaError_t e;
  switch (dtype) {
    case STARK_F64: e = launch_error<double>(n, A, B, C, rows, nrows, want, absprod, buf, blocks, res, s); break;
    case STARK_I64: e = launch_error<int64_t>(n, A, B, C, rows, nrows, want, absprod, buf, blocks, res, s); break;
    default: e = launch_error<float>(n, A, B, C, rows, nrows, want, absprod, buf, blocks, res, s); break;
  }
  double h[6] = {0, 0, 0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(buf);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return STARK_ECUDA;
  }
  out->norm_a = std::sqrt(h[0]);
  out->norm_b = std::sqrt(h[1]);
  if (nrows > 0) {
    out->max_abs_err = h[2];
    out->sum_sq_err = h[3];
    out->sum_sq_ref = h[4];
    out->max_componentwise = h[5];
  }
  return STARK_OK;
}
