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
// One generic sub-block product C (+)= A B with strides; a 256-thread block
// computes a TM x TN tile, each thread (TM/16) x (TN/16) elements (rows
// ty + 16 i, columns tx + 16 j), K in steps of 16 through shared memory.
// Tile shapes follow the edge: 64 x 64 in general, 256 x 16 for a thin
// right edge, 16 x 256 for a thin bottom edge, so an edge of a few columns
// does not pay for a 64-wide tile.
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

template <typename T, int TM, int TN>
__global__ void __launch_bounds__(256) border_kernel(BorderArgs a) {
  using Acc = typename BorderAcc<T>::Acc;
  constexpr int RM = TM / 16, RN = TN / 16;
  __shared__ Acc As[BKb][TM];
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

  for (int64_t k0 = 0; k0 < a.K; k0 += BKb) {
    // A tile TM x 16 (read along k), B tile 16 x TN (read along n); zeros
    // outside the sub-blocks
    for (int idx = threadIdx.x; idx < TM * BKb; idx += 256) {
      const int am = idx / BKb, ak = idx % BKb;
      const int64_t row = m0 + am, k = k0 + ak;
      As[ak][am] = (row < a.M && k < a.K) ? (Acc)A[row * a.lda + k] : Acc(0);
    }
    for (int idx = threadIdx.x; idx < TN * BKb; idx += 256) {
      const int bk = idx / TN, bn = idx % TN;
      const int64_t k = k0 + bk, col = n0 + bn;
      Bs[bk][bn] = (k < a.K && col < a.N) ? (Acc)B[k * a.ldb + col] : Acc(0);
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
      if (a.accumulate)
        *dst = (T)((Acc)*dst + acc[i][j]);
      else
        *dst = (T)acc[i][j];
    }
  }
}

template <typename T, int TM, int TN>
cudaError_t launch_tiles(const BorderArgs& a, cudaStream_t st) {
  const int64_t gx = (a.N + TN - 1) / TN, gy = (a.M + TM - 1) / TM;
  if (gx > 0x7FFFFFFF || gy > 65535) return cudaErrorInvalidValue;
  border_kernel<T, TM, TN><<<dim3((unsigned)gx, (unsigned)gy), 256, 0, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_typed(const BorderArgs& a, cudaStream_t st) {
  if (a.N <= 16 && a.M > 16) return launch_tiles<T, 256, 16>(a, st);  // thin right edge
  if (a.M <= 16 && a.N > 16) return launch_tiles<T, 16, 256>(a, st);  // thin bottom edge
  return launch_tiles<T, 64, 64>(a, st);
}

}  // namespace

cudaError_t launch_border(const BorderArgs& a, InType t, cudaStream_t st) {
  if (a.M < 0 || a.N < 0 || a.K < 0) return cudaErrorInvalidValue;
  if (a.M == 0 || a.N == 0) return cudaSuccess;
  if (a.lda < a.K || a.ldb < a.N || a.ldc < a.N) return cudaErrorInvalidValue;
  switch (t) {
    case kInF32: return launch_typed<float>(a, st);
    case kInF64: return launch_typed<double>(a, st);
    case kInI64: return launch_typed<int64_t>(a, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace stark
