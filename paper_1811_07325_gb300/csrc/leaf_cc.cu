// leaf_cc.cu -- leaf products on the CUDA cores for the paths the tensor
// cores cannot serve exactly: fp64 (no tcgen05 fp64 kind) and int64 (exact
// modulo 2^64).  Same structure as the tensor-core path: one launch covers
// every leaf (grid z = leaf), and the epilogue adds the finished tile into
// every C target of the leaf with its sign (Alg. 4 + Alg. 5 fused).
//
// Tiling: 64 x 64 output tile per 256-thread block, K step 16, each thread a
// 4 x 4 register tile (rows ty + 16 i, cols tx + 16 j), operands staged in
// shared memory (A transposed to [k][m] so both reads broadcast).
#include "stark_internal.h"

namespace stark {
namespace {

constexpr int BT = 64;
constexpr int BKc = 16;

template <typename T>
struct CcTraits;
template <>
struct CcTraits<double> {
  using Acc = double;
  __device__ static void add(double* dst, double v, int sign) { atomicAdd(dst, sign > 0 ? v : -v); }
};
template <>
struct CcTraits<int64_t> {
  using Acc = unsigned long long;
  __device__ static void add(int64_t* dst, unsigned long long v, int sign) {
    atomicAdd(reinterpret_cast<unsigned long long*>(dst), sign > 0 ? v : 0ull - v);
  }
};

template <typename T>
__global__ void __launch_bounds__(256) leaf_cc_kernel(LeafCcArgs p) {
  using Acc = typename CcTraits<T>::Acc;
  __shared__ Acc As[2][BKc][BT];
  __shared__ Acc Bs[2][BKc][BT];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int leaf = p.leaf_begin + blockIdx.z;
  const int64_t L = p.L;
  const int64_t m0 = (int64_t)blockIdx.y * BT, n0 = (int64_t)blockIdx.x * BT;
  const int plane = leaf - p.plane_base;  // workspace plane of this leaf
  const Acc* __restrict__ X = static_cast<const Acc*>(p.X) + (int64_t)plane * L * L;
  const Acc* __restrict__ Y = static_cast<const Acc*>(p.Y) + (int64_t)plane * L * L;

  Acc acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = Acc(0);

  // loader mapping: 1024 elements of each tile, 4 per thread
  auto load = [&](int buf, int64_t k0) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = threadIdx.x + 256 * e;
      // A tile: 64 rows x 16 k, read along k
      const int am = idx / BKc, ak = idx % BKc;
      As[buf][ak][am] = X[(m0 + am) * L + k0 + ak];
      // B tile: 16 k x 64 cols, read along n
      const int bk = idx / BT, bn = idx % BT;
      Bs[buf][bk][bn] = Y[(k0 + bk) * L + n0 + bn];
    }
  };

  const int kt = (int)(L / BKc);
  load(0, 0);
  __syncthreads();
  for (int t = 0; t < kt; ++t) {
    const int cur = t & 1;
    if (t + 1 < kt) load(cur ^ 1, (int64_t)(t + 1) * BKc);
#pragma unroll
    for (int k = 0; k < BKc; ++k) {
      Acc a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[cur][k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[cur][k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }

  const int nt = p.ccount[leaf];
  const CTarget* tg = p.ctab + (int64_t)leaf * p.maxT;
  T* C = static_cast<T*>(p.C);
  for (int t = 0; t < nt; ++t) {
    const CTarget c = tg[t];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t row = c.row_off + m0 + ty + 16 * i;
      if (row >= p.n) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t col = c.col_off + n0 + tx + 16 * j;
        if (col < p.n) CcTraits<T>::add(C + row * p.ldc + col, acc[i][j], c.sign);
      }
    }
  }
}

template <typename T>
cudaError_t launch(const LeafCcArgs& a, cudaStream_t st) {
  if (a.L % BT != 0) return cudaErrorInvalidValue;
  const int leaves = a.leaf_end - a.leaf_begin;
  if (leaves <= 0) return cudaSuccess;
  if (leaves > 65535 || a.L / BT > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)(a.L / BT), (unsigned)(a.L / BT), (unsigned)leaves);
  leaf_cc_kernel<T><<<grid, 256, 0, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_leaf_f64(const LeafCcArgs& a, cudaStream_t st) { return launch<double>(a, st); }
cudaError_t launch_leaf_i64(const LeafCcArgs& a, cudaStream_t st) { return launch<int64_t>(a, st); }

}  // namespace stark
