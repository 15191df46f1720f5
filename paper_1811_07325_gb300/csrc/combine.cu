// combine.cu -- the combine of Alg. 5 as a separate, deterministic pass.
//
// With the fused epilogue every leaf tile is added into C by L2 reductions
// whose order depends on scheduling, so float results can differ in the
// last bits from run to run.  In the deterministic mode the leaf kernel
// stores each product M_l, and this kernel writes every C element once as
// the signed sum of its contributions in ascending leaf order:
//   C at quadrant path q, position (r, c) = sum_l W_d[q, l] * M_l[r][c],
// W_d the d-fold Kronecker power of the 2x2 combine table (C11 = M1+M4-M5+M7,
// C12 = M3+M5, C21 = M2+M4, C22 = M1-M2+M3+M6).  A thread owns VEC columns
// of one (r, c) position for all 4^d quadrants: it reads each M_l vector
// once and adds it into its targets' registers.
#include "stark_internal.h"

namespace stark {
namespace {

__host__ __device__ constexpr int pow4i(int k) { return k <= 0 ? 1 : 4 * pow4i(k - 1); }
__host__ __device__ constexpr int pow7i_(int k) { return k <= 0 ? 1 : 7 * pow7i_(k - 1); }

template <int D, int VEC>
__global__ void __launch_bounds__(256) combine_kernel(const float* __restrict__ M, int64_t L, int64_t npad, int64_t n,
                                                      float* __restrict__ C, int64_t ldc) {
  constexpr int Q = pow4i(D);
  constexpr int P = pow7i_(D);
  const int64_t per_row = L / VEC;
  const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= L * per_row) return;
  const int64_t r = pos / per_row, c = (pos % per_row) * VEC;
  float out[Q][VEC];
#pragma unroll
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int e = 0; e < VEC; ++e) out[q][e] = 0.f;

#pragma unroll
  for (int l = 0; l < P; ++l) {
    float v[VEC];
    const float* src = M + (int64_t)l * L * L + r * L + c;
    if constexpr (VEC == 4) {
      const float4 x = __ldcs(reinterpret_cast<const float4*>(src));
      v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else {
#pragma unroll
      for (int e = 0; e < VEC; ++e) v[e] = __ldcs(src + e);
    }
    // targets of leaf l: per level, product m feeds one or two C quadrants
    int dig[D > 0 ? D : 1];
    {
      int x = l;
#pragma unroll
      for (int k = D - 1; k >= 0; --k) {
        dig[k] = x % 7;
        x /= 7;
      }
    }
#pragma unroll
    for (int t = 0; t < (1 << D); ++t) {
      int q = 0, sign = 1;
      bool valid = true;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const int pick = (t >> (D - 1 - k)) & 1;  // first or second target at level k
        int found = -1, count = 0;
#pragma unroll
        for (int cq = 0; cq < 4; ++cq)
          if (coef_c(dig[k], cq) != 0) {
            if (count == pick) found = cq;
            ++count;
          }
        if (found < 0) {
          valid = false;
        } else {
          q = q * 4 + found;
          sign *= coef_c(dig[k], found);
        }
      }
      if (valid) {
#pragma unroll
        for (int e = 0; e < VEC; ++e) out[q][e] = sign > 0 ? out[q][e] + v[e] : out[q][e] - v[e];
      }
    }
  }

#pragma unroll
  for (int q = 0; q < Q; ++q) {
    int64_t ro = 0, co = 0;
#pragma unroll
    for (int k = 1; k <= D; ++k) {
      const int digit = (q >> (2 * (D - k))) & 3;
      ro += (int64_t)(digit >> 1) * (npad >> k);
      co += (int64_t)(digit & 1) * (npad >> k);
    }
    const int64_t row = ro + r;
    if (row >= n) continue;
#pragma unroll
    for (int e = 0; e < VEC; ++e)
      if (co + c + e < n) C[row * ldc + co + c + e] = out[q][e];
  }
}

template <int D, int VEC>
cudaError_t launch_d(const float* M, int64_t L, int64_t npad, int64_t n, float* C, int64_t ldc, cudaStream_t s) {
  if (L % VEC != 0) return cudaErrorInvalidValue;
  const int64_t threads = L * (L / VEC);
  const int64_t blocks = (threads + 255) / 256;
  combine_kernel<D, VEC><<<(unsigned)blocks, 256, 0, s>>>(M, L, npad, n, C, ldc);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_combine(const float* M, int depth, int64_t L, int64_t npad, int64_t n, float* C, int64_t ldc,
                           cudaStream_t s) {
  switch (depth) {
    case 0: return launch_d<0, 4>(M, L, npad, n, C, ldc, s);
    case 1: return launch_d<1, 4>(M, L, npad, n, C, ldc, s);
    case 2: return launch_d<2, 4>(M, L, npad, n, C, ldc, s);
    case 3: return launch_d<3, 1>(M, L, npad, n, C, ldc, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace stark
