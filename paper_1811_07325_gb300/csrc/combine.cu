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

// Targets of product M_m (m = 0..6 for M1..M7) at one level: the C
// quadrants (0 = C11, 1 = C12, 2 = C21, 3 = C22) it is added to, with signs
// (Alg. 1 with C22 = M1 - M2 + M3 + M6).  Constant folding of these, with
// the loops below fully unrolled, fixes every accumulator index at compile
// time, so the 4^d partial sums stay in registers.
__host__ __device__ constexpr int tgt_n(int m) { return m >= 5 ? 1 : 2; }
__host__ __device__ constexpr int tgt_q(int m, int a) {
  // M1: 11 22, M2: 21 22, M3: 12 22, M4: 11 21, M5: 11 12, M6: 22, M7: 11
  return m == 0 ? (a ? 3 : 0) : m == 1 ? (a ? 3 : 2) : m == 2 ? (a ? 3 : 1) : m == 3 ? (a ? 2 : 0)
       : m == 4 ? (a ? 1 : 0) : m == 5 ? 3 : 0;
}
__host__ __device__ constexpr int tgt_s(int m, int a) { return (m == 1 && a == 1) || (m == 4 && a == 0) ? -1 : 1; }

template <int D, int VEC>
__global__ void __launch_bounds__(256) combine_kernel(const float* __restrict__ M, int64_t L, int64_t npad, int64_t n,
                                                      float* __restrict__ C, int64_t ldc) {
  static_assert(D <= 3, "depth");
  constexpr int Q = pow4i(D);
  constexpr int N1 = D >= 1 ? 7 : 1, N2 = D >= 2 ? 7 : 1, N3 = D >= 3 ? 7 : 1;
  const int64_t per_row = L / VEC;
  const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= L * per_row) return;
  const int64_t r = pos / per_row, c = (pos % per_row) * VEC;
  float out[Q][VEC];
#pragma unroll
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int e = 0; e < VEC; ++e) out[q][e] = 0.f;

  // leaves in ascending order: digits i1 (top level) .. i3, l = i1 i2 i3 in base 7
#pragma unroll
  for (int i1 = 0; i1 < N1; ++i1)
#pragma unroll
    for (int i2 = 0; i2 < N2; ++i2)
#pragma unroll
      for (int i3 = 0; i3 < N3; ++i3) {
        const int l = (i1 * N2 + i2) * N3 + i3;
        float v[VEC];
        const float* src = M + (int64_t)l * L * L + r * L + c;
        if constexpr (VEC == 4) {
          const float4 x = __ldcs(reinterpret_cast<const float4*>(src));
          v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
        } else if constexpr (VEC == 2) {
          const float2 x = __ldcs(reinterpret_cast<const float2*>(src));
          v[0] = x.x; v[1] = x.y;
        } else {
#pragma unroll
          for (int e = 0; e < VEC; ++e) v[e] = __ldcs(src + e);
        }
        // every combination of one target per level: quadrant path and sign
#pragma unroll
        for (int a1 = 0; a1 < 2; ++a1)
#pragma unroll
          for (int a2 = 0; a2 < 2; ++a2)
#pragma unroll
            for (int a3 = 0; a3 < 2; ++a3) {
              if (D < 1 && a1) continue;
              if (D < 2 && a2) continue;
              if (D < 3 && a3) continue;
              if (D >= 1 && a1 >= tgt_n(i1)) continue;
              if (D >= 2 && a2 >= tgt_n(i2)) continue;
              if (D >= 3 && a3 >= tgt_n(i3)) continue;
              int q = 0, sign = 1;
              if (D >= 1) {
                q = tgt_q(i1, a1);
                sign = tgt_s(i1, a1);
              }
              if (D >= 2) {
                q = q * 4 + tgt_q(i2, a2);
                sign *= tgt_s(i2, a2);
              }
              if (D >= 3) {
                q = q * 4 + tgt_q(i3, a3);
                sign *= tgt_s(i3, a3);
              }
#pragma unroll
              for (int e = 0; e < VEC; ++e) out[q][e] = sign > 0 ? out[q][e] + v[e] : out[q][e] - v[e];
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

// Depth 3 with the planes streamed through shared memory.  At depth 3 a
// thread holds 64 partial sums, which leaves too few registers for enough
// plane loads in flight to stream at HBM bandwidth; here a block of 128
// threads owns 128 consecutive positions of one row and cp.async copies
// the planes' row segments into a ring of kRing stages, one sibling group
// (the 7 leaves below one depth-2 product, 3.5 KB) per stage, kRing - 1
// groups in flight.  Each thread adds its position's values in ascending
// leaf order, exactly as combine_kernel<3, 1> does.
constexpr int kRing = 12;
constexpr int kTW3 = 128;

__device__ __forceinline__ void cp_async_16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__global__ void __launch_bounds__(kTW3, 4) combine3_staged_kernel(const float* __restrict__ M, int64_t L, int64_t npad,
                                                                int64_t n, float* __restrict__ C, int64_t ldc) {
  __shared__ __align__(16) float ring[kRing][7][kTW3];
  const int64_t tiles = L / kTW3;
  const int64_t r = (int64_t)blockIdx.x / tiles;
  const int64_t j0 = ((int64_t)blockIdx.x % tiles) * kTW3;
  const int t = threadIdx.x;
  const int64_t plane = L * L;
  // group g (leaves 7g .. 7g + 6) into stage g % kRing: 7 x 32 copies of 16 bytes
  auto issue = [&](int g) {
    float* st = &ring[g % kRing][0][0];
    for (int k = t; k < 7 * (kTW3 / 4); k += kTW3) {
      const int leaf = k / (kTW3 / 4), c4 = (k % (kTW3 / 4)) * 4;
      cp_async_16(static_cast<uint32_t>(__cvta_generic_to_shared(st + leaf * kTW3 + c4)),
                  M + (int64_t)(7 * g + leaf) * plane + r * L + j0 + c4);
    }
  };
#pragma unroll 1
  for (int g = 0; g < kRing - 1; ++g) {
    issue(g);
    cp_async_commit();
  }
  float out[64];
#pragma unroll
  for (int q = 0; q < 64; ++q) out[q] = 0.f;
#pragma unroll
  for (int g = 0; g < 49; ++g) {
    cp_async_wait<kRing - 2>();  // group g has landed (this thread's copies)
    __syncthreads();             // ... and every thread's
    const int i1 = g / 7, i2 = g % 7;
#pragma unroll
    for (int i3 = 0; i3 < 7; ++i3) {
      const float v = ring[g % kRing][i3][t];
#pragma unroll
      for (int a1 = 0; a1 < 2; ++a1)
#pragma unroll
        for (int a2 = 0; a2 < 2; ++a2)
#pragma unroll
          for (int a3 = 0; a3 < 2; ++a3) {
            if (a1 >= tgt_n(i1) || a2 >= tgt_n(i2) || a3 >= tgt_n(i3)) continue;
            const int q = (tgt_q(i1, a1) * 4 + tgt_q(i2, a2)) * 4 + tgt_q(i3, a3);
            const int sign = tgt_s(i1, a1) * tgt_s(i2, a2) * tgt_s(i3, a3);
            out[q] = sign > 0 ? out[q] + v : out[q] - v;
          }
    }
    __syncthreads();  // stage g % kRing is free again
    if (g + kRing - 1 < 49) issue(g + kRing - 1);
    cp_async_commit();  // (an empty group past the end keeps the count uniform)
  }
  cp_async_wait<0>();
#pragma unroll
  for (int q = 0; q < 64; ++q) {
    int64_t ro = 0, co = 0;
#pragma unroll
    for (int k = 1; k <= 3; ++k) {
      const int digit = (q >> (2 * (3 - k))) & 3;
      ro += (int64_t)(digit >> 1) * (npad >> k);
      co += (int64_t)(digit & 1) * (npad >> k);
    }
    const int64_t row = ro + r, col = co + j0 + t;
    if (row < n && col < n) C[row * ldc + col] = out[q];
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
    case 2: return launch_d<2, 2>(M, L, npad, n, C, ldc, s);  // 16 partial sums of 2: 64 registers, 4 blocks per SM
    case 3:
      if (L % kTW3 == 0) {
        const int64_t blocks = L * (L / kTW3);
        combine3_staged_kernel<<<(unsigned)blocks, kTW3, 0, s>>>(M, L, npad, n, C, ldc);
        count_launch();
        return cudaGetLastError();
      }
      return launch_d<3, 1>(M, L, npad, n, C, ldc, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace stark
