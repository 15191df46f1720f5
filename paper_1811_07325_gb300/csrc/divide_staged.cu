// divide_staged.cu -- the depth-3 divide of the split-fp32 operands (Alg. 1 /
// Alg. 3 over three levels) in one pass per operand, the input tile staged
// in shared memory.
//
// A block owns TW consecutive positions (i, j0 .. j0+TW-1) of the L x L leaf
// grid.  The 64 input row segments it needs (one per quadrant path of the
// three levels) are copied to shared memory with cp.async, 16 bytes per
// copy and all in flight at once; copies that fall in the virtual padding
// beyond n are zero-filled by the copy itself.  Each thread then takes two
// adjacent positions: per top-level product M_m it forms the level-1 sums of
// its 16 sub-quadrant vectors from shared memory and runs the last two
// levels in registers (divide_impl.cuh's Tree), storing the hi/lo split of
// the 49 leaf operands below M_m.  Every input element is read from HBM
// once; every sum is the two-term addition of Alg. 1 in level order, so the
// planes are bit-identical to the per-top-product form.
#include "divide_impl.cuh"

namespace stark {
namespace {

constexpr int kStagedVec = 2;

__device__ __forceinline__ void cp_async_16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_4(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int OUT, int SIDE, int TW>
__global__ void __launch_bounds__(TW / kStagedVec) divide_staged_kernel(DivideArgs a, int vec_ok) {
  constexpr int T = TW / kStagedVec;  // threads
  extern __shared__ __align__(16) float tile[];  // [64][TW]: quadrant path (q1 q2 q3, top first), column
  const int64_t L = a.L, npad = a.npad;
  const int64_t tiles_per_row = L / TW;
  const int64_t i = (int64_t)blockIdx.x / tiles_per_row;
  const int64_t j0 = ((int64_t)blockIdx.x % tiles_per_row) * TW;
  const float* X = static_cast<const float*>(a.X);
  const uint32_t sbase = smem_u32(tile);

  // ---- stage the 64 segments (row, col0 .. col0 + TW - 1) of the input
  auto seg_origin = [&](int g, int64_t* row, int64_t* col) {
    int64_t r = i, c = j0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int digit = (g >> (2 * (2 - k))) & 3;
      r += (int64_t)(digit >> 1) * (npad >> (k + 1));
      c += (int64_t)(digit & 1) * (npad >> (k + 1));
    }
    *row = r;
    *col = c;
  };
  if (vec_ok) {
    constexpr int CH = TW / 4;  // 16-byte copies per segment
    for (int k = threadIdx.x; k < 64 * CH; k += T) {
      const int g = k / CH, c4 = (k % CH) * 4;
      int64_t row, col;
      seg_origin(g, &row, &col);
      col += c4;
      const int64_t left = a.n - col;  // elements of this row still inside the input
      const uint32_t bytes = row < a.n && left > 0 ? (uint32_t)(left >= 4 ? 16 : 4 * left) : 0u;
      const float* src = bytes ? X + row * a.ld + col : X;
      cp_async_16(sbase + (uint32_t)((g * TW + c4) * 4), src, bytes);
    }
  } else {
    for (int k = threadIdx.x; k < 64 * TW; k += T) {
      const int g = k / TW, c = k % TW;
      int64_t row, col;
      seg_origin(g, &row, &col);
      col += c;
      const bool in = row < a.n && col < a.n;
      cp_async_4(sbase + (uint32_t)((g * TW + c) * 4), in ? X + row * a.ld + col : X, in ? 4u : 0u);
    }
  }
  cp_async_wait_all();
  __syncthreads();

  // ---- the three levels: level 1 from shared memory, levels 2 and 3 in registers
  using V = Vec<float, kStagedVec>;
  const int p = threadIdx.x * kStagedVec;
  const Emitter<OUT, float, kStagedVec> emit{a.out_hi, a.out_lo, L * L, i * L + j0 + p, a.range_flag};
  auto in = [&](int g) {
    const float2 x = *reinterpret_cast<const float2*>(tile + g * TW + p);
    V v;
    v.v[0] = x.x;
    v.v[1] = x.y;
    return v;
  };
#pragma unroll 1
  for (int m = 0; m < 7; ++m) {
    V s1[16];
#pragma unroll
    for (int h = 0; h < 16; ++h) s1[h] = level_sum<SIDE, V>(m, [&](int q) { return in(q * 16 + h); });
    Tree<float, SIDE, 2, kStagedVec>::run(s1, m, emit);
  }
}

template <int OUT, int SIDE>
cudaError_t launch_staged(const DivideArgs& a, cudaStream_t st) {
  constexpr int TW = 128;
  constexpr int SMEM = 64 * TW * 4;
  if (a.L % TW != 0 || a.ld < a.n || a.top >= 0) return cudaErrorInvalidValue;
  const int vec_ok = (a.ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(a.X) & 15) == 0);
  auto kern = divide_staged_kernel<OUT, SIDE, TW>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
  if (e != cudaSuccess) return e;
  const int64_t blocks = a.L * (a.L / TW);
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7FFFFFFF) return cudaErrorInvalidValue;
  kern<<<(unsigned)blocks, TW / kStagedVec, SMEM, st>>>(a, vec_ok);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

bool divide_staged_fits(int64_t L) { return L > 0 && L % 128 == 0; }

cudaError_t launch_divide_staged(const DivideArgs& a, int side, OutMode out, cudaStream_t st) {
  if (out == kOutSplitBf16) return side == 0 ? launch_staged<kOutSplitBf16, 0>(a, st) : launch_staged<kOutSplitBf16, 1>(a, st);
  if (out == kOutSplitTf32) return side == 0 ? launch_staged<kOutSplitTf32, 0>(a, st) : launch_staged<kOutSplitTf32, 1>(a, st);
  if (out == kOutSplitFp16) return side == 0 ? launch_staged<kOutSplitFp16, 0>(a, st) : launch_staged<kOutSplitFp16, 1>(a, st);
  return cudaErrorInvalidValue;
}

}  // namespace stark
