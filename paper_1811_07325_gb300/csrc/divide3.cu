// divide3.cu -- the breadth-first divide at depth 3 for fp32 input with
// 3xBF16 split output: one pass over the operand that reads every input
// element from HBM once and writes all 343 leaf operand planes (Alg. 3 with
// every level at once, as in divide.cu).
//
// A thread owns two consecutive columns (i, j..j+1) of the L x L leaf grid:
// it loads the matching 8-byte vector of each of the 64 depth-3 quadrant
// paths of the input (all loads independent and issued up front), then runs
// the three levels of two-term sums of Alg. 1 in registers and stores its
// two values of every leaf plane (hi and lo planes; 4-byte bf16 pairs,
// coalesced across the warp).  Two columns per thread keep the 64 input
// vectors within the register file (128 values, 168 registers in all); four
// would spill, and so does the tf32 split's rounding, so 3xTF32 keeps the
// per-top-product launches.  The sums are the same two-term additions per
// level as the depth <= 2 kernel, so the operands are bit-identical to the
// level-by-level form.  Padding is virtual (reads beyond n give zero).
#include "divide_impl.cuh"

namespace stark {
namespace {

constexpr int kThreads3 = 128;

template <int OUT, int SIDE>
__global__ void __launch_bounds__(kThreads3) divide3_kernel(DivideArgs a, int vec_ok) {
  constexpr int VEC = 2;
  constexpr int D = 3;
  const int64_t per_row = a.L / VEC;
  const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= a.L * per_row) return;
  const int64_t i = pos / per_row;
  const int64_t j = (pos % per_row) * VEC;
  const Loader<float, VEC> ld{static_cast<const float*>(a.X), a.n, a.ld, vec_ok != 0};
  const Emitter<OUT, float, VEC> emit{a.out_hi, a.out_lo, a.L * a.L, i * a.L + j, a.range_flag};
  const int64_t L = a.L;
  Vec<float, VEC> in[pow4c(D)];
#pragma unroll
  for (int g = 0; g < pow4c(D); ++g) {
    // quadrant path g = (q1, q2, q3), top level most significant: row and
    // column offsets of 4L, 2L and L per level
    const int q1 = (g >> 4) & 3, q2 = (g >> 2) & 3, q3 = g & 3;
    const int64_t r = i + (int64_t)((q1 >> 1) * 4 + (q2 >> 1) * 2 + (q3 >> 1)) * L;
    const int64_t c = j + (int64_t)((q1 & 1) * 4 + (q2 & 1) * 2 + (q3 & 1)) * L;
    in[g] = ld(r, c);
  }
  Tree<float, SIDE, D, VEC>::run(in, 0, emit);
}

template <int OUT, int SIDE>
cudaError_t launch3(const DivideArgs& a, cudaStream_t st) {
  constexpr int VEC = 2;
  if (a.L % VEC != 0 || a.ld < a.n || a.npad != 8 * a.L) return cudaErrorInvalidValue;
  const int vec_ok = (a.ld % VEC == 0) && ((reinterpret_cast<uintptr_t>(a.X) & 7) == 0);
  const int64_t threads = a.L * (a.L / VEC);
  const int64_t blocks = (threads + kThreads3 - 1) / kThreads3;
  if (blocks > 0x7FFFFFFF) return cudaErrorInvalidValue;
  divide3_kernel<OUT, SIDE><<<(unsigned)blocks, kThreads3, 0, st>>>(a, vec_ok);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_divide3(const DivideArgs& a, int side, OutMode out, cudaStream_t st) {
  if (a.top >= 0) return cudaErrorInvalidValue;
  if (out == kOutSplitBf16) return side == 0 ? launch3<kOutSplitBf16, 0>(a, st) : launch3<kOutSplitBf16, 1>(a, st);
  return cudaErrorInvalidValue;
}

}  // namespace stark
