// divide.cu -- the divide phase (Alg. 1 / Alg. 3, Sec. III-C): one streaming
// pass over an operand that writes the operand sums of all 7^depth leaf
// products.
//
// Stark forms these sums level by level, with a Spark shuffle per level
// (replicate A11 and A22 four times and A12, A21 twice, group by M-index,
// add).  Here one kernel does every level at once.  A thread owns VEC
// consecutive columns (i, j..j+VEC-1) of the L x L leaf grid; it reads the
// matching element vector of every quadrant path of the input (each input
// element is read from HBM once, with vector loads), forms the sums of the
// recursion tree in registers and stores its VEC values of every leaf plane
// (one contiguous 8- or 16-byte store per plane, coalesced across the warp).
//
// For depth <= 2 all 4^depth quadrant vectors sit in registers.  Deeper
// trees give each prefix of M-indices over the first depth-2 levels its own
// grid row: the 16 sub-quadrant sums below the prefix are evaluated from
// global memory in the same level-by-level order, then the last two levels
// run in registers.  Every sum is a two-term addition per level exactly as in
// Alg. 1, so results do not depend on evaluation order.
// Padding to n_pad is virtual: reads beyond n return zero.
// The kernel templates are in divide_impl.cuh; this file instantiates the
// breadth-first launches, divide_top.cu the depth-first ones.
#include "divide_impl.cuh"

namespace stark {
namespace {

template <typename Tin, int OUT, int SIDE>
cudaError_t by_depth(const DivideArgs& a, int depth, cudaStream_t st) {
  switch (depth) {
    case 0: return launch_one<Tin, OUT, 0, SIDE, 0>(a, st);
    case 1: return launch_one<Tin, OUT, 1, SIDE, 0>(a, st);
    case 2: return launch_one<Tin, OUT, 2, SIDE, 0>(a, st);
    case 3: return launch_one<Tin, OUT, 3, SIDE, 0>(a, st);
    case 4: return launch_one<Tin, OUT, 4, SIDE, 0>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_divide(const DivideArgs& a, int depth, int side, InType in, OutMode out, cudaStream_t st) {
  if (a.top >= 0) return launch_divide_top(a, depth, side, in, out, st);  // depth-first subtree (divide_top.cu)
  if (in == kInF32 && out == kOutSplitBf16)
    return side == 0 ? by_depth<float, kOutSplitBf16, 0>(a, depth, st) : by_depth<float, kOutSplitBf16, 1>(a, depth, st);
  if (in == kInF32 && out == kOutSplitTf32)
    return side == 0 ? by_depth<float, kOutSplitTf32, 0>(a, depth, st) : by_depth<float, kOutSplitTf32, 1>(a, depth, st);
  if (in == kInF32 && out == kOutSplitFp16)
    return side == 0 ? by_depth<float, kOutSplitFp16, 0>(a, depth, st) : by_depth<float, kOutSplitFp16, 1>(a, depth, st);
  if (in == kInF64 && out == kOutPlain)
    return side == 0 ? by_depth<double, kOutPlain, 0>(a, depth, st) : by_depth<double, kOutPlain, 1>(a, depth, st);
  if (in == kInI64 && out == kOutPlain)
    return side == 0 ? by_depth<int64_t, kOutPlain, 0>(a, depth, st) : by_depth<int64_t, kOutPlain, 1>(a, depth, st);
  if (in == kInI64 && out == kOutBf16Exact)
    return side == 0 ? by_depth<int64_t, kOutBf16Exact, 0>(a, depth, st)
                     : by_depth<int64_t, kOutBf16Exact, 1>(a, depth, st);
  return cudaErrorInvalidValue;
}

}  // namespace stark
