// divide_top.cu -- the divide phase of one depth-first subtree (Alg. 3 below
// the top one or two recursion levels): the input is read through the
// operand sums of the levels above the subtree (formed on the fly, in the
// order of Alg. 1) and the subtree's leaf operands are written to the
// workspace.  Instantiated apart from the breadth-first launches so the two
// translation units compile in parallel.
#include "divide_impl.cuh"

namespace stark {
namespace {

template <typename Tin, int OUT, int SIDE>
cudaError_t by_depth_top(const DivideArgs& a, int depth, cudaStream_t st) {
  if (a.top_levels == 1) {  // below the top level, subtree depth <= 2
    switch (depth) {
      case 0: return launch_one<Tin, OUT, 0, SIDE, 1>(a, st);
      case 1: return launch_one<Tin, OUT, 1, SIDE, 1>(a, st);
      case 2: return launch_one<Tin, OUT, 2, SIDE, 1>(a, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (a.top_levels == 2) {  // below two levels: split-fp32 dtypes, depth <= 3
    if constexpr (std::is_same_v<Tin, float>) {
      switch (depth) {
        case 0: return launch_one<Tin, OUT, 0, SIDE, 2>(a, st);
        case 1: return launch_one<Tin, OUT, 1, SIDE, 2>(a, st);
        default: return cudaErrorInvalidValue;
      }
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_divide_top(const DivideArgs& a, int depth, int side, InType in, OutMode out, cudaStream_t st) {
  if (a.top < 0) return cudaErrorInvalidValue;
  if (in == kInF32 && out == kOutSplitBf16)
    return side == 0 ? by_depth_top<float, kOutSplitBf16, 0>(a, depth, st)
                     : by_depth_top<float, kOutSplitBf16, 1>(a, depth, st);
  if (in == kInF32 && out == kOutSplitTf32)
    return side == 0 ? by_depth_top<float, kOutSplitTf32, 0>(a, depth, st)
                     : by_depth_top<float, kOutSplitTf32, 1>(a, depth, st);
  if (in == kInF32 && out == kOutSplitFp16)
    return side == 0 ? by_depth_top<float, kOutSplitFp16, 0>(a, depth, st)
                     : by_depth_top<float, kOutSplitFp16, 1>(a, depth, st);
  if (in == kInF64 && out == kOutPlain)
    return side == 0 ? by_depth_top<double, kOutPlain, 0>(a, depth, st) : by_depth_top<double, kOutPlain, 1>(a, depth, st);
  if (in == kInI64 && out == kOutPlain)
    return side == 0 ? by_depth_top<int64_t, kOutPlain, 0>(a, depth, st)
                     : by_depth_top<int64_t, kOutPlain, 1>(a, depth, st);
  if (in == kInI64 && out == kOutBf16Exact)
    return side == 0 ? by_depth_top<int64_t, kOutBf16Exact, 0>(a, depth, st)
                     : by_depth_top<int64_t, kOutBf16Exact, 1>(a, depth, st);
  return cudaErrorInvalidValue;
}

}  // namespace stark
