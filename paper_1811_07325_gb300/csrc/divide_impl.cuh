// divide_impl.cuh -- the divide kernel templates (see divide.cu), shared by
// the breadth-first launches (divide.cu) and the depth-first ones
// (divide_top.cu), which are compiled as separate translation units.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "ptx.cuh"
#include "stark_internal.h"

namespace stark {
namespace {  // internal to each translation unit that includes this

__host__ __device__ constexpr int pow4c(int k) { return k <= 0 ? 1 : 4 * pow4c(k - 1); }
__host__ __device__ constexpr int pow7c(int k) { return k <= 0 ? 1 : 7 * pow7c(k - 1); }

template <typename T>
struct AccOf {
  using type = T;
};
template <>
struct AccOf<int64_t> {
  using type = unsigned long long;  // wraps modulo 2^64
};

// The two-term sums of Alg. 1 for product m (0..6 = M1..M7), quadrant values
// from g(q), q = 0:11, 1:12, 2:21, 3:22.
template <int SIDE, typename V, class Get>
__device__ __forceinline__ V level_sum(int m, const Get& g) {
  if constexpr (SIDE == 0) {
    switch (m) {
      case 0: return g(0) + g(3);  // A11 + A22
      case 1: return g(2) + g(3);  // A21 + A22
      case 2: return g(0);         // A11
      case 3: return g(3);         // A22
      case 4: return g(0) + g(1);  // A11 + A12
      case 5: return g(2) - g(0);  // A21 - A11
      default: return g(1) - g(3); // A12 - A22
    }
  } else {
    switch (m) {
      case 0: return g(0) + g(3);  // B11 + B22
      case 1: return g(0);         // B11
      case 2: return g(1) - g(3);  // B12 - B22
      case 3: return g(2) - g(0);  // B21 - B11
      case 4: return g(3);         // B22
      case 5: return g(0) + g(1);  // B11 + B12
      default: return g(2) + g(3); // B21 + B22
    }
  }
}

// Round-to-nearest-even of an fp32 value to TF32 (10 stored mantissa bits),
// on the bit pattern: add half an ulp minus one plus the lowest kept bit,
// then clear the 13 dropped bits.  Inf/NaN pass through.
__device__ __forceinline__ float rn_tf32(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7F800000u) != 0x7F800000u) {
    u += 0x0FFFu + ((u >> 13) & 1u);
    u &= 0xFFFFE000u;
  }
  return __uint_as_float(u);
}

// A short vector of accumulator values with elementwise + and -.
template <typename Acc, int VEC>
struct Vec {
  Acc v[VEC];
  __device__ __forceinline__ Vec operator+(const Vec& o) const {
    Vec r;
#pragma unroll
    for (int e = 0; e < VEC; ++e) r.v[e] = v[e] + o.v[e];
    return r;
  }
  __device__ __forceinline__ Vec operator-(const Vec& o) const {
    Vec r;
#pragma unroll
    for (int e = 0; e < VEC; ++e) r.v[e] = v[e] - o.v[e];
    return r;
  }
};

template <int OUT, typename Tin, int VEC>
struct Emitter {
  using Acc = typename AccOf<Tin>::type;
  void* hi;
  void* lo;
  int64_t plane_elems;  // L * L
  int64_t offset;       // row * L + col of this thread's first element
  int* range_flag;

  __device__ __forceinline__ void operator()(int leaf, const Vec<Acc, VEC>& x) const {
    const int64_t at = (int64_t)leaf * plane_elems + offset;
    if constexpr (OUT == kOutBf16Exact) {
      // integer operand sums, exact in bf16 while |v| <= 256 (8 significant bits)
      __nv_bfloat16 h[VEC];
      bool bad = false;
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const long long v = (long long)x.v[e];
        bad |= (v > 256 || v < -256);
        h[e] = __float2bfloat16_rn((float)v);
      }
      if (bad) record_error(range_flag, kDevIntRange);
      store_vec(reinterpret_cast<__nv_bfloat16*>(hi) + at, h);
    } else if constexpr (OUT == kOutSplitBf16 && VEC % 2 == 0) {
      // two values per conversion (round to nearest even each, as below)
      __nv_bfloat162 h[VEC / 2], l[VEC / 2];
#pragma unroll
      for (int e = 0; e < VEC / 2; ++e) {
        h[e] = __floats2bfloat162_rn(x.v[2 * e], x.v[2 * e + 1]);
        const float2 hf = __bfloat1622float2(h[e]);
        l[e] = __floats2bfloat162_rn(x.v[2 * e] - hf.x, x.v[2 * e + 1] - hf.y);
      }
      store_vec(reinterpret_cast<__nv_bfloat162*>(hi) + at / 2, h);
      store_vec(reinterpret_cast<__nv_bfloat162*>(lo) + at / 2, l);
    } else if constexpr (OUT == kOutSplitBf16) {
      __nv_bfloat16 h[VEC], l[VEC];
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        h[e] = __float2bfloat16_rn(x.v[e]);
        l[e] = __float2bfloat16_rn(x.v[e] - __bfloat162float(h[e]));
      }
      store_vec(reinterpret_cast<__nv_bfloat16*>(hi) + at, h);
      store_vec(reinterpret_cast<__nv_bfloat16*>(lo) + at, l);
    } else if constexpr (OUT == kOutSplitFp16) {
      // hi = RN_fp16(x), lo = RN_fp16(x - hi) (x - hi exact in fp32); a sum
      // beyond the fp16 range (hi infinite) raises the plan's range flag
      __half2 h[(VEC + 1) / 2], l[(VEC + 1) / 2];
      bool bad = false;
#pragma unroll
      for (int e = 0; e < VEC / 2; ++e) {
        h[e] = __floats2half2_rn(x.v[2 * e], x.v[2 * e + 1]);
        const float2 hf = __half22float2(h[e]);
        bad |= !(fabsf(hf.x) <= 65504.f) || !(fabsf(hf.y) <= 65504.f);
        l[e] = __floats2half2_rn(x.v[2 * e] - hf.x, x.v[2 * e + 1] - hf.y);
      }
      static_assert(VEC % 2 == 0, "fp16 halves are stored in pairs");
      if (bad) record_error(range_flag, kDevFp16Range);
      store_vec(reinterpret_cast<__half2*>(hi) + at / 2, h);
      store_vec(reinterpret_cast<__half2*>(lo) + at / 2, l);
    } else if constexpr (OUT == kOutSplitTf32) {
      float h[VEC], l[VEC];
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        h[e] = rn_tf32(x.v[e]);
        l[e] = rn_tf32(x.v[e] - h[e]);
      }
      store_vec(reinterpret_cast<float*>(hi) + at, h);
      store_vec(reinterpret_cast<float*>(lo) + at, l);
    } else {
      Tin o[VEC];
#pragma unroll
      for (int e = 0; e < VEC; ++e) o[e] = (Tin)x.v[e];
      store_vec(reinterpret_cast<Tin*>(hi) + at, o);
    }
  }

  template <typename E, int N>
  __device__ __forceinline__ static void store_vec(E* p, const E (&x)[N]) {
    constexpr int bytes = (int)sizeof(E) * N;
    if constexpr (bytes % 16 == 0) {
#pragma unroll
      for (int k = 0; k < bytes / 16; ++k) __stcs(reinterpret_cast<int4*>(p) + k, reinterpret_cast<const int4*>(x)[k]);
    } else if constexpr (bytes == 8) {
      __stcs(reinterpret_cast<int2*>(p), *reinterpret_cast<const int2*>(x));
    } else if constexpr (bytes == 4) {
      __stcs(reinterpret_cast<int*>(p), *reinterpret_cast<const int*>(x));
    } else {
#pragma unroll
      for (int e = 0; e < N; ++e) p[e] = x[e];
    }
  }
};

// Register tree over the last LV levels: `in` holds the 4^LV sub-quadrant
// vectors (base-4 path, top level most significant).
template <typename Acc, int SIDE, int LV, int VEC>
struct Tree {
  template <class Emit>
  __device__ __forceinline__ static void run(const Vec<Acc, VEC> (&in)[pow4c(LV)], int prefix, const Emit& emit) {
    if constexpr (LV == 0) {
      emit(prefix, in[0]);
    } else {
      constexpr int Q = pow4c(LV - 1);
#pragma unroll
      for (int m = 0; m < 7; ++m) {
        Vec<Acc, VEC> o[Q];
#pragma unroll
        for (int h = 0; h < Q; ++h) o[h] = level_sum<SIDE, Vec<Acc, VEC>>(m, [&](int q) { return in[q * Q + h]; });
        Tree<Acc, SIDE, LV - 1, VEC>::run(o, prefix * 7 + m, emit);
      }
    }
  }
};

template <typename Tin, int VEC>
struct Loader {
  using Acc = typename AccOf<Tin>::type;
  const Tin* __restrict__ X;
  int64_t n;    // rows and columns read; zeros beyond
  int64_t ld;   // row stride
  bool vec_ok;  // rows are VEC-aligned: vector loads allowed where in bounds

  __device__ __forceinline__ Vec<Acc, VEC> operator()(int64_t row, int64_t col) const {
    Vec<Acc, VEC> r;
    if (row < n && col + VEC <= n && vec_ok) {
      const Tin* p = X + row * ld + col;
      if constexpr (sizeof(Tin) * VEC == 16) {
        const int4 raw = __ldcs(reinterpret_cast<const int4*>(p));
        const Tin* t = reinterpret_cast<const Tin*>(&raw);
#pragma unroll
        for (int e = 0; e < VEC; ++e) r.v[e] = (Acc)t[e];
      } else {
#pragma unroll
        for (int e = 0; e < VEC; ++e) r.v[e] = (Acc)__ldcs(p + e);
      }
    } else {
#pragma unroll
      for (int e = 0; e < VEC; ++e)
        r.v[e] = (row < n && col + e < n) ? (Acc)__ldcs(X + row * ld + col + e) : Acc(0);
    }
    return r;
  }
};

// The same two-term sums for a product index known only at run time:
// value = x_qa, then (+ or -) x_qb when the product has a second term, in
// the order written in level_sum (so the rounding is identical).
struct TermPair {
  int8_t qa, qb, sb;  // qb < 0: single term
};
template <int SIDE>
__device__ __forceinline__ TermPair terms_of(int m) {
  // A: M1 11+22, M2 21+22, M3 11, M4 22, M5 11+12, M6 21-11, M7 12-22
  // B: M1 11+22, M2 11, M3 12-22, M4 21-11, M5 22, M6 11+12, M7 21+22
  constexpr int8_t ta[7][3] = {{0, 3, 1}, {2, 3, 1}, {0, -1, 0}, {3, -1, 0}, {0, 1, 1}, {2, 0, -1}, {1, 3, -1}};
  constexpr int8_t tb[7][3] = {{0, 3, 1}, {0, -1, 0}, {1, 3, -1}, {2, 0, -1}, {3, -1, 0}, {0, 1, 1}, {2, 3, 1}};
  const int8_t* t = SIDE == 0 ? ta[m] : tb[m];
  return TermPair{t[0], t[1], t[2]};
}

// Depth-first traversal: the subproblem's input is the level-K operand sum
// along the M-index path dig[0..K) (top level first), formed on the fly
// from the full (padded) input, level by level in the same order as the
// breadth-first divide: S_k = two-term sum of quadrants of S_{k-1} (the
// outermost evaluation is the deepest level), S_0 = the input.
template <typename Tin, int VEC, int SIDE, int K>
struct TopLoader {
  using Acc = typename AccOf<Tin>::type;
  Loader<Tin, VEC> ld;
  int dig[K];
  int64_t npad;  // side of the full problem

  // level_sum switches on the (block-uniform) product and calls the
  // quadrant accessor with constant quadrants, so every address offset is
  // a compile-time multiple of h
  template <int F>
  __device__ __forceinline__ Vec<Acc, VEC> at(int64_t row, int64_t col) const {
    if constexpr (F == 0) {
      return ld(row, col);
    } else {
      const int64_t h = npad >> F;  // quadrant side at level F
      return level_sum<SIDE, Vec<Acc, VEC>>(
          dig[F - 1], [&](int q) { return at<F - 1>(row + (q >> 1) * h, col + (q & 1) * h); });
    }
  }
  __device__ __forceinline__ Vec<Acc, VEC> operator()(int64_t row, int64_t col) const { return at<K>(row, col); }
};

// Value at position (row, col) of the level-F operand sum S_F selected by the
// M-indices dig[0..F) (top level first).  S_k(p) = level_sum(i_k, quadrant q
// of S_{k-1} at p), S_0 = the input: the outermost sum is the deepest level,
// so the rounding is exactly that of forming the levels one after another.
template <int SIDE, typename Acc, int VEC, int F, class Load>
struct Prefix {
  __device__ __forceinline__ static Vec<Acc, VEC> eval(const Load& ld, const int* dig, int64_t npad, int64_t row,
                                                       int64_t col) {
    if constexpr (F == 0) {
      return ld(row, col);
    } else {
      const int64_t h = npad >> F;  // quadrant side at level F
      const TermPair t = terms_of<SIDE>(dig[F - 1]);
      Vec<Acc, VEC> v = Prefix<SIDE, Acc, VEC, F - 1, Load>::eval(ld, dig, npad, row + (t.qa >> 1) * h,
                                                                   col + (t.qa & 1) * h);
      if (t.qb >= 0) {
        const Vec<Acc, VEC> w = Prefix<SIDE, Acc, VEC, F - 1, Load>::eval(ld, dig, npad, row + (t.qb >> 1) * h,
                                                                         col + (t.qb & 1) * h);
        v = t.sb > 0 ? v + w : v - w;
      }
      return v;
    }
  }
};

// K > 0: a depth-first subtree below K levels (input read through TopLoader).
template <typename Tin, int OUT, int D, int SIDE, int VEC, int K>
__global__ void __launch_bounds__(256, 2) divide_kernel(DivideArgs a, int vec_ok) {
  using Acc = typename AccOf<Tin>::type;
  constexpr int R = D < 2 ? D : 2;  // levels done in registers
  constexpr int F = D - R;          // levels walked as an outer loop
  const int64_t per_row = a.L / VEC;
  const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= a.L * per_row) return;
  const int64_t i = pos / per_row;
  const int64_t j = (pos % per_row) * VEC;
  const Loader<Tin, VEC> ld0{static_cast<const Tin*>(a.X), a.n, a.ld, vec_ok != 0};
  using LoadT = std::conditional_t<(K > 0), TopLoader<Tin, VEC, SIDE, (K > 0 ? K : 1)>, Loader<Tin, VEC>>;
  LoadT ld;
  if constexpr (K > 0) {
    ld.ld = ld0;
    int x = a.top;  // base-7 path, top level most significant
#pragma unroll
    for (int k = K - 1; k >= 0; --k) {
      ld.dig[k] = x % 7;
      x /= 7;
    }
    ld.npad = a.npad << K;  // a.npad is the subproblem's side
  } else {
    ld = ld0;
  }
  const Emitter<OUT, Tin, VEC> emit{a.out_hi, a.out_lo, a.L * a.L, i * a.L + j, a.range_flag};
  const int64_t npad = a.npad;

  auto leaf_block = [&](const int* dig, int prefix) {
    // the 4^R sub-quadrant vectors below this prefix, then the register tree
    Vec<Acc, VEC> in[pow4c(R)];
#pragma unroll
    for (int g = 0; g < pow4c(R); ++g) {
      int64_t r = i, c = j;
#pragma unroll
      for (int k = 0; k < R; ++k) {
        const int digit = (g >> (2 * (R - 1 - k))) & 3;
        r += (int64_t)(digit >> 1) * (npad >> (F + k + 1));
        c += (int64_t)(digit & 1) * (npad >> (F + k + 1));
      }
      in[g] = Prefix<SIDE, Acc, VEC, F, LoadT>::eval(ld, dig, npad, r, c);
    }
    Tree<Acc, SIDE, R, VEC>::run(in, prefix, emit);
  };

  if constexpr (F == 0) {
    leaf_block(nullptr, 0);
  } else {
    // one prefix of the outer levels per grid row: the blocks in flight at a
    // time write the 2 * 7^R planes of one prefix (sequential write streams),
    // at the price of reading each prefix's input quadrants again
    const int p = (int)blockIdx.y;
    int dig[F > 0 ? F : 1];
    int x = p;
#pragma unroll
    for (int k = F - 1; k >= 0; --k) {
      dig[k] = x % 7;
      x /= 7;
    }
    leaf_block(dig, p);
  }
}

template <typename Tin, int OUT, int D, int SIDE, int K>
cudaError_t launch_one(const DivideArgs& a, cudaStream_t st) {
  constexpr int VEC = 16 / (int)sizeof(Tin);  // one 16-byte load per quadrant
  if (a.L % VEC != 0) return cudaErrorInvalidValue;
  if (a.ld < a.n) return cudaErrorInvalidValue;
  const int vec_ok = (a.ld % VEC == 0) && ((reinterpret_cast<uintptr_t>(a.X) & 15) == 0);
  const int64_t threads = a.L * (a.L / VEC);
  const int64_t blocks = (threads + 255) / 256;
  if (blocks > 0x7FFFFFFF) return cudaErrorInvalidValue;
  constexpr int F = D < 2 ? 0 : D - 2;  // outer levels: one grid row per prefix
  divide_kernel<Tin, OUT, D, SIDE, VEC, K><<<dim3((unsigned)blocks, (unsigned)pow7c(F)), 256, 0, st>>>(a, vec_ok);
  count_launch();
  return cudaGetLastError();
}

}  // namespace
}  // namespace stark
