// divide.cu -- the divide phase (Alg. 1 / Alg. 3, Sec. III-C): one pass over
// an operand that writes the operand sums of all 7^depth leaf products.
//
// Stark forms these sums level by level with a Spark shuffle per level
// (replicate A11, A22 four times and A12, A21 twice, group by M-index, add).
// Here one kernel does every level for a T x T tile position of all leaf
// planes at once: each element of the input is read from HBM once, and
// each leaf operand element is written once.
//
// Per block (output tile origin (r0, c0) inside an L x L leaf plane):
//   for each level-1 product m1 in M1..M7:
//     stage the level-1 sums  S = sum_q1 coef(m1, q1) * X_{q1, g}  for every
//     sub-path g of the remaining depth-1 levels into shared memory (two fp32
//     terms at most, exactly the additions of Alg. 1, so the result does not
//     depend on summation order), transposed for B when requested;
//   each thread then walks the remaining levels of the tree in registers and
//   writes its leaf values (bf16 hi/lo, tf32 hi/lo, or the plain value).
// Padding to n_pad is virtual: reads beyond n return zero.
#include <cuda_bf16.h>

#include "stark_internal.h"

namespace stark {
namespace {

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
template <int SIDE, typename Acc, class Get>
__device__ __forceinline__ Acc level_sum(int m, const Get& g) {
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

template <typename Acc, int Q, int VEC>
struct RegSrc {
  const Acc (&v)[Q][VEC];
  __device__ __forceinline__ Acc get(int g, int e) const { return v[g][e]; }
};

template <typename Acc, int T, int VEC>
struct SmemSrc {
  const Acc* s;
  int base;  // cr * LD + cc
  __device__ __forceinline__ Acc get(int g, int e) const { return s[g * T * (T + 1) + base + e]; }
};

// Walk LV more recursion levels of product sums, calling emit(leaf, vals)
// for every leaf below; leaf numbers extend `prefix` in base 7.
template <typename Acc, int SIDE, int LV, int VEC>
struct Tree {
  template <class Src, class Emit>
  __device__ __forceinline__ static void run(const Src& src, int prefix, Emit& emit) {
    if constexpr (LV == 0) {
      Acc v[VEC];
#pragma unroll
      for (int e = 0; e < VEC; ++e) v[e] = src.get(0, e);
      emit(prefix, v);
    } else {
      constexpr int Q = pow4c(LV - 1);
#pragma unroll
      for (int m = 0; m < 7; ++m) {
        Acc o[Q][VEC];
#pragma unroll
        for (int h = 0; h < Q; ++h)
#pragma unroll
          for (int e = 0; e < VEC; ++e)
            o[h][e] = level_sum<SIDE, Acc>(m, [&](int q) { return src.get(q * Q + h, e); });
        RegSrc<Acc, Q, VEC> rs{o};
        Tree<Acc, SIDE, LV - 1, VEC>::run(rs, prefix * 7 + m, emit);
      }
    }
  }
};

template <int OUT, typename Tin, int VEC>
struct Emitter {
  void* hi;
  void* lo;
  int64_t plane_elems;  // L * L
  int64_t offset;       // row * L + col of this thread's first element

  __device__ __forceinline__ void operator()(int leaf, const typename AccOf<Tin>::type (&v)[VEC]) const {
    const int64_t at = (int64_t)leaf * plane_elems + offset;
    if constexpr (OUT == kOutSplitBf16) {
      __nv_bfloat16 h[VEC], l[VEC];
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        h[e] = __float2bfloat16_rn(v[e]);
        l[e] = __float2bfloat16_rn(v[e] - __bfloat162float(h[e]));
      }
      store_vec(reinterpret_cast<__nv_bfloat16*>(hi) + at, h);
      store_vec(reinterpret_cast<__nv_bfloat16*>(lo) + at, l);
    } else if constexpr (OUT == kOutSplitTf32) {
      float h[VEC], l[VEC];
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        h[e] = rn_tf32(v[e]);
        l[e] = rn_tf32(v[e] - h[e]);
      }
      store_vec(reinterpret_cast<float*>(hi) + at, h);
      store_vec(reinterpret_cast<float*>(lo) + at, l);
    } else {
      Tin o[VEC];
#pragma unroll
      for (int e = 0; e < VEC; ++e) o[e] = (Tin)v[e];
      store_vec(reinterpret_cast<Tin*>(hi) + at, o);
    }
  }

  template <typename E>
  __device__ __forceinline__ static void store_vec(E* p, const E (&x)[VEC]) {
    constexpr int bytes = (int)sizeof(E) * VEC;
    if constexpr (bytes % 16 == 0) {
#pragma unroll
      for (int k = 0; k < bytes / 16; ++k) reinterpret_cast<int4*>(p)[k] = reinterpret_cast<const int4*>(x)[k];
    } else if constexpr (bytes == 8) {
      *reinterpret_cast<int2*>(p) = *reinterpret_cast<const int2*>(x);
    } else if constexpr (bytes == 4) {
      *reinterpret_cast<int*>(p) = *reinterpret_cast<const int*>(x);
    } else {
#pragma unroll
      for (int e = 0; e < VEC; ++e) p[e] = x[e];
    }
  }
};

template <typename Tin, int OUT, int D, int T, int SIDE, bool TRANS>
__global__ void __launch_bounds__(T * 8) divide_kernel(DivideArgs a) {
  using Acc = typename AccOf<Tin>::type;
  constexpr int NT = T * 8;
  constexpr int VEC = T / 8;
  constexpr int G = (D == 0) ? 1 : pow4c(D - 1);
  constexpr int LD = T + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Acc* s = reinterpret_cast<Acc*>(smem_raw);

  const int t = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.y * T;
  const int64_t c0 = (int64_t)blockIdx.x * T;
  const int64_t i0 = TRANS ? c0 : r0;
  const int64_t j0 = TRANS ? r0 : c0;
  const Tin* __restrict__ X = static_cast<const Tin*>(a.X);
  const int64_t n = a.n, npad = a.npad;

  const int cr = t / 8;
  const int cc = (t % 8) * VEC;
  Emitter<OUT, Tin, VEC> emit{a.out_hi, a.out_lo, a.L * a.L, (r0 + cr) * a.L + c0 + cc};
  const SmemSrc<Acc, T, VEC> src{s, cr * LD + cc};

  auto load = [&](int64_t row, int64_t col) -> Acc {
    return (row < n && col < n) ? (Acc)__ldg(&X[row * n + col]) : Acc(0);
  };

  if constexpr (D == 0) {
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      const int idx = t + e * NT;
      const int ii = idx / T, jj = idx % T;
      const Acc v = load(i0 + ii, j0 + jj);
      s[(TRANS ? jj : ii) * LD + (TRANS ? ii : jj)] = v;
    }
    __syncthreads();
    Tree<Acc, SIDE, 0, VEC>::run(src, 0, emit);
  } else {
    const int64_t half = npad >> 1;
    for (int m1 = 0; m1 < 7; ++m1) {
      if (m1) __syncthreads();
#pragma unroll 4
      for (int g = 0; g < G; ++g) {
        int64_t sub_r = 0, sub_c = 0;
#pragma unroll
        for (int k = 2; k <= D; ++k) {
          const int digit = (g / pow4c(D - k)) & 3;
          sub_r += (int64_t)(digit >> 1) * (npad >> k);
          sub_c += (int64_t)(digit & 1) * (npad >> k);
        }
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
          const int idx = t + e * NT;
          const int ii = idx / T, jj = idx % T;
          const int64_t row = sub_r + i0 + ii, col = sub_c + j0 + jj;
          const Acc v = level_sum<SIDE, Acc>(
              m1, [&](int q1) { return load(row + (q1 >> 1) * half, col + (q1 & 1) * half); });
          s[(g * T + (TRANS ? jj : ii)) * LD + (TRANS ? ii : jj)] = v;
        }
      }
      __syncthreads();
      Tree<Acc, SIDE, D - 1, VEC>::run(src, m1, emit);
    }
  }
}

constexpr int pick_tile(int D, int esz) {
  // largest T in {32, 16, 8} whose staging buffer fits 100 KB
  return ((D == 0 ? 1 : pow4c(D - 1)) * 32 * 33 * esz <= 100 * 1024)   ? 32
         : ((D == 0 ? 1 : pow4c(D - 1)) * 16 * 17 * esz <= 100 * 1024) ? 16
                                                                        : 8;
}

template <typename Tin, int OUT, int D, int SIDE, bool TRANS>
cudaError_t launch_one(const DivideArgs& a, cudaStream_t st) {
  using Acc = typename AccOf<Tin>::type;
  constexpr int T = pick_tile(D, (int)sizeof(Acc));
  constexpr int G = (D == 0) ? 1 : pow4c(D - 1);
  constexpr int smem = G * T * (T + 1) * (int)sizeof(Acc);
  auto kern = divide_kernel<Tin, OUT, D, T, SIDE, TRANS>;
  if (a.L % T != 0) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t tiles = a.L / T;
  if (tiles > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)tiles, (unsigned)tiles, 1);
  kern<<<grid, T * 8, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <typename Tin, int OUT, int SIDE, bool TRANS>
cudaError_t by_depth(const DivideArgs& a, int depth, cudaStream_t st) {
  switch (depth) {
    case 0: return launch_one<Tin, OUT, 0, SIDE, TRANS>(a, st);
    case 1: return launch_one<Tin, OUT, 1, SIDE, TRANS>(a, st);
    case 2: return launch_one<Tin, OUT, 2, SIDE, TRANS>(a, st);
    case 3: return launch_one<Tin, OUT, 3, SIDE, TRANS>(a, st);
    case 4: return launch_one<Tin, OUT, 4, SIDE, TRANS>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_divide(const DivideArgs& a, int depth, int side, InType in, OutMode out, bool trans,
                          cudaStream_t st) {
  if (in == kInF32 && out == kOutSplitBf16) {
    if (side == 0 && !trans) return by_depth<float, kOutSplitBf16, 0, false>(a, depth, st);
    if (side == 1 && trans) return by_depth<float, kOutSplitBf16, 1, true>(a, depth, st);
  } else if (in == kInF32 && out == kOutSplitTf32) {
    if (side == 0 && !trans) return by_depth<float, kOutSplitTf32, 0, false>(a, depth, st);
    if (side == 1 && trans) return by_depth<float, kOutSplitTf32, 1, true>(a, depth, st);
  } else if (in == kInF64 && out == kOutPlain && !trans) {
    return side == 0 ? by_depth<double, kOutPlain, 0, false>(a, depth, st)
                     : by_depth<double, kOutPlain, 1, false>(a, depth, st);
  } else if (in == kInI64 && out == kOutPlain && !trans) {
    return side == 0 ? by_depth<int64_t, kOutPlain, 0, false>(a, depth, st)
                     : by_depth<int64_t, kOutPlain, 1, false>(a, depth, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace stark
