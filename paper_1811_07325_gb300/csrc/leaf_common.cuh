// leaf_common.cuh -- pieces shared by the single-CTA and the CTA-pair leaf
// kernels: decoding a work item (one output tile of one leaf product) and
// the epilogue that adds a finished accumulator tile into C (Alg. 5 fused).
#pragma once
#include "ptx.cuh"
#include "stark_internal.h"

namespace stark {

constexpr int kBM = 128;  // accumulator rows held by one CTA (TMEM lanes)

// Everything one work item (a BM x BN tile of one leaf product) needs.
struct ItemInfo {
  const CUtensorMap* tA;
  const CUtensorMap* tB;
  const CUtensorMap* tC;
  int leaf, P, m0, n0, kblocks;
  const CTarget* tg;
  int nt;
  float* C;
  int64_t n, ldc;
  int use_tma_c;
  int sib;     // sibling-folded combine: this leaf's M-index digit at the last level (0..6 = M1..M7)
  int parent;  // and its parent's plane (relative to leaf_begin / 7)
  bool valid;  // false: a padding item of the sibling-major order (no work)
};

// Sibling-major order of the CTA-pair items (LeafTcArgs::sib): with U pairs
// launched and T pair tiles per leaf, item k*U + u is tile position
// tp = (k / 7) * U + u of the parents' tile grid (parent tp / T, tile tp % T)
// for sibling k % 7.  Pair u (which takes items u, u + U, ...) so runs the
// seven children of one parent at one tile position back to back (their
// parent-quadrant tiles stay in L2 between them), while the U pairs at one
// step share a sibling leaf, as in the leaf-major order.
__device__ __forceinline__ int64_t sib_items(const LeafTcArgs& p, int BN, int units) {
  const int64_t T = (int64_t)(p.L / (2 * kBM)) * (p.L / BN);
  const int64_t tp = (int64_t)(p.leaf_end - p.leaf_begin) / 7 * T;
  return (tp + units - 1) / units * 7 * units;
}

template <int BN, int BK>
__device__ __forceinline__ ItemInfo decode_sib(int item, const LeafTcArgs& p, const CUtensorMap* tmA,
                                               const CUtensorMap* tmB, const CUtensorMap* tmC, uint32_t rank,
                                               int units) {
  ItemInfo it;
  const int tiles_n = p.L / BN;
  const int T = (p.L / (2 * kBM)) * tiles_n;
  const int parents = (p.leaf_end - p.leaf_begin) / 7;
  const int k = item / units, u = item % units;
  const int64_t tp = (int64_t)(k / 7) * units + u;
  it.valid = tp < (int64_t)parents * T;
  it.sib = k % 7;
  it.parent = it.valid ? (int)(tp / T) : 0;
  const int tile = it.valid ? (int)(tp % T) : 0;
  it.tA = tmA;
  it.tB = tmB;
  it.tC = tmC;
  it.leaf = p.leaf_begin + it.parent * 7 + it.sib;
  it.P = p.P;
  it.m0 = ((tile / tiles_n) * 2 + (int)rank) * kBM;
  it.n0 = (tile % tiles_n) * BN;
  it.kblocks = p.L / BK;
  it.tg = nullptr;
  it.nt = 0;
  it.C = p.C;
  it.n = p.n;
  it.ldc = p.ldc;
  it.use_tma_c = 0;
  return it;
}

// First and last sibling (product M_{m+1}) that adds into quadrant q of the
// parent (C11 = M1+M4-M5+M7, C12 = M3+M5, C21 = M2+M4, C22 = M1-M2+M3+M6):
// the first stores its tile (its sign is + in every quadrant), the others add.
__host__ __device__ constexpr int sib_first(int q) {
  return coef_c(0, q) ? 0 : coef_c(1, q) ? 1 : coef_c(2, q) ? 2 : 3;
}
__host__ __device__ constexpr int sib_last(int q) {
  return coef_c(6, q) ? 6 : coef_c(5, q) ? 5 : coef_c(4, q) ? 4 : 3;
}
static_assert(coef_c(sib_first(0), 0) > 0 && coef_c(sib_first(1), 1) > 0 && coef_c(sib_first(2), 2) > 0 &&
                  coef_c(sib_first(3), 3) > 0,
              "the first contribution to each quadrant is a plain store");

// coef_c for a sibling index known only at run time, from bit masks (one
// byte per quadrant: which products add into it, and which of them with a
// minus sign), so no table is read from memory.
__host__ __device__ constexpr int sib_coef(int m, int q) {
  constexpr uint32_t nz = 0x59u | (0x14u << 8) | (0x0Au << 16) | (0x27u << 24);
  constexpr uint32_t ng = (1u << 4) | (1u << 25);
  const uint32_t bit = 1u << (q * 8 + m);
  return (nz & bit) ? ((ng & bit) ? -1 : 1) : 0;
}
__host__ __device__ constexpr bool sib_coef_matches(int k = 0) {
  return k == 28 || (sib_coef(k % 7, k / 7) == coef_c(k % 7, k / 7) && sib_coef_matches(k + 1));
}
static_assert(sib_coef_matches(), "the bit masks encode the combine table");

template <int BN, int BK, bool GROUPED, bool PAIR>
__device__ __forceinline__ ItemInfo decode_item(int item, const LeafTcArgs& p, const CUtensorMap* tmA,
                                                const CUtensorMap* tmB, const CUtensorMap* tmC, uint32_t rank) {
  ItemInfo it;
  if constexpr (GROUPED) {
    // member owning this item: the last one whose item_base <= item
    int lo = 0, hi = p.ngroups - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (p.groups[mid].item_base <= item) lo = mid; else hi = mid - 1;
    }
    const GroupDesc* g = p.groups + lo;
    const int L = g->L;
    const int tiles_n = L / BN;
    const int per_leaf = (L / kBM / (PAIR ? 2 : 1)) * tiles_n;
    const int rem = item - g->item_base;
    it.tA = &g->tmA;
    it.tB = &g->tmB;
    it.tC = &g->tmC;
    it.leaf = rem / per_leaf;
    it.P = g->P;
    it.m0 = PAIR ? (((rem % per_leaf) / tiles_n) * 2 + (int)rank) * kBM : ((rem % per_leaf) / tiles_n) * kBM;
    it.n0 = ((rem % per_leaf) % tiles_n) * BN;
    it.kblocks = L / BK;
    it.tg = g->ctab + (int64_t)it.leaf * g->maxT;
    it.nt = g->ccount[it.leaf];
    it.C = g->C;
    it.n = g->n;
    it.ldc = g->ldc;
    it.use_tma_c = g->use_tma_c;
  } else {
    // (both branches) PAIR: an item is a pair of vertically adjacent 128-row
    // tiles sharing one B tile; this CTA (cluster rank 0 or 1) computes the
    // upper or lower one
    const int tiles_n = p.L / BN;
    const int tiles_m = p.L / kBM / (PAIR ? 2 : 1);
    const int per_leaf = tiles_m * tiles_n;
    const int rem = item % per_leaf;
    int row, col;
    if (p.band > 0 && p.band < tiles_n && tiles_n % p.band == 0) {
      // bands of p.band tile columns: the tiles that run at the same time
      // share fewer B panels (L2 reuse of a leaf's Y planes)
      const int per_band = tiles_m * p.band;
      const int w = rem % per_band;
      row = w / p.band;
      col = (rem / per_band) * p.band + w % p.band;
    } else {
      row = rem / tiles_n;
      col = rem % tiles_n;
    }
    it.tA = tmA;
    it.tB = tmB;
    it.tC = tmC;
    it.leaf = p.leaf_begin + item / per_leaf;
    it.P = p.P;
    it.m0 = PAIR ? (row * 2 + (int)rank) * kBM : row * kBM;
    it.n0 = col * BN;
    it.kblocks = p.L / BK;
    it.tg = p.ctab + (int64_t)it.leaf * p.maxT;
    it.nt = p.ccount[it.leaf];
    it.C = p.C;
    it.n = p.n;
    it.ldc = p.ldc;
    it.use_tma_c = p.use_tma_c;
  }
  it.sib = -1;
  it.parent = 0;
  it.valid = true;
  return it;
}

// Epilogue of one item on one CTA: the CTA's 128 x BN accumulator tile,
// TMEM columns acc_col .. acc_col + BN - 1, read 32 columns at a time by the
// four epilogue warps (warp quarter q holds TMEM lanes 32q .. 32q + 31).
// Combine (Alg. 5) fused here: the tile of leaf l is added, with its sign,
// into every C target of l.  Fast path: each warp stages its 32 x 32 fp32
// box (and its negation when a target needs it) in shared memory at `ebuf`
// with the 128-byte swizzle and issues one TMA bulk add-reduction per target
// (the add happens at L2).  Fallback (C not 16-byte addressable by TMA):
// signed vector atomics from registers.  With p.store_m the tile is stored
// to the leaf's M plane instead (deterministic, unfused combine).
template <int BN, bool INT1>
__device__ __forceinline__ void epilogue_item(const ItemInfo& it, const LeafTcArgs& p, uint32_t tmem_base,
                                              uint32_t acc_col, int quarter, int lane, uint32_t ebuf,
                                              uint64_t pol_c) {
  const int row_in_tile = quarter * 32 + lane;
  const int m0 = it.m0, n0 = it.n0, nt = it.nt;
  const CTarget* tg = it.tg;
  bool has_pos = false, has_neg = false;
  for (int t = 0; t < nt; ++t) (tg[t].sign > 0 ? has_pos : has_neg) = true;
  const bool vec_ok = ((reinterpret_cast<uintptr_t>(it.C) & 15) == 0) && ((it.ldc & 3) == 0);
  // sibling-folded combine: the previous sibling's stores and reductions
  // into the same parent boxes (issued by this lane) have completed
  if (it.sib >= 0 && lane == 0) bulk_wait_group<0>();
#pragma unroll 1
  for (int chunk = 0; chunk < BN / 32; ++chunk) {
    uint32_t r[32];
    tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(quarter * 32) << 16) + acc_col + (uint32_t)(chunk * 32), r);
    tmem_ld_wait();
    if constexpr (INT1) {
      // exact integers held in fp32: signed 64-bit adds into C (wrap mod
      // 2^64).  A whole, 16-byte-aligned row segment goes as one bulk
      // add-reduction of 256 bytes from this thread's slot of `ebuf`
      // (staged once per sign); ragged or unaligned segments use atomics.
      unsigned long long* Ci = reinterpret_cast<unsigned long long*>(it.C);
      const uint32_t slot = ebuf + (uint32_t)lane * 256u;
      const bool aligned = ((reinterpret_cast<uintptr_t>(it.C) & 15) == 0) && ((it.ldc & 1) == 0);
      int staged = 0;  // sign of the values in the slot (0: none)
#pragma unroll 1
      for (int t = 0; t < nt; ++t) {
        const CTarget c = tg[t];
        const int64_t grow = (int64_t)c.row_off + m0 + row_in_tile;
        const int64_t gcol = (int64_t)c.col_off + n0 + chunk * 32;
        if (grow >= it.n || gcol >= it.n) continue;
        unsigned long long* dst = Ci + grow * it.ldc + gcol;
        const int64_t lim = it.n - gcol;
        if (aligned && lim >= 32) {
          if (staged != c.sign) {
            bulk_wait_group_read<0>();  // the previous reduction has read the slot
#pragma unroll
            for (int w = 0; w < 16; ++w) {
              long long v0 = __float2ll_rn(__uint_as_float(r[2 * w]));
              long long v1 = __float2ll_rn(__uint_as_float(r[2 * w + 1]));
              if (c.sign < 0) {
                v0 = -v0;
                v1 = -v1;
              }
              asm volatile("st.shared.v2.u64 [%0], {%1, %2};" ::"r"(slot + 16u * (uint32_t)w), "l"(v0), "l"(v1)
                           : "memory");
            }
            fence_proxy_async_smem();
            staged = c.sign;
          }
          bulk_reduce_add_u64(dst, slot, 256u);
          bulk_commit_group();
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const long long v = __float2ll_rn(__uint_as_float(r[j]));
            if (j < lim && v != 0) atomicAdd(dst + j, (unsigned long long)(c.sign > 0 ? v : -v));
          }
        }
      }
      bulk_wait_group_read<0>();  // the slot is free for the next chunk
    } else if (it.sib >= 0) {
      // sibling-folded combine: the tile goes into the parent's quadrants
      // with the sign of W (a plain store from the first sibling of each
      // quadrant, add-reductions after it).  The same lane issues every
      // operation on these boxes, sibling after sibling; the wait at the
      // start of the item (below) orders them.
      if (lane == 0) bulk_wait_group_read<0>();
      __syncwarp();
      const bool any_neg = sib_coef(it.sib, 0) < 0 || sib_coef(it.sib, 1) < 0 || sib_coef(it.sib, 2) < 0 ||
                           sib_coef(it.sib, 3) < 0;
#pragma unroll
      for (int sg = 0; sg < 2; ++sg) {
        if (sg == 1 && !any_neg) continue;
        const uint32_t row_addr = ebuf + (uint32_t)sg * 4096u + (uint32_t)lane * 128u;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          float4 v = make_float4(__uint_as_float(r[4 * c]), __uint_as_float(r[4 * c + 1]),
                                 __uint_as_float(r[4 * c + 2]), __uint_as_float(r[4 * c + 3]));
          if (sg == 1) v = make_float4(-v.x, -v.y, -v.z, -v.w);
          const uint32_t addr = row_addr + ((uint32_t)(c ^ (lane & 7)) << 4);
          asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z),
                       "f"(v.w)
                       : "memory");
        }
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        const uint64_t keep = policy_evict_last();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int w = sib_coef(it.sib, q);
          if (w == 0) continue;
          const int32_t x = n0 + chunk * 32 + (q & 1) * p.L;
          const int32_t y = m0 + quarter * 32 + (q >> 1) * p.L;
          const uint64_t pol = it.sib == sib_last(q) ? pol_c : keep;
          if (it.sib == sib_first(q))
            tma_store_3d_hint(it.tC, x, y, it.parent, ebuf, pol);
          else
            tma_reduce_add_3d(it.tC, x, y, it.parent, ebuf + (w > 0 ? 0u : 4096u), pol);
        }
        bulk_commit_group();
      }
    } else if (p.store_m) {
      // unfused, deterministic combine: this leaf's tile goes to its M
      // plane (tmC maps the M planes here); the combine kernel adds later
      if (lane == 0) bulk_wait_group_read<0>();
      __syncwarp();
      const uint32_t row_addr = ebuf + (uint32_t)lane * 128u;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const uint32_t addr = row_addr + ((uint32_t)(c ^ (lane & 7)) << 4);
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(r[4 * c]), "r"(r[4 * c + 1]),
                     "r"(r[4 * c + 2]), "r"(r[4 * c + 3])
                     : "memory");
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        // the planes are read back only by the combine pass, after the whole
        // launch: evict-first keeps them from displacing operand panels in L2
        tma_store_3d_hint(it.tC, n0 + chunk * 32, m0 + quarter * 32, it.leaf - p.leaf_begin, ebuf, pol_c);
        bulk_commit_group();
      }
    } else if (it.use_tma_c) {
      if (lane == 0) bulk_wait_group_read<0>();  // the previous boxes have been read
      __syncwarp();
#pragma unroll
      for (int sg = 0; sg < 2; ++sg) {
        if (sg == 0 ? !has_pos : !has_neg) continue;
        const uint32_t row_addr = ebuf + (uint32_t)sg * 4096u + (uint32_t)lane * 128u;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          float4 v = make_float4(__uint_as_float(r[4 * c]), __uint_as_float(r[4 * c + 1]),
                                 __uint_as_float(r[4 * c + 2]), __uint_as_float(r[4 * c + 3]));
          if (sg == 1) v = make_float4(-v.x, -v.y, -v.z, -v.w);
          const uint32_t addr = row_addr + ((uint32_t)(c ^ (lane & 7)) << 4);
          asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z),
                       "f"(v.w)
                       : "memory");
        }
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        for (int t = 0; t < nt; ++t) {
          const CTarget c = tg[t];
          const int64_t y = (int64_t)c.row_off + m0 + quarter * 32;
          const int64_t x = (int64_t)c.col_off + n0 + chunk * 32;
          if (y >= it.n || x >= it.n) continue;
          tma_reduce_add_2d(it.tC, (int32_t)x, (int32_t)y, ebuf + (c.sign > 0 ? 0u : 4096u), pol_c);
        }
        bulk_commit_group();
      }
    } else {
#pragma unroll 1
      for (int t = 0; t < nt; ++t) {
        const CTarget c = tg[t];
        const int64_t grow = (int64_t)c.row_off + m0 + row_in_tile;
        const int64_t gcol = (int64_t)c.col_off + n0 + chunk * 32;
        if (grow >= it.n || gcol >= it.n) continue;
        float* dst = it.C + grow * it.ldc + gcol;
        const float sg = (float)c.sign;
        if (vec_ok && gcol + 32 <= it.n) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float4 v = make_float4(sg * __uint_as_float(r[4 * j]), sg * __uint_as_float(r[4 * j + 1]),
                                   sg * __uint_as_float(r[4 * j + 2]), sg * __uint_as_float(r[4 * j + 3]));
            atomicAdd(reinterpret_cast<float4*>(dst) + j, v);
          }
        } else {
          const int64_t lim = it.n - gcol;
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j < lim) atomicAdd(dst + j, sg * __uint_as_float(r[j]));
        }
      }
    }
  }
}

// One 32 x 32 fp32 box of a tile held in registers (the accumulator-promotion
// path: a warp holds 32 rows x 128 columns of the promoted sum), combined as
// epilogue_item does: stored to the leaf's M plane, added into C by TMA bulk
// reductions (the positive and the negative box one after the other through
// a single 4 KB staging box), or added by vector atomics.  col0: the box's
// first column within the tile.
__device__ __forceinline__ void epilogue_box_regs(const ItemInfo& it, const LeafTcArgs& p, const uint32_t (&r)[32],
                                                  int col0, int quarter, int lane, uint32_t ebuf, uint64_t pol_c,
                                                  bool has_pos, bool has_neg, bool vec_ok) {
  const int m0 = it.m0, n0 = it.n0, nt = it.nt;
  const CTarget* tg = it.tg;
  const uint32_t row_addr = ebuf + (uint32_t)lane * 128u;
  if (p.store_m) {
    if (lane == 0) bulk_wait_group_read<0>();  // the previous box has been read
    __syncwarp();
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const uint32_t addr = row_addr + ((uint32_t)(c ^ (lane & 7)) << 4);
      asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(r[4 * c]), "r"(r[4 * c + 1]),
                   "r"(r[4 * c + 2]), "r"(r[4 * c + 3])
                   : "memory");
    }
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) {
      tma_store_3d_hint(it.tC, n0 + col0, m0 + quarter * 32, it.leaf - p.leaf_begin, ebuf, pol_c);
      bulk_commit_group();
    }
  } else if (it.use_tma_c) {
#pragma unroll
    for (int sg = 0; sg < 2; ++sg) {
      if (sg == 0 ? !has_pos : !has_neg) continue;
      if (lane == 0) bulk_wait_group_read<0>();
      __syncwarp();
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        float4 v = make_float4(__uint_as_float(r[4 * c]), __uint_as_float(r[4 * c + 1]), __uint_as_float(r[4 * c + 2]),
                               __uint_as_float(r[4 * c + 3]));
        if (sg == 1) v = make_float4(-v.x, -v.y, -v.z, -v.w);
        const uint32_t addr = row_addr + ((uint32_t)(c ^ (lane & 7)) << 4);
        asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                     : "memory");
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        for (int t = 0; t < nt; ++t) {
          const CTarget c = tg[t];
          if ((c.sign > 0) != (sg == 0)) continue;
          const int64_t y = (int64_t)c.row_off + m0 + quarter * 32;
          const int64_t x = (int64_t)c.col_off + n0 + col0;
          if (y >= it.n || x >= it.n) continue;
          tma_reduce_add_2d(it.tC, (int32_t)x, (int32_t)y, ebuf, pol_c);
        }
        bulk_commit_group();
      }
    }
  } else {
    const int row_in_tile = quarter * 32 + lane;
#pragma unroll 1
    for (int t = 0; t < nt; ++t) {
      const CTarget c = tg[t];
      const int64_t grow = (int64_t)c.row_off + m0 + row_in_tile;
      const int64_t gcol = (int64_t)c.col_off + n0 + col0;
      if (grow >= it.n || gcol >= it.n) continue;
      float* dst = it.C + grow * it.ldc + gcol;
      const float sg = (float)c.sign;
      if (vec_ok && gcol + 32 <= it.n) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float4 v = make_float4(sg * __uint_as_float(r[4 * j]), sg * __uint_as_float(r[4 * j + 1]),
                                 sg * __uint_as_float(r[4 * j + 2]), sg * __uint_as_float(r[4 * j + 3]));
          atomicAdd(reinterpret_cast<float4*>(dst) + j, v);
        }
      } else {
        const int64_t lim = it.n - gcol;
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (j < lim) atomicAdd(dst + j, sg * __uint_as_float(r[j]));
      }
    }
  }
}

// Persistent launch of a leaf kernel on clusters of two CTAs: as many
// clusters as can be resident at once (at most one per SM pair), never more
// than there are work items (items > 0).
template <typename Kern>
cudaError_t launch_cta_pairs(Kern kern, int threads, int smem, int64_t items, int num_sms, cudaStream_t st,
                             const CUtensorMap& tmA, const CUtensorMap& tmB, const CUtensorMap& tmC,
                             const LeafTcArgs& a) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = num_sms / 2;
  cfg.gridDim = dim3((unsigned)(2 * clusters), 1, 1);
  int active = 0;
  if (cudaOccupancyMaxActiveClusters(&active, kern, &cfg) == cudaSuccess && active > 0 && active < clusters)
    clusters = active;
  cudaGetLastError();
  if (items < clusters) clusters = (int)items;
  cfg.gridDim = dim3((unsigned)(2 * clusters), 1, 1);
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, tmA, tmB, tmC, a);
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace stark
