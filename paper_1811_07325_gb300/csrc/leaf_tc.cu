// leaf_tc.cu -- the leaf products M_l = X_l * Y_l of every leaf (Alg. 4,
// "MulBlockMat") on the tcgen05 tensor cores, with the combine of Alg. 5
// fused into the epilogue: each finished accumulator tile is added, with its
// sign, into every C quadrant the leaf contributes to (the C targets of the
// quadrant-index table), so no M_l is ever written to memory.
//
// Operands come from the divide kernel as split planes: X = X_hi + X_lo,
// Y = Y_hi + Y_lo (bf16 halves, or tf32 halves in fp32 containers), and
//   M ~= X_lo Y_hi + X_hi Y_lo + X_hi Y_hi
// accumulates in fp32 in tensor memory (the lo*lo term is below fp32
// resolution of the result and is dropped).  X planes (M x K, row-major) are
// a K-major operand.  The Y planes stay row-major (K x N) and are an
// MN-major operand, loaded in 128-byte-wide N chunks (bf16: 128-byte
// swizzle; tf32: 128-byte swizzle of 32-byte atoms); the optional K-major
// tf32 layout transposes them to N x K beforehand.
//
// This is the single-CTA form: leaf sides that are not a multiple of 256,
// the 128-wide grouped launches of batches and the server, the exact int64
// leaves, and the opt-in schedules (single CTAs on 256-wide tiles, 64-byte
// rows).  Leaf sides that are multiples of 256 run on CTA pairs
// (leaf_tc2.cu).
//
// Persistent kernel, one CTA per SM, warp-specialised:
//   warp 0      TMA producer: per k-block, 4 tiles (X_hi, X_lo, Y_hi, Y_lo)
//               into a STAGES-deep shared-memory ring
//   warp 1      TMEM allocator + single-thread MMA issuer (3 MMAs per K=16
//               (bf16) or K=8 (tf32) step), double-buffered accumulators
//   warps 2..5  epilogue (leaf_common.cuh): tcgen05.ld the accumulator and
//               add it into C for every target of the leaf
// Every mbarrier wait is bounded; on expiry the kernel records an error,
// drains its in-flight copies and MMAs, frees TMEM and returns.
#include <cstring>

#include "leaf_common.cuh"

namespace stark {
namespace {

constexpr int kThreads = 192;

// RB: bytes of one swizzled smem row (128: K = 64 bf16 per stage; 64: K = 32
// bf16 per stage, twice the stages in the same space).
// INT1: one exact bf16 product per K step (integer leaf operands), no lo
// planes, int64 combine.
// TMN: tf32 with the Y planes row-major (K x N), read MN-major in 128-byte
// boxes with the 32-byte-atom swizzle (no transpose pass).
template <int BN, int STAGES, bool TF32, int RB = 128, bool INT1 = false, bool TMN = false>
struct TcCfg {
  static constexpr int ESZ = TF32 ? 4 : 2;
  static constexpr int BK = RB / ESZ;                // K per stage: one swizzled A row
  static constexpr int A_BYTES = kBM * RB;           // one operand half tile (K-major)
  static constexpr bool B_MN = !TF32 || TMN;         // B operand MN-major (bf16, tf32 TMN) or K-major
  static constexpr int B_SWZ = TF32 ? 1 : 0;         // MN descriptor swizzle (tf32: 32-byte atoms)
  static constexpr int W = B_MN ? RB / ESZ : BN;     // N elements per B TMA box
  static constexpr int NCHUNK = BN / W;              // B boxes per half tile
  static constexpr int CH_BYTES = B_MN ? BK * RB : BN * RB;  // bytes per B box
  static constexpr int B_BYTES = NCHUNK * CH_BYTES;  // == BN * RB
  static constexpr int NHALF = INT1 ? 1 : 2;         // operand planes per side (hi, lo)
  static constexpr int STAGE_BYTES = NHALF * (A_BYTES + B_BYTES);
  static constexpr int MMA_K = 32 / ESZ;             // K of one MMA (16 bf16 / 8 tf32)
  static constexpr int KSTEPS = BK / MMA_K;          // MMAs (x3) per stage
  static constexpr int A_KSTEP = 32;                 // bytes along a K-major row
  static constexpr int B_KSTEP = B_MN ? MMA_K * RB : 32;  // bytes per MMA K step in a B box
  static constexpr int TMEM_COLS = 2 * BN;           // two accumulators
  static constexpr int EPI_BYTES = 4 * 2 * 4096;     // per epilogue warp: a +/- pair of 32x32 fp32 boxes
  static constexpr int BAR_BYTES = 8 * (2 * STAGES + 4) + 16;
  static constexpr int SMEM = STAGES * STAGE_BYTES + EPI_BYTES + 1024 + BAR_BYTES;
  static constexpr uint32_t IDESC = make_idesc<kBM, BN, TF32, B_MN>();
};

template <int BN, int STAGES, bool TF32, bool GROUPED, int RB, bool INT1, bool TMN>
__global__ void __launch_bounds__(kThreads, 1)
    leaf_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmC, const LeafTcArgs p) {
  using Cfg = TcCfg<BN, STAGES, TF32, RB, INT1, TMN>;
  static_assert(!INT1 || (!TF32 && !GROUPED), "integer mode: bf16, single problem");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment for the 128-byte swizzle atoms
  const uint32_t raw_addr = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024 - (raw_addr & 1023)) & 1023);
  const uint32_t sbase = smem_u32(smem);
  const uint32_t epi_base = sbase + STAGES * Cfg::STAGE_BYTES;
  const uint32_t bar_base = epi_base + Cfg::EPI_BYTES;
  auto full_bar = [&](int s) { return bar_base + 8 * s; };
  auto empty_bar = [&](int s) { return bar_base + 8 * (STAGES + s); };
  auto accf_bar = [&](int a) { return bar_base + 8 * (2 * STAGES + a); };
  auto acce_bar = [&](int a) { return bar_base + 8 * (2 * STAGES + 2 + a); };
  uint32_t* tmem_slot =
      reinterpret_cast<uint32_t*>(smem + STAGES * Cfg::STAGE_BYTES + Cfg::EPI_BYTES + 8 * (2 * STAGES + 4));

  const int warp = threadIdx.x / 32;
  const int lane = threadIdx.x % 32;

  const uint32_t cta_rank = 0u;
  const int unit = (int)blockIdx.x;
  const int units = (int)gridDim.x;
  const int num_items = GROUPED ? p.total_items : (p.leaf_end - p.leaf_begin) * (p.L / kBM) * (p.L / BN);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(accf_bar(a), 1);
      mbar_init(acce_bar(a), 128);
    }
    fence_mbar_init();
    if (!GROUPED) {
      prefetch_tmap(&tmA);
      prefetch_tmap(&tmB);
      if (p.use_tma_c) prefetch_tmap(&tmC);
    }
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), Cfg::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      // L2 priorities: a leaf's B panels are re-read by every row of tiles,
      // so they should stay; A panels stream through once per row of tiles
      // X panels: reused by the tiles of one tile row, which run in the same
      // wave (LRU keeps them; an evict-first hint made each tile re-read its
      // panel from DRAM: 49.5 instead of 27.4 GB per launch at n = 16384);
      // Y panels: reused across the waves of a leaf, kept preferentially
      const uint64_t pol_a = policy_evict_normal();
      const uint64_t pol_b = policy_evict_last();
      int s = 0;
      uint32_t phase = 0;
      uint32_t armed = 0, armed_phase = 0;  // per-stage: ever armed / parity of last arming
      bool ok = true;
      for (int item = unit; ok && item < num_items; item += units) {
        const ItemInfo it = decode_item<BN, Cfg::BK, GROUPED, false>(item, p, &tmA, &tmB, &tmC, cta_rank);
        // plane of this leaf in the workspace (depth-first traversal keeps
        // one subtree's leaves, numbered from plane_base)
        const int leaf = GROUPED ? it.leaf : it.leaf - p.plane_base;
        const int m0 = it.m0, n0 = it.n0;
        for (int kb = 0; kb < it.kblocks; ++kb) {
          if (!mbar_wait_bounded(empty_bar(s), phase ^ 1, p.err, kDevTimeoutEmpty, p.timeout_ns)) {
            ok = false;
            break;
          }
          const uint32_t st = sbase + s * Cfg::STAGE_BYTES;
          mbar_arrive_expect_tx(full_bar(s), Cfg::STAGE_BYTES);
          const int k0 = kb * Cfg::BK;
          tma_load_3d(st, it.tA, k0, m0, leaf, full_bar(s), pol_a);
          if constexpr (!INT1) tma_load_3d(st + Cfg::A_BYTES, it.tA, k0, m0, it.P + leaf, full_bar(s), pol_a);
          if constexpr (Cfg::B_MN) {
#pragma unroll
            for (int c = 0; c < Cfg::NCHUNK; ++c) {
              tma_load_3d(st + Cfg::NHALF * Cfg::A_BYTES + c * Cfg::CH_BYTES, it.tB, n0 + c * Cfg::W, k0, leaf, full_bar(s),
                          pol_b);
              if constexpr (!INT1)
                tma_load_3d(st + Cfg::NHALF * Cfg::A_BYTES + Cfg::B_BYTES + c * Cfg::CH_BYTES, it.tB, n0 + c * Cfg::W,
                            k0, it.P + leaf, full_bar(s), pol_b);
            }
          } else {
            tma_load_3d(st + Cfg::NHALF * Cfg::A_BYTES, it.tB, k0, n0, leaf, full_bar(s), pol_b);
            tma_load_3d(st + Cfg::NHALF * Cfg::A_BYTES + Cfg::B_BYTES, it.tB, k0, n0, it.P + leaf, full_bar(s), pol_b);
          }
          armed |= 1u << s;
          armed_phase = (armed_phase & ~(1u << s)) | (phase << s);
          if (++s == STAGES) {
            s = 0;
            phase ^= 1;
          }
        }
      }
      if (!ok) {
        // let every copy already issued land before the CTA can exit
        for (int t = 0; t < STAGES; ++t)
          if (armed & (1u << t)) mbar_wait_bounded(full_bar(t), (armed_phase >> t) & 1, nullptr, 0, 200000000ull);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int s = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      bool ok = true;
      bool issued = false;
      for (int item = unit; ok && item < num_items; item += units) {
        const int kblocks = GROUPED ? decode_item<BN, Cfg::BK, GROUPED, false>(item, p, &tmA, &tmB, &tmC, cta_rank).kblocks
                                    : p.L / Cfg::BK;
        if (!mbar_wait_bounded(acce_bar(acc), acc_phase ^ 1, p.err, kDevTimeoutAccEmpty, p.timeout_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN);
        for (int kb = 0; kb < kblocks; ++kb) {
          if (!mbar_wait_bounded(full_bar(s), phase, p.err, kDevTimeoutFull, p.timeout_ns)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = sbase + s * Cfg::STAGE_BYTES;
#pragma unroll
          for (int k = 0; k < Cfg::KSTEPS; ++k) {
            const uint32_t aoff = k * Cfg::A_KSTEP, boff = k * Cfg::B_KSTEP;
            const uint64_t a_hi = smem_desc_k<RB>(st + aoff);
            const uint64_t a_lo = smem_desc_k<RB>(st + Cfg::A_BYTES + aoff);
            uint64_t b_hi, b_lo;
            if constexpr (Cfg::B_MN) {
              b_hi = smem_desc_mn<RB, Cfg::B_SWZ>(st + Cfg::NHALF * Cfg::A_BYTES + boff, Cfg::CH_BYTES);
              b_lo = smem_desc_mn<RB, Cfg::B_SWZ>(st + Cfg::NHALF * Cfg::A_BYTES + Cfg::B_BYTES + boff,
                                                  Cfg::CH_BYTES);
            } else {
              b_hi = smem_desc_k<RB>(st + Cfg::NHALF * Cfg::A_BYTES + boff);
              b_lo = smem_desc_k<RB>(st + Cfg::NHALF * Cfg::A_BYTES + Cfg::B_BYTES + boff);
            }
            const uint32_t first = (kb == 0 && k == 0) ? 0u : 1u;
            if constexpr (INT1) {
              mma_f16(d_tmem, a_hi, b_hi, Cfg::IDESC, first);
            } else if constexpr (TF32) {
              mma_tf32(d_tmem, a_lo, b_hi, Cfg::IDESC, first);
              mma_tf32(d_tmem, a_hi, b_lo, Cfg::IDESC, 1u);
              mma_tf32(d_tmem, a_hi, b_hi, Cfg::IDESC, 1u);
            } else {
              const uint32_t idesc = p.fp16 ? idesc_as_fp16(Cfg::IDESC) : Cfg::IDESC;  // fp16 or bf16 halves
              mma_f16(d_tmem, a_lo, b_hi, idesc, first);
              mma_f16(d_tmem, a_hi, b_lo, idesc, 1u);
              mma_f16(d_tmem, a_hi, b_hi, idesc, 1u);
            }
          }
          issued = true;
          mma_commit(empty_bar(s));  // stage free once these MMAs have read it
          if (++s == STAGES) {
            s = 0;
            phase ^= 1;
          }
        }
        if (!ok) break;
        mma_commit(accf_bar(acc));  // accumulator complete
        if (++acc == 2) {
          acc = 0;
          acc_phase ^= 1;
        }
      }
      if (!ok && issued) {
        // Let the MMAs in flight finish before TMEM is released: commit to
        // the accumulator-full barrier of the current buffer (whose pending
        // phase has parity acc_phase) and wait for that phase, briefly.
        mma_commit(accf_bar(acc));
        mbar_wait_bounded(accf_bar(acc), acc_phase, nullptr, 0, 200000000ull);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // (combine fused: epilogue_item adds each finished tile into its C targets)
    const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
    const uint32_t ebuf = epi_base + (uint32_t)(warp - 2) * 8192u;  // [+ box][- box]
    const uint64_t pol_c = policy_evict_first();  // C lines: add and move on
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int item = unit; item < num_items; item += units) {
      if (!mbar_wait_bounded(accf_bar(acc), acc_phase, p.err, kDevTimeoutAccFull, p.timeout_ns)) break;
      tc_fence_after();
      const ItemInfo it = decode_item<BN, Cfg::BK, GROUPED, false>(item, p, &tmA, &tmB, &tmC, cta_rank);
      epilogue_item<BN, INT1>(it, p, tmem_base, (uint32_t)(acc * BN), quarter, lane, ebuf, pol_c);
      tc_fence_before();
      mbar_arrive(acce_bar(acc));
      if (++acc == 2) {
        acc = 0;
        acc_phase ^= 1;
      }
    }
    // every bulk reduction issued by this warp completes before the CTA exits
    // (each lane waits for its own; lanes that issued none return at once)
    bulk_wait_group<0>();
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem_base, Cfg::TMEM_COLS);
}

template <int BN, int STAGES, bool TF32, bool GROUPED, int RB = 128, bool INT1 = false, bool TMN = false>
cudaError_t launch_cfg(const LeafTcArgs& a, const CUtensorMap* tmA, const CUtensorMap* tmB, const CUtensorMap* tmC,
                       int num_sms, cudaStream_t st) {
  using Cfg = TcCfg<BN, STAGES, TF32, RB, INT1, TMN>;
  static_assert(Cfg::B_BYTES == BN * RB, "B tile size");
  int64_t items;
  if constexpr (GROUPED) {
    items = a.total_items;
    if (!a.groups || a.ngroups <= 0) return cudaErrorInvalidValue;
  } else {
    if (a.L % kBM != 0 || a.L % BN != 0 || a.L % Cfg::BK != 0) return cudaErrorInvalidValue;
    items = (int64_t)(a.leaf_end - a.leaf_begin) * (a.L / kBM) * (a.L / BN);
  }
  auto kern = leaf_tc_kernel<BN, STAGES, TF32, GROUPED, RB, INT1, TMN>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
  if (e != cudaSuccess) return e;
  if (items <= 0) return cudaSuccess;
  if (items > 0x7FFFFFFF) return cudaErrorInvalidValue;
  const int grid = (int)(items < num_sms ? items : num_sms);
  kern<<<grid, kThreads, Cfg::SMEM, st>>>(*tmA, *tmB, *tmC, a);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_leaf_tc(const LeafTcArgs& a, const CUtensorMap* tmA, const CUtensorMap* tmB,
                           const CUtensorMap* tmC, bool tf32, int bn, int num_sms, cudaStream_t st) {
  // bf16, 256-wide tiles, 64-byte rows: four 48 KB stages instead of two 96 KB
  if (bn == 256 && !tf32 && a.row_bytes == 64)
    return launch_cfg<256, 4, false, false, 64>(a, tmA, tmB, tmC, num_sms, st);
  if (tf32 && a.b_mn) {
    if (bn == 256) return launch_cfg<256, 2, true, false, 128, false, true>(a, tmA, tmB, tmC, num_sms, st);
    if (bn == 128) return launch_cfg<128, 3, true, false, 128, false, true>(a, tmA, tmB, tmC, num_sms, st);
    return cudaErrorInvalidValue;
  }
  if (bn == 256) {
    return tf32 ? launch_cfg<256, 2, true, false>(a, tmA, tmB, tmC, num_sms, st)
                : launch_cfg<256, 2, false, false>(a, tmA, tmB, tmC, num_sms, st);
  }
  if (bn == 128) {
    return tf32 ? launch_cfg<128, 3, true, false>(a, tmA, tmB, tmC, num_sms, st)
                : launch_cfg<128, 3, false, false>(a, tmA, tmB, tmC, num_sms, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_leaf_tc_int(const LeafTcArgs& a, const CUtensorMap* tmA, const CUtensorMap* tmB, int bn,
                               int num_sms, cudaStream_t st) {
  CUtensorMap none;
  memset(&none, 0, sizeof(none));
  if (bn == 256) return launch_cfg<256, 4, false, false, 128, true>(a, tmA, tmB, &none, num_sms, st);
  if (bn == 128) return launch_cfg<128, 6, false, false, 128, true>(a, tmA, tmB, &none, num_sms, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_leaf_tc_grouped(const LeafTcArgs& a, bool tf32, int bn, int num_sms, cudaStream_t st) {
  // 256-wide members run on CTA pairs (launch_leaf_tc2_grouped)
  CUtensorMap none;
  memset(&none, 0, sizeof(none));
  if (bn == 128) {
    if (tf32 && a.b_mn) return launch_cfg<128, 3, true, true, 128, false, true>(a, &none, &none, &none, num_sms, st);
    return tf32 ? launch_cfg<128, 3, true, true>(a, &none, &none, &none, num_sms, st)
                : launch_cfg<128, 3, false, true>(a, &none, &none, &none, num_sms, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace stark
