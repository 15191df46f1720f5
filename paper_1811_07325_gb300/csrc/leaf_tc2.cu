// leaf_tc2.cu -- the 3xBF16 / 3xTF32 leaf products (Alg. 4) with the fused
// combine (Alg. 5) on CTA pairs: the two CTAs of a cluster share one cta_group::2
// tcgen05 MMA of 256 x 256 per K step.  Each CTA stages its own 128 rows of
// the X tile and its own 128 columns of the Y tile, so one CTA holds 64 KB
// per pipeline stage instead of the 96 KB a single-CTA 128 x 256 tile needs
// for the same arithmetic, and three stages fit where two did.
//
// Roles (both CTAs run all four, the MMA issuer only acts in the even CTA):
//   warp 0      TMA producer: X_hi, X_lo rows and Y_hi, Y_lo column chunks of
//               this CTA into its ring; the byte counts of both CTAs go to
//               the even CTA's full barrier (cta_group::2 loads)
//   warp 1      TMEM allocation for the pair (cta_group::2); in the even CTA
//               the single-thread issuer of the pair MMAs, whose commits
//               free the stage in both CTAs and announce the accumulator to
//               both CTAs' epilogues
//   warps 2..5  epilogue of this CTA's 128 accumulator rows (shared with the
//               single-CTA kernel); each warp reports the drained accumulator
//               to the even CTA's accumulator-empty barrier
// Every wait is bounded as in the single-CTA kernel; on expiry the kernel
// records an error, lets its copies and MMAs in flight land, frees TMEM and
// returns.
#include <cstring>

#include "leaf_common.cuh"

namespace stark {
namespace {

constexpr int kThreads2 = 192;

// Y tile layouts: bf16 and tf32 with TMN (the default) keep the Y planes
// row-major and read them MN-major in 128-byte-wide column boxes (bf16:
// 128-byte swizzle; tf32: 128-byte swizzle of 32-byte atoms); tf32 without
// TMN reads planes transposed to N x K beforehand, K-major like X (one
// 128-row box per half tile).
template <bool TF32, bool TMN = false>
struct Tc2Cfg {
  static constexpr int ESZ = TF32 ? 4 : 2;
  static constexpr int RB = 128;                        // bytes of one swizzled smem row
  static constexpr int BK = RB / ESZ;                   // K per stage (64 bf16 / 32 tf32)
  static constexpr int BN = 256;                        // N of the pair MMA (accumulator columns)
  static constexpr int BNH = BN / 2;                    // Y columns staged by each CTA
  static constexpr int A_BYTES = kBM * RB;              // one X half tile (K-major), 16 KB
  static constexpr bool B_MN = !TF32 || TMN;
  static constexpr int B_SWZ = TF32 ? 1 : 0;            // MN descriptor swizzle (tf32: 32-byte atoms)
  static constexpr int W = B_MN ? RB / ESZ : BNH;       // Y columns per TMA box
  static constexpr int NCHUNK = BNH / W;                // Y boxes per half tile
  static constexpr int CH_BYTES = B_MN ? BK * RB : BNH * RB;
  static constexpr int B_BYTES = NCHUNK * CH_BYTES;     // one Y half tile, 16 KB
  static constexpr int STAGES = 3;
  static constexpr int STAGE_BYTES = 2 * (A_BYTES + B_BYTES);  // hi and lo: 64 KB
  static constexpr int MMA_K = 32 / ESZ;                // K of one MMA (16 bf16 / 8 tf32)
  static constexpr int KSTEPS = BK / MMA_K;
  static constexpr int A_KSTEP = 32;                    // bytes along a K-major row
  static constexpr int B_KSTEP = B_MN ? MMA_K * RB : 32;
  static constexpr int TMEM_COLS = 2 * BN;              // two accumulators
  static constexpr int EPI_BYTES = 4 * 2 * 4096;
  static constexpr int BAR_BYTES = 8 * (2 * STAGES + 4) + 16;
  static constexpr int SMEM = STAGES * STAGE_BYTES + EPI_BYTES + 1024 + BAR_BYTES;
  static constexpr uint32_t IDESC = make_idesc<2 * kBM, BN, TF32, B_MN>();
  static_assert(B_BYTES == BNH * RB, "Y half tile");
  static_assert(SMEM <= 232448, "shared memory per CTA");
};

// Accumulator promotion (LeafTcArgs::promo_kb): a tile's K range is cut
// into chunks of promo_kb K blocks, each accumulated by the tensor core from
// zero in one of the CTA's two TMEM accumulators, which alternate from chunk
// to chunk as they alternate from tile to tile otherwise.  Eight epilogue
// warps (two per TMEM lane quarter, one per 128-column half) load each
// chunk and add it into a running fp32 sum held in their registers (round
// to nearest, chunk 0 first), release the accumulator, and after the last
// chunk combine the sum from registers.  The tensor core's own accumulation
// so spans promo_kb K blocks instead of the whole leaf side, and the MMAs
// never wait for the additions: the next chunk goes to the other
// accumulator.
constexpr int kThreads2P = 320;  // with promotion: producer, MMA, 8 epilogue warps

// GROUPED: items of several problems (GroupDesc array, tensor maps in global
// memory), as in the single-CTA kernel's grouped mode.  SIB: sibling-major
// item order with the sibling-folded combine (LeafTcArgs::sib).  PROMO:
// accumulator promotion (above; one problem, not with SIB).
template <bool TF32, bool GROUPED, bool TMN, bool SIB, bool PROMO = false>
__global__ void __launch_bounds__(PROMO ? kThreads2P : kThreads2, 1)
    leaf_tc2_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const __grid_constant__ CUtensorMap tmC, const LeafTcArgs p) {
  using Cfg = Tc2Cfg<TF32, TMN>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024 - (raw_addr & 1023)) & 1023);
  const uint32_t sbase = smem_u32(smem);
  const uint32_t epi_base = sbase + Cfg::STAGES * Cfg::STAGE_BYTES;
  const uint32_t bar_base = epi_base + Cfg::EPI_BYTES;
  auto full_bar = [&](int s) { return bar_base + 8 * s; };
  auto empty_bar = [&](int s) { return bar_base + 8 * (Cfg::STAGES + s); };
  auto accf_bar = [&](int a) { return bar_base + 8 * (2 * Cfg::STAGES + a); };
  auto acce_bar = [&](int a) { return bar_base + 8 * (2 * Cfg::STAGES + 2 + a); };
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + Cfg::STAGES * Cfg::STAGE_BYTES + Cfg::EPI_BYTES +
                                                    8 * (2 * Cfg::STAGES + 4));

  const int warp = threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  const uint32_t rank = cluster_ctarank();
  const bool leader = rank == 0;
  const int unit = (int)(blockIdx.x >> 1);
  const int units = (int)(gridDim.x >> 1);
  const int num_items = GROUPED ? p.total_items
                        : SIB   ? (int)sib_items(p, Cfg::BN, units)
                                : (p.leaf_end - p.leaf_begin) * (p.L / (2 * kBM)) * (p.L / Cfg::BN);
  auto decode = [&](int item) {
    if constexpr (SIB)
      return decode_sib<Cfg::BN, Cfg::BK>(item, p, &tmA, &tmB, &tmC, rank, units);
    else
      return decode_item<Cfg::BN, Cfg::BK, GROUPED, true>(item, p, &tmA, &tmB, &tmC, rank);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::STAGES; ++s) {
      mbar_init(full_bar(s), 1);   // even CTA: its producer's arrive + both CTAs' bytes
      mbar_init(empty_bar(s), 1);  // the pair MMA commit
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(accf_bar(a), 1);
      mbar_init(acce_bar(a), PROMO ? 16 : 8);  // even CTA: the epilogue warps of each CTA
    }
    fence_mbar_init();
    if (!GROUPED) {
      prefetch_tmap(&tmA);
      prefetch_tmap(&tmB);
      if (p.use_tma_c || p.store_m || SIB) prefetch_tmap(&tmC);
    }
  }
  if (warp == 1) {
    tmem_alloc2(smem_u32(tmem_slot), Cfg::TMEM_COLS);
    tmem_relinquish2();
  }
  tc_fence_before();
  cluster_sync();  // barriers of both CTAs initialised, TMEM address published
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      // X panels: reused by the tiles of one tile row, which run in the same
      // wave (LRU keeps them; an evict-first hint made each tile re-read its
      // panel from DRAM: 49.5 instead of 27.4 GB per launch at n = 16384);
      // Y panels: reused across the waves of a leaf, kept preferentially
      const uint64_t pol_a = policy_evict_normal();
      const uint64_t pol_b = policy_evict_last();
      int s = 0;
      uint32_t phase = 0;
      uint32_t armed = 0, armed_phase = 0;
      bool ok = true;
      for (int item = unit; ok && item < num_items; item += units) {
        const ItemInfo it = decode(item);
        if (!it.valid) continue;
        const int leaf = GROUPED ? it.leaf : it.leaf - p.plane_base;  // workspace plane
        const int m0 = it.m0;                                 // this CTA's 128 rows
        const int nb = it.n0 + (int)rank * Cfg::BNH;          // this CTA's 128 columns
        for (int kb = 0; kb < it.kblocks; ++kb) {
          if (!mbar_wait_bounded(empty_bar(s), phase ^ 1, p.err, kDevTimeoutEmpty, p.timeout_ns)) {
            ok = false;
            break;
          }
          const uint32_t st = sbase + s * Cfg::STAGE_BYTES;
          const uint32_t fb = mapa_shared(full_bar(s), 0);
          if (leader) mbar_arrive_expect_tx(full_bar(s), 2 * Cfg::STAGE_BYTES);
          const int k0 = kb * Cfg::BK;
          tma_load_3d_cg2(st, it.tA, k0, m0, leaf, fb, pol_a);
          tma_load_3d_cg2(st + Cfg::A_BYTES, it.tA, k0, m0, it.P + leaf, fb, pol_a);
          if constexpr (Cfg::B_MN) {
#pragma unroll
            for (int c = 0; c < Cfg::NCHUNK; ++c) {
              tma_load_3d_cg2(st + 2 * Cfg::A_BYTES + c * Cfg::CH_BYTES, it.tB, nb + c * Cfg::W, k0, leaf, fb, pol_b);
              tma_load_3d_cg2(st + 2 * Cfg::A_BYTES + Cfg::B_BYTES + c * Cfg::CH_BYTES, it.tB, nb + c * Cfg::W, k0,
                              it.P + leaf, fb, pol_b);
            }
          } else {
            tma_load_3d_cg2(st + 2 * Cfg::A_BYTES, it.tB, k0, nb, leaf, fb, pol_b);
            tma_load_3d_cg2(st + 2 * Cfg::A_BYTES + Cfg::B_BYTES, it.tB, k0, nb, it.P + leaf, fb, pol_b);
          }
          armed |= 1u << s;
          armed_phase = (armed_phase & ~(1u << s)) | (phase << s);
          if (++s == Cfg::STAGES) {
            s = 0;
            phase ^= 1;
          }
        }
      }
      if (!ok) {
        // copies already issued land before the pair can leave: the even CTA
        // waits on its armed barriers, the odd one (whose copies report to the
        // even CTA) gives them time
        if (leader) {
          for (int t = 0; t < Cfg::STAGES; ++t)
            if (armed & (1u << t)) mbar_wait_bounded(full_bar(t), (armed_phase >> t) & 1, nullptr, 0, 200000000ull);
        } else {
          spin_ns(2000000ull);
        }
      } else {
        // every commit still owed to this CTA's empty barriers lands before exit
        for (int t = 0; t < Cfg::STAGES; ++t) {
          if (!mbar_wait_bounded(empty_bar(s), phase ^ 1, p.err, kDevTimeoutEmpty, p.timeout_ns)) break;
          if (++s == Cfg::STAGES) {
            s = 0;
            phase ^= 1;
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (leader && lane == 0) {
      int s = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      bool ok = true;
      bool issued = false;
      // K blocks [kb0, kb1) of the current item into the accumulator at
      // d_tmem (the first one overwrites it); false when a wait expired
      auto run_kblocks = [&](uint32_t d_tmem, int kb0, int kb1) -> bool {
        for (int kb = kb0; kb < kb1; ++kb) {
          if (!mbar_wait_bounded(full_bar(s), phase, p.err, kDevTimeoutFull, p.timeout_ns)) return false;
          tc_fence_after();
          const uint32_t st = sbase + s * Cfg::STAGE_BYTES;
#pragma unroll
          for (int k = 0; k < Cfg::KSTEPS; ++k) {
            const uint32_t aoff = k * Cfg::A_KSTEP, boff = k * Cfg::B_KSTEP;
            const uint64_t a_hi = smem_desc_k<Cfg::RB>(st + aoff);
            const uint64_t a_lo = smem_desc_k<Cfg::RB>(st + Cfg::A_BYTES + aoff);
            uint64_t b_hi, b_lo;
            if constexpr (Cfg::B_MN) {
              b_hi = smem_desc_mn<Cfg::RB, Cfg::B_SWZ>(st + 2 * Cfg::A_BYTES + boff, Cfg::CH_BYTES);
              b_lo = smem_desc_mn<Cfg::RB, Cfg::B_SWZ>(st + 2 * Cfg::A_BYTES + Cfg::B_BYTES + boff, Cfg::CH_BYTES);
            } else {
              b_hi = smem_desc_k<Cfg::RB>(st + 2 * Cfg::A_BYTES + boff);
              b_lo = smem_desc_k<Cfg::RB>(st + 2 * Cfg::A_BYTES + Cfg::B_BYTES + boff);
            }
            const uint32_t first = (kb == kb0 && k == 0) ? 0u : 1u;
            if constexpr (TF32) {
              mma2_tf32(d_tmem, a_lo, b_hi, Cfg::IDESC, first);
              mma2_tf32(d_tmem, a_hi, b_lo, Cfg::IDESC, 1u);
              mma2_tf32(d_tmem, a_hi, b_hi, Cfg::IDESC, 1u);
            } else {
              const uint32_t idesc = p.fp16 ? idesc_as_fp16(Cfg::IDESC) : Cfg::IDESC;  // fp16 or bf16 halves
              mma2_f16(d_tmem, a_lo, b_hi, idesc, first);
              mma2_f16(d_tmem, a_hi, b_lo, idesc, 1u);
              mma2_f16(d_tmem, a_hi, b_hi, idesc, 1u);
            }
          }
          issued = true;
          mma2_commit_mc(empty_bar(s), 0x3);  // the stage is free in both CTAs
          if (++s == Cfg::STAGES) {
            s = 0;
            phase ^= 1;
          }
        }
        return true;
      };
      if constexpr (PROMO) {
        // the two accumulators alternate over the chunks of every item
        const int kblocks = p.L / Cfg::BK, ck = p.promo_kb;
        for (int item = unit; ok && item < num_items; item += units) {
          for (int kc = 0; kc < kblocks; kc += ck) {
            if (!mbar_wait_bounded_cluster(acce_bar(acc), acc_phase ^ 1, p.err, kDevTimeoutAccEmpty, p.timeout_ns)) {
              ok = false;
              break;
            }
            tc_fence_after();
            if (!run_kblocks(tmem_base + (uint32_t)(acc * Cfg::BN), kc, kc + ck < kblocks ? kc + ck : kblocks)) {
              ok = false;
              break;
            }
            mma2_commit_mc(accf_bar(acc), 0x3);  // this chunk is complete in both CTAs
            if (++acc == 2) {
              acc = 0;
              acc_phase ^= 1;
            }
          }
        }
        if (!ok && issued) {
          mma2_commit_mc(accf_bar(acc), 0x1);
          mbar_wait_bounded(accf_bar(acc), acc_phase, nullptr, 0, 200000000ull);
        }
      } else {
        for (int item = unit; ok && item < num_items; item += units) {
          if (SIB && !decode(item).valid) continue;
          const int kblocks = GROUPED ? decode(item).kblocks : p.L / Cfg::BK;
          // both CTAs' epilogues have drained this accumulator
          if (!mbar_wait_bounded_cluster(acce_bar(acc), acc_phase ^ 1, p.err, kDevTimeoutAccEmpty, p.timeout_ns)) {
            ok = false;
            break;
          }
          tc_fence_after();
          if (!run_kblocks(tmem_base + (uint32_t)(acc * Cfg::BN), 0, kblocks)) {
            ok = false;
            break;
          }
          mma2_commit_mc(accf_bar(acc), 0x3);  // both halves of the accumulator complete
          if (++acc == 2) {
            acc = 0;
            acc_phase ^= 1;
          }
        }
        if (!ok && issued) {
          // MMAs in flight finish before TMEM is released (own barrier only)
          mma2_commit_mc(accf_bar(acc), 0x1);
          mbar_wait_bounded(accf_bar(acc), acc_phase, nullptr, 0, 200000000ull);
        }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
    const uint32_t ebuf = epi_base + (uint32_t)(warp - 2) * 8192u;
    const uint64_t pol_c = policy_evict_first();
    if constexpr (PROMO) {
      // warps 2..9: lane quarter warp % 4, columns (warp - 2) / 4 * 128 + 0..127
      const int half = (warp - 2) >> 2;
      const uint32_t pbuf = epi_base + (uint32_t)(warp - 2) * 4096u;  // one 32 x 32 fp32 box
      const uint32_t lane_base = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 128);
      const int kblocks = p.L / Cfg::BK, ck = p.promo_kb;
      const int nch = (kblocks + ck - 1) / ck;
      int acc = 0;
      uint32_t acc_phase = 0;
      bool ok = true;
      for (int item = unit; ok && item < num_items; item += units) {
        float run[128];
        for (int c = 0; c < nch; ++c) {
          if (!mbar_wait_bounded(accf_bar(acc), acc_phase, p.err, kDevTimeoutAccFull, p.timeout_ns)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t col = lane_base + (uint32_t)(acc * Cfg::BN);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            uint32_t r[16];
            tmem_ld_32x32b_x16(col + (uint32_t)(j * 16), r);
            tmem_ld_wait();
#pragma unroll
            for (int e = 0; e < 16; ++e)
              run[j * 16 + e] = c == 0 ? __uint_as_float(r[e]) : __fadd_rn(run[j * 16 + e], __uint_as_float(r[e]));
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive_cluster(mapa_shared(acce_bar(acc), 0));  // the chunk is in registers
          if (++acc == 2) {
            acc = 0;
            acc_phase ^= 1;
          }
        }
        if (!ok) break;
        const ItemInfo it = decode(item);  // (after the chunks: its registers are not live while they add)
        bool has_pos = false, has_neg = false;
        for (int t = 0; t < it.nt; ++t) (it.tg[t].sign > 0 ? has_pos : has_neg) = true;
        const bool vec_ok = ((reinterpret_cast<uintptr_t>(it.C) & 15) == 0) && ((it.ldc & 3) == 0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          uint32_t r[32];
#pragma unroll
          for (int e = 0; e < 32; ++e) r[e] = __float_as_uint(run[j * 32 + e]);
          epilogue_box_regs(it, p, r, half * 128 + j * 32, quarter, lane, pbuf, pol_c, has_pos, has_neg, vec_ok);
        }
      }
    } else {
      int acc = 0;
      uint32_t acc_phase = 0;
      for (int item = unit; item < num_items; item += units) {
        const ItemInfo it = decode(item);
        if (!it.valid) continue;
        if (!mbar_wait_bounded(accf_bar(acc), acc_phase, p.err, kDevTimeoutAccFull, p.timeout_ns)) break;
        tc_fence_after();
        epilogue_item<Cfg::BN, false>(it, p, tmem_base, (uint32_t)(acc * Cfg::BN), quarter, lane, ebuf, pol_c);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(mapa_shared(acce_bar(acc), 0));
        if (++acc == 2) {
          acc = 0;
          acc_phase ^= 1;
        }
      }
    }
    bulk_wait_group<0>();  // each lane's own bulk reductions
  }

  tc_fence_before();
  cluster_sync();  // both CTAs done with TMEM, shared memory and barriers
  tc_fence_after();
  if (warp == 1) tmem_dealloc2(tmem_base, Cfg::TMEM_COLS);
  cluster_sync();
}

template <bool TF32, bool GROUPED, bool TMN = false, bool SIB = false, bool PROMO = false>
cudaError_t launch2(const LeafTcArgs& a, const CUtensorMap* tmA, const CUtensorMap* tmB, const CUtensorMap* tmC,
                    int num_sms, cudaStream_t st) {
  using Cfg = Tc2Cfg<TF32, TMN>;
  auto kern = leaf_tc2_kernel<TF32, GROUPED, TMN, SIB, PROMO>;
  if (PROMO && a.promo_kb <= 0) return cudaErrorInvalidValue;
  int64_t items;
  if constexpr (GROUPED) {
    if (!a.groups || a.ngroups <= 0) return cudaErrorInvalidValue;
    items = a.total_items;
  } else {
    if (SIB && (a.leaf_begin % 7 != 0 || (a.leaf_end - a.leaf_begin) % 7 != 0)) return cudaErrorInvalidValue;
    // (sibling-major: the padded item count follows the pairs launched; the
    // kernel derives it, and any count >= the pairs gives the same launch)
    items = (int64_t)(a.leaf_end - a.leaf_begin) * (a.L / (2 * kBM)) * (a.L / Cfg::BN);
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
  if (e != cudaSuccess) return e;
  if (items <= 0) return cudaSuccess;
  if (items > 0x7FFFFFFF) return cudaErrorInvalidValue;
  return launch_cta_pairs(kern, PROMO ? kThreads2P : kThreads2, Cfg::SMEM, items, num_sms, st, *tmA, *tmB, *tmC, a);
}

}  // namespace

// Leaf sides the pair kernel tiles exactly (both dtypes: 256-row pair tiles,
// 256 columns, whole K blocks).
bool leaf_tc2_fits(const LeafTcArgs& a) { return a.L % 256 == 0; }

cudaError_t launch_leaf_tc2(const LeafTcArgs& a, const CUtensorMap* tmA, const CUtensorMap* tmB,
                            const CUtensorMap* tmC, bool tf32, int num_sms, cudaStream_t st) {
  if (!leaf_tc2_fits(a)) return cudaErrorInvalidValue;
  if (a.promo_kb > 0) {
    // accumulator promotion: bf16 and MN-major tf32, not with the sibling fold
    if (a.sib || (tf32 && !a.b_mn)) return cudaErrorInvalidValue;
    return tf32 ? launch2<true, false, true, false, true>(a, tmA, tmB, tmC, num_sms, st)
                : launch2<false, false, false, false, true>(a, tmA, tmB, tmC, num_sms, st);
  }
  if (a.sib) {
    if (tf32 && !a.b_mn) return cudaErrorInvalidValue;  // sibling fold: bf16 and MN-major tf32 only
    return tf32 ? launch2<true, false, true, true>(a, tmA, tmB, tmC, num_sms, st)
                : launch2<false, false, false, true>(a, tmA, tmB, tmC, num_sms, st);
  }
  if (tf32 && a.b_mn) return launch2<true, false, true>(a, tmA, tmB, tmC, num_sms, st);
  return tf32 ? launch2<true, false>(a, tmA, tmB, tmC, num_sms, st)
              : launch2<false, false>(a, tmA, tmB, tmC, num_sms, st);
}

cudaError_t launch_leaf_tc2_grouped(const LeafTcArgs& a, bool tf32, int num_sms, cudaStream_t st) {
  CUtensorMap none;
  memset(&none, 0, sizeof(none));
  if (tf32 && a.b_mn) return launch2<true, true, true>(a, &none, &none, &none, num_sms, st);
  return tf32 ? launch2<true, true>(a, &none, &none, &none, num_sms, st)
              : launch2<false, true>(a, &none, &none, &none, num_sms, st);
}

}  // namespace stark
