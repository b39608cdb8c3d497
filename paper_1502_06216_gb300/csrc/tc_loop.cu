// tc_loop.cu -- the scaling loop as one persistent tensor-core kernel per chunk
// of (odd, even) pairs.
//
// The four passes of a pair (see tc_gemm.cu: K_x and K_y contractions of a and
// b with the b-update + residual and the prox + a-update epilogues) depend on
// each other through whole images, so a pair needs a grid-wide barrier between
// passes.  Launched one kernel per pass, every pass pays a launch, the CTA
// set-up (barriers, TMEM allocation, descriptor fetch) and a cold operand
// pipeline, and the next pass cannot start early: a CTA holds ~200 KB of
// shared memory, so no CTA of the next kernel fits beside it on an SM.
//
// Here one cooperative launch with one CTA per SM runs up to `pairs` pairs:
//   * warp 16 (one lane) is the TMA producer, warp 17 (one lane) issues
//     tcgen05.mma, warps 0-15 drain TMEM through the epilogue;
//   * a CTA takes the tiles blockIdx.x, blockIdx.x + G, ... of every pass;
//   * between passes the epilogue warps meet every other CTA at a grid
//     barrier: one release-add on a 64-bit arrival counter in Ctrl that never
//     resets within a step (barrier b is complete at G b arrivals) and a
//     bounded acquire poll; a CTA that met NaN/Inf or gave up a wait sets the
//     flag slot of that barrier, and every CTA reads the slot after the
//     barrier and acts on it at the next one, so all stop at the same pass;
//   * before the barrier the producer has already loaded what does not depend
//     on the previous pass: the Gibbs-factor K-blocks of its next tile (only
//     the MMA reads them) and the epilogue tiles (q and e^{-sigma w} are fixed
//     during the step; the old b is this CTA's own tile), so after it only the
//     image K-blocks remain to be fetched;
//   * the stop rule (Sec. 3.4) uses the per-tile residual partials of the
//     b-update pass, added in a fixed order by every CTA while pass 2 (the
//     x-contraction of xi b) runs, and takes effect at the barrier before the
//     prox pass: when it fires, pass 2 has only rewritten the intermediate
//     image, and p, a, b are those of the pair the residual belongs to.
// The arithmetic of each tile is that of tc_pass_kernel with 64-wide tiles,
// so the two forms give the same bits when the per-pass form also uses them.
#include "tc_common.cuh"

namespace jko {

namespace {

constexpr int LBN = 64;                      // output tile width of every pass
constexpr int EK_CROWD_PLAIN = 3;            // EK_CROWD, scalar kappa, no mask or binary
constexpr int NEPI = 512;                    // epilogue threads: 16 warps, 4 per TMEM quadrant
constexpr int NTL = NEPI + 64;               // + producer warp + MMA warp
constexpr int WARP_PROD = 16;
constexpr int WARP_MMA = 17;
constexpr int EPI_BAR = 1;                   // named barrier of the epilogue warps
constexpr uint32_t LOOP_SMEM_BUDGET = 224 * 1024;
constexpr uint32_t kGoSpinLimit = 1u << 27;

// Resident-factor mode (BF16, one tile per CTA, the same 1-D factor in every
// pass): the CTA keeps its band of at most RES_KB factor K-blocks in shared
// memory for the whole launch and streams only image K-blocks.
constexpr int RES_KB = 8;
constexpr int RES_STAGES = 4;

// output staging tile (operand type: hi + lo, or one tf32 tile of the same
// bytes) and epilogue region: q | old b in the b-update pass, e^{-sigma w} | p
// in the prox pass (two fp32 tiles).  In resident mode the factor band leaves
// no room for the epilogue tiles: the epilogue reads q, old b and
// e^{-sigma w} from global memory, and p is staged in the idle image stages.
__host__ __device__ constexpr uint32_t loop_staging_bytes(int) {
  return 2u * (uint32_t)LBN * BM * 2u;
}
__host__ __device__ constexpr uint32_t loop_epi_bytes(bool res) {
  return res ? 0u : 2u * LBN * BM * 4u;
}
__host__ __device__ constexpr uint32_t loop_res_bytes(bool res) {
  return res ? (uint32_t)RES_KB * BM * KB_BYTES : 0u;
}
__host__ __device__ constexpr uint32_t loop_stage_bytes(int mode, bool res) {
  return res ? (img_split(mode) ? 2u : 1u) * (uint32_t)LBN * KB_BYTES : stage_bytes(mode, LBN);
}
__host__ __device__ constexpr int loop_stages(int mode, bool res) {
  return res ? RES_STAGES
         : (LOOP_SMEM_BUDGET - loop_epi_bytes(false) - loop_staging_bytes(mode)) /
                       stage_bytes(mode, LBN) <
                   (uint32_t)MAX_STAGES
             ? (int)((LOOP_SMEM_BUDGET - loop_epi_bytes(false) - loop_staging_bytes(mode)) /
                     stage_bytes(mode, LBN))
             : MAX_STAGES;
}
__host__ __device__ constexpr size_t loop_smem_bytes(int mode, bool res) {
  return (size_t)loop_res_bytes(res) + (size_t)loop_stages(mode, res) * loop_stage_bytes(mode, res) +
         loop_staging_bytes(mode) + loop_epi_bytes(res) + 1024 +
         (size_t)(2 * loop_stages(mode, res) + 8) * 8 + 16;
}

struct LoopPass {
  int M, N;          // output D is M x N (M along the contracted axis)
  int tiles_n;       // tiles along N
  int ntiles;        // tiles of the pass
  const int4* kbt;   // per 128-row tile: band of the factor (band_tile)
};

struct LoopArgs {
  LoopPass pass[4];
  Ctrl* ctrl;
  ProxArgs<float> P;
  double* part;      // residual partial of each tile of the b-update pass
  int nparts;
  int pairs;         // pairs this launch may run
  // resident mode: the epilogue's global reads (q and e^{-sigma w} as
  // [ny][nx] fp32, b as the operand pair [ny][pitch_b])
  const float* q;
  const void* b_hi;
  const void* b_lo;
  int pitch_b;
};

// Tensor maps of the four passes: factor (A), image (B) and output of each
// pass (hi, lo), and the fp32 fields.
struct LoopMaps {
  CUtensorMap K[4][2];
  CUtensorMap B[4][2];
  CUtensorMap O[4][2];
  CUtensorMap Q, E, P;
};

// Bounded wait until the epilogue leader has published the barrier of pass q.
__device__ __forceinline__ bool wait_go(const int* s_go, int q) {
  for (uint32_t i = 0; i < kGoSpinLimit; ++i) {
    if (*(const volatile int*)s_go >= q) {
      __threadfence_block();
      return true;
    }
  }
  return false;
}

template <int MODE, int EK, bool RES>
__global__ void __launch_bounds__(NTL, 1)
tc_loop_kernel(const __grid_constant__ LoopMaps maps, const __grid_constant__ LoopArgs args) {
  // EK_CROWD_PLAIN: the congestion/potential kind with a scalar bound and no
  // mask or binary constraint, compiled without the per-cell field checks
  constexpr bool PLAIN = EK == EK_CROWD_PLAIN;
  constexpr int EKP = PLAIN ? EK_CROWD : EK;
  using T = typename OpT<MODE>::T;
  constexpr int KE = OpT<MODE>::kElems;
  constexpr int NSPLIT = img_split(MODE) ? 2 : 1;         // image hi (+ lo) blocks
  constexpr uint32_t A_BYTES = BM * KB_BYTES;
  constexpr uint32_t B_BYTES = LBN * KB_BYTES;
  constexpr uint32_t STAGE_BYTES = loop_stage_bytes(MODE, RES);
  constexpr int STAGES = loop_stages(MODE, RES);
  constexpr uint32_t B_OFF = RES ? 0u : A_BYTES;          // image blocks within a stage
  constexpr uint32_t ALO_OFF = A_BYTES + NSPLIT * B_BYTES; // factor lo (BF16X3)
  static_assert(STAGES >= 2, "at least two stages");
  static_assert(!RES || MODE == MODE_BF16, "resident factors: BF16 only");
  constexpr uint32_t STG_BYTES = loop_staging_bytes(MODE);
  constexpr uint32_t F32_TILE = (uint32_t)LBN * BM * 4u;
  // resident mode keeps each thread's cells of the last b (operand value) in
  // TMEM columns BPREV_COL .. +63 beside the accumulator, for the next residual
  constexpr uint32_t BPREV_COL = 128;
  static_assert(!RES || acc_cols(MODE, LBN) <= BPREV_COL, "accumulator below the old b");
  constexpr uint32_t TMEM_COLS = RES ? 256u : acc_cols(MODE, LBN);
  constexpr int CB = LBN * (int)sizeof(T) / 128;   // 128-byte column blocks of an operand tile
  constexpr uint32_t OUT_BLOCK = BM * 128;
  static_assert((uint32_t)NSPLIT * CB * OUT_BLOCK <= STG_BYTES, "staging tile");
  static_assert((uint32_t)NSPLIT * CB * OUT_BLOCK <= F32_TILE, "old b fits its tile");
  constexpr uint32_t EPI_B_LOAD = F32_TILE + (uint32_t)NSPLIT * CB * OUT_BLOCK;
  constexpr uint32_t EPI_A_LOAD = F32_TILE;
  // epilogue tiles moved by the producer: q and the old b for the b-update
  // pass, e^{-sigma w} for the prox pass of the congestion/potential kind.  In
  // resident mode the factor band leaves no room for a region of their own:
  // the q or e^{-sigma w} tile goes into the output staging region, idle while
  // the MMAs run, and the old b stays in the registers of the thread that
  // computed it (every pair gives a thread the same cells of its one tile)
  constexpr bool EPI1 = true;
  constexpr bool EPI3 = EKP == EK_CROWD;

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* res_a = smem;                               // resident factor band
  unsigned char* stages = smem + loop_res_bytes(RES);        // operand stages
  unsigned char* st_hi = stages + STAGES * STAGE_BYTES;      // output staging
  unsigned char* st_lo = st_hi + CB * OUT_BLOCK;
  unsigned char* epi_f = RES ? st_hi : st_hi + STG_BYTES;    // q or e^{-sigma w}
  unsigned char* epi_g = epi_f + F32_TILE;                   // old b (or p)
  unsigned char* p_st = RES ? stages : epi_g;                // staged p of the prox pass
  static_assert(!RES || STAGES * STAGE_BYTES >= F32_TILE, "p fits the image stages");
  uint64_t* full_bar = (uint64_t*)(epi_f + loop_epi_bytes(RES)); // A + B arrivals of a stage
  uint64_t* empty_bar = full_bar + STAGES;                   // stage consumed by the MMAs
  uint64_t* accum_bar = empty_bar + STAGES;                  // accumulator of a tile complete
  uint64_t* tmem_free_bar = accum_bar + 1;                   // accumulator drained (16 warps)
  uint64_t* epi_full_bar = accum_bar + 2;                    // epilogue tiles loaded
  uint64_t* epi_free_bar = accum_bar + 3;                    // epilogue region free again
  uint64_t* res_bar = accum_bar + 4;                         // resident band loaded
  uint32_t* tmem_slot = (uint32_t*)(accum_bar + 5);

  __shared__ int s_go;          // last pass whose barrier the epilogue has crossed
  __shared__ int s_stop;        // 1: the loop ends at pass s_go
  __shared__ int s_fault;       // 1: a bounded wait gave up; 4: NaN/Inf met
  __shared__ int s_it0, s_maxit;
  __shared__ unsigned s_base;   // barriers completed in this step before this launch
  __shared__ double s_tol;
  __shared__ float s_red[NEPI / 32];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = gridDim.x;
  Ctrl* ctrl = args.ctrl;
  const int nq = 4 * args.pairs;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], RES ? 1 : 2);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(accum_bar, 1);
    mbar_init(tmem_free_bar, NEPI / 32);
    mbar_init(epi_full_bar, 1);
    mbar_init(epi_free_bar, 1);
    mbar_init(res_bar, 1);
    fence_mbar_init();
    const int done = *(volatile int*)&ctrl->done;
    const int nonfinite = *(volatile int*)&ctrl->nonfinite;
    s_stop = (done != RUNNING || nonfinite) ? 1 : 0;
    if (done == RUNNING && nonfinite && blockIdx.x == 0) ctrl->done = NONFINITE;
    s_it0 = ctrl->it;
    s_maxit = ctrl->max_iter;
    s_tol = ctrl->tol;
    s_base = ctrl->bar_base;
    s_go = 0;
    s_fault = 0;
  }
  if (warp == WARP_MMA) {
    tmem_alloc(tmem_slot, TMEM_COLS);
    tmem_relinquish();
  }
  if (warp == WARP_PROD && lane == 0) {
    for (int p = 0; p < 4; ++p) {
      tma_prefetch_desc(&maps.K[p][0]);
      tma_prefetch_desc(&maps.B[p][0]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const bool stopped_at_start = s_stop != 0;
  int pairs_done = 0;
  unsigned nbar = 0;             // grid barriers crossed by this launch (epilogue thread 0)

  if (stopped_at_start) {
    // nothing to do: the step has already stopped
  } else if (warp == WARP_PROD) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t kc = 0;   // K-blocks issued (position in the stage ring)
      uint32_t ec = 0;   // epilogue-tile loads issued
      bool ok = true;
      if constexpr (RES) {
        // this CTA's factor band: the same m-tile and factor in every pass
        const LoopPass& P0 = args.pass[0];
        const int mt = (int)blockIdx.x / P0.tiles_n;
        const int4 kb = P0.kbt[mt];
        mbar_arrive_expect_tx(res_bar, (uint32_t)kb.y * A_BYTES);
        for (int i = 0; i < kb.y; ++i)
          tma_load_2d(res_a + i * A_BYTES, &maps.K[0][0], res_bar, kb.x + i * KE, mt * BM);
      }
      for (int q = 0; q < nq && ok; ++q) {
        const int p = q & 3;
        const LoopPass& PS = args.pass[p];
        const bool epi_pass = (p == 1 && EPI1) || (p == 3 && EPI3);
        int pre = 0;              // K-blocks of the first tile whose A half is in flight
        bool epi_pending = false; // epilogue tiles of the first tile issued before the barrier
        for (int t = blockIdx.x; t < PS.ntiles && ok; t += G) {
          const bool first = t == (int)blockIdx.x;
          const int mt = t / PS.tiles_n;
          const int m0 = mt * BM, n0 = (t - mt * PS.tiles_n) * LBN;
          const int4 kb = PS.kbt[mt];
          if (epi_pass) {
            // resident mode: the staging region is free once the stores of
            // the previous pass have read it (one arrival before every grid
            // barrier, the q-th before barrier q)
            if (RES) ok = mbar_wait(epi_free_bar, (uint32_t)(q - 1) & 1);
            else if (ec > 0) ok = mbar_wait(epi_free_bar, (ec - 1) & 1);
            if (!ok) break;
            if (p == 1) {
              mbar_arrive_expect_tx(epi_full_bar, RES ? F32_TILE : EPI_B_LOAD);
#pragma unroll
              for (int cb = 0; cb < LBN / 32; ++cb)
                tma_load_2d(epi_f + cb * (BM * 128), &maps.Q, epi_full_bar, n0 + cb * 32, m0);
              constexpr int KEO = 128 / (int)sizeof(T);
#pragma unroll
              for (int cb = 0; cb < (RES ? 0 : CB); ++cb) {
                tma_load_2d(epi_g + cb * OUT_BLOCK, &maps.O[1][0], epi_full_bar, n0 + cb * KEO, m0);
                if constexpr (NSPLIT == 2)
                  tma_load_2d(epi_g + (CB + cb) * OUT_BLOCK, &maps.O[1][1], epi_full_bar,
                              n0 + cb * KEO, m0);
              }
            } else {
              mbar_arrive_expect_tx(epi_full_bar, EPI_A_LOAD);
#pragma unroll
              for (int cb = 0; cb < LBN / 32; ++cb)
                tma_load_2d(epi_f + cb * (BM * 128), &maps.E, epi_full_bar, n0 + cb * 32, m0);
            }
            ++ec;
            epi_pending = first;
          }
          if (first && q > 0) {
            // factor halves of the first K-blocks: independent of the previous pass
            pre = RES ? 0 : (kb.y < STAGES ? kb.y : STAGES);
            for (int i = 0; i < pre && ok; ++i) {
              const uint32_t k = kc + i;
              const int s = (int)(k % STAGES);
              if (k >= (uint32_t)STAGES) ok = mbar_wait(&empty_bar[s], ((k / STAGES) - 1) & 1);
              if (!ok) break;
              unsigned char* st = stages + s * STAGE_BYTES;
              mbar_arrive_expect_tx(&full_bar[s], (fac_split(MODE) ? 2u : 1u) * A_BYTES);
              const int kx = kb.x + i * KE;
              tma_load_2d(st, &maps.K[p][0], &full_bar[s], kx, m0);
              if constexpr (fac_split(MODE))
                tma_load_2d(st + ALO_OFF, &maps.K[p][1], &full_bar[s], kx, m0);
            }
            if (!ok) break;
            ok = wait_go(&s_go, q);
            if (!ok) break;
            if (s_stop) {
              // the loop ends here: let the loads in flight land, then leave
              for (int i = 0; i < pre && ok; ++i) {
                const uint32_t k = kc + i;
                mbar_arrive(&full_bar[k % STAGES]);
                ok = mbar_wait(&full_bar[k % STAGES], (k / STAGES) & 1);
              }
              if (ok && epi_pending) ok = mbar_wait(epi_full_bar, (ec - 1) & 1);
              if (ok && RES) ok = mbar_wait(res_bar, 0);
              q = nq;
              break;
            }
            fence_proxy_async_global();
          }
          for (int i = 0; i < kb.y && ok; ++i) {
            const uint32_t k = kc + i;
            const int s = (int)(k % STAGES);
            unsigned char* st = stages + s * STAGE_BYTES;
            const int kx = kb.x + i * KE;
            if (RES) {
              if (k >= (uint32_t)STAGES) ok = mbar_wait(&empty_bar[s], ((k / STAGES) - 1) & 1);
              if (!ok) break;
            } else if (!(first && i < pre)) {
              if (k >= (uint32_t)STAGES) ok = mbar_wait(&empty_bar[s], ((k / STAGES) - 1) & 1);
              if (!ok) break;
              mbar_arrive_expect_tx(&full_bar[s], (fac_split(MODE) ? 2u : 1u) * A_BYTES);
              tma_load_2d(st, &maps.K[p][0], &full_bar[s], kx, m0);
              if constexpr (fac_split(MODE))
                tma_load_2d(st + ALO_OFF, &maps.K[p][1], &full_bar[s], kx, m0);
            }
            mbar_arrive_expect_tx(&full_bar[s], NSPLIT * B_BYTES);
            tma_load_2d(st + B_OFF, &maps.B[p][0], &full_bar[s], kx, n0);
            if constexpr (NSPLIT == 2)
              tma_load_2d(st + B_OFF + B_BYTES, &maps.B[p][1], &full_bar[s], kx, n0);
          }
          kc += kb.y;
        }
        if (ok && q > 0 && q < nq && (int)blockIdx.x >= PS.ntiles) {
          // no tile in this pass: follow the barriers all the same
          ok = wait_go(&s_go, q);
          if (ok && s_stop) q = nq;
        }
      }
      if (!ok) atomicOr(&s_fault, 1);
    }
  } else if (warp == WARP_MMA) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t kc = 0, tc = 0;
      bool ok = true;
      if constexpr (RES) ok = mbar_wait(res_bar, 0);
      for (int q = 0; q < nq && ok; ++q) {
        const int p = q & 3;
        const LoopPass& PS = args.pass[p];
        if (q > 0) {
          ok = wait_go(&s_go, q);
          if (!ok || s_stop) break;
        }
        for (int t = blockIdx.x; t < PS.ntiles && ok; t += G) {
          const int nkb = PS.kbt[t / PS.tiles_n].y;
          if (tc > 0) ok = mbar_wait(tmem_free_bar, (tc - 1) & 1);
          if (!ok) break;
          tc_fence_after();
          for (int i = 0; i < nkb && ok; ++i) {
            const uint32_t k = kc + i;
            const int s = (int)(k % STAGES);
            ok = mbar_wait(&full_bar[s], (k / STAGES) & 1);
            if (!ok) break;
            tc_fence_after();
            const uint32_t sa = smem_u32(stages + s * STAGE_BYTES);
            const uint64_t a_hi = sdesc_sw128(RES ? smem_u32(res_a + i * A_BYTES) : sa);
            const uint64_t a_lo = sdesc_sw128(sa + ALO_OFF);
            const uint64_t b = sdesc_sw128(sa + B_OFF);
#pragma unroll
            for (int kk = 0; kk < KB_BYTES / 32; ++kk)
              umma_kstep<MODE, LBN>(tmem_base, a_hi, a_lo, b, kk, (i > 0 || kk > 0) ? 1u : 0u);
            umma_commit(&empty_bar[s]);
          }
          umma_commit(accum_bar);
          kc += nkb;
          ++tc;
        }
      }
      if (!ok) atomicOr(&s_fault, 1);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int quad = warp & 3;
    const int grp = warp >> 2;
    const int rl = quad * 32 + lane;
    const ProxArgs<float> P = args.P;
    // congestion/potential cells with a scalar bound and no mask: the common
    // case, evaluated without the per-cell field checks
    constexpr bool crowd_plain = PLAIN;
    uint32_t tc = 0, ec = 0;
    int bad = 0;
    bool free_pending = false;   // epi_free owed once the last stores have read smem
    int dec_stop = 0;            // stop rule of this pair, taken during pass 2
    unsigned flag_prev = 0;      // flag slot of the previous barrier (thread 0)
    // resident mode: whether this thread's cells of b (operand value hi + lo)
    // from the last b-update pass are in TMEM (BPREV_COL), the old b of the
    // next residual: registers would spill at this kernel's register cap
    bool bprev_ok = false;
    for (int q = 0; q < nq; ++q) {
      const int p = q & 3;
      const int pair = q >> 2;
      const LoopPass& PS = args.pass[p];
      if (q > 0) {
        // ---- grid barrier: the previous pass is complete everywhere ----
        if (threadIdx.x == 0) {
          if (p == 0) {
            // after the prox pass: its a tiles are in global memory; the p
            // tiles (their own, last, bulk group) are read by no pass and
            // need only have left the stages, which the next loads refill
            bulk_wait_read_all();
            bulk_wait_all_but_last();
          } else {
            bulk_wait_all();               // this CTA's output tiles are in global memory
          }
          fence_proxy_async_global();
          if (free_pending) mbar_arrive(epi_free_bar);
          if (s_fault & 3) atomicOr(&ctrl->nonfinite, 2);
        }
        free_pending = false;
        bad = warp_or(bad);
        if (lane == 0 && bad) {
          atomicOr(&ctrl->nonfinite, 1);
          atomicOr(&s_fault, 4);
        }
        bad = 0;
        named_bar_sync(EPI_BAR, NEPI);
        if (threadIdx.x == 0) {
          const unsigned b = s_base + (++nbar);
          const bool ok = grid_barrier(ctrl, (unsigned)G, b, s_fault != 0);
          // flags of the previous barrier: every CTA has read the same value
          int stop = flag_prev != 0 || !ok;
          if (!ok) {
            atomicOr(&s_fault, 1);
            atomicOr(&ctrl->nonfinite, 2);
          }
          if (stop && blockIdx.x == 0) ctrl->done = NONFINITE;
          if (!stop && p == 3) stop = dec_stop;
          s_stop = stop;
          __threadfence_block();
          *(volatile int*)&s_go = q;
          // slot of this barrier, final now; the slot of barrier b + 2 (read
          // after barrier b - 1 by every CTA) is cleared for its next use
          flag_prev = *(volatile unsigned*)&ctrl->bar_flag[b % 3];
          if (blockIdx.x == 0) ctrl->bar_flag[(b + 2) % 3] = 0u;
        }
        named_bar_sync(EPI_BAR, NEPI);
        if (p == 0) pairs_done = pair;   // the pairs before this one are complete
        if (s_stop) break;
        if (p == 2 && warp == 0) {
          // stop rule from the residual partials of the b-update pass, in a
          // fixed order; it takes effect at the next barrier
          double v = 0.0;
          for (int i = lane; i < args.nparts; i += 32) v += __ldcg(args.part + i);
          v = warp_sum(v);
          const int it = s_it0 + pair;   // pairs completed before this one
          int d = RUNNING;
          if (it > 0 && !isfinite(v)) d = NONFINITE;
          else if (it > 0 && v <= s_tol) d = CONVERGED;
          else if (it >= s_maxit) d = MAX_ITER;
          else if (stall_rule(ctrl, it, v, lane == 0 && blockIdx.x == 0)) d = STALLED;
          if (lane == 0 && blockIdx.x == 0) {
            if (it > 0) ctrl->res_last = v;
            if (d != RUNNING) ctrl->done = d;
          }
          dec_stop = d != RUNNING;
        }
      }
      const bool have_prev = p == 1 && (s_it0 + pair) > 0;
      const bool epi_pass = (p == 1 && EPI1) || (p == 3 && EPI3);
      bool first = true;
      for (int t = blockIdx.x; t < PS.ntiles; t += G) {
        const int mt = t / PS.tiles_n;
        const int m0 = mt * BM, n0 = (t - mt * PS.tiles_n) * LBN;
        if (!first) {
          // the previous tile's stores must have read the staging and
          // epilogue tiles; the producer waits for that before it refills them
          if (threadIdx.x == 0) {
            bulk_wait_read_all();
            if (free_pending) mbar_arrive(epi_free_bar);
          }
          free_pending = false;
          named_bar_sync(EPI_BAR, NEPI);
        }
        const int c = grp;                      // 16-column chunk of the tile
        const int m = m0 + rl;
        const int nb = n0 + c * 16;
        int cnt = PS.N - nb;
        cnt = (m >= PS.M || cnt < 0) ? 0 : (cnt > 16 ? 16 : cnt);
        float bo[16];
        if constexpr (RES) {
          // the first b-update pass of a launch that continues a step: the
          // old b from global memory (this CTA's own tile, read past L1) into
          // the TMEM columns where the b-update passes keep it
          if (p == 1 && have_prev && !bprev_ok) {
            load_op16_cg<MODE>((const T*)args.b_hi, (const T*)args.b_lo,
                               cnt ? (size_t)m * args.pitch_b + nb : 0, cnt, bo);
            uint32_t rb[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) rb[j] = __float_as_uint(bo[j]);
            tmem_st16(tmem_base + ((uint32_t)(quad * 32) << 16) + BPREV_COL + (uint32_t)(grp * 16),
                      rb);
            tmem_wait_st();
            bprev_ok = true;
          }
        }
        bool have = mbar_wait(accum_bar, tc & 1);
        if (have && epi_pass) have = mbar_wait(epi_full_bar, ec & 1);
        if (!have && lane == 0) atomicOr(&s_fault, 1);
        __syncwarp();
        tc_fence_after();
        float v[16], o[16];
        // resident mode: the old b of the residual from TMEM
        const bool ld_old = RES && p == 1 && have_prev;
        const uint32_t t_old = tmem_base + ((uint32_t)(quad * 32) << 16) + BPREV_COL + (uint32_t)(grp * 16);
        tmem_tile16<MODE, LBN>(tmem_base + ((uint32_t)(quad * 32) << 16), grp * 16, v);
        if (ld_old) tmem_wait_st();   // this thread's store of it, one pair ago
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tmem_free_bar);
        float res_f = 0.0f;
        if (p == 0 || p == 2) {
#pragma unroll
          for (int j = 0; j < 16; ++j) o[j] = v[j];
        } else if (p == 1) {
          if constexpr (RES) {
            // the old b from TMEM; q four columns at a time from the staging
            // region (the layout of smem_ld_f32x16), to stay within the
            // register cap of this kernel's 18 warps
            const unsigned char* qrow = epi_f + (c >> 1) * (BM * 128) + rl * 128;
            const int k0 = (c & 1) * 4;
            uint32_t rb[8];
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {
              if (ld_old && (q4 & 1) == 0) {   // the old b, eight columns at a time
                tmem_ld8_issue(t_old + (uint32_t)(4 * q4), rb);
                tmem_wait_ld();
                reg_fence8(rb);
              }
              const float4 t = *reinterpret_cast<const float4*>(qrow + (((k0 + q4) ^ (rl & 7)) << 4));
              const float qq[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int j = 4 * q4 + u;
                if (j < cnt) {
                  if (have_prev)
                    res_f += abs_residual<float>(__uint_as_float(rb[4 * (q4 & 1) + u]), v[j], qq[u]);
                  o[j] = b_update<float>(qq[u], v[j]);
                  bad |= !isfinite(o[j]);
                } else {
                  o[j] = 0.0f;
                }
              }
            }
          } else {
            // q and the old b four columns at a time
#pragma unroll
            for (int g4 = 0; g4 < 4; ++g4) {
              const float4 t = smem_ld_f32x4(epi_f, rl, c, g4);
              const float qq[4] = {t.x, t.y, t.z, t.w};
              float bb[4] = {0.0f, 0.0f, 0.0f, 0.0f};
              if (have_prev) smem_ld_op4<MODE>(epi_g, epi_g + CB * OUT_BLOCK, rl, c, g4, bb);
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int j = 4 * g4 + u;
                if (j < cnt) {
                  if (have_prev) res_f += abs_residual<float>(bb[u], v[j], qq[u]);
                  o[j] = b_update<float>(qq[u], v[j]);
                  bad |= !isfinite(o[j]);
                } else {
                  o[j] = 0.0f;
                }
              }
            }
          }
        } else {
          const int irow = m * PS.N + nb;
          if (crowd_plain) {
            // e^{-sigma w} in, p out, four columns at a time (the layout of
            // smem_ld_f32x16 / smem_st_f32x16), to stay within the register
            // cap of this kernel's 18 warps
            const bool hk = P.has_kappa != 0;
            const float kap = P.kappa_s;
            const int k0 = (c & 1) * 4;
            const unsigned char* erow = epi_f + (c >> 1) * (BM * 128) + rl * 128;
            unsigned char* prow = p_st + (c >> 1) * (BM * 128) + rl * 128;
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {
              const int off = ((k0 + q4) ^ (rl & 7)) << 4;
              const float4 t = *reinterpret_cast<const float4*>(erow + off);
              const float ee[4] = {t.x, t.y, t.z, t.w};
              float pp[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int j = 4 * q4 + u;
                float a = ee[u];
                if (hk && a * v[j] > kap) a = ratio_div<float>(kap, v[j]);
                if (j >= cnt) a = 0.0f;
                bad |= !isfinite(a);
                o[j] = a;
                pp[u] = a * v[j];
              }
              *reinterpret_cast<float4*>(prow + off) = make_float4(pp[0], pp[1], pp[2], pp[3]);
            }
          } else {
            // the general prox, four columns at a time as above
            const int k0 = (c & 1) * 4;
            const unsigned char* erow = epi_f + (c >> 1) * (BM * 128) + rl * 128;
            unsigned char* prow = p_st + (c >> 1) * (BM * 128) + rl * 128;
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {
              const int off = ((k0 + q4) ^ (rl & 7)) << 4;
              float ee[4] = {0.0f, 0.0f, 0.0f, 0.0f};
              if (EKP == EK_CROWD) {
                const float4 t = *reinterpret_cast<const float4*>(erow + off);
                ee[0] = t.x; ee[1] = t.y; ee[2] = t.z; ee[3] = t.w;
              }
              float pp[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int j = 4 * q4 + u;
                if (j < cnt) {
                  const float a = prox_ratio_e<float, EKP>(P, irow + j, v[j], ee[u]);
                  bad |= !isfinite(a);
                  o[j] = a;
                  pp[u] = a * v[j];
                } else {
                  o[j] = 0.0f;
                  pp[u] = 0.0f;
                }
              }
              *reinterpret_cast<float4*>(prow + off) = make_float4(pp[0], pp[1], pp[2], pp[3]);
            }
          }
        }
        if constexpr (RES) {
          // every thread has read the q / e^{-sigma w} tile in the staging
          // region before any writes its output there
          if (epi_pass) named_bar_sync(EPI_BAR, NEPI);
          if (p == 1) {
            uint32_t rs[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) rs[j] = __float_as_uint(op_value<MODE>(o[j]));
            tmem_st16(tmem_base + ((uint32_t)(quad * 32) << 16) + BPREV_COL + (uint32_t)(grp * 16),
                      rs);
            bprev_ok = true;   // (waited for before the next load and before the end)
          }
        }
        stage16<MODE>(st_hi, st_lo, rl, c, o);
        fence_proxy_async_smem();
        double res = 0.0;
        if (p == 1)   // includes the barrier
          res = (double)tile_sum16(res_f, s_red, [] { named_bar_sync(EPI_BAR, NEPI); });
        else
          named_bar_sync(EPI_BAR, NEPI);
        if (threadIdx.x == 0) {
          if (p == 1) args.part[t] = res;
          constexpr int KEo = 128 / (int)sizeof(T);
#pragma unroll
          for (int cb = 0; cb < CB; ++cb) {
            tma_store_2d(&maps.O[p][0], st_hi + cb * OUT_BLOCK, n0 + cb * KEo, m0);
            if constexpr (NSPLIT == 2) tma_store_2d(&maps.O[p][1], st_lo + cb * OUT_BLOCK, n0 + cb * KEo, m0);
          }
          if (p == 3) {
            bulk_commit();                 // the a tiles, then the p tiles as their own group
#pragma unroll
            for (int cb = 0; cb < LBN / 32; ++cb)
              tma_store_2d(&maps.P, p_st + cb * (BM * 128), n0 + cb * 32, m0);
          }
          bulk_commit();
        }
        // resident mode: every pass's stores free the staging region that
        // the producer refills before the next barrier
        free_pending = RES ? true : epi_pass;
        first = false;
        ++tc;
        if (epi_pass) ++ec;
      }
      if (p == 3 && q == nq - 1) pairs_done = pair + 1;
    }
    if (threadIdx.x == 0) bulk_wait_all();
    if (RES) tmem_wait_st();   // the old b's stores, before the columns are freed
    bad = warp_or(bad);
    if (lane == 0 && bad) atomicOr(&ctrl->nonfinite, 1);
  }

  tc_fence_before();
  __syncthreads();
  __syncwarp();
  if (warp == WARP_MMA) tmem_dealloc(tmem_base, TMEM_COLS);
  if (threadIdx.x == 0 && !stopped_at_start) {
    if (s_fault & 3) atomicOr(&ctrl->nonfinite, 2);
    if (blockIdx.x == 0) {
      ctrl->it = s_it0 + pairs_done;
      ctrl->bar_base = s_base + nbar;   // every CTA crossed the same barriers
    }
  }
}

// ------------------------------------------------------------ grouped batch
// One cooperative launch runs the scaling loop of every flow of a batch that
// shares the operand precision and the energy kind (the prox of the epilogue
// is compiled for one kind: a run-time choice among the three inlines all of
// them at the 96-register cap of 19 warps and made the element math of a tile
// several times slower).  The tiles of all flows form one list per
// pass, walked by the CTAs between the same grid barriers as above; each tile
// names its flow, whose tensor maps and descriptor live in device memory.
// Every flow keeps its own stop rule: during pass 2 the flow's designated CTA
// (f mod G) adds its residual partials in the same order as the loop kernel,
// records the decision in the flow's Ctrl and sets the flow's bit in a stop
// word; after the barrier before the prox pass every CTA reads the words, so
// all skip the flow's tiles from that pass on, exactly where the loop kernel
// alone would stop.  The per-tile arithmetic is that of tc_loop_kernel, so a
// flow of a grouped launch gives the bits of the same flow on the loop kernel.
// NaN/Inf in a flow is recorded in its Ctrl and stops that flow at its next
// decision; a wait that gives up stops the whole launch.
constexpr int MAXF = 2048;                   // flows per grouped launch

struct FlowDesc {
  int M[4], N[4];           // output geometry of each pass
  Ctrl* ctrl;               // it, done, max_iter, tol, res_last, nonfinite of the flow
  double* part;             // residual partial of each b-update tile
  int nparts;
  int ek;
  ProxArgs<float> P;
};

// Tile g of pass p: items[p][2g] = {flow, m0, n0, 8 t + 2 ek + e} (t: index
// of the tile in the flow's pass, ek: energy kind, e: 1 if the tile loads
// epilogue tiles), items[p][2g + 1] = {first K element of the factor band of
// its 128-row block, K-blocks of the band, M, N of the flow's pass}.  Every
// role loads a tile's two int4 one tile ahead, so no per-tile global load
// chain sits on the critical path.
struct BatchArgs {
  const FlowDesc* flows;
  const LoopMaps* maps;     // tensor maps of each flow
  const int4* items[4];
  int ntiles[4];
  Ctrl* bctrl;              // grid-barrier words of the launch
  unsigned* gstop;          // bit f: flow f stopped by a decision of this launch
  int F;
  int pairs;
};

__device__ __forceinline__ bool flow_stopped(const unsigned* mask, int f) {
  return (*(const volatile unsigned*)&mask[f >> 5] >> (f & 31)) & 1u;
}

struct TileItem {
  int4 a, b;
};

__device__ __forceinline__ TileItem load_item(const int4* items, int g, int nt) {
  TileItem r;
  if (g < nt) {
    r.a = __ldg(items + 2 * g);
    r.b = __ldg(items + 2 * g + 1);
  } else {
    r.a = make_int4(0, 0, 0, 0);
    r.b = make_int4(0, 0, 0, 0);
  }
  return r;
}

constexpr int NTB = NTL + 32;               // + warp 18, which loads the epilogue tiles
constexpr int WARP_EPILD = 18;

template <int MODE, int EK>
__global__ void __launch_bounds__(NTB, 1) tc_batch_kernel(const __grid_constant__ BatchArgs args) {
  using T = typename OpT<MODE>::T;
  constexpr int KE = OpT<MODE>::kElems;
  constexpr int NSPLIT = img_split(MODE) ? 2 : 1;         // image hi (+ lo) blocks
  constexpr uint32_t A_BYTES = BM * KB_BYTES;
  constexpr uint32_t B_BYTES = LBN * KB_BYTES;
  constexpr uint32_t STAGE_BYTES = loop_stage_bytes(MODE, false);
  constexpr uint32_t ALO_OFF = A_BYTES + NSPLIT * B_BYTES; // factor lo (BF16X3)
  constexpr int STAGES = loop_stages(MODE, false);
  static_assert(STAGES >= 2, "at least two stages");
  constexpr uint32_t STG_BYTES = loop_staging_bytes(MODE);
  constexpr uint32_t F32_TILE = (uint32_t)LBN * BM * 4u;
  constexpr uint32_t TMEM_COLS = acc_cols(MODE, LBN);
  constexpr int CB = LBN * (int)sizeof(T) / 128;
  constexpr uint32_t OUT_BLOCK = BM * 128;
  constexpr uint32_t EPI_B_LOAD = F32_TILE + (uint32_t)NSPLIT * CB * OUT_BLOCK;
  constexpr uint32_t EPI_A_LOAD = F32_TILE;

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* stages = smem;
  unsigned char* st_hi = stages + STAGES * STAGE_BYTES;
  unsigned char* st_lo = st_hi + CB * OUT_BLOCK;
  unsigned char* epi_f = st_hi + STG_BYTES;
  unsigned char* epi_g = epi_f + F32_TILE;
  uint64_t* full_bar = (uint64_t*)(epi_f + loop_epi_bytes(false));
  uint64_t* empty_bar = full_bar + STAGES;
  uint64_t* accum_bar = empty_bar + STAGES;
  uint64_t* tmem_free_bar = accum_bar + 1;
  uint64_t* epi_full_bar = accum_bar + 2;
  uint64_t* epi_free_bar = accum_bar + 3;
  uint32_t* tmem_slot = (uint32_t*)(accum_bar + 5);

  __shared__ int s_go, s_stop, s_fault, s_gfault;
  __shared__ unsigned s_base;
  __shared__ float s_red[NEPI / 32];
  __shared__ unsigned s_fstop[MAXF / 32];   // flows whose tiles are skipped
  __shared__ unsigned s_itpos[MAXF / 32];   // flows with pairs done before this launch

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = gridDim.x;
  const int F = args.F;
  const int nwords = (F + 31) >> 5;
  Ctrl* bctrl = args.bctrl;
  const int nq = 4 * args.pairs;

  for (int i = threadIdx.x; i < MAXF / 32; i += NTB) {
    s_fstop[i] = 0u;
    s_itpos[i] = 0u;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(accum_bar, 1);
    mbar_init(tmem_free_bar, NEPI / 32);
    mbar_init(epi_full_bar, 1);
    mbar_init(epi_free_bar, 1);
    fence_mbar_init();
    s_base = bctrl->bar_base;
    s_go = 0;
    s_fault = 0;
    s_gfault = 0;
  }
  if (warp == WARP_MMA) {
    tmem_alloc(tmem_slot, TMEM_COLS);
    tmem_relinquish();
  }
  __syncthreads();
  // flows that stopped in an earlier launch of the step (their Ctrl changes
  // only in pass 2, after two grid barriers, so every CTA reads the same)
  for (int f = threadIdx.x; f < F; f += NTB) {
    Ctrl* c = args.flows[f].ctrl;
    const int done = *(volatile int*)&c->done;
    const int nf = *(volatile int*)&c->nonfinite;
    if (done != RUNNING || nf) atomicOr(&s_fstop[f >> 5], 1u << (f & 31));
    if (c->it > 0) atomicOr(&s_itpos[f >> 5], 1u << (f & 31));
    if (done == RUNNING && nf && f % G == (int)blockIdx.x) c->done = NONFINITE;
  }
  // the stop words of this launch start empty (first read after barrier 3)
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < nwords; i += NTB) args.gstop[i] = 0u;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x == 0) {
    bool all = true;
    for (int w = 0; w < nwords && all; ++w) {
      const int nb = F - 32 * w;
      all = s_fstop[w] == (nb >= 32 ? 0xffffffffu : ((1u << nb) - 1u));
    }
    s_stop = all ? 1 : 0;
  }
  __syncthreads();
  const uint32_t tmem_base = *tmem_slot;
  const bool stopped_at_start = s_stop != 0;
  int pairs_done = 0;
  unsigned nbar = 0;

  if (stopped_at_start) {
    // every flow has already stopped
  } else if (warp == WARP_PROD || warp == WARP_EPILD) {
    // ------------------------------------------------------------ producers
    // warp 16 streams the operand K-blocks, warp 18 the epilogue tiles, each
    // as soon as its own buffer is free, so the next tile's operands load
    // while the epilogue still holds the current tile's q / old b /
    // e^{-sigma w} (two lanes of one warp would wait on each other)
    const bool kload = warp == WARP_PROD;
    if (lane == 0) {
      uint32_t kc = 0, ec = 0;
      bool ok = true;
      for (int q = 0; q < nq && ok; ++q) {
        const int p = q & 3;
        const int nt = args.ntiles[p];
        TileItem nx = load_item(args.items[p], blockIdx.x, nt);
        if (q > 0) {
          ok = wait_go(&s_go, q);
          if (!ok || s_stop) break;
          fence_proxy_async_global();
        }
        for (int g = blockIdx.x; g < nt && ok; g += G) {
          const TileItem cur = nx;
          nx = load_item(args.items[p], g + G, nt);
          const int4 it = cur.a;
          if (flow_stopped(s_fstop, it.x)) continue;
          const LoopMaps* mp = args.maps + it.x;
          const int m0 = it.y, n0 = it.z;
          if (kload) {
            const int4 kb = cur.b;
            for (int i = 0; i < kb.y && ok; ++i) {
              const uint32_t k = kc + i;
              const int s = (int)(k % STAGES);
              if (k >= (uint32_t)STAGES) ok = mbar_wait(&empty_bar[s], ((k / STAGES) - 1) & 1);
              if (!ok) break;
              unsigned char* st = stages + s * STAGE_BYTES;
              const int kx = kb.x + i * KE;
              mbar_arrive_expect_tx(&full_bar[s], STAGE_BYTES);
              tma_load_2d(st, &mp->K[p][0], &full_bar[s], kx, m0);
              tma_load_2d(st + A_BYTES, &mp->B[p][0], &full_bar[s], kx, n0);
              if constexpr (NSPLIT == 2)
                tma_load_2d(st + A_BYTES + B_BYTES, &mp->B[p][1], &full_bar[s], kx, n0);
              if constexpr (fac_split(MODE))
                tma_load_2d(st + ALO_OFF, &mp->K[p][1], &full_bar[s], kx, m0);
            }
            kc += kb.y;
          } else if (it.w & 1) {
            if (ec > 0) ok = mbar_wait(epi_free_bar, (ec - 1) & 1);
            if (!ok) break;
            if (p == 1) {
              mbar_arrive_expect_tx(epi_full_bar, EPI_B_LOAD);
#pragma unroll
              for (int cb = 0; cb < LBN / 32; ++cb)
                tma_load_2d(epi_f + cb * (BM * 128), &mp->Q, epi_full_bar, n0 + cb * 32, m0);
              constexpr int KEO = 128 / (int)sizeof(T);
#pragma unroll
              for (int cb = 0; cb < CB; ++cb) {
                tma_load_2d(epi_g + cb * OUT_BLOCK, &mp->O[1][0], epi_full_bar, n0 + cb * KEO, m0);
                if constexpr (NSPLIT == 2)
                  tma_load_2d(epi_g + (CB + cb) * OUT_BLOCK, &mp->O[1][1], epi_full_bar,
                              n0 + cb * KEO, m0);
              }
            } else {
              mbar_arrive_expect_tx(epi_full_bar, EPI_A_LOAD);
#pragma unroll
              for (int cb = 0; cb < LBN / 32; ++cb)
                tma_load_2d(epi_f + cb * (BM * 128), &mp->E, epi_full_bar, n0 + cb * 32, m0);
            }
            ++ec;
          }
        }
      }
      if (!ok) atomicOr(&s_fault, 1);
    }
  } else if (warp == WARP_MMA) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t kc = 0, tc = 0;
      bool ok = true;
      for (int q = 0; q < nq && ok; ++q) {
        const int p = q & 3;
        const int nt = args.ntiles[p];
        TileItem nx = load_item(args.items[p], blockIdx.x, nt);
        if (q > 0) {
          ok = wait_go(&s_go, q);
          if (!ok || s_stop) break;
        }
        for (int g = blockIdx.x; g < nt && ok; g += G) {
          const TileItem cur = nx;
          nx = load_item(args.items[p], g + G, nt);
          if (flow_stopped(s_fstop, cur.a.x)) continue;
          const int nkb = cur.b.y;
          if (tc > 0) ok = mbar_wait(tmem_free_bar, (tc - 1) & 1);
          if (!ok) break;
          tc_fence_after();
          for (int i = 0; i < nkb && ok; ++i) {
            const uint32_t k = kc + i;
            const int s = (int)(k % STAGES);
            ok = mbar_wait(&full_bar[s], (k / STAGES) & 1);
            if (!ok) break;
            tc_fence_after();
            const uint32_t sa = smem_u32(stages + s * STAGE_BYTES);
            const uint64_t a_hi = sdesc_sw128(sa);
            const uint64_t a_lo = sdesc_sw128(sa + ALO_OFF);
            const uint64_t b = sdesc_sw128(sa + A_BYTES);
#pragma unroll
            for (int kk = 0; kk < KB_BYTES / 32; ++kk)
              umma_kstep<MODE, LBN>(tmem_base, a_hi, a_lo, b, kk, (i > 0 || kk > 0) ? 1u : 0u);
            umma_commit(&empty_bar[s]);
          }
          umma_commit(accum_bar);
          kc += nkb;
          ++tc;
        }
      }
      if (!ok) atomicOr(&s_fault, 1);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int quad = warp & 3;
    const int grp = warp >> 2;
    const int rl = quad * 32 + lane;
    uint32_t tc = 0, ec = 0;
    bool free_pending = false;
    unsigned flag_prev = 0;      // flag slot of the previous barrier (warp 0)
    for (int q = 0; q < nq; ++q) {
      const int p = q & 3;
      const int pair = q >> 2;
      const int nt = args.ntiles[p];
      TileItem nx = load_item(args.items[p], blockIdx.x, nt);
      if (q > 0) {
        // ---- grid barrier ----
        if (threadIdx.x == 0) {
          bulk_wait_all();
          fence_proxy_async_global();
          if (free_pending) mbar_arrive(epi_free_bar);
          if (s_fault & 3) atomicOr(&bctrl->nonfinite, 2);
        }
        free_pending = false;
        named_bar_sync(EPI_BAR, NEPI);
        if (warp == 0) {
          int stop = 0;
          unsigned b = 0;
          if (lane == 0) {
            b = s_base + (++nbar);
            const bool ok = grid_barrier(bctrl, (unsigned)G, b, (s_fault & 3) != 0);
            stop = flag_prev != 0 || !ok;
            if (!ok) {
              atomicOr(&s_fault, 1);
              atomicOr(&bctrl->nonfinite, 2);
            }
            if (stop) s_gfault = 1;
          }
          stop = __shfl_sync(0xffffffffu, stop, 0);
          __syncwarp();
          if (!stop && p == 3) {
            // the decisions of pass 2 take effect now, in every CTA alike
            bool all = true;
            for (int w = lane; w < nwords; w += 32) {
              const unsigned m = s_fstop[w] | __ldcg(args.gstop + w);
              s_fstop[w] = m;
              const int nb = F - 32 * w;
              all = all && m == (nb >= 32 ? 0xffffffffu : ((1u << nb) - 1u));
            }
            stop = __all_sync(0xffffffffu, all) ? 1 : 0;
          }
          if (lane == 0) {
            s_stop = stop;
            __threadfence_block();
            *(volatile int*)&s_go = q;
            flag_prev = *(volatile unsigned*)&bctrl->bar_flag[b % 3];
            if (blockIdx.x == 0) bctrl->bar_flag[(b + 2) % 3] = 0u;
          }
        }
        named_bar_sync(EPI_BAR, NEPI);
        if (p == 0) pairs_done = pair;
        if (s_stop) break;
        if (p == 2) {
          // stop rule of this CTA's flows (f = blockIdx.x + G k, warp by warp),
          // the partials added in the loop kernel's order
          for (int f = (int)blockIdx.x + warp * G; f < F; f += (NEPI / 32) * G) {
            if (flow_stopped(s_fstop, f)) continue;
            const FlowDesc& FD = args.flows[f];
            const int np = FD.nparts;
            double v = 0.0;
            for (int i = lane; i < np; i += 32) v += __ldcg(FD.part + i);
            v = warp_sum(v);
            Ctrl* c = FD.ctrl;
            const int it = *(const volatile int*)&c->it + pair;
            int d = RUNNING;
            if (*(const volatile int*)&c->nonfinite & 1) d = NONFINITE;
            else if (it > 0 && !isfinite(v)) d = NONFINITE;
            else if (it > 0 && v <= c->tol) d = CONVERGED;
            else if (it >= c->max_iter) d = MAX_ITER;
            else if (stall_rule(c, it, v, lane == 0)) d = STALLED;
            if (lane == 0) {
              if (it > 0) c->res_last = v;
              if (d != RUNNING) {
                c->done = d;
                c->it = it;
                atomicOr(args.gstop + (f >> 5), 1u << (f & 31));
              }
              __threadfence();
            }
          }
        }
      }
      bool first = true;
      for (int g = blockIdx.x; g < nt; g += G) {
        const TileItem cur = nx;
        nx = load_item(args.items[p], g + G, nt);
        const int4 itm = cur.a;
        if (flow_stopped(s_fstop, itm.x)) continue;
        const FlowDesc& FD = args.flows[itm.x];
        const LoopMaps* mp = args.maps + itm.x;
        const int t = itm.w >> 3;
        const bool epi_pass = (itm.w & 1) != 0;
        const int m0 = itm.y, n0 = itm.z;
        const int PM = cur.b.z, PN = cur.b.w;
        const bool have_prev =
            p == 1 && (pair > 0 || ((s_itpos[itm.x >> 5] >> (itm.x & 31)) & 1u) != 0);
        // per-flow values, loaded while the tile's MMAs run
        ProxArgs<float> P{};
        double* part = nullptr;
        if (p == 3) P = FD.P;
        if (p == 1) part = FD.part;
        if (!first) {
          if (threadIdx.x == 0) {
            bulk_wait_read_all();
            if (free_pending) mbar_arrive(epi_free_bar);
          }
          free_pending = false;
          named_bar_sync(EPI_BAR, NEPI);
        }
        bool have = mbar_wait(accum_bar, tc & 1);
        if (have && epi_pass) have = mbar_wait(epi_full_bar, ec & 1);
        if (!have && lane == 0) atomicOr(&s_fault, 1);
        __syncwarp();
        tc_fence_after();
        float v[16], o[16];
        tmem_tile16<MODE, LBN>(tmem_base + ((uint32_t)(quad * 32) << 16), grp * 16, v);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tmem_free_bar);
        const int c = grp;
        const int m = m0 + rl;
        const int nb = n0 + c * 16;
        int cnt = PN - nb;
        cnt = (m >= PM || cnt < 0) ? 0 : (cnt > 16 ? 16 : cnt);
        float res_f = 0.0f;
        int bad = 0;
        if (p == 0 || p == 2) {
#pragma unroll
          for (int j = 0; j < 16; ++j) o[j] = v[j];
        } else if (p == 1) {
          float qv[16], bo[16];
          smem_ld_f32x16(epi_f, rl, c, qv);
          if (have_prev) smem_ld_op16<MODE>(epi_g, epi_g + CB * OUT_BLOCK, rl, c, bo);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            if (j < cnt) {
              if (have_prev) res_f += abs_residual<float>(bo[j], v[j], qv[j]);
              o[j] = b_update<float>(qv[j], v[j]);
              bad |= !isfinite(o[j]);
            } else {
              o[j] = 0.0f;
            }
          }
        } else {
          const int irow = m * PN + nb;
          float ev[16], pv[16];
          if (EK == EK_CROWD) smem_ld_f32x16(epi_f, rl, c, ev);
          if (EK == EK_CROWD && P.mask == nullptr && P.kappa == nullptr && P.binary == 0) {
            const bool hk = P.has_kappa != 0;
            const float kap = P.kappa_s;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              float a = ev[j];
              if (hk && a * v[j] > kap) a = ratio_div<float>(kap, v[j]);
              if (j >= cnt) a = 0.0f;
              bad |= !isfinite(a);
              o[j] = a;
              pv[j] = a * v[j];
            }
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              float a = 0.0f;
              if (j < cnt) {
                a = prox_ratio_e<float, EK>(P, irow + j, v[j], EK == EK_CROWD ? ev[j] : 0.0f);
                bad |= !isfinite(a);
              }
              o[j] = a;
              pv[j] = j < cnt ? a * v[j] : 0.0f;
            }
          }
          smem_st_f32x16(epi_g, rl, c, pv);
        }
        bad = warp_or(bad);
        if (lane == 0 && bad) atomicOr(&FD.ctrl->nonfinite, 1);
        stage16<MODE>(st_hi, st_lo, rl, c, o);
        fence_proxy_async_smem();
        double res = 0.0;
        if (p == 1)
          res = (double)tile_sum16(res_f, s_red, [] { named_bar_sync(EPI_BAR, NEPI); });
        else
          named_bar_sync(EPI_BAR, NEPI);
        if (threadIdx.x == 0) {
          if (p == 1) part[t] = res;
          constexpr int KEo = 128 / (int)sizeof(T);
#pragma unroll
          for (int cb = 0; cb < CB; ++cb) {
            tma_store_2d(&mp->O[p][0], st_hi + cb * OUT_BLOCK, n0 + cb * KEo, m0);
            if constexpr (NSPLIT == 2) tma_store_2d(&mp->O[p][1], st_lo + cb * OUT_BLOCK, n0 + cb * KEo, m0);
          }
          if (p == 3) {
#pragma unroll
            for (int cb = 0; cb < LBN / 32; ++cb)
              tma_store_2d(&mp->P, epi_g + cb * (BM * 128), n0 + cb * 32, m0);
          }
          bulk_commit();
        }
        free_pending = epi_pass;
        first = false;
        ++tc;
        if (epi_pass) ++ec;
      }
      if (p == 3 && q == nq - 1) pairs_done = pair + 1;
    }
    if (threadIdx.x == 0) bulk_wait_all();
  }

  tc_fence_before();
  __syncthreads();
  __syncwarp();
  if (warp == WARP_MMA) tmem_dealloc(tmem_base, TMEM_COLS);
  if (threadIdx.x == 0 && !stopped_at_start) {
    if (s_fault & 3) atomicOr(&bctrl->nonfinite, 2);
    // the designated CTA records the pairs of its flows still running
    for (int f = blockIdx.x; f < F; f += G) {
      Ctrl* c = args.flows[f].ctrl;
      if (*(volatile int*)&c->done != RUNNING) continue;
      c->it = *(volatile int*)&c->it + pairs_done;
      if (s_gfault) {
        atomicOr(&c->nonfinite, 2);
        c->done = NONFINITE;
      }
    }
    if (blockIdx.x == 0) bctrl->bar_base = s_base + nbar;
  }
}

template <int MODE, int EK, bool RES>
cudaError_t set_loop_attr() {
  return cudaFuncSetAttribute(tc_loop_kernel<MODE, EK, RES>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)loop_smem_bytes(MODE, RES));
}

template <int MODE, int EK, bool RES>
cudaError_t launch_loop(const LoopMaps& maps, const LoopArgs& args, int grid, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(NTL);
  cfg.dynamicSmemBytes = loop_smem_bytes(MODE, RES);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, tc_loop_kernel<MODE, EK, RES>, maps, args);
}

template <int MODE, bool RES>
cudaError_t dispatch_loop(int ek, const LoopMaps& maps, const LoopArgs& args, int grid,
                          cudaStream_t st) {
  const ProxArgs<float>& P = args.P;
  if (ek == EK_CROWD && P.mask == nullptr && P.kappa == nullptr && P.binary == 0)
    return launch_loop<MODE, EK_CROWD_PLAIN, RES>(maps, args, grid, st);
  if (ek == EK_CROWD) return launch_loop<MODE, EK_CROWD, RES>(maps, args, grid, st);
  if (ek == EK_ENTROPY) return launch_loop<MODE, EK_ENTROPY, RES>(maps, args, grid, st);
  return launch_loop<MODE, EK_POWER, RES>(maps, args, grid, st);
}

template <int MODE, int EK, bool RES>
int blocks_per_sm() {
  int nb = 0;
  if (set_loop_attr<MODE, EK, RES>() != cudaSuccess) return 0;
  if (EK == EK_CROWD && set_loop_attr<MODE, EK_CROWD_PLAIN, RES>() != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tc_loop_kernel<MODE, EK, RES>, NTL,
                                                    loop_smem_bytes(MODE, RES)) != cudaSuccess)
    return 0;
  return nb;
}

template <int MODE, bool RES>
int loop_blocks_per_sm(int ek) {
  if (ek == EK_CROWD) return blocks_per_sm<MODE, EK_CROWD, RES>();
  if (ek == EK_ENTROPY) return blocks_per_sm<MODE, EK_ENTROPY, RES>();
  return blocks_per_sm<MODE, EK_POWER, RES>();
}

// Geometry of pass `which` (0..3) with 64-wide tiles.
LoopPass loop_pass(const TcPlan* P, int which) {
  const TcConfig& c = P->cfg;
  const bool over_x = (which & 1) == 0;
  const int side = P->absorbed ? (which >> 1) : 0;
  LoopPass L;
  L.M = over_x ? c.nx : c.ny;
  L.N = over_x ? c.ny : c.nx;
  L.tiles_n = (L.N + LBN - 1) / LBN;
  L.ntiles = L.tiles_n * ((L.M + BM - 1) / BM);
  L.kbt = P->kbt[over_x ? 0 : 1][side];
  return L;
}

}  // namespace

int tc_loop_setup(TcPlan* P, std::string* msg) {
  P->loop_ok = 0;
  if (!P->tma_epi) return 0;   // fp32 fields must be TMA tiles (nx % 4 == 0)
  int dev = 0, sms = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop || sms < 1) return 0;
  const int ek = P->cfg.ek;
  const int nb = P->mode == MODE_TF32 ? loop_blocks_per_sm<MODE_TF32, false>(ek)
                 : P->mode == MODE_BF16X3 ? loop_blocks_per_sm<MODE_BF16X3, false>(ek)
                                          : loop_blocks_per_sm<MODE_BF16, false>(ek);
  cudaGetLastError();
  if (nb < 1) return 0;
  int maxt = 0;
  for (int w = 0; w < 4; ++w) maxt = std::max(maxt, loop_pass(P, w).ntiles);
  P->loop_grid = std::min(maxt, sms * nb);
  // resident factors: BF16, the same factor and band table in every pass
  // (square grid, equal lengths, no absorption), one tile per CTA and a band
  // of at most RES_KB K-blocks per 128-row tile
  P->loop_res = 0;
  const TcConfig& cc = P->cfg;
  if (P->mode == MODE_BF16 && !P->absorbed && cc.nx == cc.ny && cc.lx == cc.ly &&
      maxt <= P->loop_grid && loop_blocks_per_sm<MODE_BF16, true>(ek) >= 1) {
    const LoopPass L0 = loop_pass(P, 0), L1 = loop_pass(P, 1);
    std::vector<int4> t0((L0.M + BM - 1) / BM), t1((L1.M + BM - 1) / BM);
    bool same = t0.size() == t1.size() &&
                cudaMemcpy(t0.data(), L0.kbt, t0.size() * sizeof(int4), cudaMemcpyDeviceToHost) == cudaSuccess &&
                cudaMemcpy(t1.data(), L1.kbt, t1.size() * sizeof(int4), cudaMemcpyDeviceToHost) == cudaSuccess;
    for (size_t i = 0; same && i < t0.size(); ++i)
      same = t0[i].x == t1[i].x && t0[i].y == t1[i].y && t0[i].z == t1[i].z &&
             t0[i].w == t1[i].w && t0[i].y <= RES_KB;
    P->loop_res = same ? 1 : 0;
  }
  cudaGetLastError();
  static_assert(LBN == 64, "the plan's 64-row image maps serve the loop kernel");
  // executed flops of one pair with 64-wide tiles
  const int KE = P->mode == MODE_TF32 ? 32 : 64;
  const double mult = P->mode == MODE_BF16X3 ? 3.0 : (P->mode == MODE_BF16 ? 2.0 : 1.0);
  double f = 0.0;
  for (int w = 0; w < 4; ++w) {
    const LoopPass L = loop_pass(P, w);
    std::vector<int4> tab((L.M + BM - 1) / BM);
    if (cudaMemcpy(tab.data(), L.kbt, tab.size() * sizeof(int4), cudaMemcpyDeviceToHost) !=
        cudaSuccess) {
      *msg = "reading the band tables";
      return 2;
    }
    for (const int4& t : tab) f += band_tile_flops(t, KE, LBN, mult) * L.tiles_n;
  }
  P->loop_flops_pair = f;
  P->loop_ok = 1;
  return 0;
}

int tc_loop_supported(const TcPlan* P) { return P && P->loop_ok; }

int tc_loop_resident(const TcPlan* P) { return P && P->loop_ok && P->loop_res; }

double tc_loop_flops(const TcPlan* P, int pairs) { return P->loop_flops_pair * pairs; }

// Tensor maps of the four passes of plan P with 64-wide tiles.
static void loop_maps_of(const TcPlan* P, LoopMaps* maps) {
  for (int w = 0; w < 4; ++w) {
    const bool over_x = (w & 1) == 0;
    const int half = w >> 1;
    const int side = P->absorbed ? half : 0;
    for (int sp = 0; sp < 2; ++sp) {
      maps->K[w][sp] = P->mK[over_x ? 0 : 1][side][sp];
      if (over_x) {
        maps->B[w][sp] = half == 0 ? P->lA[sp] : P->lB[sp];
        maps->O[w][sp] = P->sT[sp];
      } else {
        maps->B[w][sp] = P->lT[sp];
        maps->O[w][sp] = half == 0 ? P->sB[sp] : P->sA[sp];
      }
    }
  }
  maps->Q = P->fQ;
  maps->E = P->fE;
  maps->P = P->fP;
}

cudaError_t tc_enqueue_loop(TcPlan* P, int pairs, cudaStream_t st) {
  if (!P->loop_ok || pairs < 1) return cudaErrorInvalidValue;
  const TcConfig& c = P->cfg;
  LoopMaps maps;
  loop_maps_of(P, &maps);
  LoopArgs args{};
  for (int w = 0; w < 4; ++w) args.pass[w] = loop_pass(P, w);
  args.ctrl = c.ctrl;
  args.P = c.prox;
  args.part = c.part;
  args.nparts = args.pass[1].ntiles;
  args.pairs = pairs;
  args.q = c.q;
  args.b_hi = P->img_b[0];
  args.b_lo = P->img_b[1];
  args.pitch_b = P->px;
  switch (P->mode) {
    case MODE_TF32: return dispatch_loop<MODE_TF32, false>(c.ek, maps, args, P->loop_grid, st);
    case MODE_BF16X3: return dispatch_loop<MODE_BF16X3, false>(c.ek, maps, args, P->loop_grid, st);
    default:
      return P->loop_res ? dispatch_loop<MODE_BF16, true>(c.ek, maps, args, P->loop_grid, st)
                         : dispatch_loop<MODE_BF16, false>(c.ek, maps, args, P->loop_grid, st);
  }
}

// ------------------------------------------------------------ grouped batch (host)
namespace {

template <int MODE, int EK>
cudaError_t set_batch_attr() {
  return cudaFuncSetAttribute(tc_batch_kernel<MODE, EK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)loop_smem_bytes(MODE, false));
}

template <int MODE, int EK>
int batch_blocks_per_sm() {
  int nb = 0;
  if (set_batch_attr<MODE, EK>() != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tc_batch_kernel<MODE, EK>, NTB,
                                                    loop_smem_bytes(MODE, false)) != cudaSuccess)
    return 0;
  return nb;
}

template <int MODE, int EK>
cudaError_t launch_batch(const BatchArgs& args, int grid, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(NTB);
  cfg.dynamicSmemBytes = loop_smem_bytes(MODE, false);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, tc_batch_kernel<MODE, EK>, args);
}

template <int MODE>
int batch_blocks_ek(int ek) {
  return ek == EK_CROWD ? batch_blocks_per_sm<MODE, EK_CROWD>()
         : ek == EK_ENTROPY ? batch_blocks_per_sm<MODE, EK_ENTROPY>()
                            : batch_blocks_per_sm<MODE, EK_POWER>();
}

template <int MODE>
cudaError_t launch_batch_ek(int ek, const BatchArgs& args, int grid, cudaStream_t st) {
  return ek == EK_CROWD ? launch_batch<MODE, EK_CROWD>(args, grid, st)
         : ek == EK_ENTROPY ? launch_batch<MODE, EK_ENTROPY>(args, grid, st)
                            : launch_batch<MODE, EK_POWER>(args, grid, st);
}

}  // namespace

struct TcGroup {
  int mode = 0, ek = 0, F = 0, grid = 0;
  FlowDesc* flows = nullptr;
  LoopMaps* maps = nullptr;
  int4* items[4] = {nullptr, nullptr, nullptr, nullptr};
  int ntiles[4] = {0, 0, 0, 0};
  Ctrl* bctrl = nullptr;
  unsigned* gstop = nullptr;
  double flops_pair = 0.0;
};

void tc_group_destroy(TcGroup* g) {
  if (!g) return;
  cudaFree(g->flows);
  cudaFree(g->maps);
  for (auto* it : g->items) cudaFree(it);
  cudaFree(g->bctrl);
  cudaFree(g->gstop);
  delete g;
}

int tc_group_create(TcPlan* const* plans, int n, TcGroup** out, std::string* msg) {
  *out = nullptr;
  if (n < 1 || n > MAXF) {
    *msg = "a grouped launch takes 1 to 2048 flows";
    return 1;
  }
  const int mode = plans[0]->mode, ek = plans[0]->cfg.ek;
  for (int f = 0; f < n; ++f)
    if (!plans[f]->loop_ok || plans[f]->mode != mode || plans[f]->cfg.ek != ek) {
      *msg = "every flow of a group needs the loop kernel, the group's precision and energy kind";
      return 1;
    }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int nb = mode == MODE_TF32 ? batch_blocks_ek<MODE_TF32>(ek)
                 : mode == MODE_BF16X3 ? batch_blocks_ek<MODE_BF16X3>(ek)
                                       : batch_blocks_ek<MODE_BF16>(ek);
  cudaGetLastError();
  if (nb < 1 || sms < 1) {
    *msg = "the grouped kernel does not fit an SM";
    return 1;
  }
  TcGroup* g = new TcGroup();
  g->mode = mode;
  g->ek = ek;
  g->F = n;
  std::vector<FlowDesc> fd(n);
  std::vector<LoopMaps> mp(n);
  std::vector<int4> items[4];
  for (int f = 0; f < n; ++f) {
    TcPlan* P = plans[f];
    const TcConfig& c = P->cfg;
    loop_maps_of(P, &mp[f]);
    FlowDesc& d = fd[f];
    for (int w = 0; w < 4; ++w) {
      const LoopPass L = loop_pass(P, w);
      d.M[w] = L.M;
      d.N[w] = L.N;
      std::vector<int4> tab((L.M + BM - 1) / BM);
      if (cudaMemcpy(tab.data(), L.kbt, tab.size() * sizeof(int4), cudaMemcpyDeviceToHost) !=
          cudaSuccess) {
        tc_group_destroy(g);
        *msg = "reading the band tables";
        return 2;
      }
      const int epi = (w == 1 || (w == 3 && c.ek == EK_CROWD)) ? 1 : 0;
      for (int t = 0; t < L.ntiles; ++t) {
        const int mt = t / L.tiles_n;
        items[w].push_back(make_int4(f, mt * BM, (t - mt * L.tiles_n) * LBN, 8 * t + 2 * c.ek + epi));
        items[w].push_back(make_int4(tab[mt].x, tab[mt].y, L.M, L.N));
      }
    }
    d.ctrl = c.ctrl;
    d.part = c.part;
    d.nparts = loop_pass(P, 1).ntiles;
    d.ek = c.ek;
    d.P = c.prox;
    g->flops_pair += P->loop_flops_pair;
  }
  int maxt = 0;
  for (int w = 0; w < 4; ++w) {
    g->ntiles[w] = (int)items[w].size() / 2;
    maxt = std::max(maxt, g->ntiles[w]);
  }
  g->grid = std::min(maxt, sms * nb);
  cudaError_t e = cudaMalloc((void**)&g->flows, sizeof(FlowDesc) * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&g->maps, sizeof(LoopMaps) * n);
  for (int w = 0; w < 4 && e == cudaSuccess; ++w)
    e = cudaMalloc((void**)&g->items[w], sizeof(int4) * items[w].size());
  if (e == cudaSuccess) e = cudaMalloc((void**)&g->bctrl, sizeof(Ctrl));
  if (e == cudaSuccess) e = cudaMalloc((void**)&g->gstop, sizeof(unsigned) * (MAXF / 32));
  if (e == cudaSuccess) e = cudaMemcpy(g->flows, fd.data(), sizeof(FlowDesc) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->maps, mp.data(), sizeof(LoopMaps) * n, cudaMemcpyHostToDevice);
  for (int w = 0; w < 4 && e == cudaSuccess; ++w)
    e = cudaMemcpy(g->items[w], items[w].data(), sizeof(int4) * items[w].size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(g->bctrl, 0, sizeof(Ctrl));
  if (e == cudaSuccess) e = cudaMemset(g->gstop, 0, sizeof(unsigned) * (MAXF / 32));
  if (e != cudaSuccess) {
    tc_group_destroy(g);
    *msg = std::string("grouped launch set-up: ") + cudaGetErrorName(e);
    return 2;
  }
  *out = g;
  return 0;
}

cudaError_t tc_group_begin_step(TcGroup* g, cudaStream_t st) {
  return cudaMemsetAsync(g->bctrl, 0, sizeof(Ctrl), st);
}

cudaError_t tc_group_enqueue(TcGroup* g, int pairs, cudaStream_t st) {
  if (!g || pairs < 1) return cudaErrorInvalidValue;
  BatchArgs a{};
  a.flows = g->flows;
  a.maps = g->maps;
  for (int w = 0; w < 4; ++w) {
    a.items[w] = g->items[w];
    a.ntiles[w] = g->ntiles[w];
  }
  a.bctrl = g->bctrl;
  a.gstop = g->gstop;
  a.F = g->F;
  a.pairs = pairs;
  switch (g->mode) {
    case MODE_TF32: return launch_batch_ek<MODE_TF32>(g->ek, a, g->grid, st);
    case MODE_BF16X3: return launch_batch_ek<MODE_BF16X3>(g->ek, a, g->grid, st);
    default: return launch_batch_ek<MODE_BF16>(g->ek, a, g->grid, st);
  }
}

int tc_group_flows(const TcGroup* g) { return g ? g->F : 0; }

double tc_group_flops(const TcGroup* g, int pairs) { return g ? g->flops_pair * pairs : 0.0; }


}  // namespace jko
