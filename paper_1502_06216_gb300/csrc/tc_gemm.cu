// tc_gemm.cu -- tensor-core form of the Gibbs-kernel application (tcgen05 +
// TMA + TMEM, sm_103a) with the scaling and proximal updates fused into the
// GEMM epilogues.
//
// xi X = K_y X K_x^T (Sec. 4.1) is two dense contractions.  Each pass computes
//     D[m][n] = sum_k K[m][k] B[n][k]
// with K a 1-D Gibbs factor (symmetric, n_k x n_k) and B an image stored with
// its contracted axis contiguous, so both operands are K-major:
//   pass 0 / 2:  K = K_x, B = a / b as [ny][nx]   ->  D = T^T  as [nx][ny]
//   pass 1 / 3:  K = K_y, B = T^T as [nx][ny]     ->  D = xi a / xi b as [ny][nx]
// Pass 1 carries  b = q / xi a  and the residual (Eq. update-formula-1, the
// stopping rule of Sec. 3.4); pass 3 carries  p = Prox_{sigma f}(s),  a = p / s
// (Eq. update-formula-2, Eq. defn-pell).
//
// One CTA computes a 128 x BN tile: warp 0 (one lane) streams K-blocks of the
// kernel factor and of the image through a ring of shared-memory stages with
// TMA (128-byte swizzle), warp 1 (one lane) issues tcgen05.mma into a TMEM
// accumulator and commits each stage back to the producer, and all four warps
// then drain TMEM (tcgen05.ld) through the epilogue.  Only the K-blocks that
// meet the band |m - k| <= r are visited, r being the last offset at which the
// factor is a normal number in the operand precision (entries beyond it are
// stored as exact zeros), so the skipped tiles contribute exactly zero.
//
// Precision modes (see img_split / fac_split in tc_common.cuh): TF32
// (kind::tf32, operands rounded to tf32), BF16 (bf16 factor times the image
// as a bf16 pair hi + lo: one MMA of width 2 BN), BF16X3 (that plus the
// factor's lo part times the image's hi part).  Accumulation is FP32 in TMEM
// throughout.
#include "tc_common.cuh"

namespace jko {

namespace {

struct TcPassArgs {
  int M, N, Kdim;         // D is M x N, contraction length Kdim (= M)
  int pitch_out;          // row pitch (elements) of the operand-typed output image
  void* out_hi;           // EPI_STORE: T^T ; EPI_B: b ; EPI_A: a   (operand type)
  void* out_lo;           // BF16X3 low parts
  float* p;               // EPI_A
  const float* q;         // EPI_B
  Ctrl* ctrl;
  ProxArgs<float> P;
  int tma_epi;            // 1: epilogue tiles moved by TMA (fp32 fields with nx % 4 == 0)
  const int4* kbt;        // per 128-row tile: band of the factor (band_tile)
  double* part;           // residual partials, one per block of the b-update pass
  int nparts;             // partials read by the deciding pass
  int decide;             // 1: this pass takes the stop decision (stop_gate)
};

template <int MODE, int EPI, int EK, int BN>
__global__ void __launch_bounds__(NT, 1)
tc_pass_kernel(const __grid_constant__ CUtensorMap mapA_hi, const __grid_constant__ CUtensorMap mapA_lo,
               const __grid_constant__ CUtensorMap mapB_hi, const __grid_constant__ CUtensorMap mapB_lo,
               const __grid_constant__ CUtensorMap mapO_hi, const __grid_constant__ CUtensorMap mapO_lo,
               const __grid_constant__ CUtensorMap mapF, const __grid_constant__ CUtensorMap mapP,
               TcPassArgs args) {
  using T = typename OpT<MODE>::T;
  constexpr int KE = OpT<MODE>::kElems;                  // elements per K-block
  constexpr int UK = (MODE == MODE_TF32) ? 8 : 16;      // K per MMA
  constexpr int NSPLIT = img_split(MODE) ? 2 : 1;        // image hi (+ lo) tiles
  constexpr uint32_t A_BYTES = BM * KB_BYTES;
  constexpr uint32_t B_BYTES = BN * KB_BYTES;
  constexpr uint32_t STAGE_BYTES = stage_bytes(MODE, BN);
  constexpr uint32_t ALO_OFF = A_BYTES + NSPLIT * B_BYTES;  // factor lo (BF16X3)
  constexpr int STAGES = num_stages(MODE, EPI, BN);
  constexpr uint32_t EPI_BYTES = epi_bytes(MODE, EPI, BN);
  // the prox pass loads e^{-sigma w} only for the congestion/potential kind
  constexpr uint32_t EPI_LOAD =
      (EPI == EPI_A && EK != EK_CROWD) ? 0u : epi_load_bytes(MODE, EPI, BN);
  constexpr uint32_t F32_TILE = (uint32_t)BN * BM * 4u;   // one fp32 epilogue tile
  static_assert(STAGES >= 2, "at least two stages");
  constexpr uint32_t TMEM_COLS = acc_cols(MODE, BN);

  Ctrl* ctrl = args.ctrl;
  __shared__ int s_it;

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* epi_f = smem + STAGES * STAGE_BYTES;   // q (b pass) or e^{-sigma w} (prox)
  unsigned char* epi_g = epi_f + F32_TILE;                // old b (b pass) or p (prox)
  uint64_t* full_bar = (uint64_t*)(smem + STAGES * STAGE_BYTES + EPI_BYTES);
  uint64_t* empty_bar = full_bar + STAGES;
  uint64_t* accum_bar = empty_bar + STAGES;
  uint64_t* epi_bar = accum_bar + 1;
  uint32_t* tmem_slot = (uint32_t*)(epi_bar + 1);
  __shared__ int s_fault;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN;
  const int m0 = blockIdx.y * BM;

  // K-blocks holding the non-zero band of rows [m0, m0 + BM) of the factor
  const int4 kb = args.kbt[blockIdx.y];
  const int nkb = kb.y;

  if (threadIdx.x == 0) {
    s_fault = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(accum_bar, 1);
    mbar_init(epi_bar, 1);
    fence_mbar_init();
    tma_prefetch_desc(&mapA_hi);
    tma_prefetch_desc(&mapB_hi);
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  // Everything above touches no data of the preceding kernel, so it overlaps
  // that kernel's tail; from here on its results are read.
  pdl_launch_dependents();
  pdl_wait();
  if (stop_gate(ctrl, args.part, args.nparts, args.decide != 0, &s_it)) {
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem_base, TMEM_COLS);
    return;
  }

  const bool tma_epi = EPI != EPI_STORE && args.tma_epi;
  bool ok = true;
  if (warp == 0 && lane == 0) {
    // ---- TMA producer: epilogue tiles first (independent of the MMAs) ----
    if (tma_epi) {
      mbar_arrive_expect_tx(epi_bar, EPI_LOAD);
      if (EPI == EPI_B || EK == EK_CROWD) {
#pragma unroll
        for (int cb = 0; cb < BN / 32; ++cb)
          tma_load_2d(epi_f + cb * (BM * 128), &mapF, epi_bar, n0 + cb * 32, m0);
      }
      if constexpr (EPI == EPI_B) {
        constexpr int CBO = BN * (int)sizeof(T) / 128;
        constexpr int KEO = 128 / (int)sizeof(T);
#pragma unroll
        for (int cb = 0; cb < CBO; ++cb) {
          tma_load_2d(epi_g + cb * (BM * 128), &mapO_hi, epi_bar, n0 + cb * KEO, m0);
          if constexpr (NSPLIT == 2)
            tma_load_2d(epi_g + (CBO + cb) * (BM * 128), &mapO_lo, epi_bar, n0 + cb * KEO, m0);
        }
      }
    }
    for (int i = 0; i < nkb && ok; ++i) {
      const int s = i % STAGES;
      if (i >= STAGES) ok = mbar_wait(&empty_bar[s], ((i / STAGES) - 1) & 1);
      if (!ok) break;
      unsigned char* st = smem + s * STAGE_BYTES;
      mbar_arrive_expect_tx(&full_bar[s], STAGE_BYTES);
      const int kx = kb.x + i * KE;
      tma_load_2d(st, &mapA_hi, &full_bar[s], kx, m0);
      tma_load_2d(st + A_BYTES, &mapB_hi, &full_bar[s], kx, n0);
      if constexpr (NSPLIT == 2) tma_load_2d(st + A_BYTES + B_BYTES, &mapB_lo, &full_bar[s], kx, n0);
      if constexpr (fac_split(MODE)) tma_load_2d(st + ALO_OFF, &mapA_lo, &full_bar[s], kx, m0);
    }
    if (!ok) atomicOr(&s_fault, 1);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    for (int i = 0; i < nkb && ok; ++i) {
      const int s = i % STAGES;
      ok = mbar_wait(&full_bar[s], (i / STAGES) & 1);
      if (!ok) break;
      tc_fence_after();
      const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
      const uint64_t a_hi = sdesc_sw128(sa);
      const uint64_t a_lo = sdesc_sw128(sa + ALO_OFF);
      const uint64_t b = sdesc_sw128(sa + A_BYTES);
#pragma unroll
      for (int kk = 0; kk < KB_BYTES / 32; ++kk)   // 32 bytes of K per MMA
        umma_kstep<MODE, BN>(tmem_base, a_hi, a_lo, b, kk, (i > 0 || kk > 0) ? 1u : 0u);
      umma_commit(&empty_bar[s]);   // frees the stage once these MMAs have read it
    }
    umma_commit(accum_bar);          // accumulator complete
    if (!ok) atomicOr(&s_fault, 1);
  }
  (void)UK;
  __syncwarp();

  // ---- epilogue: all four warps, warp w owns TMEM lanes 32w .. 32w+31 ----
  bool have = mbar_wait(accum_bar, 0);
  if (have && tma_epi) have = mbar_wait(epi_bar, 0);
  if (!have) atomicOr(&s_fault, 1);
  __syncwarp();
  tc_fence_after();

  // The operand-typed output tile is staged in shared memory (the pipeline
  // stages are free once the accumulator is complete) and written with TMA.
  constexpr int CB = BN * (int)sizeof(T) / 128;       // 128-byte column blocks
  constexpr uint32_t OUT_BLOCK = BM * 128;
  static_assert((NSPLIT * CB) * OUT_BLOCK <= STAGES * STAGE_BYTES, "staging fits the stages");
  unsigned char* st_hi = smem;
  unsigned char* st_lo = smem + CB * OUT_BLOCK;
  // warp w reads TMEM lanes 32 (w % 4) .. +31 (its quadrant) and the column
  // group w / 4 of the tile: chunks [g CPG, (g + 1) CPG) of 16 columns
  const int quad = warp & 3;
  const int grp = warp >> 2;
  const int rl = quad * 32 + lane;
  const int m = m0 + rl;
  const bool row_ok = m < args.M;
  const bool vec_in = (args.N & 3) == 0;
  float res_f = 0.0f;  // this thread's residual terms (FP32, one rounding each)
  int bad = 0;
  const bool have_prev = (EPI == EPI_B) ? (s_it > 0) : false;
  const T* cur_hi = (const T*)args.out_hi;
  const T* cur_lo = (const T*)args.out_lo;
  if (have) {
    // all TMEM loads of this thread's row first, one wait, then the chunks
    // unrolled so that their shared-memory loads and arithmetic overlap
    constexpr int NCH = BN / 16 / NWG;   // chunks per thread
    static_assert(NCH >= 1 && NCH * 16 * NWG == BN, "column groups cover the tile");
    static_assert(NCH == 1 || !img_split(MODE), "split images: one chunk per thread");
    uint32_t racc[NCH][16];
    float vsum[16];
    if constexpr (img_split(MODE)) {
      tmem_tile16<MODE, BN>(tmem_base + ((uint32_t)(quad * 32) << 16), grp * 16, vsum);
    } else {
#pragma unroll
      for (int cc = 0; cc < NCH; ++cc)
        tmem_ld16_issue(tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)((grp * NCH + cc) * 16),
                        racc[cc]);
      tmem_wait_ld();
#pragma unroll
      for (int cc = 0; cc < NCH; ++cc) reg_fence16(racc[cc]);
    }
#pragma unroll
    for (int cc = 0; cc < NCH; ++cc) {
      const int c = grp * NCH + cc;
      float v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = img_split(MODE) ? vsum[j] : __uint_as_float(racc[cc][j]);
      const int nb = n0 + c * 16;
      int cnt = args.N - nb;
      cnt = !row_ok || cnt < 0 ? 0 : (cnt > 16 ? 16 : cnt);
      float o[16];
      if (EPI == EPI_STORE) {
#pragma unroll
        for (int j = 0; j < 16; ++j) o[j] = v[j];
      } else if (EPI == EPI_B) {
        const size_t irow = (size_t)m * args.N + nb;   // q is [M][N] unpadded
        float qv[16], bo[16];
        if (tma_epi) {
          smem_ld_f32x16(epi_f, rl, c, qv);
          if (have_prev)
            smem_ld_op16<MODE>(epi_g, epi_g + (BN * (int)sizeof(T) / 128) * (BM * 128), rl, c, bo);
        } else {
          load_f32x16(args.q + (cnt ? irow : 0), cnt, vec_in, qv);
          if (have_prev)
            load_op16<MODE>(cur_hi, cur_lo, cnt ? (size_t)m * args.pitch_out + nb : 0, cnt, bo);
        }
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
      } else {  // EPI_A
        const size_t irow = (size_t)m * args.N + nb;
        float ev[16], pv[16];
        if (EK == EK_CROWD) {
          if (tma_epi) smem_ld_f32x16(epi_f, rl, c, ev);
          else load_f32x16(args.P.E + (cnt ? irow : 0), cnt, vec_in, ev);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          if (j < cnt) {
            const float a = prox_ratio_e<float, EK>(args.P, (int)(irow + j), v[j],
                                                     EK == EK_CROWD ? ev[j] : 0.0f);
            bad |= !isfinite(a);
            o[j] = a;
            pv[j] = a * v[j];
          } else {
            o[j] = 0.0f;
            pv[j] = 0.0f;
          }
        }
        if (tma_epi) smem_st_f32x16(epi_g, rl, c, pv);
        else if (cnt) store_f32x16(args.p + irow, cnt, vec_in, pv);
      }
      stage16<MODE>(st_hi, st_lo, rl, c, o);
    }
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && have) {
    constexpr int KEo = 128 / (int)sizeof(T);  // columns per block
#pragma unroll
    for (int cb = 0; cb < CB; ++cb) {
      tma_store_2d(&mapO_hi, st_hi + cb * OUT_BLOCK, n0 + cb * KEo, m0);
      if constexpr (NSPLIT == 2) tma_store_2d(&mapO_lo, st_lo + cb * OUT_BLOCK, n0 + cb * KEo, m0);
    }
    if (EPI == EPI_A && tma_epi) {
#pragma unroll
      for (int cb = 0; cb < BN / 32; ++cb)
        tma_store_2d(&mapP, epi_g + cb * (BM * 128), n0 + cb * 32, m0);
    }
    bulk_commit();
    bulk_wait_all();
  }
  if (warp == 1) tmem_dealloc(tmem_base, TMEM_COLS);

  if (EPI == EPI_STORE) {
    if (threadIdx.x == 0 && s_fault) atomicOr(&ctrl->nonfinite, 2);
    return;
  }
  // ---- residual partial / flags / pair counter (see stop_gate) ----
  bad = warp_or(bad);
  if (EPI == EPI_B) {
    __shared__ float s_redf[16];
    const double res = (double)tile_sum16(res_f, s_redf, [] { __syncthreads(); });
    if (threadIdx.x == 0) args.part[blockIdx.y * gridDim.x + blockIdx.x] = res;
  }
  if (lane == 0 && bad) atomicOr(&ctrl->nonfinite, 1);
  if (threadIdx.x == 0 && s_fault) atomicOr(&ctrl->nonfinite, 2);
  if (EPI == EPI_A && threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0) ctrl->it = s_it + 1;
}

// The plan's scaling images (operand type, [ny][pitch]) as fp32 [ny][nx]:
// the operand value hi (+ lo) the passes multiply with.
template <typename T>
__global__ void export_op_kernel(const T* hi, const T* lo, int pitch, float* dst, int nx, int ny) {
  const long long n = (long long)nx * ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long y = i / nx, x = i - y * nx;
    const long long k = y * pitch + x;
    if constexpr (sizeof(T) == 4) dst[i] = hi[k];
    else dst[i] = __bfloat162float(hi[k]) + __bfloat162float(lo[k]);
  }
}

// a = 1 in operand precision (cold start), padded columns included.
template <typename T>
__global__ void fill_op_kernel(T* hi, T* lo, long long n, float v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if constexpr (sizeof(T) == 4) {
      hi[i] = v;
    } else {
      hi[i] = __float2bfloat16_rn(v);
      if (lo) lo[i] = __float2bfloat16_rn(0.0f);
    }
  }
}


}  // namespace

namespace {

template <int MODE, int EPI, int EK, int BN>
size_t smem_bytes() {
  constexpr int ST = num_stages(MODE, EPI, BN);
  return (size_t)ST * stage_bytes(MODE, BN) + epi_bytes(MODE, EPI, BN) + 1024 + (2 * ST + 2) * 8 +
         16;
}

struct Maps {
  const CUtensorMap *a_hi, *a_lo, *b_hi, *b_lo, *o_hi, *o_lo, *f, *pm;
};

template <int MODE, int EPI, int EK, int BN>
cudaError_t launch_pass(const Maps& M, const TcPassArgs& args, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((args.N + BN - 1) / BN, (args.M + BM - 1) / BM);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem_bytes<MODE, EPI, EK, BN>();
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, tc_pass_kernel<MODE, EPI, EK, BN>, *M.a_hi, *M.a_lo, *M.b_hi,
                            *M.b_lo, *M.o_hi, *M.o_lo, *M.f, *M.pm, args);
}

template <int MODE, int EPI, int EK, int BN>
cudaError_t set_attr() {
  return cudaFuncSetAttribute(tc_pass_kernel<MODE, EPI, EK, BN>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_bytes<MODE, EPI, EK, BN>());
}

template <int MODE, int BN>
cudaError_t set_attrs_bn() {
  cudaError_t e;
  if ((e = set_attr<MODE, EPI_STORE, EK_CROWD, BN>()) != cudaSuccess) return e;
  if ((e = set_attr<MODE, EPI_B, EK_CROWD, BN>()) != cudaSuccess) return e;
  if ((e = set_attr<MODE, EPI_A, EK_CROWD, BN>()) != cudaSuccess) return e;
  if ((e = set_attr<MODE, EPI_A, EK_ENTROPY, BN>()) != cudaSuccess) return e;
  return set_attr<MODE, EPI_A, EK_POWER, BN>();
}

// 128-wide tiles exist for the forms whose epilogue tiles leave room for at
// least two pipeline stages: TF32 (the image pairs of BF16 / BF16X3 double
// the image blocks and the old-b tile).
template <int MODE>
constexpr bool has_bn128() { return !img_split(MODE); }

template <int MODE>
cudaError_t set_attrs() {
  cudaError_t e = set_attrs_bn<MODE, 64>();
  if (e != cudaSuccess) return e;
  if constexpr (has_bn128<MODE>()) return set_attrs_bn<MODE, 128>();
  return cudaSuccess;
}

template <int MODE, int BN>
cudaError_t dispatch_epi(int epi, int ek, const Maps& M, const TcPassArgs& args, cudaStream_t st) {
  if (epi == EPI_STORE) return launch_pass<MODE, EPI_STORE, EK_CROWD, BN>(M, args, st);
  if (epi == EPI_B) return launch_pass<MODE, EPI_B, EK_CROWD, BN>(M, args, st);
  if (ek == EK_CROWD) return launch_pass<MODE, EPI_A, EK_CROWD, BN>(M, args, st);
  if (ek == EK_ENTROPY) return launch_pass<MODE, EPI_A, EK_ENTROPY, BN>(M, args, st);
  return launch_pass<MODE, EPI_A, EK_POWER, BN>(M, args, st);
}

template <int MODE>
cudaError_t dispatch_bn(int bn, int epi, int ek, const Maps& M, const TcPassArgs& args,
                        cudaStream_t st) {
  if constexpr (has_bn128<MODE>()) {
    if (bn == 128) return dispatch_epi<MODE, 128>(epi, ek, M, args, st);
  }
  return dispatch_epi<MODE, 64>(epi, ek, M, args, st);
}

// Smallest normal FP32 (and BF16) number: factor entries below it are stored
// as exact zeros, so the K-blocks that hold none of the rest contribute nothing.
constexpr double kNormalMin = 1.1754943508222875e-38;

// Log-scale of one axis for the absorption: beta_axis(i) = -sigma (w_axis(i) -
// mean(w)/2), w_axis = mean of w over the other axis, so beta_x(x) + beta_y(y)
// = -sigma (additive separable fit of w).  Zero without absorption.
void axis_logscale(const TcConfig& c, int axis, std::vector<double>& beta) {
  const int nx = c.nx, ny = c.ny;
  const int n = axis == 0 ? nx : ny;
  beta.assign(n, 0.0);
  if (!c.absorb || !c.w_host) return;
  double tot = 0.0;
  for (long long i = 0; i < (long long)nx * ny; ++i) tot += c.w_host[i];
  const double mean = tot / ((double)nx * ny);
  for (int i = 0; i < n; ++i) {
    double acc = 0.0;
    if (axis == 0) for (int y = 0; y < ny; ++y) acc += c.w_host[(size_t)y * nx + i];
    else for (int x = 0; x < nx; ++x) acc += c.w_host[(size_t)i * nx + x];
    const double wm = acc / (axis == 0 ? ny : nx);
    beta[i] = -c.sigma * (wm - 0.5 * mean);
  }
}

// Factor of one axis and side in operand precision, hi (+ lo) [n][pitch]:
//   a side  K~[i][j] = exp(-(i-j)^2 h^2 / gamma + beta(j) - beta(i))
//   b side  the transpose.
// Also the per-tile K-block ranges of its non-zero entries.  Returns false if
// an entry would overflow FP32.
template <typename T>
bool build_factor(std::vector<T>& hi, std::vector<T>& lo, std::vector<int4>& kbt, int n,
                  int pitch, double length, double gamma, const std::vector<double>& beta,
                  bool transpose, int KE) {
  const double h = length / n;
  hi.assign((size_t)n * pitch, T(0.0f));
  lo.assign((size_t)n * pitch, T(0.0f));
  const int tiles = (n + BM - 1) / BM;
  std::vector<int> kmin(tiles, n), kmax(tiles, -1);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double d = (i - j) * h;
      const double ex = -(d * d) / gamma + (transpose ? beta[i] - beta[j] : beta[j] - beta[i]);
      if (ex > 88.0) return false;
      const double v = std::exp(ex);
      if (v < kNormalMin) continue;
      const int t = i / BM;
      kmin[t] = std::min(kmin[t], j);
      kmax[t] = std::max(kmax[t], j);
      if constexpr (sizeof(T) == 4) {
        // round to tf32 (10 mantissa bits, nearest-away as cvt.rna)
        float f = (float)v;
        uint32_t u;
        std::memcpy(&u, &f, 4);
        u = (u + 0x1000u) & 0xFFFFE000u;
        std::memcpy(&f, &u, 4);
        hi[(size_t)i * pitch + j] = f;
      } else {
        const float f = (float)v;
        const __nv_bfloat16 bh = __float2bfloat16_rn(f);
        hi[(size_t)i * pitch + j] = bh;
        lo[(size_t)i * pitch + j] = __float2bfloat16_rn(f - __bfloat162float(bh));
      }
    }
  // K-blocks from the first non-zero column rounded down to a whole 128-byte
  // block: a box row that straddles two 128-byte lines costs the TMA two L2
  // requests (measured: 380 instead of 160 ns per 64-row box), which more
  // than cancels the block saved.
  constexpr int ALIGN = 128 / (int)sizeof(T);
  kbt.assign(tiles, make_int4(0, 0, 0, -1));
  for (int t = 0; t < tiles; ++t)
    if (kmax[t] >= 0) {
      const int k0 = kmin[t] / ALIGN * ALIGN;
      kbt[t] = make_int4(k0, (kmax[t] - k0) / KE + 1, kmin[t], kmax[t]);
    }
  return true;
}

template <typename T>
cudaError_t alloc_img(void** p, size_t elems) {
  cudaError_t e = cudaMalloc(p, elems * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemset(*p, 0, elems * sizeof(T));
}

// The absorbed energy: e^{-(sigma w + beta)} (congestion) or sigma w + beta.
int absorbed_energy(TcPlan* P, const std::vector<double>& bx, const std::vector<double>& by,
                    std::string* msg) {
  TcConfig& c = P->cfg;
  const int nx = c.nx, ny = c.ny;
  std::vector<float> v((size_t)nx * ny);
  const bool crowd = c.ek == EK_CROWD;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const double t = c.sigma * c.w_host[(size_t)y * nx + x] + bx[x] + by[y];
      v[(size_t)y * nx + x] = crowd ? (float)std::exp(-t) : (float)t;
    }
  float** dst = crowd ? &P->E_abs : &P->sw_abs;
  if (cudaMalloc((void**)dst, v.size() * sizeof(float)) != cudaSuccess ||
      cudaMemcpy(*dst, v.data(), v.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
    *msg = "upload of the absorbed energy";
    return 2;
  }
  if (crowd) c.prox.E = P->E_abs;
  else c.prox.sw = P->sw_abs;
  return 0;
}

// Executed flops of each pass for the current tile widths, from the band tables.
void pass_flops_of(TcPlan* P) {
  const TcConfig& c = P->cfg;
  const int KE = P->mode == MODE_TF32 ? 32 : 64;
  const double mult = P->mode == MODE_BF16X3 ? 3.0 : (P->mode == MODE_BF16 ? 2.0 : 1.0);
  for (int pass = 0; pass < 4; ++pass) {
    const int axis = (pass & 1) == 0 ? 0 : 1;
    const int side = P->absorbed ? (pass >> 1) : 0;
    const int M = axis == 0 ? c.nx : c.ny, N = axis == 0 ? c.ny : c.nx;
    const int bn = axis == 0 ? P->bn_x : P->bn_y;
    std::vector<int4> tab((M + BM - 1) / BM);
    cudaMemcpy(tab.data(), P->kbt[axis][side], tab.size() * sizeof(int4), cudaMemcpyDeviceToHost);
    double f = 0.0;
    for (const int4& t : tab) f += band_tile_flops(t, KE, bn, mult) * ((N + bn - 1) / bn);
    P->flops[pass] = f;
  }
}

template <typename T>
int create_typed(TcPlan* P, std::string* msg) {
  TcConfig& c = P->cfg;
  const int nx = c.nx, ny = c.ny;
  const int align = 16 / (int)sizeof(T);
  P->px = round_up(nx, align);
  P->py = round_up(ny, align);
  const int nsplit = img_split(P->mode) ? 2 : 1;        // image hi (+ lo)
  const int ksplit = fac_split(P->mode) ? 2 : 1;        // factor hi (+ lo)
  const int KE = P->mode == MODE_TF32 ? 32 : 64;
  P->absorbed = c.absorb && c.w_host ? 1 : 0;
  std::vector<double> beta[2];
  axis_logscale(c, 0, beta[0]);
  axis_logscale(c, 1, beta[1]);
  std::vector<T> hi, lo;
  std::vector<int4> kbt;
  for (int axis = 0; axis < 2; ++axis) {
    const int n = axis == 0 ? nx : ny;
    const int pitch = axis == 0 ? P->px : P->py;
    for (int side = 0; side < (P->absorbed ? 2 : 1); ++side) {
      if (!build_factor<T>(hi, lo, kbt, n, pitch, axis == 0 ? c.lx : c.ly, c.gamma, beta[axis],
                           side == 1, KE)) {
        *msg = "absorbed Gibbs factor overflows FP32 (potential too steep for gamma)";
        return 1;
      }
      for (int sp = 0; sp < ksplit; ++sp) {
        const auto& src = sp == 0 ? hi : lo;
        if (cudaMalloc(&P->k[axis][side][sp], src.size() * sizeof(T)) != cudaSuccess ||
            cudaMemcpy(P->k[axis][side][sp], src.data(), src.size() * sizeof(T),
                       cudaMemcpyHostToDevice) != cudaSuccess) {
          *msg = "upload of a Gibbs factor";
          return 2;
        }
      }
      if (cudaMalloc((void**)&P->kbt[axis][side], kbt.size() * sizeof(int4)) != cudaSuccess ||
          cudaMemcpy(P->kbt[axis][side], kbt.data(), kbt.size() * sizeof(int4),
                     cudaMemcpyHostToDevice) != cudaSuccess) {
        *msg = "upload of the band tables";
        return 2;
      }
    }
  }
  if (P->absorbed) {
    const int rc = absorbed_energy(P, beta[0], beta[1], msg);
    if (rc) return rc;
  }
  for (int sp = 0; sp < nsplit; ++sp) {
    if (alloc_img<T>(&P->img_a[sp], (size_t)ny * P->px) != cudaSuccess ||
        alloc_img<T>(&P->img_b[sp], (size_t)ny * P->px) != cudaSuccess ||
        alloc_img<T>(&P->img_t[sp], (size_t)nx * P->py) != cudaSuccess) {
      *msg = "cudaMalloc operand images";
      return 2;
    }
  }
  // tile widths: BN = 128 when that still fills the GPU, else 64
  auto pick = [](int M, int N) { return ((M + BM - 1) / BM) * ((N + 127) / 128) >= 152 ? 128 : 64; };
  P->bn_x = pick(nx, ny);  // pass over x: M = nx, N = ny
  P->bn_y = pick(ny, nx);  // pass over y: M = ny, N = nx
  if (img_split(P->mode)) P->bn_x = P->bn_y = 64;
  // tensor maps (hi and lo; lo maps alias hi when unused; b side aliases a side)
  const int m = P->mode;
  for (int sp = 0; sp < 2; ++sp) {
    const int si = sp < nsplit ? sp : 0;
    const int ki = sp < ksplit ? sp : 0;
    bool ok = true;
    for (int axis = 0; axis < 2 && ok; ++axis)
      for (int side = 0; side < 2 && ok; ++side) {
        const int sd = P->absorbed ? side : 0;
        const int n = axis == 0 ? nx : ny;
        ok = make_map(&P->mK[axis][side][sp], P->k[axis][sd][ki], m, n, n,
                      axis == 0 ? P->px : P->py, BM);
      }
    // image operand loads: boxes of 64 rows (64-wide tiles) and, where the
    // mode has them, 128 rows (128-wide tiles)
    const int wide = img_split(m) ? 64 : 128;
    ok = ok && make_map(&P->lA[sp], P->img_a[si], m, ny, nx, P->px, 64) &&
         make_map(&P->lB[sp], P->img_b[si], m, ny, nx, P->px, 64) &&
         make_map(&P->lT[sp], P->img_t[si], m, nx, ny, P->py, 64) &&
         make_map(&P->mA[sp], P->img_a[si], m, ny, nx, P->px, wide) &&
         make_map(&P->mB[sp], P->img_b[si], m, ny, nx, P->px, wide) &&
         make_map(&P->mT[sp], P->img_t[si], m, nx, ny, P->py, wide) &&
         make_map(&P->sA[sp], P->img_a[si], m, ny, nx, P->px, BM) &&
         make_map(&P->sB[sp], P->img_b[si], m, ny, nx, P->px, BM) &&
         make_map(&P->sT[sp], P->img_t[si], m, nx, ny, P->py, BM);
    if (!ok) { *msg = "cuTensorMapEncodeTiled failed"; return 2; }
  }
  if (!P->absorbed)
    for (int axis = 0; axis < 2; ++axis) P->kbt[axis][1] = P->kbt[axis][0];
  // fp32 fields [ny][nx] (q, e^{-sigma w}, p) as TMA tiles when rows are 16-byte multiples
  P->tma_epi = (nx % 4 == 0) ? 1 : 0;
  P->fQ = P->fE = P->fP = P->mK[0][0][0];
  if (P->tma_epi) {
    bool ok = make_map(&P->fQ, (void*)c.q, MODE_TF32, ny, nx, nx, BM) &&
              make_map(&P->fP, (void*)c.p, MODE_TF32, ny, nx, nx, BM);
    if (ok && c.ek == EK_CROWD && c.prox.E)
      ok = make_map(&P->fE, (void*)c.prox.E, MODE_TF32, ny, nx, nx, BM);
    if (!ok) { *msg = "cuTensorMapEncodeTiled failed (fields)"; return 2; }
  }
  pass_flops_of(P);
  cudaError_t ea = m == MODE_TF32 ? set_attrs<MODE_TF32>()
                                  : (m == MODE_BF16X3 ? set_attrs<MODE_BF16X3>() : set_attrs<MODE_BF16>());
  if (ea != cudaSuccess) { *msg = "cudaFuncSetAttribute (shared memory)"; return 2; }
  return tc_loop_setup(P, msg);
}

}  // namespace

int tc_create(const TcConfig& cfg, TcPlan** out, std::string* msg) {
  *out = nullptr;
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) {
    *msg = "tensor-core precisions need an sm_103 GPU (GB300)";
    return 1;
  }
  if (!get_encode()) { *msg = "cuTensorMapEncodeTiled is unavailable"; return 1; }
  TcPlan* P = new TcPlan();
  P->cfg = cfg;
  P->mode = cfg.precision == JKO_TF32 ? MODE_TF32 : (cfg.precision == JKO_BF16X3 ? MODE_BF16X3 : MODE_BF16);
  const int rc = P->mode == MODE_TF32 ? create_typed<float>(P, msg) : create_typed<__nv_bfloat16>(P, msg);
  if (rc != 0) { tc_destroy(P); return rc; }
  *out = P;
  return 0;
}

cudaError_t tc_log_begin_step(TcPlan* P, cudaStream_t st);
cudaError_t tc_log_enqueue_pass(TcPlan* P, int which, cudaStream_t st);

int tc_logdomain(const TcPlan* P) { return P ? P->logd : 0; }

cudaError_t tc_begin_step(TcPlan* P, cudaStream_t st) {
  if (P->logd) {
    cudaError_t e = tc_log_begin_step(P, st);
    if (e != cudaSuccess) return e;
  }
  const long long n = (long long)P->cfg.ny * P->px;
  if (P->mode == MODE_TF32)
    fill_op_kernel<float><<<152 * 4, 256, 0, st>>>((float*)P->img_a[0], nullptr, n, 1.0f);
  else
    fill_op_kernel<__nv_bfloat16><<<152 * 4, 256, 0, st>>>(
        (__nv_bfloat16*)P->img_a[0], (__nv_bfloat16*)P->img_a[1], n, 1.0f);
  return cudaGetLastError();
}

cudaError_t tc_export_scalings(const TcPlan* P, float* a, float* b, cudaStream_t st) {
  const int nx = P->cfg.nx, ny = P->cfg.ny;
  if (P->mode == MODE_TF32) {
    export_op_kernel<float><<<152 * 4, 256, 0, st>>>((const float*)P->img_a[0], nullptr, P->px, a, nx, ny);
    export_op_kernel<float><<<152 * 4, 256, 0, st>>>((const float*)P->img_b[0], nullptr, P->px, b, nx, ny);
  } else {
    export_op_kernel<__nv_bfloat16><<<152 * 4, 256, 0, st>>>(
        (const __nv_bfloat16*)P->img_a[0], (const __nv_bfloat16*)P->img_a[1], P->px, a, nx, ny);
    export_op_kernel<__nv_bfloat16><<<152 * 4, 256, 0, st>>>(
        (const __nv_bfloat16*)P->img_b[0], (const __nv_bfloat16*)P->img_b[1], P->px, b, nx, ny);
  }
  return cudaGetLastError();
}

cudaError_t tc_enqueue_pass(TcPlan* P, int which, cudaStream_t st) {
  if (P->logd) return tc_log_enqueue_pass(P, which, st);
  const TcConfig& c = P->cfg;
  const bool over_x = (which & 1) == 0;
  const int half = which >> 1;
  TcPassArgs a{};
  a.ctrl = c.ctrl;
  a.P = c.prox;   // absorbed energy images when the plan absorbs the potential
  a.q = c.q;
  a.p = c.p;
  a.part = c.part;
  a.nparts = ((c.nx + P->bn_y - 1) / P->bn_y) * ((c.ny + BM - 1) / BM);  // b-update grid
  Maps mp{};
  int bn, epi;
  const int side = P->absorbed ? half : 0;  // xi a uses K~, xi b its transpose
  if (over_x) {  // K_x . image^T -> T^T [nx][ny]
    a.M = c.nx; a.N = c.ny; a.Kdim = c.nx;
    a.kbt = P->kbt[0][side];
    a.pitch_out = P->py;
    a.out_hi = P->img_t[0]; a.out_lo = P->img_t[1];
    mp.a_hi = &P->mK[0][side][0]; mp.a_lo = &P->mK[0][side][1];
    const bool w = P->bn_x != 64;   // image boxes of the tile width
    mp.b_hi = half == 0 ? (w ? &P->mA[0] : &P->lA[0]) : (w ? &P->mB[0] : &P->lB[0]);
    mp.b_lo = half == 0 ? (w ? &P->mA[1] : &P->lA[1]) : (w ? &P->mB[1] : &P->lB[1]);
    mp.o_hi = &P->sT[0]; mp.o_lo = &P->sT[1];
    mp.f = mp.pm = &P->mK[0][0][0];   // unused by the plain pass
    a.decide = half == 1 ? 1 : 0;  // the pass after the b-update decides
    bn = P->bn_x;
    epi = EPI_STORE;
  } else {       // K_y . T^T^T -> [ny][nx] with the epilogue
    a.M = c.ny; a.N = c.nx; a.Kdim = c.ny;
    a.kbt = P->kbt[1][side];
    a.pitch_out = P->px;
    a.out_hi = half == 0 ? P->img_b[0] : P->img_a[0];
    a.out_lo = half == 0 ? P->img_b[1] : P->img_a[1];
    mp.a_hi = &P->mK[1][side][0]; mp.a_lo = &P->mK[1][side][1];
    const bool w = P->bn_y != 64;
    mp.b_hi = w ? &P->mT[0] : &P->lT[0];
    mp.b_lo = w ? &P->mT[1] : &P->lT[1];
    mp.o_hi = half == 0 ? &P->sB[0] : &P->sA[0];
    mp.o_lo = half == 0 ? &P->sB[1] : &P->sA[1];
    mp.f = half == 0 ? &P->fQ : &P->fE;
    mp.pm = &P->fP;
    a.tma_epi = P->tma_epi;
    bn = P->bn_y;
    epi = half == 0 ? EPI_B : EPI_A;
  }
  switch (P->mode) {
    case MODE_TF32: return dispatch_bn<MODE_TF32>(bn, epi, c.ek, mp, a, st);
    case MODE_BF16X3: return dispatch_bn<MODE_BF16X3>(bn, epi, c.ek, mp, a, st);
    default: return dispatch_bn<MODE_BF16>(bn, epi, c.ek, mp, a, st);
  }
}

double tc_pass_flops(const TcPlan* P, int which) { return P->flops[which & 3]; }

int tc_tile(const TcPlan* P) { return P->bn_x == P->bn_y ? P->bn_x : 0; }

int tc_set_tile(TcPlan* P, int bn) {
  if (bn != 64 && !(bn == 128 && !img_split(P->mode))) return 1;
  P->bn_x = P->bn_y = bn;
  pass_flops_of(P);
  return 0;
}

int tc_absorbed(const TcPlan* P) { return P ? P->absorbed : 0; }

int tc_partials(int nx, int ny) {
  // upper bound over the tile widths: the log-domain form's 32-column tiles
  // give the most blocks
  return ((nx + 31) / 32) * ((ny + BM - 1) / BM);
}

void tc_destroy(TcPlan* P) {
  if (!P) return;
  void* bufs[] = {P->img_a[0], P->img_a[1], P->img_b[0], P->img_b[1], P->img_t[0],
                  P->img_t[1], P->E_abs, P->sw_abs, P->sh_a, P->sh_b, P->sh_t, P->lwm,
                  P->lwe, P->k_log[0], P->k_log[1], P->sk[0], P->sk[1], P->kbt_log[0],
                  P->kbt_log[1]};
  for (void* b : bufs) if (b) cudaFree(b);
  for (int axis = 0; axis < 2; ++axis)
    for (int side = 0; side < 2; ++side) {
      for (int sp = 0; sp < 2; ++sp)
        if (P->k[axis][side][sp]) cudaFree(P->k[axis][side][sp]);
      if (P->kbt[axis][side] && (side == 0 || P->absorbed)) cudaFree(P->kbt[axis][side]);
    }
  delete P;
}

}  // namespace jko
