// tc_log.cu -- the tensor-core passes in the log domain (TF32): every image
// operand carries base-2 exponents per row and per group of 32 cells, and the
// factor per row and K-block, so the scalings keep their range however far
// the potential spreads them.
//
// The scalings of a step span e^{sigma (max w - min w)} (Prop. 4.1: a =
// min(e^{-sigma w}, kappa / s)); past ~87 e-folds they leave the FP32 range.
// The separable absorption of tc_gemm.cu removes the part of the potential
// that is a sum of a function of x and one of y; what is left must fit the
// range.  Here each image X (a, b and the intermediate T, all [rows][cols])
// is stored as a TF32 mantissa M and an int32 exponent E per row and group of
// 32 consecutive columns (one TF32 K-block), X[r][c] = M[r][c] 2^{E[r][c / 32]},
// with the largest |M| of a group in [1, 2).  The factor is stored the same
// way per row and K-block, K[m][k] = K'[m][k] 2^{s[m][k / 32]}, so that a
// product K' M of the kernel's far tail (K ~ e^{-100}: where a steep
// potential puts the mass that dominates a sum) stays a normal number.  A
// pass D[m][n] = sum_k K[m][k] X[n][k] runs one MMA accumulator per K-block g
// of its band (32 TMEM columns each, at most 16),
// P_g[m][n] = sum_{k in g} K'[m][k] M[n][k], and the epilogue adds the groups
// with exact power-of-two scalings in the frame of the largest term,
// D = 2^F sum_g P_g 2^{E[n][g] + s[m][g] - F}: only terms below 2^-126 of the
// largest are lost.  Its output is renormalised the same way (one exponent
// per output row and 32-column tile, which is the next pass's group) and the
// b-update and the congestion prox (Prop. 4.1) run on mantissa and exponent.
// A group's products keep every term that matters as long as the image spans
// at most ~70 e-folds inside its 32 cells; the set-up refuses potentials
// that change faster (sigma times the largest step of w between neighbours,
// over 32 cells).  The arithmetic of a group inside the MMA is that of the
// TF32 form.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "tc_common.cuh"

namespace jko {

namespace {

constexpr int LGC = 32;      // cells per exponent group (one TF32 K-block)
constexpr int MAXG = 16;     // groups per tile (16 x 32 TMEM columns)
constexpr int LBNL = 32;     // output tile width (= the next pass's group)
constexpr int NTL = 256;     // threads: 8 warps, 2 per TMEM lane quadrant
constexpr int kNoExp = -100000;   // exponent of an all-zero group / value

struct LogPassArgs {
  int M, N;                 // output D is M x N
  int pitch_out;            // row pitch (elements) of the output mantissa image
  float* out;               // output mantissa image (tf32 values)
  const int4* kbt;          // band of the factor per 128-row tile (TF32 K-blocks of 32)
  const int* sk;            // factor exponents [M][gk] per row and K-block
  int gk;
  const int* sh_in;         // exponents of the input image [N][gin]
  int gin;
  int* sh_out;              // exponents of the output image [M][gout]
  int gout;
  const float* q;           // EPI_B: q [M][N] (fp32, unpadded)
  float* p;                 // EPI_A: p [M][N]
  const float* lwm;         // EPI_A: lw2 = -sigma w log2(e) [M][N] as 2^{lw2} =
  const int* lwe;           //   lwm 2^{lwe}, lwm = 2^{lw2 - floor(lw2)}, lwe = floor(lw2)
  Ctrl* ctrl;
  ProxArgs<float> P;        // kappa, mask
  double* part;
  int nparts;
  int decide;
};

// 2^k as a float for k in [-126, 127]; 0 below (a term that small against
// the frame is dropped), +inf above.
__device__ __forceinline__ float pow2i(int k) {
  if (k < -126) return 0.0f;
  if (k > 127) return __int_as_float(0x7f800000);
  return __int_as_float((k + 127) << 23);
}
// Unbiased exponent of a finite non-zero float (subnormals: -127).
__device__ __forceinline__ int expo(float x) {
  return (int)((__float_as_uint(x) >> 23) & 0xffu) - 127;
}
// Sum of one float per thread over the 8 warps in a fixed order (warp
// butterflies, then warp 0 over the 8 warp sums); valid in thread 0.
__device__ __forceinline__ float log_tile_sum(float v, float* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum_f(v);
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  float t = 0.0f;
  if (warp == 0) {
    t = lane < NTL / 32 ? scratch[lane] : 0.0f;
    t = warp_sum_f(t);
  }
  return t;
}

__device__ __forceinline__ void tmem_ld2_issue(uint32_t taddr, uint32_t (&r)[2]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(taddr));
}
__device__ __forceinline__ void reg_fence2(uint32_t (&r)[2]) {
  asm volatile("" : "+r"(r[0]), "+r"(r[1]));
}

template <int EPI>
__global__ void __launch_bounds__(NTL, 1)
tc_log_pass_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   const __grid_constant__ CUtensorMap mapO, LogPassArgs args) {
  constexpr int KE = 32;                                  // TF32 elements per K-block
  constexpr uint32_t A_BYTES = BM * KB_BYTES;
  constexpr uint32_t B_BYTES = LBNL * KB_BYTES;
  constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
  constexpr int STAGES = 6;
  constexpr uint32_t TMEM_COLS = MAXG * LBNL;             // 512
  constexpr uint32_t IDESC = make_idesc<MODE_TF32>(BM, LBNL);
  constexpr int CB = 1;                                    // one 128-byte column block per tile
  constexpr uint32_t OUT_BLOCK = BM * 128;
  static_assert(CB * OUT_BLOCK <= STAGES * STAGE_BYTES, "staging fits the stages");

  Ctrl* ctrl = args.ctrl;
  __shared__ int s_it;
  __shared__ int s_fault;
  __shared__ int s_shin[LBNL][MAXG];    // input exponents of the tile's columns and groups
  __shared__ int s_rowx[2][BM];         // per column-group warp: row maximum of output exponents
  __shared__ float s_redf[16];

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full_bar = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty_bar = full_bar + STAGES;
  uint64_t* accum_bar = empty_bar + STAGES;
  uint32_t* tmem_slot = (uint32_t*)(accum_bar + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * LBNL;
  const int m0 = blockIdx.y * BM;
  const int4 kb = args.kbt[blockIdx.y];
  const int nkb = kb.y;
  const int g0 = kb.x / LGC;           // K-blocks start on 32-element boundaries
  const int ngrp = nkb;

  if (threadIdx.x == 0) {
    s_fault = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(accum_bar, 1);
    fence_mbar_init();
    tma_prefetch_desc(&mapA);
    tma_prefetch_desc(&mapB);
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  pdl_launch_dependents();
  pdl_wait();
  if (stop_gate(ctrl, args.part, args.nparts, args.decide != 0, &s_it)) {
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem_base, TMEM_COLS);
    return;
  }
  // exponents of the input rows n0 .. n0+31 for the tile's groups
  for (int e = threadIdx.x; e < LBNL * MAXG; e += NTL) {
    const int r = e / MAXG, g = e - r * MAXG;
    const int n = n0 + r, gg = g0 + g;
    s_shin[r][g] = (g < ngrp && n < args.N && gg < args.gin) ? args.sh_in[(size_t)n * args.gin + gg]
                                                              : kNoExp;
  }

  bool ok = true;
  if (warp == 0 && lane == 0) {
    for (int i = 0; i < nkb && ok; ++i) {
      const int s = i % STAGES;
      if (i >= STAGES) ok = mbar_wait(&empty_bar[s], ((i / STAGES) - 1) & 1);
      if (!ok) break;
      unsigned char* st = smem + s * STAGE_BYTES;
      mbar_arrive_expect_tx(&full_bar[s], STAGE_BYTES);
      const int kx = kb.x + i * KE;
      tma_load_2d(st, &mapA, &full_bar[s], kx, m0);
      tma_load_2d(st + A_BYTES, &mapB, &full_bar[s], kx, n0);
    }
    if (!ok) atomicOr(&s_fault, 1);
  } else if (warp == 1 && lane == 0) {
    // one accumulator per exponent group: K-block i into group i
    for (int i = 0; i < nkb && ok; ++i) {
      const int s = i % STAGES;
      ok = mbar_wait(&full_bar[s], (i / STAGES) & 1);
      if (!ok) break;
      tc_fence_after();
      const int g = i;
      const bool first = true;
      const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
      const uint64_t a = sdesc_sw128(sa);
      const uint64_t b = sdesc_sw128(sa + A_BYTES);
#pragma unroll
      for (int kk = 0; kk < KB_BYTES / 32; ++kk) {
        const uint64_t adv = (uint64_t)(kk * 2);
        umma<MODE_TF32>(tmem_base + (uint32_t)(g * LBNL), a + adv, b + adv, IDESC,
                        (first && kk == 0) ? 0u : 1u);
      }
      umma_commit(&empty_bar[s]);
    }
    umma_commit(accum_bar);
    if (!ok) atomicOr(&s_fault, 1);
  }
  __syncwarp();
  __syncthreads();   // s_shin complete

  // ---- epilogue: warp w: TMEM lanes 32 (w % 4) .., 16 columns (w / 4) of the tile ----
  bool have = mbar_wait(accum_bar, 0);
  if (!have) atomicOr(&s_fault, 1);
  __syncwarp();
  tc_fence_after();
  const int quad = warp & 3, grp = warp >> 2;
  const int rl = quad * 32 + lane;
  const int m = m0 + rl;
  const bool row_ok = m < args.M;
  const uint32_t lane_base = tmem_base + ((uint32_t)(quad * 32) << 16);
  // this row's factor exponents for the tile's K-blocks
  int skr[MAXG];
#pragma unroll
  for (int g = 0; g < MAXG; ++g)
    skr[g] = (g < ngrp && row_ok) ? args.sk[(size_t)m * args.gk + g0 + g] : 0;
  // this thread's 16 values as (mantissa S in [1, 2 ngrp), exponent F)
  float S[16];
  int F[16];
  if (have) {
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) {
      // the chunk's 2 columns of every group: all loads issued, one wait
      // (ngrp is the same in the whole CTA, so the warp-wide loads stay uniform)
      uint32_t r[MAXG][2];
#pragma unroll
      for (int g = 0; g < MAXG; ++g) {
        if (g < ngrp) tmem_ld2_issue(lane_base + (uint32_t)(g * LBNL + grp * 16 + ch * 2), r[g]);
        else r[g][0] = r[g][1] = 0u;
      }
      tmem_wait_ld();
      float v[MAXG][2];
#pragma unroll
      for (int g = 0; g < MAXG; ++g) {
        reg_fence2(r[g]);
        v[g][0] = __uint_as_float(r[g][0]);
        v[g][1] = __uint_as_float(r[g][1]);
      }
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) {
        const int c = grp * 16 + ch * 2 + jj;   // column within the tile
        int fr = kNoExp;
#pragma unroll
        for (int g = 0; g < MAXG; ++g) {
          const float x = v[g][jj];
          if (x != 0.0f) fr = max(fr, expo(x) + s_shin[c][g] + skr[g]);
        }
        float sum = 0.0f;
        if (fr != kNoExp) {
#pragma unroll
          for (int g = 0; g < MAXG; ++g) {
            const float x = v[g][jj];
            if (x != 0.0f) sum += x * pow2i(s_shin[c][g] + skr[g] - fr);
          }
        }
        S[ch * 2 + jj] = sum;
        F[ch * 2 + jj] = sum != 0.0f ? fr : kNoExp;
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) { S[j] = 0.0f; F[j] = kNoExp; }
  }
  tc_fence_before();

  // ---- the epilogue arithmetic on (S, F), the output value as (o, e) ----
  const int nb = n0 + grp * 16;
  int cnt = args.N - nb;
  cnt = !row_ok || cnt < 0 ? 0 : (cnt > 16 ? 16 : cnt);
  float (&o)[16] = S;     // the output value (o, oe) replaces (S, F) in place
  int (&oe)[16] = F;
  float res_f = 0.0f;
  int bad = 0;
  const int tile_g = blockIdx.x;   // the output tile's group in the output image
  if (EPI == EPI_STORE) {
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (j >= cnt) { o[j] = 0.0f; oe[j] = kNoExp; }
  } else if (EPI == EPI_B) {
    // b = q / Y; the residual of the previous b: |b_old Y - q| (the old b is
    // this tile's mantissa and row exponent, read before they are rewritten)
    const bool have_prev = s_it > 0;
    const int bold_e = (row_ok && have_prev) ? args.sh_out[(size_t)m * args.gout + tile_g] : kNoExp;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float Sj = S[j];
      const int Fj = F[j];
      o[j] = 0.0f;
      oe[j] = kNoExp;
      if (j < cnt) {
        const size_t idx = (size_t)m * args.N + nb + j;
        const float qv = args.q[idx];
        if (have_prev) {
          const float bom = args.out[(size_t)m * args.pitch_out + nb + j];
          float bY = 0.0f;
          // (far from the fixed point b_old Y can exceed the FP32 range: a
          // large finite term keeps the sum finite and the pair running)
          if (bom != 0.0f && Sj != 0.0f) bY = fminf((bom * Sj) * pow2i(bold_e + Fj), 1e30f);
          res_f += fabsf(bY - qv);
        }
        if (qv != 0.0f && Sj != 0.0f) {
          o[j] = qv / Sj;
          oe[j] = -Fj;
          bad |= !isfinite(o[j]);
        }
      }
    }
  } else {
    // congestion prox (Prop. 4.1) in log2: a = min(2^{lw2}, kappa / s), 0 on
    // the mask; p = a s.  2^{lw2} = lm 2^{le}, s = S 2^F: the comparison takes
    // the integer exponents apart from the logarithms of the mantissas
    const ProxArgs<float>& P = args.P;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float Sj = S[j];
      const int Fj = F[j];
      o[j] = 0.0f;
      oe[j] = kNoExp;
      if (j < cnt) {
        const size_t idx = (size_t)m * args.N + nb + j;
        float pv = 0.0f;
        const bool masked = P.mask && P.mask[idx];
        if (!masked) {
          const float lm = args.lwm[idx];
          const int le = args.lwe[idx];
          const float kap = P.kappa ? P.kappa[idx] : P.kappa_s;
          const bool hk = P.kappa ? isfinite(kap) : P.has_kappa != 0;
          if (hk && Sj != 0.0f && (float)(le + Fj) + __log2f(lm * Sj) > __log2f(kap)) {
            o[j] = kap / Sj;                      // a = kappa / s
            oe[j] = -Fj;
            pv = kap;
          } else {
            o[j] = lm;                            // a = 2^{lw2}
            oe[j] = le;
            if (Sj != 0.0f) pv = (lm * Sj) * pow2i(le + Fj);
          }
          bad |= !isfinite(o[j]);
        }
        args.p[idx] = pv;
      }
    }
  }
  // ---- the output row exponent of this tile: the largest over its 32 columns ----
  int rx = kNoExp;
#pragma unroll
  for (int j = 0; j < 16; ++j)
    if (o[j] != 0.0f) rx = max(rx, expo(o[j]) + oe[j]);
  s_rowx[grp][rl] = rx;
  __syncthreads();
  const int R = max(s_rowx[0][rl], s_rowx[1][rl]);
#pragma unroll
  for (int j = 0; j < 16; ++j)
    o[j] = (o[j] != 0.0f && R != kNoExp) ? o[j] * pow2i(oe[j] - R) : 0.0f;
  if (grp == 0 && row_ok) args.sh_out[(size_t)m * args.gout + tile_g] = R == kNoExp ? 0 : R;
  // the mantissa tile, staged in the free stages and stored with TMA
  stage16<MODE_TF32>(smem, smem, rl, grp, o);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && have) {
#pragma unroll
    for (int cb = 0; cb < CB; ++cb) tma_store_2d(&mapO, smem + cb * OUT_BLOCK, n0 + cb * 32, m0);
    bulk_commit();
    bulk_wait_all();
  }
  if (warp == 1) tmem_dealloc(tmem_base, TMEM_COLS);
  if (EPI == EPI_STORE) {
    if (threadIdx.x == 0 && s_fault) atomicOr(&ctrl->nonfinite, 2);
    return;
  }
  bad = warp_or(bad);
  if (EPI == EPI_B) {
    const double res = (double)log_tile_sum(res_f, s_redf);
    if (threadIdx.x == 0) args.part[blockIdx.y * gridDim.x + blockIdx.x] = res;
  }
  if (lane == 0 && bad) atomicOr(&ctrl->nonfinite, 1);
  if (threadIdx.x == 0 && s_fault) atomicOr(&ctrl->nonfinite, 2);
  if (EPI == EPI_A && threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0) ctrl->it = s_it + 1;
}

size_t log_smem_bytes() { return 6 * (size_t)(BM + LBNL) * KB_BYTES + 1024 + 16 * 8 + 16; }
// (six stages of a 128-row factor block and a 32-row image block)

template <int EPI>
cudaError_t launch_log(const CUtensorMap& A, const CUtensorMap& B, const CUtensorMap& O,
                       const LogPassArgs& args, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((args.N + LBNL - 1) / LBNL, (args.M + BM - 1) / BM);
  cfg.blockDim = dim3(NTL);
  cfg.dynamicSmemBytes = log_smem_bytes();
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, tc_log_pass_kernel<EPI>, A, B, O, args);
}

__global__ void fill_int_kernel(int* x, long long n, int v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = v;
}

constexpr double kLog2e = 1.4426950408889634;
constexpr double kGroupRange = 70.0;   // e-folds an image may span inside one group
constexpr double kCut = 50.0;          // e-folds below the diagonal where the band ends

// The largest change of w between neighbouring cells along one axis (w: [ny][nx]).
double axis_step(const double* w, int nx, int ny, int axis) {
  double m = 0.0;
  if (!w) return m;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const size_t i = (size_t)y * nx + x;
      if (axis == 0 && x + 1 < nx) m = std::max(m, std::fabs(w[i + 1] - w[i]));
      if (axis == 1 && y + 1 < ny) m = std::max(m, std::fabs(w[i + nx] - w[i]));
    }
  return m;
}

float tf32_rna_host(double v) {
  float f = (float)v;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u = (u + 0x1000u) & 0xFFFFE000u;
  std::memcpy(&f, &u, 4);
  return f;
}

// The scaled factor of one axis: K[i][j] = exp(-(i-j)^2 h^2 / gamma) for
// |i - j| <= r, stored as K'[i][j] = K[i][j] 2^{-s[i][j / 32]} in TF32 with
// s[i][g] = floor(log2 of the row's largest entry in K-block g); entries of
// K' below 2^-126 are dropped.  Also the K-block range of every 128-row tile.
int build_log_factor(int n, int pitch, double h, double gamma, int r, std::vector<float>* fac,
                     std::vector<int>* sk, int gk, std::vector<int4>* kbt, std::string* msg) {
  fac->assign((size_t)n * pitch, 0.0f);
  sk->assign((size_t)n * gk, 0);
  const int tiles = (n + BM - 1) / BM;
  std::vector<int> kmin(tiles, n), kmax(tiles, -1);
  for (int i = 0; i < n; ++i) {
    const int j0 = std::max(0, i - r), j1 = std::min(n - 1, i + r);
    for (int g = j0 / LGC; g <= j1 / LGC; ++g) {
      const int lo = std::max(j0, g * LGC), hi = std::min(j1, g * LGC + LGC - 1);
      const int jc = std::min(std::max(i, lo), hi);   // the block's entry nearest the diagonal
      const double dc = (i - jc) * h;
      const int e = (int)std::floor(-(dc * dc) / gamma * kLog2e);
      (*sk)[(size_t)i * gk + g] = e;
      for (int j = lo; j <= hi; ++j) {
        const double d = (i - j) * h;
        const double v = std::exp2(-(d * d) / gamma * kLog2e - e);
        if (v < 1.1754943508222875e-38) continue;
        (*fac)[(size_t)i * pitch + j] = tf32_rna_host(v);
        kmin[i / BM] = std::min(kmin[i / BM], j);
        kmax[i / BM] = std::max(kmax[i / BM], j);
      }
    }
  }
  kbt->assign(tiles, make_int4(0, 0, 0, -1));
  for (int t = 0; t < tiles; ++t)
    if (kmax[t] >= 0) {
      const int k0 = kmin[t] / LGC * LGC;
      const int nkb = (kmax[t] - k0) / LGC + 1;
      if (nkb > MAXG) {
        *msg = "the log-domain form keeps at most 16 K-blocks of 32 cells per band (the band "
               "that the potential's slope asks for is wider)";
        return 1;
      }
      (*kbt)[t] = make_int4(k0, nkb, kmin[t], kmax[t]);
    }
  return 0;
}

}  // namespace

// Set-up of the log-domain form on a TF32 plan: the scaled factors and their
// bands, exponent images, and the log2 potential.
//
// Band: a cell at distance d contributes K(d) a(k) to an output whose own
// term is a(m); with a's log-slope bounded by lambda = sigma max|dw| / h
// (e-folds per unit length), the contributions beyond the first d with
// d^2 / gamma - lambda d > 50 are below e^{-50} of that term, so the band
// stops there (where the potential is flat this is the Gaussian's own e^{-50}).
int tc_log_setup(TcPlan* P, const double* w_host, double sigma, std::string* msg) {
  const TcConfig& c = P->cfg;
  if (P->mode != MODE_TF32 || P->absorbed) {
    *msg = "the log-domain form runs on the TF32 tensor-core form without separable absorption";
    return 1;
  }
  std::vector<float> fac;
  std::vector<int> skh;
  std::vector<int4> kbt;
  for (int axis = 0; axis < 2; ++axis) {
    const int n = axis == 0 ? c.nx : c.ny;
    const int pitch = axis == 0 ? P->px : P->py;
    const double h = (axis == 0 ? c.lx : c.ly) / n;
    const double step = axis_step(w_host, c.nx, c.ny, axis);
    if (sigma * step * LGC > kGroupRange) {
      *msg = "the log-domain form needs sigma times the largest step of w between neighbouring "
             "cells to stay below 70 / 32 e-folds (a finer grid)";
      return 1;
    }
    const double lg = sigma * step / h * c.gamma;
    const double dcut = 0.5 * (lg + std::sqrt(lg * lg + 4.0 * kCut * c.gamma));
    const int r = (int)std::min<double>(n - 1, std::ceil(dcut / h));
    P->gk[axis] = (n + LGC - 1) / LGC;
    const int rc = build_log_factor(n, pitch, h, c.gamma, r, &fac, &skh, P->gk[axis], &kbt, msg);
    if (rc) return rc;
    if (cudaMalloc(&P->k_log[axis], fac.size() * sizeof(float)) != cudaSuccess ||
        cudaMemcpy(P->k_log[axis], fac.data(), fac.size() * sizeof(float), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMalloc((void**)&P->sk[axis], skh.size() * sizeof(int)) != cudaSuccess ||
        cudaMemcpy(P->sk[axis], skh.data(), skh.size() * sizeof(int), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMalloc((void**)&P->kbt_log[axis], kbt.size() * sizeof(int4)) != cudaSuccess ||
        cudaMemcpy(P->kbt_log[axis], kbt.data(), kbt.size() * sizeof(int4), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
      *msg = "upload of the scaled factors";
      return 2;
    }
    if (!make_map(&P->mKl[axis], P->k_log[axis], MODE_TF32, n, n, pitch, BM)) {
      *msg = "cuTensorMapEncodeTiled failed (scaled factor)";
      return 2;
    }
    // executed flops of the passes over this axis
    const int N = axis == 0 ? c.ny : c.nx;
    double f = 0.0;
    for (const int4& t : kbt) f += band_tile_flops(t, LGC, LBNL, 1.0) * ((N + LBNL - 1) / LBNL);
    P->flops[axis] = P->flops[axis + 2] = f;
  }
  P->gx = (c.nx + LGC - 1) / LGC;
  P->gy = (c.ny + LGC - 1) / LGC;
  if (cudaMalloc((void**)&P->sh_a, sizeof(int) * (size_t)c.ny * P->gx) != cudaSuccess ||
      cudaMalloc((void**)&P->sh_b, sizeof(int) * (size_t)c.ny * P->gx) != cudaSuccess ||
      cudaMalloc((void**)&P->sh_t, sizeof(int) * (size_t)c.nx * P->gy) != cudaSuccess ||
      cudaMemset(P->sh_b, 0, sizeof(int) * (size_t)c.ny * P->gx) != cudaSuccess ||
      cudaMemset(P->sh_t, 0, sizeof(int) * (size_t)c.nx * P->gy) != cudaSuccess) {
    *msg = "cudaMalloc exponent images";
    return 2;
  }
  const size_t N = (size_t)c.nx * c.ny;
  std::vector<float> lm(N);
  std::vector<int> le(N);
  for (size_t i = 0; i < N; ++i) {
    const double x = -sigma * (w_host ? w_host[i] : 0.0) * kLog2e;
    const double e = std::floor(x);
    le[i] = (int)e;
    lm[i] = (float)std::exp2(x - e);
    if (lm[i] >= 2.0f) { lm[i] = 1.0f; le[i] += 1; }
  }
  if (cudaMalloc((void**)&P->lwm, N * sizeof(float)) != cudaSuccess ||
      cudaMemcpy(P->lwm, lm.data(), N * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMalloc((void**)&P->lwe, N * sizeof(int)) != cudaSuccess ||
      cudaMemcpy(P->lwe, le.data(), N * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
    *msg = "upload of the log2 potential";
    return 2;
  }
  if (cudaFuncSetAttribute(tc_log_pass_kernel<EPI_STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)log_smem_bytes()) != cudaSuccess ||
      cudaFuncSetAttribute(tc_log_pass_kernel<EPI_B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)log_smem_bytes()) != cudaSuccess ||
      cudaFuncSetAttribute(tc_log_pass_kernel<EPI_A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)log_smem_bytes()) != cudaSuccess) {
    *msg = "cudaFuncSetAttribute (log-domain passes)";
    return 2;
  }
  // image loads in 32-row boxes (the log form's tile width)
  bool okm = make_map(&P->l32[0], P->img_a[0], MODE_TF32, c.ny, c.nx, P->px, LBNL) &&
             make_map(&P->l32[1], P->img_b[0], MODE_TF32, c.ny, c.nx, P->px, LBNL) &&
             make_map(&P->l32[2], P->img_t[0], MODE_TF32, c.nx, c.ny, P->py, LBNL);
  if (!okm) {
    *msg = "cuTensorMapEncodeTiled failed (log-domain image maps)";
    return 2;
  }
  P->logd = 1;
  P->loop_ok = 0;   // the persistent loop kernel does not carry exponents
  return 0;
}

cudaError_t tc_log_begin_step(TcPlan* P, cudaStream_t st) {
  fill_int_kernel<<<64, 256, 0, st>>>(P->sh_a, (long long)P->cfg.ny * P->gx, 0);
  return cudaGetLastError();
}

cudaError_t tc_log_enqueue_pass(TcPlan* P, int which, cudaStream_t st) {
  const TcConfig& c = P->cfg;
  const bool over_x = (which & 1) == 0;
  const int half = which >> 1;
  LogPassArgs a{};
  a.ctrl = c.ctrl;
  a.P = c.prox;
  a.part = c.part;
  a.nparts = ((c.nx + LBNL - 1) / LBNL) * ((c.ny + BM - 1) / BM);   // b-update grid
  a.q = c.q;
  a.p = c.p;
  a.lwm = P->lwm;
  a.lwe = P->lwe;
  if (over_x) {   // K_x . image^T -> T [nx][ny]
    a.M = c.nx; a.N = c.ny;
    a.kbt = P->kbt_log[0];
    a.sk = P->sk[0];
    a.gk = P->gk[0];
    a.pitch_out = P->py;
    a.out = (float*)P->img_t[0];
    a.sh_in = half == 0 ? P->sh_a : P->sh_b;
    a.gin = P->gx;
    a.sh_out = P->sh_t;
    a.gout = P->gy;
    a.decide = half == 1 ? 1 : 0;
    const CUtensorMap& B = half == 0 ? P->l32[0] : P->l32[1];
    return launch_log<EPI_STORE>(P->mKl[0], B, P->sT[0], a, st);
  }
  a.M = c.ny; a.N = c.nx;
  a.kbt = P->kbt_log[1];
  a.sk = P->sk[1];
  a.gk = P->gk[1];
  a.pitch_out = P->px;
  a.out = (float*)(half == 0 ? P->img_b[0] : P->img_a[0]);
  a.sh_in = P->sh_t;
  a.gin = P->gy;
  a.sh_out = half == 0 ? P->sh_b : P->sh_a;
  a.gout = P->gx;
  const CUtensorMap& O = half == 0 ? P->sB[0] : P->sA[0];
  return half == 0 ? launch_log<EPI_B>(P->mKl[1], P->l32[2], O, a, st)
                   : launch_log<EPI_A>(P->mKl[1], P->l32[2], O, a, st);
}

}  // namespace jko
