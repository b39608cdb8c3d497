// tc_multi.cu -- the Gibbs-kernel passes of the steps with several couplings
// (Sec. 5.1 generic diagonal scaling: the Wasserstein attraction of Sec. 5.2,
// the two species and the pairwise attraction of Sec. 5.3) on the tensor
// cores: TF32; BF16 (the factor in bf16, images as bf16 pairs hi + lo, one
// product K_hi . (x_hi + x_lo)); BF16x3 (the factor as a pair too, plus
// K_lo . x_hi), the products of the single-density forms.
//
// Those steps apply the same separable xi to M = 2 or 3 images per half-step
// and meet at a joint proximal map (attraction.cu) that couples the images
// cell by cell.  Here one launch runs one pass of xi for all M images
// (blockIdx.z = image):
//     D_z[m][n] = sum_k K[m][k] X_z[n][k]
// with the factor K of the pass (K_x or K_y of the handle's plan, the same band
// tables) and the image X_z stored with its contracted axis contiguous, as
// the single-density passes of tc_gemm.cu.  Epilogues:
//   EPI_STORE  D as the operand (rounded to tf32, or the bf16 pair): the
//              intermediate, next pass's operand;
//   EPI_B      b_z = q_z / D (rounded to tf32 in the TF32 form; fp32 in the
//              bf16 forms, split into its pair before the next pass), and the
//              residual |b_old D - q_z| partial of the tile (part + z * tiles);
//   EPI_RAW    D as fp32: xi b_z for the joint prox, which reads it at full
//              precision (the single-density TF32 form's prox reads the
//              accumulator itself).
// The joint prox kernels round their scalings to tf32 when they feed the TF32
// form, as the single-density TF32 epilogue does; the bf16 forms take fp32
// scalings and split every image of the first pass into its bf16 pair
// (tc_split_pairs).
#include "tc_common.cuh"

namespace jko {

namespace {

constexpr int MBN = 64;                  // output tile width
constexpr int MNT = 128;                 // 4 warps, one per TMEM lane quadrant
constexpr int MAXZ = 3;
constexpr int EPI_RAW = TC_EPI_RAW;

// pipeline stages: 24 KB (TF32), 32 KB (BF16: image pairs), 48 KB (BF16x3:
// factor and image pairs)
__host__ __device__ constexpr int multi_stages(int mode) { return mode == MODE_BF16X3 ? 4 : 6; }

struct MultiMaps {
  CUtensorMap A[2];       // factor of the pass (hi; lo: BF16x3)
  CUtensorMap B[MAXZ][2]; // images (64-row boxes), hi [+ lo]
  CUtensorMap O[MAXZ][2]; // outputs (128-row boxes), hi [+ lo] when operand-typed
};

struct MultiArgs {
  int M, N;               // each output D_z is M x N
  int pitch_out;          // row pitch of the outputs
  float* out[MAXZ];
  const float* q[MAXZ];   // EPI_B: q_z [M][N]
  const int4* kbt;        // per 128-row tile: band of the factor
  Ctrl* ctrl;
  double* part;           // EPI_B: residual partials, image z at part + z * tiles
  int nparts;             // partials read by the deciding pass
  int decide;
};

// 16 fp32 values of row r, chunk c (16 columns) into a 128-byte swizzled
// output tile, rounded to tf32 (ROUND) or as they are.
template <bool ROUND>
__device__ __forceinline__ void stage16_f32(unsigned char* st, int r, int c, const float (&o)[16]) {
  constexpr uint32_t BLK = BM * 128;
  const int cb = c >> 1, k0 = (c & 1) * 4;
  unsigned char* row = st + cb * BLK + r * 128;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint4 u;
    u.x = __float_as_uint(ROUND ? tf32_round(o[4 * q]) : o[4 * q]);
    u.y = __float_as_uint(ROUND ? tf32_round(o[4 * q + 1]) : o[4 * q + 1]);
    u.z = __float_as_uint(ROUND ? tf32_round(o[4 * q + 2]) : o[4 * q + 2]);
    u.w = __float_as_uint(ROUND ? tf32_round(o[4 * q + 3]) : o[4 * q + 3]);
    *reinterpret_cast<uint4*>(row + (((k0 + q) ^ (r & 7)) << 4)) = u;
  }
}

template <int MODE, int EPI>
__global__ void __launch_bounds__(MNT, 1)
tc_multi_kernel(const __grid_constant__ MultiMaps maps, MultiArgs args) {
  constexpr int KE = OpT<MODE>::kElems;                   // elements per K-block
  constexpr int MSTAGES = multi_stages(MODE);
  constexpr int NSPLIT = img_split(MODE) ? 2 : 1;         // image hi (+ lo) blocks
  constexpr uint32_t A_BYTES = BM * KB_BYTES;
  constexpr uint32_t B_BYTES = MBN * KB_BYTES;
  constexpr uint32_t STAGE_BYTES = stage_bytes(MODE, MBN);
  constexpr uint32_t ALO_OFF = A_BYTES + NSPLIT * B_BYTES; // factor lo (BF16x3)
  constexpr uint32_t TMEM_COLS = acc_cols(MODE, MBN);
  constexpr uint32_t IDESC = make_idesc<MODE_TF32>(BM, MBN);
  constexpr int CB = MBN * 4 / 128;                        // 128-byte column blocks (fp32)
  constexpr uint32_t OUT_BLOCK = BM * 128;
  // an operand-typed output (EPI_STORE) of the bf16 forms: hi and lo tiles
  constexpr bool PAIR_OUT = EPI == EPI_STORE && MODE != MODE_TF32;
  static_assert(CB * OUT_BLOCK <= MSTAGES * STAGE_BYTES, "staging fits the stages");

  Ctrl* ctrl = args.ctrl;
  __shared__ int s_it;
  __shared__ int s_fault;
  __shared__ float s_redf[MNT / 32];
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full_bar = (uint64_t*)(smem + MSTAGES * STAGE_BYTES);
  uint64_t* empty_bar = full_bar + MSTAGES;
  uint64_t* accum_bar = empty_bar + MSTAGES;
  uint32_t* tmem_slot = (uint32_t*)(accum_bar + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int z = blockIdx.z;
  const int n0 = blockIdx.x * MBN;
  const int m0 = blockIdx.y * BM;
  const int4 kb = args.kbt[blockIdx.y];
  const int nkb = kb.y;
  const CUtensorMap* mapB = &maps.B[z][0];

  if (threadIdx.x == 0) {
    s_fault = 0;
    for (int s = 0; s < MSTAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(accum_bar, 1);
    fence_mbar_init();
    tma_prefetch_desc(&maps.A[0]);
    tma_prefetch_desc(mapB);
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

  bool ok = true;
  if (warp == 0 && lane == 0) {
    for (int i = 0; i < nkb && ok; ++i) {
      const int s = i % MSTAGES;
      if (i >= MSTAGES) ok = mbar_wait(&empty_bar[s], ((i / MSTAGES) - 1) & 1);
      if (!ok) break;
      unsigned char* st = smem + s * STAGE_BYTES;
      mbar_arrive_expect_tx(&full_bar[s], STAGE_BYTES);
      const int kx = kb.x + i * KE;
      tma_load_2d(st, &maps.A[0], &full_bar[s], kx, m0);
      tma_load_2d(st + A_BYTES, mapB, &full_bar[s], kx, n0);
      if constexpr (NSPLIT == 2)
        tma_load_2d(st + A_BYTES + B_BYTES, &maps.B[z][1], &full_bar[s], kx, n0);
      if constexpr (fac_split(MODE)) tma_load_2d(st + ALO_OFF, &maps.A[1], &full_bar[s], kx, m0);
    }
    if (!ok) atomicOr(&s_fault, 1);
  } else if (warp == 1 && lane == 0) {
    for (int i = 0; i < nkb && ok; ++i) {
      const int s = i % MSTAGES;
      ok = mbar_wait(&full_bar[s], (i / MSTAGES) & 1);
      if (!ok) break;
      tc_fence_after();
      const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
      const uint64_t a = sdesc_sw128(sa);
      const uint64_t b = sdesc_sw128(sa + A_BYTES);
      if constexpr (MODE == MODE_TF32) {
#pragma unroll
        for (int kk = 0; kk < KB_BYTES / 32; ++kk) {
          const uint64_t adv = (uint64_t)(kk * 2);
          umma<MODE_TF32>(tmem_base, a + adv, b + adv, IDESC, (i > 0 || kk > 0) ? 1u : 0u);
        }
      } else {
        const uint64_t a_lo = sdesc_sw128(sa + ALO_OFF);
#pragma unroll
        for (int kk = 0; kk < KB_BYTES / 32; ++kk)
          umma_kstep<MODE, MBN>(tmem_base, a, a_lo, b, kk, (i > 0 || kk > 0) ? 1u : 0u);
      }
      umma_commit(&empty_bar[s]);
    }
    umma_commit(accum_bar);
    if (!ok) atomicOr(&s_fault, 1);
  }
  __syncwarp();

  // ---- epilogue: warp w drains TMEM lanes 32w .. 32w+31 (its rows) ----
  bool have = mbar_wait(accum_bar, 0);
  if (!have) atomicOr(&s_fault, 1);
  __syncwarp();
  tc_fence_after();
  const int rl = warp * 32 + lane;
  const int m = m0 + rl;
  const bool row_ok = m < args.M;
  const bool have_prev = EPI == EPI_B && s_it > 0;
  float res_f = 0.0f;
  int bad = 0;
  if (have) {
    const uint32_t t_lane = tmem_base + ((uint32_t)(warp * 32) << 16);
    uint32_t racc[MODE == MODE_TF32 ? MBN / 16 : 1][16];
    if constexpr (MODE == MODE_TF32) {
#pragma unroll
      for (int c = 0; c < MBN / 16; ++c) tmem_ld16_issue(t_lane + (uint32_t)(c * 16), racc[c]);
      tmem_wait_ld();
    }
#pragma unroll
    for (int c = 0; c < MBN / 16; ++c) {
      float acc[16];
      if constexpr (MODE == MODE_TF32) {
        reg_fence16(racc[c]);
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = __uint_as_float(racc[c][j]);
      } else {
        tmem_tile16<MODE, MBN>(t_lane, c * 16, acc);   // hi and lo products added
      }
      const int nb = n0 + c * 16;
      int cnt = args.N - nb;
      cnt = !row_ok || cnt < 0 ? 0 : (cnt > 16 ? 16 : cnt);
      float o[16];
      if (EPI == EPI_B) {
        const float* q = args.q[z] + (size_t)m * args.N + nb;
        const float* bold = args.out[z] + (size_t)m * args.pitch_out + nb;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          o[j] = 0.0f;
          if (j < cnt) {
            const float v = acc[j];
            const float qv = q[j];
            if (have_prev) res_f += abs_residual<float>(bold[j], v, qv);
            o[j] = b_update<float>(qv, v);
            bad |= !isfinite(o[j]);
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) o[j] = j < cnt ? acc[j] : 0.0f;
      }
      if constexpr (PAIR_OUT) stage16<MODE>(smem, smem + OUT_BLOCK, rl, c, o);
      else stage16_f32<EPI != EPI_RAW && MODE == MODE_TF32>(smem, rl, c, o);
    }
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && have) {
    if constexpr (PAIR_OUT) {
      tma_store_2d(&maps.O[z][0], smem, n0, m0);
      tma_store_2d(&maps.O[z][1], smem + OUT_BLOCK, n0, m0);
    } else {
#pragma unroll
      for (int cb = 0; cb < CB; ++cb)
        tma_store_2d(&maps.O[z][0], smem + cb * OUT_BLOCK, n0 + cb * 32, m0);
    }
    bulk_commit();
    bulk_wait_all();
  }
  if (warp == 1) tmem_dealloc(tmem_base, TMEM_COLS);
  bad = warp_or(bad);
  if (EPI == EPI_B) {
    const float w = warp_sum_f(res_f);
    if (lane == 0) s_redf[warp] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.0f;
#pragma unroll
      for (int i = 0; i < MNT / 32; ++i) t += s_redf[i];
      const int tiles = gridDim.x * gridDim.y;
      args.part[(size_t)z * tiles + blockIdx.y * gridDim.x + blockIdx.x] = (double)t;
    }
  }
  if (lane == 0 && bad) atomicOr(&ctrl->nonfinite, 1);
  if (threadIdx.x == 0 && s_fault) atomicOr(&ctrl->nonfinite, 2);
}

constexpr size_t multi_smem_bytes(int mode) {
  return (size_t)multi_stages(mode) * stage_bytes(mode, MBN) + 1024 +
         (2 * multi_stages(mode) + 2) * 8 + 16;
}
static_assert(multi_smem_bytes(MODE_BF16X3) <= 227 * 1024 &&
                  multi_smem_bytes(MODE_BF16) <= 227 * 1024 &&
                  multi_smem_bytes(MODE_TF32) <= 227 * 1024,
              "the stages fit shared memory");

template <int MODE, int EPI>
cudaError_t launch_multi(const MultiMaps& maps, const MultiArgs& a, int nz, cudaStream_t st) {
  static bool attr_set = false;   // per process: the attribute belongs to the function
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(tc_multi_kernel<MODE, EPI>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)multi_smem_bytes(MODE));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((a.N + MBN - 1) / MBN, (a.M + BM - 1) / BM, nz);
  cfg.blockDim = dim3(MNT);
  cfg.dynamicSmemBytes = multi_smem_bytes(MODE);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, tc_multi_kernel<MODE, EPI>, maps, a);
}

template <int MODE>
cudaError_t launch_multi_epi(const MultiMaps& maps, const MultiArgs& a, int nz, int epi,
                             cudaStream_t st) {
  if (epi == EPI_STORE) return launch_multi<MODE, EPI_STORE>(maps, a, nz, st);
  if (epi == EPI_B) return launch_multi<MODE, EPI_B>(maps, a, nz, st);
  return launch_multi<MODE, EPI_RAW>(maps, a, nz, st);
}

// x -> (hi, lo) = (bf16(x), bf16(x - hi)) for nz images of n elements each
__global__ void split_pairs_kernel(const float* x0, const float* x1, const float* x2,
                                   __nv_bfloat16* h0, __nv_bfloat16* h1, __nv_bfloat16* h2,
                                   long long n) {
  const float* x = blockIdx.y == 0 ? x0 : blockIdx.y == 1 ? x1 : x2;
  __nv_bfloat16* h = blockIdx.y == 0 ? h0 : blockIdx.y == 1 ? h1 : h2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float v = x[i];
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    h[i] = hi;
    h[n + i] = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
}

}  // namespace

int tc_mode(const TcPlan* P) { return P ? P->mode : -1; }

int tc_multi_tiles(int nx, int ny, int axis) {
  const int M = axis == 0 ? nx : ny, N = axis == 0 ? ny : nx;
  return ((N + MBN - 1) / MBN) * ((M + BM - 1) / BM);
}

cudaError_t tc_split_pairs(int nz, const float* const* x, void* const* pairs, long long n,
                           cudaStream_t st) {
  if (nz < 1 || nz > MAXZ) return cudaErrorInvalidValue;
  const float* xs[MAXZ];
  __nv_bfloat16* hs[MAXZ];
  for (int z = 0; z < MAXZ; ++z) {
    xs[z] = x[z < nz ? z : 0];
    hs[z] = (__nv_bfloat16*)pairs[z < nz ? z : 0];
  }
  long long g = (n + 255) / 256;
  if (g > 152 * 4) g = 152 * 4;
  split_pairs_kernel<<<dim3((unsigned)(g < 1 ? 1 : g), nz), 256, 0, st>>>(
      xs[0], xs[1], xs[2], hs[0], hs[1], hs[2], n);
  return cudaGetLastError();
}

cudaError_t tc_multi_pass(TcPlan* P, int axis, int nz, const void* const* in, void* const* out,
                          int epi, const float* const* q, double* part, int nparts, int decide,
                          cudaStream_t st) {
  const TcConfig& c = P->cfg;
  const int mode = P->mode;
  if (P->absorbed || nz < 1 || nz > MAXZ) return cudaErrorInvalidValue;
  const int row_unit = mode == MODE_TF32 ? 4 : 8;       // 16-byte rows of the operands
  if (c.nx % row_unit != 0 || c.ny % row_unit != 0) return cudaErrorInvalidValue;
  MultiMaps maps;
  MultiArgs a{};
  // axis 0: in [ny][nx] -> out [nx][ny] (M = nx); axis 1: in [nx][ny] -> out [ny][nx].
  // Operand images (every input; the output of EPI_STORE) in the bf16 forms:
  // the pair as one buffer, hi [rows][pitch] then lo [rows][pitch].
  const int M = axis == 0 ? c.nx : c.ny, N = axis == 0 ? c.ny : c.nx;
  const bool pair_out = epi == EPI_STORE && mode != MODE_TF32;
  maps.A[0] = P->mK[axis][0][0];
  maps.A[1] = mode == MODE_BF16X3 ? P->mK[axis][0][1] : P->mK[axis][0][0];
  const size_t lo_in = (size_t)N * M * 2, lo_out = (size_t)M * N * 2;   // bytes to the lo half
  for (int z = 0; z < MAXZ; ++z) {
    const int zz = z < nz ? z : 0;
    unsigned char* ib = (unsigned char*)in[zz];
    unsigned char* ob = (unsigned char*)out[zz];
    bool ok = make_map(&maps.B[z][0], ib, mode, N, M, M, MBN);
    ok = ok && (mode == MODE_TF32 ? (maps.B[z][1] = maps.B[z][0], true)
                                  : make_map(&maps.B[z][1], ib + lo_in, mode, N, M, M, MBN));
    if (pair_out) {
      ok = ok && make_map(&maps.O[z][0], ob, mode, M, N, N, BM) &&
           make_map(&maps.O[z][1], ob + lo_out, mode, M, N, N, BM);
    } else {
      ok = ok && make_map(&maps.O[z][0], ob, MODE_TF32, M, N, N, BM);
      maps.O[z][1] = maps.O[z][0];
    }
    if (!ok) return cudaErrorInvalidValue;
    a.out[z] = (float*)out[zz];
    a.q[z] = q ? q[zz] : nullptr;
  }
  a.M = M;
  a.N = N;
  a.pitch_out = N;
  a.kbt = P->kbt[axis][0];
  a.ctrl = c.ctrl;
  a.part = part;
  a.nparts = nparts;
  a.decide = decide;
  if (mode == MODE_BF16X3) return launch_multi_epi<MODE_BF16X3>(maps, a, nz, epi, st);
  if (mode == MODE_BF16) return launch_multi_epi<MODE_BF16>(maps, a, nz, epi, st);
  return launch_multi_epi<MODE_TF32>(maps, a, nz, epi, st);
}

}  // namespace jko
