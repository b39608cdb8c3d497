// simt_filter.cu -- plain CUDA-core (FP32 / FP64) form of the Gibbs-kernel
// application and the fused scaling / proximal epilogues.
//
// xi = e^{-|x-y|^2/gamma} on a uniform grid is separable (Sec. 4.1):
// xi X = K_y X K_x^T.  One "pass" filters an image along its strided axis and
// writes the result transposed:
//     out[j][i'] = sum_i k(|i' - i|) in[i][j],   in: [n_i][n_j], out: [n_j][n_i]
// Two passes (y then x) give xi X back in the original [ny][nx] layout.  The
// second pass of each half-iteration carries the elementwise work:
//   EPI_B  b-update + residual (Eq. update-formula-1 and the stopping rule of
//          Sec. 3.4):  r += |b_old Y - q| ;  b = q / Y  (0 where q = 0)
//   EPI_A  KL prox + a-update (Eq. update-formula-2, Eq. defn-pell):
//          a = Prox_{sigma f}(s)/s ;  p = a s
//
// Thread layout: a warp spans 32 consecutive j (coalesced loads of in[i][j]);
// each thread computes RB consecutive outputs i' with a register window that
// slides along i, so each input load feeds RB multiply-adds.  RB = 16, or 4
// where 16 would leave the grid under two blocks per SM (small images: more
// threads, each tap sum in the same order, so the same bits).  The taps are
// the 2r+1 values k(d), d = -r..r, held in shared memory (broadcast reads).
// The outputs of a block are transposed through shared memory before the
// epilogue, which then runs along the output rows with coalesced accesses.
#include "jko_internal.cuh"
#include "jko_kernels.h"

namespace jko {

namespace {

constexpr int RB_MAX = 16;  // outputs per thread along the filtered axis (or 4)
constexpr int BJ = 32;   // threads along the contiguous axis
// thread rows per block (BI): 4, or 8 for the 4-output FP32 form where 8-row
// blocks still give every SM one (32 output rows then share one staged halo)

// One element global -> shared by cp.async (L1-allocating); ok = false writes 0
// and reads nothing.
template <typename T>
__device__ __forceinline__ void cp_async_zfill(T* dst, const T* src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = ok ? (int)sizeof(T) : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;"
               ::"r"(d), "l"(src), "n"((int)sizeof(T)), "r"(n) : "memory");
}
// Four consecutive taps from a 16-byte aligned shared address.
__device__ __forceinline__ void ld_shared4(const float* p, float* o) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld_shared4(const double* p, double* o) {
  const double2 v0 = reinterpret_cast<const double2*>(p)[0];
  const double2 v1 = reinterpret_cast<const double2*>(p)[1];
  o[0] = v0.x; o[1] = v0.y; o[2] = v1.x; o[3] = v1.y;
}

// 16 bytes global -> shared (L2 only); the bytes past nbytes (0..16) are zeroed.
__device__ __forceinline__ void cp_async16_zfill(void* dst, const void* src, int nbytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
               ::"r"(d), "l"(src), "r"(nbytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// One step of the sliding window: acc[o] += k[t0 + dd] x(t0 + o + dd) for
// dd < RB, the rows of the window being lo[0 .. RB) then hi[0 .. RB).
template <typename T, int RB>
__device__ __forceinline__ void tap_step(T (&acc)[RB], const T (&lo)[RB], const T (&hi)[RB],
                                         const T* taps) {
  T kk[RB];
#pragma unroll
  for (int v = 0; v < RB; v += 4) ld_shared4(taps + v, kk + v);
#pragma unroll
  for (int dd = 0; dd < RB; ++dd) {
#pragma unroll
    for (int o = 0; o < RB; ++o)
      acc[o] = fma(kk[dd], (o + dd < RB) ? lo[o + dd] : hi[o + dd - RB], acc[o]);
  }
}

// The tap loop of the untiled pass: rows base + t of the column col (row
// stride ld), three rotating windows (see the kernel); CHECK: rows outside
// [0, n_i) read as 0, else all rows read lie inside.
template <typename T, int RB, bool CHECK>
__device__ __forceinline__ void global_taps(T (&acc)[RB], const T* col, int ld, int base,
                                            int n_i, int t_lo, int t_hi, const T* s_k) {
  auto row = [&](int t) -> T {
    const int ii = base + t;
    return (!CHECK || (ii >= 0 && ii < n_i)) ? __ldg(col + (size_t)ii * ld) : T(0);
  };
  T wa[RB], wb[RB];
#pragma unroll
  for (int u = 0; u < RB; ++u) wa[u] = row(t_lo + u);
  for (int t0 = t_lo; t0 <= t_hi; t0 += RB) {
#pragma unroll
    for (int u = 0; u < RB; ++u) wb[u] = row(t0 + RB + u);
    tap_step<T, RB>(acc, wa, wb, s_k + t0);
#pragma unroll
    for (int u = 0; u < RB; ++u) wa[u] = wb[u];
  }
}

// Staged input rows of the tiled pass: the block's BI RB output rows, the
// 2r rows of the taps' reach and 2 RB more that the last window prefetch reads.
template <int RB, int BI>
__host__ __device__ constexpr int tile_rows(int r) { return BI * RB + 2 * r + 2 * RB; }
// Shared-memory slots of the taps (2r + 1 + RB, zero-padded), rounded up to
// four so that the staged rows behind them start 16-byte aligned.
template <int RB>
__host__ __device__ constexpr int tap_slots(int r) { return (2 * r + 1 + RB + 3) & ~3; }

// TILE: the block first stages its input rows [i_lo - r, i_lo + BI RB + r + 2 RB)
// of its 32 columns in shared memory (coalesced, zeros outside the image), so
// the tap loop reads shared memory with no bounds checks instead of guarded
// global loads; the same terms are added in the same order either way.
template <typename T, int EPI, int EK, int RB, bool TILE, int BI>
__global__ void __launch_bounds__(BJ * BI)
filter_pass(PassArgs<T> A, ProxArgs<T> P) {
  Ctrl* ctrl = A.ctrl;
  __shared__ int s_it;
  if (stop_gate(ctrl, A.part, A.nparts, A.decide != 0, &s_it)) return;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s_k = reinterpret_cast<T*>(smem_raw);
  __shared__ double s_red[33];
  const int tid = threadIdx.y * BJ + threadIdx.x;
  const int ntap = 2 * A.r + 1 + RB;  // taps are zero-padded by RB entries
  for (int t = tid; t < ntap; t += BJ * BI) s_k[t] = A.taps[t];
  __syncthreads();

  // the image of this block: one per launch, or blockIdx.z of a batched launch
  const T* in_img = A.in;
  T* out_img = A.out;
  const T* q_img = A.q;
  if (EPI != EPI_A && A.nz > 1) {
    const int z = blockIdx.z;
    in_img = z == 0 ? A.in_z[0] : (z == 1 ? A.in_z[1] : A.in_z[2]);
    out_img = z == 0 ? A.out_z[0] : (z == 1 ? A.out_z[1] : A.out_z[2]);
    q_img = z == 0 ? A.q_z[0] : (z == 1 ? A.q_z[1] : A.q_z[2]);
  }

  const int j = blockIdx.x * BJ + threadIdx.x;
  const int i0 = (blockIdx.y * BI + threadIdx.y) * RB;
  const bool active = (j < A.n_j) && (i0 < A.n_i);

  T acc[RB];
#pragma unroll
  for (int o = 0; o < RB; ++o) acc[o] = T(0);

  // Both forms: acc[o] = sum_t k[t] in[i0 + o + t - r][j] over t in
  // [t_lo, t_hi], rows outside [0, n_i) read as 0.  t_lo is rounded down to a
  // multiple of 4 so that the taps of a step load four at a time; the terms
  // added that way multiply zeros (rows above the image) and leave every sum
  // unchanged.  Three register windows of RB rows rotate, (a, b) -> (b, c) ->
  // (c, a): a step reads two and loads the rows of the step after next into
  // the third, so the window slides without register moves and its loads
  // are in flight during a step's multiply-adds.
  if constexpr (TILE) {
    // rows [blk_lo - r, blk_lo - r + tile_rows) of columns [blockIdx.x BJ, +BJ)
    T* s_in = s_k + tap_slots<RB>(A.r);
    const int r = A.r;
    const int n_i = A.n_i;
    const int blk_lo = blockIdx.y * BI * RB;
    const int rows = tile_rows<RB, BI>(r);
    const int c0 = blockIdx.x * BJ;
    // asynchronous copies, all in flight at once, zero-filled outside the
    // image: 16 bytes each where the rows are 16-byte aligned, else one element
    constexpr int EPC = 16 / (int)sizeof(T);   // elements per 16-byte chunk
    constexpr int CPR = BJ / EPC;              // chunks per staged row
    if (A.n_j % EPC == 0 && (reinterpret_cast<uintptr_t>(in_img) & 15) == 0) {
      for (int q = tid; q < rows * CPR; q += BJ * BI) {
        const int rr = q / CPR;
        const int jc = c0 + (q % CPR) * EPC;
        const int ii = blk_lo - r + rr;
        int nb = 0;
        if (ii >= 0 && ii < n_i && jc < A.n_j)
          nb = (A.n_j - jc < EPC ? A.n_j - jc : EPC) * (int)sizeof(T);
        cp_async16_zfill(s_in + rr * BJ + (jc - c0),
                         nb ? in_img + (size_t)ii * A.n_j + jc : in_img, nb);
      }
    } else {
      const int jc = c0 + threadIdx.x;
      for (int rr = threadIdx.y; rr < rows; rr += BI) {
        const int ii = blk_lo - r + rr;
        const bool ok = jc < A.n_j && ii >= 0 && ii < n_i;
        cp_async_zfill(s_in + rr * BJ + threadIdx.x,
                       ok ? in_img + (size_t)ii * A.n_j + jc : in_img, ok);
      }
    }
    cp_async_wait_all();
    __syncthreads();
    if (active) {
      // input row ii sits at row ii - (blk_lo - r) of s_in
      int t_lo = r - i0 - (RB - 1);
      if (t_lo < 0) t_lo = 0;
      t_lo &= ~3;
      int t_hi = n_i - 1 - i0 + r;
      if (t_hi > 2 * r) t_hi = 2 * r;
      const T* col = s_in + (i0 - blk_lo) * BJ + threadIdx.x;   // row of t = 0
      T wa[RB], wb[RB], wc[RB];
#pragma unroll
      for (int u = 0; u < RB; ++u) wa[u] = col[(t_lo + u) * BJ];
#pragma unroll
      for (int u = 0; u < RB; ++u) wb[u] = col[(t_lo + RB + u) * BJ];
      for (int t0 = t_lo;;) {
        if (t0 > t_hi) break;
#pragma unroll
        for (int u = 0; u < RB; ++u) wc[u] = col[(t0 + 2 * RB + u) * BJ];
        tap_step<T, RB>(acc, wa, wb, s_k + t0);
        t0 += RB;
        if (t0 > t_hi) break;
#pragma unroll
        for (int u = 0; u < RB; ++u) wa[u] = col[(t0 + 2 * RB + u) * BJ];
        tap_step<T, RB>(acc, wb, wc, s_k + t0);
        t0 += RB;
        if (t0 > t_hi) break;
#pragma unroll
        for (int u = 0; u < RB; ++u) wb[u] = col[(t0 + 2 * RB + u) * BJ];
        tap_step<T, RB>(acc, wc, wa, s_k + t0);
        t0 += RB;
      }
    }
  } else if (active) {
    const int r = A.r;
    const int n_i = A.n_i;
    int t_lo = r - i0 - (RB - 1);
    if (t_lo < 0) t_lo = 0;
    t_lo &= ~3;
    int t_hi = n_i - 1 - i0 + r;
    if (t_hi > 2 * r) t_hi = 2 * r;
    const T* col = in_img + j;
    // rows i0 - r + t for t in [t_lo, t_hi + 3 RB) are read (the last
    // prefetch included); where all lie inside the image no load is guarded
    if (i0 - r + t_lo >= 0 && i0 - r + t_hi + 3 * RB <= n_i)
      global_taps<T, RB, false>(acc, col, A.n_j, i0 - r, n_i, t_lo, t_hi, s_k);
    else
      global_taps<T, RB, true>(acc, col, A.n_j, i0 - r, n_i, t_lo, t_hi, s_k);
  }

  // ---- epilogue: out is [n_j][n_i].  The block's outputs out[jb, jb + BJ)
  // [ib, ib + W) pass through shared memory and are read back along i, so
  // that a warp reads and writes whole row segments (W >= 32: 128 bytes; W = 16:
  // two of 64) instead of one element in each of 32 rows ----
  // The buffer, [BJ][W + 1] (+1: conflict-free column writes), sits behind
  // the taps; in the tiled form it reuses the staged rows, whose last reads
  // the first barrier waits for (one less static buffer: four 1024^2 FP32
  // blocks per SM instead of three).
  constexpr int W = BI * RB;
  T* s_o = s_k + tap_slots<RB>(A.r);
  if constexpr (TILE) __syncthreads();
#pragma unroll
  for (int o = 0; o < RB; ++o) s_o[threadIdx.x * (W + 1) + threadIdx.y * RB + o] = acc[o];
  __syncthreads();
  const int jb = blockIdx.x * BJ;
  const int ib = blockIdx.y * W;
  T res_t = T(0);  // this thread's residual terms, in the working precision
  int bad = 0;
  const bool have_prev = s_it > 0;
  // The global reads of all RB elements (q and the old b; e^{-sigma w} of the
  // crowd prox) are issued before the first write: a write could alias a
  // later read, so in one loop they would wait one L2 round trip each.
  T ld0[RB], ld1[RB];
#pragma unroll
  for (int k = 0; k < RB; ++k) {
    const int e = tid + k * BJ * BI;
    const int jl = e / W;
    const int il = e % W;
    ld0[k] = T(0);
    ld1[k] = T(0);
    if (jb + jl < A.n_j && ib + il < A.n_i) {
      const size_t idx = (size_t)(jb + jl) * A.n_i + (ib + il);
      if (EPI == EPI_B) {
        ld0[k] = q_img[idx];
        if (have_prev) ld1[k] = out_img[idx];
      } else if (EPI == EPI_A && EK == EK_CROWD) {
        ld0[k] = P.E[idx];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < RB; ++k) {
    const int e = tid + k * BJ * BI;
    const int jl = e / W;
    const int il = e % W;
    if (jb + jl < A.n_j && ib + il < A.n_i) {
      const size_t idx = (size_t)(jb + jl) * A.n_i + (ib + il);
      const T v = s_o[jl * (W + 1) + il];
      if (EPI == EPI_STORE) {
        out_img[idx] = v;
      } else if (EPI == EPI_B) {
        const T qv = ld0[k];
        if (have_prev) res_t += abs_residual<T>(ld1[k], v, qv);
        const T bn = b_update<T>(qv, v);
        bad |= !dev_finite(bn);
        out_img[idx] = bn;
      } else {  // EPI_A
        const T a = EK == EK_CROWD ? prox_ratio_e<T, EK>(P, (int)idx, v, ld0[k])
                                   : prox_ratio<T, EK>(P, (int)idx, v);
        bad |= !dev_finite(a);
        A.out[idx] = a;
        A.p[idx] = a * v;
      }
    }
  }
  if (EPI == EPI_STORE) return;

  // ---- residual partial / flags / pair counter (see stop_gate) ----
  bad = warp_or(bad);
  if (EPI == EPI_B) {
    const double res = block_sum((double)res_t, s_red);
    if (tid == 0) A.part[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = res;
  }
  if ((threadIdx.x & 31) == 0 && bad) atomicOr(&ctrl->nonfinite, 1);
  if (EPI == EPI_A && tid == 0 && blockIdx.x == 0 && blockIdx.y == 0) ctrl->it = s_it + 1;
}

// Outputs per thread for an [n_i][n_j] pass: 16 unless that leaves fewer than
// two blocks per SM.
int rb_for(int n_i, int n_j) {
  const int blocks16 = ((n_j + BJ - 1) / BJ) * ((n_i + 4 * 16 - 1) / (4 * 16));
  return blocks16 < 2 * 152 ? 4 : 16;
}

// Thread rows per block: 8 for the 4-output form of a handle alone in FP32 where
// that grid still has a block for every SM (512^2: 256 blocks; halves the staged
// halo per output row: porous 512^2 passes 7.2-8.9 -> 6.7-8.2 us, measured), else
// 4 (at 256^2 the 8-row grid left SMs idle: 4.1 -> 4.4 us; FP64 at 512^2 215 -> 224).
int bi_for(int rb, int n_i, int n_j, int latency, bool fp32) {
  if (rb != 4 || !latency || !fp32) return 4;
  const int blocks8 = ((n_j + BJ - 1) / BJ) * ((n_i + 8 * 4 - 1) / (8 * 4));
  return blocks8 >= 152 ? 8 : 4;
}

// Shared memory of the tiled pass: taps + the staged rows.
template <typename T, int RB, int BI>
size_t tile_smem(int r) {
  return sizeof(T) * ((size_t)tap_slots<RB>(r) + (size_t)tile_rows<RB, BI>(r) * BJ);
}

template <typename T, int EPI, int EK, int RB, bool TILE, int BI>
cudaError_t launch_rb(const PassArgs<T>& A, const ProxArgs<T>& P, cudaStream_t st) {
  const size_t smem = TILE ? tile_smem<T, RB, BI>(A.r)
                           : sizeof(T) * (size_t)(tap_slots<RB>(A.r) + BJ * (BI * RB + 1));
  auto kern = filter_pass<T, EPI, EK, RB, TILE, BI>;
  // opt in well below 48 KB: the kernel's static shared memory (stop gate,
  // reductions) counts against the same default limit
  if (smem > 32 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 block(BJ, BI);
  dim3 grid((A.n_j + BJ - 1) / BJ, (A.n_i + BI * RB - 1) / (BI * RB),
            (EPI != EPI_A && A.nz > 1) ? (unsigned)A.nz : 1u);
  kern<<<grid, block, smem, st>>>(A, P);
  return cudaGetLastError();
}

// A handle alone stages its rows in shared memory: the 4-output form up to
// 160 KB a block, the 16-output form up to 72 KB (three or four blocks per
// SM; 1024^2 FP32, r = 147: 51 KB, plain pass 16.4 us against 23.3 untiled,
// measured), else the untiled 16-output form (FP64 at 1024^2).  Flows of a
// batch keep the untiled 16-output form: there the other flows fill the GPU,
// and the extra blocks and staged halos cost throughput (256-flow FP32 batch:
// 17.6k against 6.2k flow-steps/s with the 4-output tiles, measured).
template <typename T, int EPI, int EK, int RB, int BI>
cudaError_t launch_rb4(const PassArgs<T>& A, const ProxArgs<T>& P, cudaStream_t st) {
  constexpr size_t kTileMax = 160 * 1024;
  return tile_smem<T, RB, BI>(A.r) <= kTileMax ? launch_rb<T, EPI, EK, RB, true, BI>(A, P, st)
                                               : launch_rb<T, EPI, EK, RB, false, BI>(A, P, st);
}

template <typename T, int EPI, int EK>
cudaError_t launch_one(const PassArgs<T>& A, const ProxArgs<T>& P, cudaStream_t st) {
  if (A.latency && rb_for(A.n_i, A.n_j) == 4) {
    if (bi_for(4, A.n_i, A.n_j, A.latency, sizeof(T) == 4) == 8)
      return launch_rb4<T, EPI, EK, 4, 8>(A, P, st);
    return launch_rb4<T, EPI, EK, 4, 4>(A, P, st);
  }
  constexpr size_t kTile16Max = 72 * 1024;
  if (A.latency && tile_smem<T, 16, 4>(A.r) <= kTile16Max)
    return launch_rb<T, EPI, EK, 16, true, 4>(A, P, st);
  return launch_rb<T, EPI, EK, 16, false, 4>(A, P, st);
}

}  // namespace

int simt_tap_padding() { return RB_MAX; }
int simt_pass_blocks(int n_i, int n_j, int latency, int fp64) {
  const int rb = latency ? rb_for(n_i, n_j) : 16;
  const int bi = bi_for(rb, n_i, n_j, latency, fp64 == 0);
  return ((n_j + BJ - 1) / BJ) * ((n_i + bi * rb - 1) / (bi * rb));
}

template <typename T>
cudaError_t simt_pass(int epi, int ek, const PassArgs<T>& A, const ProxArgs<T>& P,
                      cudaStream_t st) {
  if (epi == EPI_STORE) return launch_one<T, EPI_STORE, EK_CROWD>(A, P, st);
  if (epi == EPI_B) return launch_one<T, EPI_B, EK_CROWD>(A, P, st);
  switch (ek) {
    case EK_CROWD: return launch_one<T, EPI_A, EK_CROWD>(A, P, st);
    case EK_ENTROPY: return launch_one<T, EPI_A, EK_ENTROPY>(A, P, st);
    default: return launch_one<T, EPI_A, EK_POWER>(A, P, st);
  }
}

template cudaError_t simt_pass<float>(int, int, const PassArgs<float>&, const ProxArgs<float>&,
                                      cudaStream_t);
template cudaError_t simt_pass<double>(int, int, const PassArgs<double>&,
                                       const ProxArgs<double>&, cudaStream_t);

}  // namespace jko
