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
constexpr int BI = 4;    // thread rows per block

// One element global -> shared by cp.async (L1-allocating); ok = false writes 0
// and reads nothing.
template <typename T>
__device__ __forceinline__ void cp_async_zfill(T* dst, const T* src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = ok ? (int)sizeof(T) : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;"
               ::"r"(d), "l"(src), "n"((int)sizeof(T)), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// TILE (small images): the block first stages its input rows [i_lo - r, i_lo + BI RB + r)
// of its 32 columns in shared memory (coalesced, zeros outside the image), so
// the tap loop reads shared memory instead of a chain of dependent global
// loads; the same terms are added in the same order either way.
template <typename T, int EPI, int EK, int RB, bool TILE>
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

  if constexpr (TILE) {
    // rows [blk_lo - r, blk_lo + BI RB + r + RB) of columns [blockIdx.x BJ, +BJ)
    // (RB rows beyond the last used one: the window's last refill reads them)
    T* s_in = s_k + ntap;
    const int r = A.r;
    const int n_i = A.n_i;
    const int blk_lo = blockIdx.y * BI * RB;
    const int rows = BI * RB + 2 * r + RB;
    const int jc = blockIdx.x * BJ + threadIdx.x;
    // asynchronous copies, all in flight at once (a load-then-store loop
    // waits one L2 round trip per row); rows outside the image are zero-filled
    for (int rr = threadIdx.y; rr < rows; rr += BI) {
      const int ii = blk_lo - r + rr;
      const bool ok = jc < A.n_j && ii >= 0 && ii < n_i;
      cp_async_zfill(s_in + rr * BJ + threadIdx.x,
                     ok ? in_img + (size_t)ii * A.n_j + jc : in_img, ok);
    }
    cp_async_wait_all();
    __syncthreads();
    if (active) {
      // the register window of the untiled pass, refilled from shared memory:
      // input row ii sits at row ii - (blk_lo - r) of s_in
      int t_lo = r - i0 - (RB - 1);
      if (t_lo < 0) t_lo = 0;
      int t_hi = n_i - 1 - i0 + r;
      if (t_hi > 2 * r) t_hi = 2 * r;
      const T* col = s_in + (i0 - blk_lo) * BJ + threadIdx.x;   // row of t = 0
      T win[2 * RB];
#pragma unroll
      for (int u = 0; u < RB; ++u) win[u] = col[(t_lo + u) * BJ];
      for (int t0 = t_lo; t0 <= t_hi; t0 += RB) {
#pragma unroll
        for (int u = 0; u < RB; ++u) win[RB + u] = col[(t0 + RB + u) * BJ];
#pragma unroll
        for (int dd = 0; dd < RB; ++dd) {
          const T k = s_k[t0 + dd];
#pragma unroll
          for (int o = 0; o < RB; ++o) acc[o] = fma(k, win[o + dd], acc[o]);
        }
#pragma unroll
        for (int u = 0; u < RB; ++u) win[u] = win[RB + u];
      }
    }
  } else if (active) {
    // acc[o] = sum_{t=0}^{2r} k[t] in[i0 + o + t - r][j]; rows outside [0, n_i) are 0.
    const int r = A.r;
    const int n_i = A.n_i;
    int t_lo = r - i0 - (RB - 1);
    if (t_lo < 0) t_lo = 0;
    int t_hi = n_i - 1 - i0 + r;
    if (t_hi > 2 * r) t_hi = 2 * r;
    const T* col = in_img + j;
    const size_t ld = (size_t)A.n_j;
    T win[2 * RB];
    int base = i0 - r + t_lo;
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const int ii = base + u;
      win[u] = (ii >= 0 && ii < n_i) ? __ldg(col + (size_t)ii * ld) : T(0);
    }
    for (int t0 = t_lo; t0 <= t_hi; t0 += RB) {
      base = i0 - r + t0;
#pragma unroll
      for (int u = 0; u < RB; ++u) {
        const int ii = base + RB + u;
        win[RB + u] = (ii >= 0 && ii < n_i) ? __ldg(col + (size_t)ii * ld) : T(0);
      }
#pragma unroll
      for (int dd = 0; dd < RB; ++dd) {
        const T k = s_k[t0 + dd];
#pragma unroll
        for (int o = 0; o < RB; ++o) acc[o] = fma(k, win[o + dd], acc[o]);
      }
#pragma unroll
      for (int u = 0; u < RB; ++u) win[u] = win[RB + u];
    }
  }

  // ---- epilogue: out is [n_j][n_i].  The block's outputs out[jb, jb + BJ)
  // [ib, ib + W) pass through shared memory and are read back along i, so
  // that a warp reads and writes whole row segments (W >= 32: 128 bytes; W = 16:
  // two of 64) instead of one element in each of 32 rows ----
  constexpr int W = BI * RB;
  __shared__ T s_o[BJ][W + 1];   // +1: conflict-free column writes
#pragma unroll
  for (int o = 0; o < RB; ++o) s_o[threadIdx.x][threadIdx.y * RB + o] = acc[o];
  __syncthreads();
  const int jb = blockIdx.x * BJ;
  const int ib = blockIdx.y * W;
  T res_t = T(0);  // this thread's residual terms, in the working precision
  int bad = 0;
  const bool have_prev = s_it > 0;
#pragma unroll
  for (int k = 0; k < RB; ++k) {
    const int e = tid + k * BJ * BI;
    const int jl = e / W;
    const int il = e % W;
    if (jb + jl < A.n_j && ib + il < A.n_i) {
      const size_t idx = (size_t)(jb + jl) * A.n_i + (ib + il);
      const T v = s_o[jl][il];
      if (EPI == EPI_STORE) {
        out_img[idx] = v;
      } else if (EPI == EPI_B) {
        const T qv = q_img[idx];
        if (have_prev) res_t += abs_residual<T>(out_img[idx], v, qv);
        const T bn = b_update<T>(qv, v);
        bad |= !dev_finite(bn);
        out_img[idx] = bn;
      } else {  // EPI_A
        const T a = prox_ratio<T, EK>(P, (int)idx, v);
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
  const int blocks16 = ((n_j + BJ - 1) / BJ) * ((n_i + BI * 16 - 1) / (BI * 16));
  return blocks16 < 2 * 152 ? 4 : 16;
}

// Shared memory of the tiled pass: taps + the staged rows.
template <typename T, int RB>
size_t tile_smem(int r) {
  return sizeof(T) * ((size_t)(2 * r + 1 + RB) + (size_t)(BI * RB + 2 * r + RB) * BJ);
}

template <typename T, int EPI, int EK, int RB, bool TILE>
cudaError_t launch_rb(const PassArgs<T>& A, const ProxArgs<T>& P, cudaStream_t st) {
  const size_t smem = TILE ? tile_smem<T, RB>(A.r) : sizeof(T) * (size_t)(2 * A.r + 1 + RB);
  auto kern = filter_pass<T, EPI, EK, RB, TILE>;
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

// Small images (the 4-output variant) stage their rows in shared memory; on
// large ones the untiled pass keeps more blocks resident and wins (1024^2
// FP32: 5.4k against 5.0k pairs/s tiled, measured).  Flows of a batch keep the
// 16-output form: there the other flows fill the GPU, and the extra blocks
// and staged halos cost throughput (256-flow FP32 batch: 17.6k against 6.2k
// flow-steps/s, measured).
template <typename T, int EPI, int EK>
cudaError_t launch_one(const PassArgs<T>& A, const ProxArgs<T>& P, cudaStream_t st) {
  constexpr size_t kTileMax = 160 * 1024;
  if (A.latency && rb_for(A.n_i, A.n_j) == 4)
    return tile_smem<T, 4>(A.r) <= kTileMax ? launch_rb<T, EPI, EK, 4, true>(A, P, st)
                                            : launch_rb<T, EPI, EK, 4, false>(A, P, st);
  return launch_rb<T, EPI, EK, 16, false>(A, P, st);
}

}  // namespace

int simt_tap_padding() { return RB_MAX; }
int simt_pass_blocks(int n_i, int n_j, int latency) {
  const int rb = latency ? rb_for(n_i, n_j) : 16;
  return ((n_j + BJ - 1) / BJ) * ((n_i + BI * rb - 1) / (BI * rb));
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
