// jko_step_kernels.cu -- per-step prologue and epilogue kernels: fill, input
// validation, and the FP64 mass / congestion statistics with the optional
// mass renormalisation of the step output.
#include <algorithm>

#include "jko_kernels.h"

namespace jko {

namespace {

constexpr int NT = 256;

template <typename T>
__global__ void fill_kernel(T* x, T v, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = v;
}

// The start of a step in one launch: the control block reset to its initial
// value, q copied into the handle's image (q_in NULL: already there) and, for
// the plain form, the cold start a = 1 (a NULL: the form sets up its own).
template <typename T>
__global__ void step_begin_kernel(Ctrl init, Ctrl* ctrl, unsigned* chunks, const T* q_in, T* q,
                                  long long nq, T* a, long long na) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *ctrl = init;
    if (chunks) *chunks = 0;
  }
  const long long n = nq > na ? nq : na;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (q_in && i < nq) q[i] = q_in[i];
    if (a && i < na) a[i] = T(1);
  }
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T kappa_at(const ProxArgs<T>& P, long long i) {
  return P.kappa ? P.kappa[i] : P.kappa_s;
}

template <typename T>
__global__ void validate_kernel(const T* q, long long n, ProxArgs<T> P, Ctrl* ctrl) {
  __shared__ double s_red[33];
  double sum = 0.0;
  unsigned long long neg = 0, bad = 0, over = 0, msk = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const T v = q[i];
    if (!isfinite(v)) { ++bad; continue; }
    sum += (double)v;
    if (v < T(0)) ++neg;
    if (P.has_kappa && (double)v > (double)kappa_at(P, i) * (1.0 + 1e-2)) ++over;
    if (P.mask && P.mask[i] && v != T(0)) ++msk;
  }
  sum = block_sum(sum, s_red);
  neg = warp_sum_u64(neg);
  bad = warp_sum_u64(bad);
  over = warp_sum_u64(over);
  msk = warp_sum_u64(msk);
  if ((threadIdx.x & 31) == 0) {
    if (neg) atomicAdd(&ctrl->q_neg, neg);
    if (bad) atomicAdd(&ctrl->q_bad, bad);
    if (over) atomicAdd(&ctrl->q_over, over);
    if (msk) atomicAdd(&ctrl->q_masked, msk);
  }
  if (threadIdx.x == 0) atomicAdd(&ctrl->q_sum, sum);
}

template <typename T>
__global__ void finalize_reduce_kernel(const T* p, long long n, ProxArgs<T> P, Ctrl* ctrl,
                                       double* part) {
  __shared__ double s_red[33];
  __shared__ int s_last;
  double sum = 0.0;
  T mx = T(0);   // max p / kappa, a diagnostic: the working precision suffices
  int bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const T v = p[i];
    bad |= !isfinite(v);
    sum += (double)v;
    if (P.has_kappa) {
      const T r = v / kappa_at(P, i);
      mx = r > mx ? r : mx;
    }
  }
  sum = block_sum(sum, s_red);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  bad = warp_or(bad);
  if ((threadIdx.x & 31) == 0) {
    const double mxd = (double)mx;
    if (mxd > 0.0) atomicMax(&ctrl->maxpk_bits, (unsigned long long)__double_as_longlong(mxd));
    if (bad) atomicOr(&ctrl->nonfinite, 1);
  }
  // The mass is summed in a fixed order, so that repeated runs give the same
  // bits: one partial per block, and the last block to arrive adds them up.
  if (threadIdx.x == 0) {
    part[blockIdx.x] = sum;
    __threadfence();
    s_last = atomicAdd(&ctrl->arrive_f, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double tot = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) tot += __ldcg(part + i);
  tot = block_sum(tot, s_red);
  if (threadIdx.x == 0) {
    ctrl->mass = tot;
    ctrl->arrive_f = 0;
  }
}

// True when the input checks of a step (validate_kernel) found q invalid.
__device__ __forceinline__ bool q_invalid(const Ctrl* ctrl) {
  return ctrl->q_bad || ctrl->q_neg || fabs(ctrl->q_sum - 1.0) > 1e-3 || ctrl->q_masked ||
         ctrl->q_over;
}

template <typename T>
__global__ void finalize_write_kernel(const T* p, T* out, long long n, int renorm,
                                      const Ctrl* ctrl, int check, Ctrl* record) {
  // the step's final control block, for a flow that reads all steps' at its end
  if (record && blockIdx.x == 0 && threadIdx.x == 0) *record = *ctrl;
  // a step whose input failed its checks leaves the output untouched
  if (check && q_invalid(ctrl)) return;
  const double mass = ctrl->mass;
  const bool scale = renorm && mass > 0.0 && isfinite(mass);
  // p / mass as p times the FP64 reciprocal (within one FP64 ulp of the
  // quotient): one multiply per cell instead of a division on the narrow FP64 pipe
  const double inv = scale ? 1.0 / mass : 1.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const T v = p[i];
    out[i] = scale ? (T)((double)v * inv) : v;
  }
}

int grid_for(long long n) {
  long long g = (n + NT - 1) / NT;
  if (g > 152 * 8) g = 152 * 8;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

template <typename T>
cudaError_t launch_step_begin(const Ctrl& init, Ctrl* ctrl, unsigned* chunks, const T* q_in,
                              T* q, long long nq, T* a, long long na, cudaStream_t st) {
  step_begin_kernel<T><<<grid_for(nq > na ? nq : na), NT, 0, st>>>(init, ctrl, chunks, q_in, q,
                                                                    nq, a, na);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fill(T* x, T v, long long n, cudaStream_t st) {
  fill_kernel<T><<<grid_for(n), NT, 0, st>>>(x, v, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_validate(const T* q, long long n, const ProxArgs<T>& P, Ctrl* ctrl,
                            cudaStream_t st) {
  validate_kernel<T><<<grid_for(n), NT, 0, st>>>(q, n, P, ctrl);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_finalize_reduce(const T* p, long long n, const ProxArgs<T>& P, Ctrl* ctrl,
                                   double* part, int part_cap, cudaStream_t st) {
  if (!part || part_cap < 1) return cudaErrorInvalidValue;
  const int g = std::min(grid_for(n), part_cap);
  finalize_reduce_kernel<T><<<g, NT, 0, st>>>(p, n, P, ctrl, part);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_finalize_write(const T* p, T* out, long long n, int renorm, const Ctrl* ctrl,
                                  cudaStream_t st, int check, Ctrl* record) {
  finalize_write_kernel<T><<<grid_for(n), NT, 0, st>>>(p, out, n, renorm, ctrl, check, record);
  return cudaGetLastError();
}

namespace {
__global__ void gather_done_kernel(Ctrl* const* ctrls, int* done, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    done[i] = ctrls[i]->done;
}
__global__ void gather_ctrl_kernel(Ctrl* const* ctrls, Ctrl* out, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = *ctrls[i];
}
}  // namespace

namespace {
__global__ void chunk_loop_cond_kernel(unsigned* chunks, const Ctrl* ctrl,
                                       cudaGraphConditionalHandle hc, unsigned max_chunks) {
  const unsigned n = *chunks + 1;
  *chunks = n;
  cudaGraphSetConditional(hc, (ctrl->done == RUNNING && n < max_chunks) ? 1u : 0u);
}
}  // namespace

cudaError_t launch_chunk_loop_cond(unsigned* chunks, const Ctrl* ctrl,
                                   cudaGraphConditionalHandle hc, unsigned max_chunks,
                                   cudaStream_t st) {
  chunk_loop_cond_kernel<<<1, 1, 0, st>>>(chunks, ctrl, hc, max_chunks);
  return cudaGetLastError();
}

namespace {
__global__ void resume_kernel(Ctrl* ctrl) {
  ctrl->done = RUNNING;
  ctrl->since[0] = 0;
  ctrl->since[1] = 0;
}
}  // namespace

cudaError_t launch_resume(Ctrl* ctrl, cudaStream_t st) {
  resume_kernel<<<1, 1, 0, st>>>(ctrl);
  return cudaGetLastError();
}

cudaError_t launch_gather_done(Ctrl* const* ctrls, int* done, int n, cudaStream_t st) {
  gather_done_kernel<<<(n + 127) / 128, 128, 0, st>>>(ctrls, done, n);
  return cudaGetLastError();
}
cudaError_t launch_gather_ctrl(Ctrl* const* ctrls, Ctrl* out, int n, cudaStream_t st) {
  gather_ctrl_kernel<<<(n + 127) / 128, 128, 0, st>>>(ctrls, out, n);
  return cudaGetLastError();
}

#define JKO_INST(T)                                                                     \
  template cudaError_t launch_fill<T>(T*, T, long long, cudaStream_t);                  \
  template cudaError_t launch_validate<T>(const T*, long long, const ProxArgs<T>&, Ctrl*, \
                                          cudaStream_t);                                \
  template cudaError_t launch_finalize_reduce<T>(const T*, long long, const ProxArgs<T>&, \
                                                 Ctrl*, double*, int, cudaStream_t);    \
  template cudaError_t launch_finalize_write<T>(const T*, T*, long long, int, const Ctrl*, \
                                                cudaStream_t, int, Ctrl*);                    \
  template cudaError_t launch_step_begin<T>(const Ctrl&, Ctrl*, unsigned*, const T*, T*,     \
                                            long long, T*, long long, cudaStream_t);
JKO_INST(float)
JKO_INST(double)
#undef JKO_INST

}  // namespace jko
