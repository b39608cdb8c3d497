// attraction.cu -- the joint proximal half-step of the Wasserstein attraction
// with congestion (Sec. 5.2) on the CUDA cores (FP32 / FP64).
//
// The step is the generic diagonal scaling of Sec. 5.1 with M = 2 couplings
// pi_m = diag(a_m) xi diag(b_m), weights lambda = (1, tau), the columns held at
// (q, r) and the rows at a common p.  With the corrections of Prop.
// prop-implementation-generic (which are 1 at the column half-steps, so the
// prox input is xi b_m alone), one iteration is
//     b_1 = q / xi a_1,  b_2 = r / xi a_2                 (filter passes, EPI_B)
//     s_m = xi b_m                                      (filter passes)
//     p = Prox^{KL}_{sigma h/(1+tau)}(s_1^{1/(1+tau)} s_2^{tau/(1+tau)})   (Eq. prox-psi-attraction)
//     a_m = p / s_m                                     (this kernel)
// The energy fields of the handle are built with sigma / (1 + tau), so the
// proximal map of h is the single-coupling one, taken at the geometric mean.
#include "jko_internal.cuh"
#include "jko_kernels.h"

namespace jko {

namespace {

constexpr int NT = 256;

template <typename T, int EK>
__global__ void __launch_bounds__(NT) attraction_prox_kernel(const T* s1, const T* s2, T* a1, T* a2,
                                                             T* p, long long n, T tau,
                                                             ProxArgs<T> P, Ctrl* ctrl, int rnd) {
  __shared__ int s_it;
  if (stop_gate(ctrl, nullptr, 0, false, &s_it)) return;
  const T w1 = T(1) / (T(1) + tau), w2 = tau / (T(1) + tau);
  int bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const T x1 = s1[i], x2 = s2[i];
    // geometric mean s_1^{1/(1+tau)} s_2^{tau/(1+tau)}, 0 where either vanishes
    const T g = (x1 > T(0) && x2 > T(0))
                    ? dev_exp<T>(w1 * dev_log<T>(x1) + w2 * dev_log<T>(x2)) : T(0);
    const T pm = prox_ratio<T, EK>(P, (int)i, g) * g;
    // a_m = p / s_m with IEEE division: s_m may be subnormal far from the
    // support of b_m, where x * rcp(s) would overflow (a_m itself stays finite,
    // ~ (s_other / s_m)^{weight})
    const T r1 = x1 > T(0) ? pm / x1 : T(0);
    const T r2 = x2 > T(0) ? pm / x2 : T(0);
    bad |= !dev_finite(r1) || !dev_finite(r2) || !dev_finite(pm);
    a1[i] = op_round<T>(r1, rnd);
    a2[i] = op_round<T>(r2, rnd);
    p[i] = pm;
  }
  bad = warp_or(bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicOr(&ctrl->nonfinite, 1);
  if (threadIdx.x == 0 && blockIdx.x == 0) ctrl->it = s_it + 1;
}

// Two densities coupled through the congestion of their sum (Sec. 5.3): with
// a~_m = s_m e^{-sigma w_m}, p_m = a~_m min(1, kappa / (a~_1 + a~_2)) and
// a_m = p_m / s_m = e^{-sigma w_m} min(1, ...) (no division by s_m).
template <typename T>
__global__ void __launch_bounds__(NT) species_prox_kernel(const T* s1, const T* s2, const T* E1,
                                                          const T* E2, T* a1, T* a2, T* p,
                                                          long long n, T kappa, int has_kappa,
                                                          Ctrl* ctrl, int rnd) {
  __shared__ int s_it;
  if (stop_gate(ctrl, nullptr, 0, false, &s_it)) return;
  int bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const T e1 = E1 ? E1[i] : T(1), e2 = E2 ? E2[i] : T(1);
    const T t1 = s1[i] * e1, t2 = s2[i] * e2;
    const T t = t1 + t2;
    const T f = (has_kappa && t > kappa) ? kappa / t : T(1);
    a1[i] = op_round<T>(e1 * f, rnd);
    a2[i] = op_round<T>(e2 * f, rnd);
    p[i] = t1 * f;
    p[n + i] = t2 * f;
    bad |= !dev_finite(t1 * f) || !dev_finite(t2 * f);
  }
  bad = warp_or(bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicOr(&ctrl->nonfinite, 1);
  if (threadIdx.x == 0 && blockIdx.x == 0) ctrl->it = s_it + 1;
}

// Pairwise attraction of two densities (Sec. 5.3, multiple densities): the
// generic scaling with 3 couplings, pi_1 (rows p_1, columns q_1), pi_2 (rows
// q_2, columns p_2), pi_3 (rows p_1, columns p_2), weights (1, 1, t), t = tau
// alpha.  By the update rules of Prop. prop-implementation-generic the prox
// inputs are xi b_m (rows) and xi^T a_m (columns) alone.

// Weighted geometric mean x^{1/(1+t)} y^{t/(1+t)}, 0 where either vanishes.
template <typename T>
__device__ __forceinline__ T weighted_geomean(T x, T y, T t) {
  return (x > T(0) && y > T(0)) ? dev_exp<T>((dev_log<T>(x) + t * dev_log<T>(y)) / (T(1) + t))
                                : T(0);
}

// p / s with IEEE division, 0 where p = 0 (s may be subnormal in the far field)
template <typename T>
__device__ __forceinline__ T safe_ratio(T p, T s) {
  return (p > T(0) && s > T(0)) ? p / s : T(0);
}

// Row half-step (psi_1): p_1 = min(e^{-sigma' w_1} g(s_1, s_3), kappa) is the
// common row marginal of pi_1 and pi_3, pi_2 keeps the rows q_2.
template <typename T>
__global__ void __launch_bounds__(NT) pairwise_rows_kernel(const T* s1, const T* s2, const T* s3,
                                                           const T* E1, const T* q2, T* a1, T* a2,
                                                           T* a3, T* p1, long long n, T t, T kappa,
                                                           int has_kappa, Ctrl* ctrl, int rnd) {
  __shared__ int s_it;
  if (stop_gate(ctrl, nullptr, 0, false, &s_it)) return;
  int bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const T x1 = s1[i], x3 = s3[i];
    T pm = weighted_geomean<T>(x1, x3, t) * (E1 ? E1[i] : T(1));
    if (has_kappa && pm > kappa) pm = kappa;
    const T r1 = safe_ratio<T>(pm, x1), r3 = safe_ratio<T>(pm, x3);
    const T r2 = b_update<T>(q2[i], s2[i]);
    bad |= !dev_finite(r1) || !dev_finite(r2) || !dev_finite(r3) || !dev_finite(pm);
    a1[i] = op_round<T>(r1, rnd);
    a2[i] = op_round<T>(r2, rnd);
    a3[i] = op_round<T>(r3, rnd);
    p1[i] = pm;
  }
  bad = warp_or(bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicOr(&ctrl->nonfinite, 1);
}

// Column half-step (psi_2): first the residual of the iterate the row
// half-step left against psi_2's affine constraints, |b_1 y_1 - q_1| +
// |b_2 y_2 - b_3 y_3| (one partial per block, summed by the next pair's first
// kernel), and its column marginal p_2 = b_2 y_2; then the prox on the columns
// of pi_2 and pi_3 and b_1 = q_1 / y_1; the pair counter.
template <typename T>
__global__ void __launch_bounds__(NT) pairwise_cols_kernel(const T* y1, const T* y2, const T* y3,
                                                           const T* E2, const T* q1, T* b1, T* b2,
                                                           T* b3, T* p2, double* part, long long n,
                                                           T t, T kappa, int has_kappa,
                                                           Ctrl* ctrl, int rnd) {
  __shared__ int s_it;
  __shared__ double s_red[33];
  if (stop_gate(ctrl, nullptr, 0, false, &s_it)) return;
  int bad = 0;
  double res = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const T v1 = y1[i], v2 = y2[i], v3 = y3[i];
    const T qq = q1[i], c1 = b1[i], c2 = b2[i], c3 = b3[i];
    res += (double)abs_residual<T>(c1, v1, qq) + (double)fabs(c2 * v2 - c3 * v3);
    p2[i] = c2 * v2;
    T pm = weighted_geomean<T>(v2, v3, t) * (E2 ? E2[i] : T(1));
    if (has_kappa && pm > kappa) pm = kappa;
    const T r1 = b_update<T>(qq, v1);
    const T r2 = safe_ratio<T>(pm, v2), r3 = safe_ratio<T>(pm, v3);
    bad |= !dev_finite(r1) || !dev_finite(r2) || !dev_finite(r3);
    b1[i] = op_round<T>(r1, rnd);
    b2[i] = op_round<T>(r2, rnd);
    b3[i] = op_round<T>(r3, rnd);
  }
  const double tot = block_sum(res, s_red);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
  bad = warp_or(bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicOr(&ctrl->nonfinite, 1);
  if (threadIdx.x == 0 && blockIdx.x == 0) ctrl->it = s_it + 1;
}

}  // namespace

int pairwise_blocks(long long n) {
  long long g = (n + NT - 1) / NT;
  if (g > 152 * 8) g = 152 * 8;
  if (g < 1) g = 1;
  return (int)g;
}

template <typename T>
cudaError_t launch_pairwise_rows(const T* s1, const T* s2, const T* s3, const T* E1, const T* q2,
                                 T* a1, T* a2, T* a3, T* p1, long long n, double t, double kappa,
                                 int has_kappa, Ctrl* ctrl, cudaStream_t st, int rnd) {
  pairwise_rows_kernel<T><<<pairwise_blocks(n), NT, 0, st>>>(
      s1, s2, s3, E1, q2, a1, a2, a3, p1, n, (T)t, (T)kappa, has_kappa, ctrl, rnd);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pairwise_cols(const T* y1, const T* y2, const T* y3, const T* E2, const T* q1,
                                 T* b1, T* b2, T* b3, T* p2, double* part, long long n, double t,
                                 double kappa, int has_kappa, Ctrl* ctrl, cudaStream_t st,
                                 int rnd) {
  pairwise_cols_kernel<T><<<pairwise_blocks(n), NT, 0, st>>>(
      y1, y2, y3, E2, q1, b1, b2, b3, p2, part, n, (T)t, (T)kappa, has_kappa, ctrl, rnd);
  return cudaGetLastError();
}

#define JKO_PW_INST(T)                                                                        \
  template cudaError_t launch_pairwise_rows<T>(const T*, const T*, const T*, const T*,       \
                                               const T*, T*, T*, T*, T*, long long, double,   \
                                               double, int, Ctrl*, cudaStream_t, int);        \
  template cudaError_t launch_pairwise_cols<T>(const T*, const T*, const T*, const T*,       \
                                               const T*, T*, T*, T*, T*, double*, long long,  \
                                               double, double, int, Ctrl*, cudaStream_t, int);
JKO_PW_INST(float)
JKO_PW_INST(double)
#undef JKO_PW_INST

template <typename T>
cudaError_t launch_species_prox(const T* s1, const T* s2, const T* E1, const T* E2, T* a1, T* a2,
                                T* p, long long n, double kappa, int has_kappa, Ctrl* ctrl,
                                cudaStream_t st, int rnd) {
  long long g = (n + NT - 1) / NT;
  if (g > 152 * 8) g = 152 * 8;
  if (g < 1) g = 1;
  species_prox_kernel<T><<<(int)g, NT, 0, st>>>(s1, s2, E1, E2, a1, a2, p, n, (T)kappa,
                                                has_kappa, ctrl, rnd);
  return cudaGetLastError();
}

template cudaError_t launch_species_prox<float>(const float*, const float*, const float*,
                                               const float*, float*, float*, float*, long long,
                                               double, int, Ctrl*, cudaStream_t, int);
template cudaError_t launch_species_prox<double>(const double*, const double*, const double*,
                                                const double*, double*, double*, double*,
                                                long long, double, int, Ctrl*, cudaStream_t, int);

template <typename T>
cudaError_t launch_attraction_prox(int ek, const T* s1, const T* s2, T* a1, T* a2, T* p,
                                   long long n, double tau, const ProxArgs<T>& P, Ctrl* ctrl,
                                   cudaStream_t st, int rnd) {
  long long g = (n + NT - 1) / NT;
  if (g > 152 * 8) g = 152 * 8;
  if (g < 1) g = 1;
  const int grid = (int)g;
  if (ek == EK_CROWD)
    attraction_prox_kernel<T, EK_CROWD><<<grid, NT, 0, st>>>(s1, s2, a1, a2, p, n, (T)tau, P, ctrl, rnd);
  else if (ek == EK_ENTROPY)
    attraction_prox_kernel<T, EK_ENTROPY><<<grid, NT, 0, st>>>(s1, s2, a1, a2, p, n, (T)tau, P, ctrl, rnd);
  else
    attraction_prox_kernel<T, EK_POWER><<<grid, NT, 0, st>>>(s1, s2, a1, a2, p, n, (T)tau, P, ctrl, rnd);
  return cudaGetLastError();
}

template cudaError_t launch_attraction_prox<float>(int, const float*, const float*, float*, float*,
                                                   float*, long long, double,
                                                   const ProxArgs<float>&, Ctrl*, cudaStream_t, int);
template cudaError_t launch_attraction_prox<double>(int, const double*, const double*, double*,
                                                    double*, double*, long long, double,
                                                    const ProxArgs<double>&, Ctrl*, cudaStream_t, int);

}  // namespace jko
