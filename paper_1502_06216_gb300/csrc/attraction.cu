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
                                                             ProxArgs<T> P, Ctrl* ctrl) {
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
    a1[i] = r1;
    a2[i] = r2;
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
                                                          Ctrl* ctrl) {
  __shared__ int s_it;
  if (stop_gate(ctrl, nullptr, 0, false, &s_it)) return;
  int bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const T e1 = E1 ? E1[i] : T(1), e2 = E2 ? E2[i] : T(1);
    const T t1 = s1[i] * e1, t2 = s2[i] * e2;
    const T t = t1 + t2;
    const T f = (has_kappa && t > kappa) ? kappa / t : T(1);
    a1[i] = e1 * f;
    a2[i] = e2 * f;
    p[i] = t1 * f;
    p[n + i] = t2 * f;
    bad |= !dev_finite(t1 * f) || !dev_finite(t2 * f);
  }
  bad = warp_or(bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicOr(&ctrl->nonfinite, 1);
  if (threadIdx.x == 0 && blockIdx.x == 0) ctrl->it = s_it + 1;
}

}  // namespace

template <typename T>
cudaError_t launch_species_prox(const T* s1, const T* s2, const T* E1, const T* E2, T* a1, T* a2,
                                T* p, long long n, double kappa, int has_kappa, Ctrl* ctrl,
                                cudaStream_t st) {
  long long g = (n + NT - 1) / NT;
  if (g > 152 * 8) g = 152 * 8;
  if (g < 1) g = 1;
  species_prox_kernel<T><<<(int)g, NT, 0, st>>>(s1, s2, E1, E2, a1, a2, p, n, (T)kappa,
                                                has_kappa, ctrl);
  return cudaGetLastError();
}

template cudaError_t launch_species_prox<float>(const float*, const float*, const float*,
                                               const float*, float*, float*, float*, long long,
                                               double, int, Ctrl*, cudaStream_t);
template cudaError_t launch_species_prox<double>(const double*, const double*, const double*,
                                                const double*, double*, double*, double*,
                                                long long, double, int, Ctrl*, cudaStream_t);

template <typename T>
cudaError_t launch_attraction_prox(int ek, const T* s1, const T* s2, T* a1, T* a2, T* p,
                                   long long n, double tau, const ProxArgs<T>& P, Ctrl* ctrl,
                                   cudaStream_t st) {
  long long g = (n + NT - 1) / NT;
  if (g > 152 * 8) g = 152 * 8;
  if (g < 1) g = 1;
  const int grid = (int)g;
  if (ek == EK_CROWD)
    attraction_prox_kernel<T, EK_CROWD><<<grid, NT, 0, st>>>(s1, s2, a1, a2, p, n, (T)tau, P, ctrl);
  else if (ek == EK_ENTROPY)
    attraction_prox_kernel<T, EK_ENTROPY><<<grid, NT, 0, st>>>(s1, s2, a1, a2, p, n, (T)tau, P, ctrl);
  else
    attraction_prox_kernel<T, EK_POWER><<<grid, NT, 0, st>>>(s1, s2, a1, a2, p, n, (T)tau, P, ctrl);
  return cudaGetLastError();
}

template cudaError_t launch_attraction_prox<float>(int, const float*, const float*, float*, float*,
                                                   float*, long long, double,
                                                   const ProxArgs<float>&, Ctrl*, cudaStream_t);
template cudaError_t launch_attraction_prox<double>(int, const double*, const double*, double*,
                                                    double*, double*, long long, double,
                                                    const ProxArgs<double>&, Ctrl*, cudaStream_t);

}  // namespace jko
