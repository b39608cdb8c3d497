// jko_adjoint.cu -- reverse-mode differentiation of the JKO flow (CUDA cores).
//
// One step maps q to p through the fixed point of the scaling loop (Prop. 3.3,
// 2-vector form): with Y = xi a, b = q / Y, s = xi b, the fixed point is
// a = r(s, w), r = Prox_{sigma f}(s)/s, and the output is p = a (.) s
// (then p / sum p when renormalising).  Implicit differentiation at the fixed
// point, xi symmetric, D = b / Y, R_s = dr/ds, R_w = dr/dw:
//   direct terms   abar = s (.) g - xi( D (.) xi(a (.) g) ),   qbar0 = xi(a (.) g) / Y
//   adjoint solve  lambda = abar - xi( D (.) xi(R_s (.) lambda) )
//                  (the transposed linearisation of the forward map a -> r(xi(q / xi a));
//                  the same contraction, so a fixed-point iteration converges like
//                  the forward loop)
//   gradients      qbar = qbar0 + xi(R_s (.) lambda) / Y,   wbar += R_w (.) lambda.
// Steps are walked backwards from a tape of each step's input q_t and final a_t
// (jko_flow_record); Y, b, s are recomputed from them.  Every xi application
// is the forward's own: the two CUDA-core filter passes (or their FFT form)
// of the Gaussian, or the Clenshaw evaluation of the heat kernel xi~, which is
// symmetric as well (Sec. 4.1, Eq. heat-kernel).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "jko.h"
#include "jko_handle.h"
#include "jko_kernels.h"

namespace {

using jko::PassArgs;

constexpr int NT = 256;

int grid_for(long long n) {
  long long g = (n + NT - 1) / NT;
  if (g > 152 * 8) g = 152 * 8;
  return (int)(g < 1 ? 1 : g);
}

#define GS(i, n)                                                                  \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); \
       i += (long long)gridDim.x * blockDim.x)

// b = q / Y with the forward's guard, and 1/Y (0 where the forward set b = 0
// because Y underflowed or where q = 0 but Y is fine: 1/Y there).
template <typename T>
__global__ void k_b_invY(const T* q, const T* Y, T* b, T* invY, long long n) {
  GS(i, n) {
    const T y = Y[i];
    const bool ok = y >= jko::NormalMin<T>::v;
    b[i] = jko::b_update<T>(q[i], y);
    invY[i] = ok ? T(1) / y : T(0);
  }
}

template <typename T>
__global__ void k_dot3(const T* x, const T* y, const T* z, double* out, long long n) {
  __shared__ double s_red[33];
  double v = 0.0;
  GS(i, n) v += (double)x[i] * (double)y[i] * (double)z[i];
  v = jko::block_sum(v, s_red);
  if (threadIdx.x == 0) atomicAdd(out, v);
}

// gt = (g - <g, a s> / m) / m  (adjoint of p / m with m = sum p);  u = a gt
template <typename T>
__global__ void k_renorm(const T* g, const T* a, const double* dot, double m, int renorm, T* gt,
                         T* u, long long n) {
  const double c = renorm ? *dot / m : 0.0;
  const double inv = renorm ? 1.0 / m : 1.0;
  GS(i, n) {
    const T v = (T)(((double)g[i] - c) * inv);
    gt[i] = v;
    u[i] = a[i] * v;
  }
}

template <typename T>
__global__ void k_mul(const T* x, const T* y, T* out, long long n) {
  GS(i, n) out[i] = x[i] * y[i];
}

// out = s gt - w2 ; qbar0 = v invY
template <typename T>
__global__ void k_abar(const T* s, const T* gt, const T* w2, const T* v, const T* invY, T* abar,
                       T* qbar0, long long n) {
  GS(i, n) {
    abar[i] = s[i] * gt[i] - w2[i];
    qbar0[i] = v[i] * invY[i];
  }
}

// u = R_s (.) lambda
template <typename T, int EK>
__global__ void k_rs(jko::ProxArgs<T> P, const T* s, const T* lam, T* u, long long n) {
  GS(i, n) {
    T rs, rw;
    jko::ratio_grad<T, EK>(P, (int)i, s[i], rs, rw);
    u[i] = rs * lam[i];
  }
}

// lambda_new = abar - w2 ; diff += |lambda_new - lambda| ; norm += |abar|
template <typename T>
__global__ void k_lambda(const T* abar, const T* w2, T* lam, double* diff, double* norm,
                         long long n) {
  __shared__ double s_red[33];
  double d = 0.0, a = 0.0;
  GS(i, n) {
    const T ln = abar[i] - w2[i];
    d += fabs((double)ln - (double)lam[i]);
    a += fabs((double)abar[i]);
    lam[i] = ln;
  }
  d = jko::block_sum(d, s_red);
  a = jko::block_sum(a, s_red);
  if (threadIdx.x == 0) {
    atomicAdd(diff, d);
    atomicAdd(norm, a);
  }
}

// g = qbar0 + v invY ;  wbar += R_w (.) lambda
template <typename T, int EK>
__global__ void k_final(jko::ProxArgs<T> P, const T* s, const T* lam, const T* qbar0, const T* v,
                        const T* invY, T* g, T* wbar, long long n) {
  GS(i, n) {
    T rs, rw;
    jko::ratio_grad<T, EK>(P, (int)i, s[i], rs, rw);
    g[i] = qbar0[i] + v[i] * invY[i];
    wbar[i] += rw * lam[i];
  }
}

// The FFT tables of the pass along x (lines of length nx) or along y.
template <typename T>
jko::FftArgs<T> fft_tables(const jko_handle* h, bool along_x) {
  jko::FftArgs<T> F;
  F.L = along_x ? h->fft_Lx : h->fft_Ly;
  F.log2L = along_x ? h->fft_lgx : h->fft_lgy;
  F.khat = (const T*)(along_x ? h->fft_khat_x : h->fft_khat_y);
  F.tw = (const T*)(along_x ? h->fft_tw_x : h->fft_tw_y);
  return F;
}

template <typename T>
cudaError_t xi_apply(jko_handle* h, const T* in, T* out, cudaStream_t st) {
  if (h->heat_L)
    return jko::heat_apply<T>(h->heat, h->hb, in, out, h->grid.nx, h->grid.ny,
                              (const uint8_t*)h->mask, h->ctrl, h->part, 0, 0, st, true);
  jko::ProxArgs<T> P = jko::prox_args<T>(h);
  PassArgs<T> A{};
  A.ctrl = h->ctrl;
  A.part = h->part;
  A.latency = h->simt_latency;
  A.in = in;
  A.out = (T*)h->t1;
  A.taps = (const T*)h->taps_y;
  A.n_i = h->grid.ny; A.n_j = h->grid.nx; A.r = h->ry;
  cudaError_t e = h->fft ? jko::fft_pass<T>(jko::EPI_STORE, h->ek, A, P, fft_tables<T>(h, false), st)
                         : jko::simt_pass<T>(jko::EPI_STORE, h->ek, A, P, st);
  if (e != cudaSuccess) return e;
  A.in = (const T*)h->t1;
  A.out = out;
  A.taps = (const T*)h->taps_x;
  A.n_i = h->grid.nx; A.n_j = h->grid.ny; A.r = h->rx;
  if (h->fft) return jko::fft_pass<T>(jko::EPI_STORE, h->ek, A, P, fft_tables<T>(h, true), st);
  return jko::simt_pass<T>(jko::EPI_STORE, h->ek, A, P, st);
}

#define ACK(call)                                                                     \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return jko::handle_error(h, e_ == cudaErrorMemoryAllocation ? JKO_ERR_OOM : JKO_ERR_CUDA, \
                               std::string(#call) + ": " + cudaGetErrorName(e_));     \
  } while (0)

template <typename T, int EK>
jko_status backward_t(jko_handle* h, const T* grad_final, T* grad_p0, T* grad_w, int* adj_iters) {
  cudaStream_t st = h->stream;
  const long long N = h->N;
  if (!h->adj) {
    ACK(cudaMalloc(&h->adj, sizeof(T) * N * 10));
    ACK(cudaMalloc((void**)&h->adj_red, sizeof(double) * 4));
  }
  T* W = (T*)h->adj;
  T *Y = W, *b = W + N, *s = W + 2 * N, *invY = W + 3 * N, *g = W + 4 * N, *gt = W + 5 * N,
    *u = W + 6 * N, *v = W + 7 * N, *lam = W + 8 * N, *abar = W + 9 * N;
  T* qbar0 = gt;  // written once gt has been consumed (k_abar)
  jko::ProxArgs<T> P = jko::prox_args<T>(h);
  // a clean control block: the filter passes only check that no stop is recorded
  ACK(cudaMemcpyAsync(h->ctrl, h->ctrl_init, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
  ACK(cudaMemcpyAsync(g, grad_final, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
  if (grad_w) ACK(cudaMemsetAsync(grad_w, 0, sizeof(T) * N, st));
  T* wbar_dev = grad_w;
  T* scratch_w = nullptr;
  if (!wbar_dev) {  // gradient in w not requested: accumulate into u-sized scratch anyway
    scratch_w = u;
  }
  const int budget = std::max(16, 10 * h->prm.max_iter);
  const double tol = std::max(h->prm.tol, h->fp64 ? 1e-15 : 1e-7);
  const int G = grid_for(N);
  T* wtmp = v;  // second xi output shares v
  for (int t = h->tape_steps - 1; t >= 0; --t) {
    const T* q = (const T*)h->tape + (size_t)(2 * t) * N;
    const T* a = q + N;
    const double m = h->tape_mass[t];
    // recompute the fixed-point quantities of step t
    ACK(xi_apply<T>(h, a, Y, st));
    k_b_invY<T><<<G, NT, 0, st>>>(q, Y, b, invY, N);
    ACK(cudaGetLastError());
    ACK(xi_apply<T>(h, b, s, st));
    // adjoint of the renormalisation, then the direct terms
    ACK(cudaMemsetAsync(h->adj_red, 0, sizeof(double) * 4, st));
    k_dot3<T><<<G, NT, 0, st>>>(g, a, s, h->adj_red, N);
    ACK(cudaGetLastError());
    k_renorm<T><<<G, NT, 0, st>>>(g, a, h->adj_red, m, h->prm.renormalize, gt, u, N);
    ACK(cudaGetLastError());
    ACK(xi_apply<T>(h, u, v, st));                 // v = xi(a gt)
    // D (.) v with D = b / Y = b invY
    k_mul<T><<<G, NT, 0, st>>>(b, invY, u, N);      // u = D
    k_mul<T><<<G, NT, 0, st>>>(u, v, lam, N);       // lam = D v (temporary)
    ACK(cudaGetLastError());
    ACK(xi_apply<T>(h, lam, abar, st));            // abar = xi(D v) (temporary)
    // D is needed in the solve: keep it in b (b itself is no longer needed)
    ACK(cudaMemcpyAsync(b, u, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
    T* D = b;
    // qbar0 needs its own storage: use gt after abar is formed
    k_abar<T><<<G, NT, 0, st>>>(s, gt, abar, v, invY, abar, gt, N);  // abar, qbar0 (in gt)
    ACK(cudaGetLastError());
    // adjoint fixed-point solve, lambda_0 = abar
    ACK(cudaMemcpyAsync(lam, abar, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
    int k = 0;
    bool conv = false;
    double host_red[4];
    for (; k < budget && !conv; ++k) {
      if ((k & 7) == 0) ACK(cudaMemsetAsync(h->adj_red, 0, sizeof(double) * 4, st));
      k_rs<T, EK><<<G, NT, 0, st>>>(P, s, lam, u, N);
      ACK(cudaGetLastError());
      ACK(xi_apply<T>(h, u, v, st));
      k_mul<T><<<G, NT, 0, st>>>(D, v, u, N);
      ACK(cudaGetLastError());
      ACK(xi_apply<T>(h, u, wtmp, st));  // wtmp aliases v: v is consumed above
      k_lambda<T><<<G, NT, 0, st>>>(abar, wtmp, lam, h->adj_red, h->adj_red + 1, N);
      ACK(cudaGetLastError());
      if ((k & 7) == 7) {
        ACK(cudaMemcpyAsync(host_red, h->adj_red, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
        ACK(cudaStreamSynchronize(st));
        // host_red holds the sums of 8 iterations; the last one dominates a
        // contracting sequence, so the test is conservative
        conv = host_red[0] <= tol * host_red[1];
        if (!std::isfinite(host_red[0]))
          return jko::handle_error(h, JKO_ERR_NUMERIC, "adjoint iterates are not finite");
      }
    }
    if (adj_iters) adj_iters[t] = k;
    // gradients of this step
    k_rs<T, EK><<<G, NT, 0, st>>>(P, s, lam, u, N);
    ACK(cudaGetLastError());
    ACK(xi_apply<T>(h, u, v, st));
    k_final<T, EK><<<G, NT, 0, st>>>(P, s, lam, qbar0, v, invY, g,
                                      wbar_dev ? wbar_dev : scratch_w, N);
    ACK(cudaGetLastError());
  }
  if (grad_p0) ACK(cudaMemcpyAsync(grad_p0, g, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
  ACK(cudaStreamSynchronize(st));
  return JKO_OK;
}

// ---- the Wasserstein attraction (Sec. 5.2), congestion/potential energy ----
// The step's fixed point over both couplings: Y_m = xi a_m, b_m = t_m / Y_m
// (t_1 = q, t_2 = r), s_m = xi b_m, p = min(E g, kappa) with the geometric mean
// g = s_1^{th1} s_2^{th2} (th1 = 1/(1+tau), th2 = tau/(1+tau), E = e^{-sigma' w},
// sigma' = sigma/(1+tau): Eq. prox-psi-attraction), a_m = p / s_m.  Per cell,
// with p unclamped: da_1/ds_1 = (th1 - 1) a_1/s_1, da_1/ds_2 = th2 a_1/s_2,
// da_2/ds_1 = th1 a_2/s_1, da_2/ds_2 = (th2 - 1) a_2/s_2, da_m/dw = -sigma' a_m;
// clamped (E g > kappa): a_m = kappa/s_m, da_m/ds_m = -a_m/s_m, no w term.
// The adjoint solve runs over both channels: u = J^T lambda cell by cell, then
// lambda_m = abar_m - xi(D_m xi u_m); p = a_1 s_1 gives the direct terms of
// channel 1 as in the single-coupling step, and q only enters through b_1.
template <typename T>
__device__ __forceinline__ bool att_jacobian(const jko::ProxArgs<T>& P, long long i, T s1, T s2,
                                             T th1, T th2, T (&J)[4], T& a1, T& a2) {
  J[0] = J[1] = J[2] = J[3] = T(0);
  a1 = a2 = T(0);
  if ((P.mask != nullptr && P.mask[i]) || !(s1 > T(0) && s2 > T(0))) return false;
  const T g = jko::dev_exp<T>(th1 * jko::dev_log<T>(s1) + th2 * jko::dev_log<T>(s2));
  const T e = P.E[i];
  if (P.has_kappa) {
    const T kap = P.kappa ? P.kappa[i] : P.kappa_s;
    if (e * g > kap) {
      a1 = kap / s1;
      a2 = kap / s2;
      J[0] = -a1 / s1;
      J[3] = -a2 / s2;
      return false;
    }
  }
  const T pm = e * g;
  a1 = pm / s1;
  a2 = pm / s2;
  J[0] = (th1 - T(1)) * a1 / s1;   // da_1/ds_1
  J[1] = th2 * a1 / s2;            // da_1/ds_2
  J[2] = th1 * a2 / s1;            // da_2/ds_1
  J[3] = (th2 - T(1)) * a2 / s2;   // da_2/ds_2
  return true;
}

// u = J^T lambda
template <typename T>
__global__ void k_att_u(jko::ProxArgs<T> P, const T* s1, const T* s2, const T* l1, const T* l2,
                        T* u1, T* u2, T th1, T th2, long long n) {
  GS(i, n) {
    T J[4], a1, a2;
    att_jacobian<T>(P, i, s1[i], s2[i], th1, th2, J, a1, a2);
    u1[i] = J[0] * l1[i] + J[2] * l2[i];
    u2[i] = J[1] * l1[i] + J[3] * l2[i];
  }
}

// g = qbar0 + v invY ;  wbar += -sigma' (a_1 lambda_1 + a_2 lambda_2) where unclamped
template <typename T>
__global__ void k_att_final(jko::ProxArgs<T> P, const T* s1, const T* s2, const T* l1,
                            const T* l2, const T* qbar0, const T* v, const T* invY, T* g, T* wbar,
                            T th1, T th2, T sigma_f, long long n) {
  GS(i, n) {
    T J[4], a1, a2;
    const bool free_ = att_jacobian<T>(P, i, s1[i], s2[i], th1, th2, J, a1, a2);
    g[i] = qbar0[i] + v[i] * invY[i];
    if (free_) wbar[i] += -sigma_f * (a1 * l1[i] + a2 * l2[i]);
  }
}

template <typename T>
jko_status backward_attraction(jko_handle* h, const T* grad_final, T* grad_p0, T* grad_w,
                               int* adj_iters) {
  cudaStream_t st = h->stream;
  const long long N = h->N;
  if (!h->adj2) ACK(cudaMalloc(&h->adj2, sizeof(T) * N * 18));
  if (!h->adj_red) ACK(cudaMalloc((void**)&h->adj_red, sizeof(double) * 4));
  T* W = (T*)h->adj2;
  T *Y1 = W, *Y2 = W + N, *b1 = W + 2 * N, *b2 = W + 3 * N, *s1 = W + 4 * N, *s2 = W + 5 * N,
    *iY1 = W + 6 * N, *iY2 = W + 7 * N, *g = W + 8 * N, *gt = W + 9 * N, *u1 = W + 10 * N,
    *u2 = W + 11 * N, *v1 = W + 12 * N, *v2 = W + 13 * N, *l1 = W + 14 * N, *l2 = W + 15 * N,
    *ab1 = W + 16 * N, *ab2 = W + 17 * N;
  const T th1 = T(1.0 / (1.0 + h->prm.tau)), th2 = T(h->prm.tau / (1.0 + h->prm.tau));
  const T sigma_f = T(h->prm.tau / h->prm.gamma / (1.0 + h->prm.tau));
  jko::ProxArgs<T> P = jko::prox_args<T>(h);
  ACK(cudaMemcpyAsync(h->ctrl, h->ctrl_init, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
  ACK(cudaMemcpyAsync(g, grad_final, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
  T* wbar = grad_w ? grad_w : v2;   // v2 is rewritten before it is read again
  if (grad_w) ACK(cudaMemsetAsync(grad_w, 0, sizeof(T) * N, st));
  const int budget = std::max(16, 10 * h->prm.max_iter);
  const double tol = std::max(h->prm.tol, h->fp64 ? 1e-15 : 1e-7);
  const int G = grid_for(N);
  const T* r = (const T*)h->tgt;
  for (int t = h->tape_steps - 1; t >= 0; --t) {
    const T* q = (const T*)h->tape + (size_t)(3 * t) * N;
    const T* a1 = q + N;
    const T* a2 = q + 2 * N;
    const double m = h->tape_mass[t];
    ACK(xi_apply<T>(h, a1, Y1, st));
    ACK(xi_apply<T>(h, a2, Y2, st));
    k_b_invY<T><<<G, NT, 0, st>>>(q, Y1, b1, iY1, N);
    k_b_invY<T><<<G, NT, 0, st>>>(r, Y2, b2, iY2, N);
    ACK(cudaGetLastError());
    ACK(xi_apply<T>(h, b1, s1, st));
    ACK(xi_apply<T>(h, b2, s2, st));
    // the renormalisation's adjoint and the direct terms of p = a_1 s_1
    ACK(cudaMemsetAsync(h->adj_red, 0, sizeof(double) * 4, st));
    k_dot3<T><<<G, NT, 0, st>>>(g, a1, s1, h->adj_red, N);
    k_renorm<T><<<G, NT, 0, st>>>(g, a1, h->adj_red, m, h->prm.renormalize, gt, u1, N);
    ACK(cudaGetLastError());
    ACK(xi_apply<T>(h, u1, v1, st));                 // v1 = xi(a_1 gt)
    k_mul<T><<<G, NT, 0, st>>>(b1, iY1, b1, N);      // b1 <- D_1
    k_mul<T><<<G, NT, 0, st>>>(b2, iY2, b2, N);      // b2 <- D_2
    k_mul<T><<<G, NT, 0, st>>>(b1, v1, u1, N);
    ACK(cudaGetLastError());
    ACK(xi_apply<T>(h, u1, ab1, st));                // xi(D_1 v1)
    k_abar<T><<<G, NT, 0, st>>>(s1, gt, ab1, v1, iY1, ab1, gt, N);   // abar_1; qbar0 in gt
    ACK(cudaGetLastError());
    ACK(cudaMemsetAsync(ab2, 0, sizeof(T) * N, st));
    ACK(cudaMemcpyAsync(l1, ab1, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
    ACK(cudaMemsetAsync(l2, 0, sizeof(T) * N, st));
    int k = 0;
    bool conv = false;
    double host_red[4];
    for (; k < budget && !conv; ++k) {
      if ((k & 7) == 0) ACK(cudaMemsetAsync(h->adj_red, 0, sizeof(double) * 4, st));
      k_att_u<T><<<G, NT, 0, st>>>(P, s1, s2, l1, l2, u1, u2, th1, th2, N);
      ACK(cudaGetLastError());
      ACK(xi_apply<T>(h, u1, v1, st));
      ACK(xi_apply<T>(h, u2, v2, st));
      k_mul<T><<<G, NT, 0, st>>>(b1, v1, u1, N);
      k_mul<T><<<G, NT, 0, st>>>(b2, v2, u2, N);
      ACK(cudaGetLastError());
      ACK(xi_apply<T>(h, u1, v1, st));
      ACK(xi_apply<T>(h, u2, v2, st));
      k_lambda<T><<<G, NT, 0, st>>>(ab1, v1, l1, h->adj_red, h->adj_red + 1, N);
      k_lambda<T><<<G, NT, 0, st>>>(ab2, v2, l2, h->adj_red, h->adj_red + 1, N);
      ACK(cudaGetLastError());
      if ((k & 7) == 7) {
        ACK(cudaMemcpyAsync(host_red, h->adj_red, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
        ACK(cudaStreamSynchronize(st));
        conv = host_red[0] <= tol * host_red[1];
        if (!std::isfinite(host_red[0]))
          return jko::handle_error(h, JKO_ERR_NUMERIC, "adjoint iterates are not finite");
      }
    }
    if (adj_iters) adj_iters[t] = k;
    // gradients of this step: q enters through b_1 only (r is fixed)
    k_att_u<T><<<G, NT, 0, st>>>(P, s1, s2, l1, l2, u1, u2, th1, th2, N);
    ACK(cudaGetLastError());
    ACK(xi_apply<T>(h, u1, v1, st));
    if (!grad_w) ACK(cudaMemsetAsync(v2, 0, sizeof(T) * N, st));
    k_att_final<T><<<G, NT, 0, st>>>(P, s1, s2, l1, l2, gt, v1, iY1, g, wbar, th1, th2, sigma_f,
                                     N);
    ACK(cudaGetLastError());
  }
  if (grad_p0) ACK(cudaMemcpyAsync(grad_p0, g, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
  ACK(cudaStreamSynchronize(st));
  return JKO_OK;
}

// ---- two species coupled through the congestion of their sum (Sec. 5.3) ----
// Fixed point over both couplings: b_m = q_m / xi a_m, s_m = xi b_m, the joint
// prox t = s_1 E_1 + s_2 E_2 (E_m = e^{-sigma w_m}), f = min(1, kappa / t),
// p_m = s_m E_m f, a_m = E_m f.  Unclamped (t <= kappa) a_m = E_m does not
// depend on s; clamped, da_m/ds_n = -a_m E_n / t, so (J^T lambda)_n =
// -E_n (a_1 lambda_1 + a_2 lambda_2) / t.  The potential w = w_1 of the first
// species: da_1/dw = -sigma a_1 (1 - s_1 E_1 / t 1[clamped]), da_2/dw =
// sigma a_2 s_1 E_1 / t 1[clamped].  Both species carry direct terms (p_m =
// a_m s_m) and their own q_m.
template <typename T>
__device__ __forceinline__ bool sp_clamped(const T* E1, const T* E2, long long i, T s1, T s2,
                                          T kappa, int has_kappa, T& t, T& a1, T& a2) {
  const T e1 = E1[i], e2 = E2 ? E2[i] : T(1);
  t = s1 * e1 + s2 * e2;
  const bool c = has_kappa && t > kappa;
  const T f = c ? kappa / t : T(1);
  a1 = e1 * f;
  a2 = e2 * f;
  return c;
}

template <typename T>
__global__ void k_sp_u(const T* E1, const T* E2, const T* s1, const T* s2, const T* l1,
                       const T* l2, T* u1, T* u2, T kappa, int has_kappa, long long n) {
  GS(i, n) {
    T t, a1, a2;
    if (sp_clamped<T>(E1, E2, i, s1[i], s2[i], kappa, has_kappa, t, a1, a2)) {
      const T c = -(a1 * l1[i] + a2 * l2[i]) / t;
      u1[i] = E1[i] * c;
      u2[i] = (E2 ? E2[i] : T(1)) * c;
    } else {
      u1[i] = T(0);
      u2[i] = T(0);
    }
  }
}

template <typename T>
__global__ void k_sp_final(const T* E1, const T* E2, const T* s1, const T* s2, const T* l1,
                           const T* l2, const T* qb1, const T* qb2, const T* v1, const T* v2,
                           const T* iY1, const T* iY2, T* g1, T* g2, T* wbar, T sigma, T kappa,
                           int has_kappa, long long n) {
  GS(i, n) {
    T t, a1, a2;
    const bool c = sp_clamped<T>(E1, E2, i, s1[i], s2[i], kappa, has_kappa, t, a1, a2);
    g1[i] = qb1[i] + v1[i] * iY1[i];
    g2[i] = qb2[i] + v2[i] * iY2[i];
    const T share = c ? s1[i] * E1[i] / t : T(0);   // the first species' part of t
    wbar[i] += -sigma * a1 * (T(1) - share) * l1[i] + sigma * a2 * share * l2[i];
  }
}

template <typename T>
jko_status backward_species(jko_handle* h, const T* grad_final, T* grad_p0, T* grad_w,
                            int* adj_iters) {
  cudaStream_t st = h->stream;
  const long long N = h->N;
  if (!h->adj2) ACK(cudaMalloc(&h->adj2, sizeof(T) * N * 20));
  if (!h->adj_red) ACK(cudaMalloc((void**)&h->adj_red, sizeof(double) * 4));
  T* W = (T*)h->adj2;
  T *Y1 = W, *Y2 = W + N, *b1 = W + 2 * N, *b2 = W + 3 * N, *s1 = W + 4 * N, *s2 = W + 5 * N,
    *iY1 = W + 6 * N, *iY2 = W + 7 * N, *g = W + 8 * N /* 2N */, *gt = W + 10 * N /* 2N */,
    *u1 = W + 12 * N, *u2 = W + 13 * N, *v1 = W + 14 * N, *v2 = W + 15 * N, *l1 = W + 16 * N,
    *l2 = W + 17 * N, *ab1 = W + 18 * N, *ab2 = W + 19 * N;
  T *g1 = g, *g2 = g + N, *gt1 = gt, *gt2 = gt + N;
  const T sigma = T(h->prm.tau / h->prm.gamma), kappa = T(h->kappa_s);
  const T* E1 = (const T*)h->E;
  const T* E2 = (const T*)h->E2;
  ACK(cudaMemcpyAsync(h->ctrl, h->ctrl_init, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
  ACK(cudaMemcpyAsync(g, grad_final, sizeof(T) * 2 * N, cudaMemcpyDeviceToDevice, st));
  T* wbar = grad_w;
  if (grad_w) ACK(cudaMemsetAsync(grad_w, 0, sizeof(T) * N, st));
  const int budget = std::max(16, 10 * h->prm.max_iter);
  const double tol = std::max(h->prm.tol, h->fp64 ? 1e-15 : 1e-7);
  const int G = grid_for(N);
  for (int t = h->tape_steps - 1; t >= 0; --t) {
    const T* q1 = (const T*)h->tape + (size_t)(4 * t) * N;
    const T* q2 = q1 + N;
    const T* a1 = q1 + 2 * N;
    const T* a2 = q1 + 3 * N;
    const double m = h->tape_mass[t];
    ACK(xi_apply<T>(h, a1, Y1, st));
    ACK(xi_apply<T>(h, a2, Y2, st));
    k_b_invY<T><<<G, NT, 0, st>>>(q1, Y1, b1, iY1, N);
    k_b_invY<T><<<G, NT, 0, st>>>(q2, Y2, b2, iY2, N);
    ACK(cudaGetLastError());
    ACK(xi_apply<T>(h, b1, s1, st));
    ACK(xi_apply<T>(h, b2, s2, st));
    // the renormalisation's adjoint over both species, then the direct terms of p_m = a_m s_m
    ACK(cudaMemsetAsync(h->adj_red, 0, sizeof(double) * 4, st));
    k_dot3<T><<<G, NT, 0, st>>>(g1, a1, s1, h->adj_red, N);
    k_dot3<T><<<G, NT, 0, st>>>(g2, a2, s2, h->adj_red, N);
    k_renorm<T><<<G, NT, 0, st>>>(g1, a1, h->adj_red, m, h->prm.renormalize, gt1, u1, N);
    k_renorm<T><<<G, NT, 0, st>>>(g2, a2, h->adj_red, m, h->prm.renormalize, gt2, u2, N);
    ACK(cudaGetLastError());
    ACK(xi_apply<T>(h, u1, v1, st));                 // v_m = xi(a_m gt_m)
    ACK(xi_apply<T>(h, u2, v2, st));
    k_mul<T><<<G, NT, 0, st>>>(b1, iY1, b1, N);      // b_m <- D_m
    k_mul<T><<<G, NT, 0, st>>>(b2, iY2, b2, N);
    k_mul<T><<<G, NT, 0, st>>>(b1, v1, u1, N);
    k_mul<T><<<G, NT, 0, st>>>(b2, v2, u2, N);
    ACK(cudaGetLastError());
    ACK(xi_apply<T>(h, u1, ab1, st));
    ACK(xi_apply<T>(h, u2, ab2, st));
    k_abar<T><<<G, NT, 0, st>>>(s1, gt1, ab1, v1, iY1, ab1, gt1, N);   // abar_1; qbar0_1 in gt1
    k_abar<T><<<G, NT, 0, st>>>(s2, gt2, ab2, v2, iY2, ab2, gt2, N);
    ACK(cudaGetLastError());
    ACK(cudaMemcpyAsync(l1, ab1, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
    ACK(cudaMemcpyAsync(l2, ab2, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
    int k = 0;
    bool conv = false;
    double host_red[4];
    for (; k < budget && !conv; ++k) {
      if ((k & 7) == 0) ACK(cudaMemsetAsync(h->adj_red, 0, sizeof(double) * 4, st));
      k_sp_u<T><<<G, NT, 0, st>>>(E1, E2, s1, s2, l1, l2, u1, u2, kappa, h->has_kappa, N);
      ACK(cudaGetLastError());
      ACK(xi_apply<T>(h, u1, v1, st));
      ACK(xi_apply<T>(h, u2, v2, st));
      k_mul<T><<<G, NT, 0, st>>>(b1, v1, u1, N);
      k_mul<T><<<G, NT, 0, st>>>(b2, v2, u2, N);
      ACK(cudaGetLastError());
      ACK(xi_apply<T>(h, u1, v1, st));
      ACK(xi_apply<T>(h, u2, v2, st));
      k_lambda<T><<<G, NT, 0, st>>>(ab1, v1, l1, h->adj_red, h->adj_red + 1, N);
      k_lambda<T><<<G, NT, 0, st>>>(ab2, v2, l2, h->adj_red, h->adj_red + 1, N);
      ACK(cudaGetLastError());
      if ((k & 7) == 7) {
        ACK(cudaMemcpyAsync(host_red, h->adj_red, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
        ACK(cudaStreamSynchronize(st));
        conv = host_red[0] <= tol * host_red[1];
        if (!std::isfinite(host_red[0]))
          return jko::handle_error(h, JKO_ERR_NUMERIC, "adjoint iterates are not finite");
      }
    }
    if (adj_iters) adj_iters[t] = k;
    k_sp_u<T><<<G, NT, 0, st>>>(E1, E2, s1, s2, l1, l2, u1, u2, kappa, h->has_kappa, N);
    ACK(cudaGetLastError());
    ACK(xi_apply<T>(h, u1, v1, st));
    ACK(xi_apply<T>(h, u2, v2, st));
    T* wacc = wbar;
    if (!grad_w) wacc = ab2;   // abar_2 is not needed any more: a scratch accumulator
    k_sp_final<T><<<G, NT, 0, st>>>(E1, E2, s1, s2, l1, l2, gt1, gt2, v1, v2, iY1, iY2, g1, g2,
                                    wacc, sigma, kappa, h->has_kappa, N);
    ACK(cudaGetLastError());
  }
  if (grad_p0) ACK(cudaMemcpyAsync(grad_p0, g, sizeof(T) * 2 * N, cudaMemcpyDeviceToDevice, st));
  ACK(cudaStreamSynchronize(st));
  return JKO_OK;
}

template <typename T>
jko_status backward_dispatch(jko_handle* h, const void* gf, void* gp, void* gw, int* it) {
  if (h->attract) return backward_attraction<T>(h, (const T*)gf, (T*)gp, (T*)gw, it);
  if (h->species == 2) return backward_species<T>(h, (const T*)gf, (T*)gp, (T*)gw, it);
  switch (h->ek) {
    case jko::EK_CROWD:
      return backward_t<T, jko::EK_CROWD>(h, (const T*)gf, (T*)gp, (T*)gw, it);
    case jko::EK_ENTROPY:
      return backward_t<T, jko::EK_ENTROPY>(h, (const T*)gf, (T*)gp, (T*)gw, it);
    default:
      return backward_t<T, jko::EK_POWER>(h, (const T*)gf, (T*)gp, (T*)gw, it);
  }
}

template <typename T, typename W>
__global__ void k_set_potential(const W* w, T* E, T* sw, double sigma, long long n) {
  GS(i, n) {
    const double wi = (double)w[i];
    if (E) E[i] = (T)exp(-sigma * wi);
    if (sw) sw[i] = (T)(sigma * wi);
  }
}

// sigma of the energy fields: tau / gamma, over (1 + tau) for the attraction's
// prox of h (Eq. prox-psi-attraction)
double field_sigma(const jko_handle* h) {
  return h->prm.tau / h->prm.gamma / (h->attract ? 1.0 + h->prm.tau : 1.0);
}

jko_status check_set_potential(jko_handle* h, const void* w) {
  if (!h || !w) return jko::handle_error(h, JKO_ERR_INVALID_ARG, "NULL handle or w");
  if (h->pair_alpha > 0)
    return jko::handle_error(h, JKO_ERR_UNSUPPORTED,
                             "the potentials of a pairwise-attraction handle are fixed at "
                             "creation");
  if (h->tc && jko::tc_absorbed(h->tc))
    return jko::handle_error(h, JKO_ERR_UNSUPPORTED,
                             "the potential is absorbed into the Gibbs factors of this handle");
  if (h->ek != jko::EK_CROWD && !h->sw)
    return jko::handle_error(h, JKO_ERR_INVALID_ARG,
                             "the handle was created without a potential (w = NULL)");
  return JKO_OK;
}

}  // namespace

extern "C" {

jko_status jko_set_potential(jko_handle* h, const double* w_host) {
  if (jko_status st = check_set_potential(h, w_host)) return st;
  const long long N = h->N;
  double lo = INFINITY, hi = -INFINITY;
  for (long long i = 0; i < N; ++i) {
    if (!std::isfinite(w_host[i])) return jko::handle_error(h, JKO_ERR_INVALID_ARG, "w must be finite");
    lo = std::min(lo, w_host[i]);
    hi = std::max(hi, w_host[i]);
  }
  // the FFT application's range rule of jko_create: e^{sigma (max w - min w)}
  // within e^8 (FP32) / e^24 (FP64)
  if (h->fft && h->prm.tau / h->prm.gamma * (hi - lo) > (h->fp64 ? 24.0 : 8.0))
    return jko::handle_error(h, JKO_ERR_UNSUPPORTED,
                             "the FFT application needs the potential's scalings within e^8 "
                             "(FP32) / e^24 (FP64)");
  double* wd = nullptr;
  ACK(cudaMalloc((void**)&wd, sizeof(double) * N));
  cudaError_t e = cudaMemcpyAsync(wd, w_host, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream);
  const double sigma = field_sigma(h);
  if (e == cudaSuccess) {
    if (h->fp64)
      k_set_potential<double, double><<<grid_for(N), NT, 0, h->stream>>>(wd, (double*)h->E, (double*)h->sw, sigma, N);
    else
      k_set_potential<float, double><<<grid_for(N), NT, 0, h->stream>>>(wd, (float*)h->E, (float*)h->sw, sigma, N);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(wd);
  ACK(e);
  return JKO_OK;
}

jko_status jko_set_potential_device(jko_handle* h, const void* w_dev) {
  if (jko_status st = check_set_potential(h, w_dev)) return st;
  const long long N = h->N;
  const double sigma = field_sigma(h);
  if (h->fp64)
    k_set_potential<double, double><<<grid_for(N), NT, 0, h->stream>>>(
        (const double*)w_dev, (double*)h->E, (double*)h->sw, sigma, N);
  else
    k_set_potential<float, float><<<grid_for(N), NT, 0, h->stream>>>(
        (const float*)w_dev, (float*)h->E, (float*)h->sw, sigma, N);
  ACK(cudaGetLastError());
  return JKO_OK;
}

jko_status jko_flow_record(jko_handle* h, const void* p0_dev, int n_steps, void* p_final_dev,
                           jko_step_info* infos) {
  if (!h || !p0_dev || n_steps < 1) return jko::handle_error(h, JKO_ERR_INVALID_ARG, "bad arguments");
  if (h->tc) return jko::handle_error(h, JKO_ERR_UNSUPPORTED, "recording needs a JKO_FP32 or JKO_FP64 handle");
  if (h->binary)
    return jko::handle_error(h, JKO_ERR_UNSUPPORTED,
                             "the binary congestion prox is discontinuous: no adjoint");
  if (h->attract && h->ek != jko::EK_CROWD)
    return jko::handle_error(h, JKO_ERR_UNSUPPORTED,
                             "the attraction's adjoint covers the congestion / potential energy");
  // Its Jacobian a_m / s_m grows like s_m^{-1 - tau/(1+tau)} where the blur
  // s_m = xi b_m of one coupling is tiny near the other's support, and the
  // band-limited FP32 factors that would cancel it are exact zeros there: the
  // FP32 adjoint overflows (measured: gradients off by 1e37), the FP64 one
  // matches the oracle.
  if (h->attract && !h->fp64)
    return jko::handle_error(h, JKO_ERR_UNSUPPORTED,
                             "the attraction's adjoint needs a JKO_FP64 handle (its Jacobian "
                             "a_m / s_m leaves the FP32 range)");
  if (h->pair_alpha > 0)
    return jko::handle_error(h, JKO_ERR_UNSUPPORTED, "no adjoint for the pairwise attraction");
  const size_t es = h->es, N = (size_t)h->N, ns = (size_t)h->ns;
  // per step: q_t (both species: 2 N) and the final scalings a_t (a_2 of the
  // second coupling or species too)
  const size_t per = h->species == 2 ? 4 : (h->attract ? 3 : 2);
  if (h->tape_cap < n_steps) {
    if (h->tape) cudaFree(h->tape);
    h->tape = nullptr;
    h->tape_cap = 0;
    ACK(cudaMalloc(&h->tape, es * N * per * n_steps));
    h->tape_cap = n_steps;
  }
  h->tape_steps = 0;
  h->tape_mass.assign(n_steps, 1.0);
  cudaStream_t st = h->stream;
  int worst = JKO_OK;
  const void* q = p0_dev;
  for (int t = 0; t < n_steps; ++t) {
    char* slot = (char*)h->tape + es * N * per * t;
    if (q != (const void*)slot)  // from step 1 on the previous step wrote its output here
      ACK(cudaMemcpyAsync(slot, q, es * ns, cudaMemcpyDeviceToDevice, st));
    jko_step_info info{};
    void* dst = (t + 1 < n_steps) ? (void*)((char*)h->tape + es * N * per * (t + 1)) : p_final_dev;
    if (!dst) {
      if (!h->stage_out) ACK(cudaMalloc(&h->stage_out, es * ns));
      dst = h->stage_out;
    }
    jko_status s = jko::step_internal(h, slot, dst, &info, t == 0);
    if (s == JKO_ERR_INVALID_ARG || s == JKO_ERR_CUDA || s == JKO_ERR_OOM || s == JKO_ERR_TIMEOUT)
      return s;
    if (infos) infos[t] = info;
    if (s == JKO_ERR_NUMERIC) worst = JKO_ERR_NUMERIC;
    else if (s == JKO_NOT_CONVERGED && worst == JKO_OK) worst = JKO_NOT_CONVERGED;
    ACK(cudaMemcpyAsync(slot + es * ns, h->a, es * N, cudaMemcpyDeviceToDevice, st));
    if (h->attract || h->species == 2)
      ACK(cudaMemcpyAsync(slot + es * (ns + N), h->a2, es * N, cudaMemcpyDeviceToDevice, st));
    h->tape_mass[t] = info.mass;
    h->tape_steps = t + 1;
    q = dst;
  }
  ACK(cudaStreamSynchronize(st));
  return (jko_status)worst;
}

jko_status jko_flow_backward(jko_handle* h, const void* grad_final_dev, void* grad_p0_dev,
                             void* grad_w_dev, int* adj_iters) {
  if (!h || !grad_final_dev) return jko::handle_error(h, JKO_ERR_INVALID_ARG, "bad arguments");
  if (h->tape_steps < 1) return jko::handle_error(h, JKO_ERR_INVALID_ARG, "no recorded flow");
  if (grad_w_dev && h->ek != jko::EK_CROWD && !h->sw)
    return jko::handle_error(h, JKO_ERR_INVALID_ARG, "the energy has no potential to differentiate");
  return h->fp64 ? backward_dispatch<double>(h, grad_final_dev, grad_p0_dev, grad_w_dev, adj_iters)
                 : backward_dispatch<float>(h, grad_final_dev, grad_p0_dev, grad_w_dev, adj_iters);
}

}  // extern "C"
