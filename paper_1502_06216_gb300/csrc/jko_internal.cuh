// jko_internal.cuh -- device-side shared pieces of the JKO path: the control
// block that carries the stopping decision between kernels, reductions, and
// the pointwise KL proximal maps evaluated in ratio form a = Prox(s)/s.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace jko {

// Stop states written into Ctrl::done.
// STALLED: the residual set no new minimum over `stall` pairs in a row (the
// iterates have reached the rounding floor of their arithmetic).
enum : int { RUNNING = 0, CONVERGED = 1, MAX_ITER = 2, NONFINITE = 3, STALLED = 4 };

// Control block in device memory, one per handle.  Kernels of the scaling loop
// read `done` when they start and return at once when it is set, so a fixed
// chunk of launched iterations becomes a no-op after the stop.  Decisions are
// taken by the last block of a kernel to finish (atomic arrival counter), so no
// kernel ever waits on another block.
struct Ctrl {
  int it;                 // (odd, even) pairs completed in this step
  int done;               // RUNNING / CONVERGED / MAX_ITER / NONFINITE
  int nonfinite;          // set when an epilogue meets NaN or Inf
  int max_iter;           // copy of the step budget
  unsigned int bar_base;  // grid barriers the persistent loop kernel completed this step
  unsigned int bar_spare;
  unsigned int arrive_f;  // arrival counter of the finalisation kernel
  unsigned int arrive_v;  // arrival counter of the validation kernel
  double tol;             // L1 residual tolerance
  double res_acc;         // residual accumulator of the running pass
  double res_last;        // residual of the last completed pair
  double mass;            // sum p (finalisation)
  unsigned long long maxpk_bits;  // max p/kappa as ordered bits (p >= 0)
  // validation of the step input q
  double q_sum;
  unsigned long long q_neg;       // count of q < 0
  unsigned long long q_bad;       // count of non-finite q
  unsigned long long q_over;      // count of q > kappa (1 + 1e-2)
  unsigned long long q_masked;    // count of q != 0 on the mask
  // grid barrier of the persistent loop kernel (all 0 at the start of a step)
  unsigned long long bar_cnt;     // arrivals, G per barrier
  unsigned int bar_flag[4];       // [b % 3]: some CTA met NaN/Inf or gave up a wait before barrier b
  // stall rule: pairs without a new minimum of the residual before the step
  // stops (0 = off); the smallest residual so far and the pairs since, kept
  // twice by pair parity (the decision of pair k reads slot k & 1 and writes
  // the other), so that every block of a deciding kernel reads the state the
  // previous decision left while one block writes the next
  int stall;
  int since[2];
  int stall_spare;
  double best[2];
};

// The stall rule for the decision after pair `it` (>= 1) with residual
// `total`: true when the residual has set no new minimum for ctrl->stall
// pairs.  `write`: this thread records the new state.
__device__ __forceinline__ bool stall_rule(Ctrl* ctrl, int it, double total, bool write) {
  const int n = *(volatile int*)&ctrl->stall;
  if (n <= 0 || it < 1) return false;
  const int rd = it & 1;
  double best = it == 1 ? INFINITY : __ldcg(&ctrl->best[rd]);
  int since = it == 1 ? 0 : *(volatile int*)&ctrl->since[rd];
  if (total < best) {
    best = total;
    since = 0;
  } else {
    ++since;
  }
  if (write) {
    ctrl->best[rd ^ 1] = best;
    ctrl->since[rd ^ 1] = since;
  }
  return since >= n;
}

// A scaling stored as the operand of the TF32 tensor-core passes (rnd = 1):
// rounded to tf32 (nearest, ties away), as the tensor-core epilogues store it.
template <typename T>
__device__ __forceinline__ T op_round(T x, int) { return x; }
template <>
__device__ __forceinline__ float op_round<float>(float x, int rnd) {
  if (!rnd) return x;
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// ---- grid-wide barrier of the persistent kernels (tc_loop.cu, heat.cu) ----
__device__ __forceinline__ unsigned long long ld_acquire_gpu_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
constexpr unsigned kGridSpinLimit = 1u << 24;   // polls of one barrier before giving up

// Grid-wide barrier number b (1, 2, ... within the step) of the G
// co-resident blocks, called by one thread per block after the block's
// writes: one release-add on a 64-bit arrival counter in Ctrl that never
// resets within a step (barrier b is complete at G b arrivals) and a bounded
// acquire poll.  `flag`: this block met NaN/Inf or gave up a wait; it is
// recorded in slot b % 3, final for every block once barrier b is complete.
// False if the poll gave up.
__device__ __forceinline__ bool grid_barrier(Ctrl* ctrl, unsigned G, unsigned b, bool flag) {
  if (flag) atomicOr(&ctrl->bar_flag[b % 3], 1u);
  red_release_add_u64(&ctrl->bar_cnt, 1ull);
  const unsigned long long target = (unsigned long long)G * b;
  for (unsigned i = 0; i < kGridSpinLimit; ++i)
    if (ld_acquire_gpu_u64(&ctrl->bar_cnt) >= target) return true;
  return false;
}

// ---- stop protocol of the scaling loop ----
// The b-update pass writes one residual partial per block (plain stores, one
// slot each).  The pass that follows it (along x of xi b) reduces the partials
// in a fixed order at its start, so every block reaches the same decision:
// converged (residual <= tol, Sec. 3.4), budget exhausted, or non-finite;
// block 0 records it in Ctrl.  The prox pass advances the pair counter from
// block 0.  Every other pass only checks the recorded state.  No block waits
// for another and no address is contended, except the rare non-finite flag.
// Must be called by all threads of the block; returns true when the kernel
// has to return at once.
__device__ __forceinline__ bool stop_gate(Ctrl* ctrl, const double* part, int nparts,
                                          bool decide, int* s_it) {
  __shared__ int s_state[2];
  __shared__ double s_total;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const bool first = tid == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0;
  if (tid == 0) {
    s_state[0] = *(volatile int*)&ctrl->done;
    s_state[1] = *(volatile int*)&ctrl->nonfinite;
    *s_it = ctrl->it;
  }
  if (decide && tid < 32) {
    double v = 0.0;
    for (int i = tid; i < nparts; i += 32) v += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (tid == 0) s_total = v;
  }
  __syncthreads();
  if (s_state[0] != RUNNING) return true;
  if (s_state[1] != 0) {
    if (first) ctrl->done = NONFINITE;
    return true;
  }
  if (!decide) return false;
  const double total = s_total;
  const int it = *s_it;
  int d = RUNNING;
  if (it > 0 && !isfinite(total)) d = NONFINITE;
  else if (it > 0 && total <= ctrl->tol) d = CONVERGED;
  else if (it >= ctrl->max_iter) d = MAX_ITER;
  else if (stall_rule(ctrl, it, total, first)) d = STALLED;
  if (first) {
    if (it > 0) ctrl->res_last = total;
    if (d != RUNNING) ctrl->done = d;
  }
  return d != RUNNING;
}

// Energy kinds of the proximal epilogue (compile-time).
enum : int { EK_CROWD = 0, EK_ENTROPY = 1, EK_POWER = 2 };

// Per-cell energy constants, precomputed at create time in working precision T.
template <typename T>
struct ProxArgs {
  const T* E;          // e^{-sigma w} (crowd) ; unused otherwise
  const T* sw;         // sigma * w (entropy, power), may be NULL (= 0)
  const T* c;          // entropy: sigma*alpha ; power: beta = sigma*alpha*m/(m-1)
  const T* kappa;      // per-cell kappa, or NULL
  T kappa_s;           // scalar kappa (+inf = none), used when kappa == NULL
  const uint8_t* mask; // 1 = obstacle, or NULL
  T m1;                // m - 1 (power)
  int newton;          // Newton steps (power)
  int has_kappa;       // 1 if any congestion bound is finite
  T sigma;             // tau / gamma (derivatives with respect to w)
  // generalised entropies with per-cell exponents (Eq. defn-gen-entropies,
  // power kind): m_i - 1 per cell, with c = sigma alpha_i m_i; NULL = scalar m
  const T* m1f = nullptr;
  // 1: the congestion is the non-convex iota_{{0,kappa}} (Eq. dfn-congestion-noncvx)
  int binary = 0;
};

template <typename T> __device__ __forceinline__ T dev_exp(T x);
template <> __device__ __forceinline__ float dev_exp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double dev_exp<double>(double x) { return exp(x); }
template <typename T> __device__ __forceinline__ T dev_log(T x);
template <> __device__ __forceinline__ float dev_log<float>(float x) { return logf(x); }
template <> __device__ __forceinline__ double dev_log<double>(double x) { return log(x); }
template <typename T> __device__ __forceinline__ T dev_expm1(T x);
template <> __device__ __forceinline__ float dev_expm1<float>(float x) { return expm1f(x); }
template <> __device__ __forceinline__ double dev_expm1<double>(double x) { return expm1(x); }

template <typename T> __device__ __forceinline__ bool dev_finite(T x) { return isfinite(x); }

// x / y for the scaling updates.  In FP32 it is x times the correctly rounded
// reciprocal of y (within about one ulp of the quotient): the IEEE division's
// slow path, taken for the extreme magnitudes the scalings reach, costs more
// than the rest of the epilogue.  FP64 keeps the true division.
template <typename T> __device__ __forceinline__ T ratio_div(T x, T y);
template <> __device__ __forceinline__ float ratio_div<float>(float x, float y) {
  return x * __frcp_rn(y);
}
template <> __device__ __forceinline__ double ratio_div<double>(double x, double y) {
  return x / y;
}

// b = q / Y of the b-update (Eq. update-formula-1), 0 where q = 0 and also
// where Y = xi^T a is below the smallest normal number of the working
// precision: there a has underflowed over the whole kernel width, the cell's
// mass is below what the scalings can represent, and q / Y would overflow.
template <typename T> struct NormalMin;
template <> struct NormalMin<float> { static constexpr float v = 1.17549435e-38f; };
template <> struct NormalMin<double> { static constexpr double v = 2.2250738585072014e-308; };
template <typename T>
__device__ __forceinline__ T b_update(T q, T Y) {
  return (q == T(0) || !(Y >= NormalMin<T>::v)) ? T(0) : ratio_div<T>(q, Y);
}

// Newton stopping threshold on the step |dy| relative to 1 + |y|.
template <typename T> struct NewtonEps;
template <> struct NewtonEps<float> { static constexpr float v = 1e-7f; };
template <> struct NewtonEps<double> { static constexpr double v = 1e-15; };

// y = log psi of the power kind for one cell with finite l = log s - sigma w,
// and k = g'(y) - 1 for the derivative (dy/dl = 1 / (1 + k)).
//  * scalar m (power form): y + beta e^{(m-1) y} = l, beta = sigma alpha m/(m-1);
//    g is increasing and convex, so Newton from y0 = l (g(l) >= 0) decreases
//    monotonically to the root without overshoot;
//  * per-cell m (the paper's e_m, Eq. prox-psi as printed):
//    y + c (e^{m1 y} - 1)/m1 = l, c = sigma alpha m, m1 = m - 1; at m1 = 0 it
//    is Eq. prox-entropy, y = l/(1 + c).  From y0 = l/(1 + c), where
//    g(y0) = c ((e^{m1 y0} - 1)/m1 - y0) >= 0, Newton again decreases
//    monotonically (g increasing and convex); expm1 keeps small m1 exact.
template <typename T>
__device__ __forceinline__ T power_log_psi(const ProxArgs<T>& P, int idx, T l, T& k) {
  const T c = P.c[idx];
  if (P.m1f != nullptr) {
    const T m1 = P.m1f[idx];
    T y = l / (T(1) + c);
    if (m1 > T(0)) {
      for (int it = 0; it < P.newton; ++it) {
        const T g = y + c * dev_expm1<T>(m1 * y) / m1 - l;
        const T dy = g / (T(1) + c * dev_exp<T>(m1 * y));
        y -= dy;
        if (!(dy > NewtonEps<T>::v * (T(1) + fabs(y)))) break;
      }
      k = c * dev_exp<T>(m1 * y);
    } else {
      k = c;
    }
    return y;
  }
  T y = l;
  for (int it = 0; it < P.newton; ++it) {
    const T e = c * dev_exp<T>(P.m1 * y);
    const T dy = (y + e - l) / (T(1) + P.m1 * e);
    y -= dy;
    if (!(dy > NewtonEps<T>::v * (T(1) + fabs(y)))) break;
  }
  k = P.m1 * c * dev_exp<T>(P.m1 * y);
  return y;
}

// Limit of psi / s as s -> 0 for the power kind: e^{-sigma w} (scalar m);
// e^{c/m1 - sigma w} for a per-cell m1 > 0, 0 at m1 = 0 (the entropy reading).
template <typename T>
__device__ __forceinline__ T power_ratio_at_zero(const ProxArgs<T>& P, int idx, T sw) {
  if (P.m1f == nullptr) return dev_exp<T>(-sw);
  const T m1 = P.m1f[idx];
  return m1 > T(0) ? dev_exp<T>(P.c[idx] / m1 - sw) : T(0);
}

// a = Prox_{sigma f}(s) / s for one cell, extended continuously at s = 0
// (Prop. 4.1, Eq. prox-entropy, Eq. prox-psi with the shift rule
// Eq. prox-calculus-shift; clamp at kappa; 0 on the mask).
// `e` is e^{-sigma w} of the cell when the caller has already loaded it (crowd
// kind only; pass P.E[idx] otherwise).
template <typename T, int EK>
__device__ __forceinline__ T prox_ratio_e(const ProxArgs<T>& P, int idx, T s, T e) {
  if (P.mask != nullptr && P.mask[idx]) return T(0);
  T a;
  if (EK == EK_CROWD) {
    if (P.binary) {
      // Eq. dfn-congestion-noncvx with the shift rule: p = kappa where
      // s e^{-sigma w} > kappa / e, else 0 (0 at the tie); a = p / s
      const T kap = P.kappa ? P.kappa[idx] : P.kappa_s;
      return (s * e > kap * T(0.36787944117144233)) ? ratio_div<T>(kap, s) : T(0);
    }
    a = e;
  } else if (EK == EK_ENTROPY) {
    // psi = (s e^{-sigma w})^{1/(1+sigma alpha)} ; a = psi / s
    if (!(s > T(0))) return T(0);
    const T c = P.c[idx];
    const T sw = P.sw ? P.sw[idx] : T(0);
    a = dev_exp<T>(-(c * dev_log<T>(s) + sw) / (T(1) + c));
  } else {
    // power kind: y = log psi from power_log_psi, l = log s - sigma w
    const T sw = P.sw ? P.sw[idx] : T(0);
    if (!(s > T(0))) {
      a = power_ratio_at_zero<T>(P, idx, sw);
    } else {
      const T ls = dev_log<T>(s);
      T k;
      const T y = power_log_psi<T>(P, idx, ls - sw, k);
      a = dev_exp<T>(y - ls);
    }
  }
  // clamp p = a s at kappa: a = min(a, kappa / s), dividing only where the
  // bound is active (a s > kappa > 0 implies s > 0)
  if (P.has_kappa) {
    const T kap = P.kappa ? P.kappa[idx] : P.kappa_s;
    if (a * s > kap) a = ratio_div<T>(kap, s);
  }
  return a;
}

// Derivatives of the ratio r(s, w) = Prox_{sigma f}(s)/s at one cell, for the
// adjoint: (dr/ds, dr/dw).  Unclamped: crowd r = e^{-sigma w}; entropy from
// Eq. prox-entropy; power from differentiating Eq. prox-psi (y = log psi):
// dy/dl = 1/(1 + k), k = (m-1) beta psi^{m-1} (scalar m) or c psi^{m_i - 1}
// (per-cell exponents), as power_log_psi returns it.  Clamped at kappa (the forward's
// test a s > kappa): r = kappa/s.  Masked cells: 0.
template <typename T, int EK>
__device__ __forceinline__ void ratio_grad(const ProxArgs<T>& P, int idx, T s, T& rs, T& rw) {
  rs = T(0);
  rw = T(0);
  if (P.mask != nullptr && P.mask[idx]) return;
  T a = T(0), ds = T(0), dw = T(0);
  if (EK == EK_CROWD) {
    a = P.E[idx];
    dw = -P.sigma * a;
  } else if (EK == EK_ENTROPY) {
    if (!(s > T(0))) return;
    const T c = P.c[idx];
    const T sw = P.sw ? P.sw[idx] : T(0);
    a = dev_exp<T>(-(c * dev_log<T>(s) + sw) / (T(1) + c));
    ds = -a * c / ((T(1) + c) * s);
    dw = -P.sigma * a / (T(1) + c);
  } else {
    const T sw = P.sw ? P.sw[idx] : T(0);
    if (!(s > T(0))) {
      a = power_ratio_at_zero<T>(P, idx, sw);
      dw = -P.sigma * a;
    } else {
      const T ls = dev_log<T>(s);
      T k;
      const T y = power_log_psi<T>(P, idx, ls - sw, k);
      a = dev_exp<T>(y - ls);
      ds = -(a / s) * k / (T(1) + k);
      dw = -P.sigma * a / (T(1) + k);
    }
  }
  if (P.has_kappa) {
    const T kap = P.kappa ? P.kappa[idx] : P.kappa_s;
    if (a * s > kap) {
      rs = -kap / (s * s);
      rw = T(0);
      return;
    }
  }
  rs = ds;
  rw = dw;
}

template <typename T, int EK>
__device__ __forceinline__ T prox_ratio(const ProxArgs<T>& P, int idx, T s) {
  return prox_ratio_e<T, EK>(P, idx, s, EK == EK_CROWD ? P.E[idx] : T(0));
}

// |b Y - q| with one rounding (fused multiply-add) in the working precision.
template <typename T>
__device__ __forceinline__ T abs_residual(T b, T Y, T q) { return fabs(fma(b, Y, -q)); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_or(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum over a 1-, 2- or 3-D block (linear thread order, whole warps);
// every thread gets the total.  `scratch` has >= 33 doubles.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int lane = tid & 31, wid = tid >> 5;
  const int nw = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    t = lane < nw ? scratch[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) scratch[32] = t;
  }
  __syncthreads();
  return scratch[32];
}

}  // namespace jko
