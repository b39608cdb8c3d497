// heat.cu -- the heat-kernel Gibbs kernel on a domain with obstacles
// (Sec. 4.1, Eq. heat-kernel) on the CUDA cores (FP32 / FP64).
//
// xi~ v = A^{-L} v with A = Id - c Delta_M, c = gamma / L, Delta_M the
// axis-aligned finite-difference Laplacian on the free cells (Neumann: a
// missing neighbour, outside the grid or on the mask, contributes nothing).
// The paper pre-factors A (sparse Cholesky) and runs L back-substitutions.
// Here A is symmetric with its spectrum in [1, lmax], lmax = 1 + 4 c/hx^2 +
// 4 c/hy^2 (Gershgorin), so A^{-L} = f(A) for f(lambda) = lambda^{-L} is
// replaced by its Chebyshev expansion p of degree D on that interval, with
// ||p(A) - A^{-L}||_2 <= max |p - f| on [1, lmax] (the sum of the dropped
// coefficients).  p(A) v is evaluated by Clenshaw's recurrence: one fused
// 5-point stencil kernel per degree, D + 1 launches for the whole operator
// (against L separate solves).  p(A) stays symmetric, as xi~ is.
// The b-update (with the residual partials of the stop rule) and the prox
// (with the pair counter) are elementwise kernels around the two xi~
// applications of a pair; every kernel passes the stop gate first.
#include <cmath>
#include <vector>

#include "jko_internal.cuh"
#include "jko_kernels.h"

namespace jko {

namespace {

constexpr int HBX = 32, HBY = 8;

struct HeatGeom {
  int nx, ny;
  double cx, cy;          // c / hx^2, c / hy^2
  const uint8_t* mask;    // 1 = obstacle, or NULL
};

__device__ __forceinline__ bool is_free(const HeatGeom& g, int i) {
  return g.mask == nullptr || g.mask[i] == 0;
}

// (A v)_i = v_i + sum over free neighbours j of c_dir (v_i - v_j)
template <typename T>
__device__ __forceinline__ T apply_A(const HeatGeom& g, const T* v, int x, int y) {
  const int i = y * g.nx + x;
  const T vi = v[i];
  T acc = vi;
  const T cx = (T)g.cx, cy = (T)g.cy;
  if (x > 0 && is_free(g, i - 1)) acc += cx * (vi - v[i - 1]);
  if (x + 1 < g.nx && is_free(g, i + 1)) acc += cx * (vi - v[i + 1]);
  if (y > 0 && is_free(g, i - g.nx)) acc += cy * (vi - v[i - g.nx]);
  if (y + 1 < g.ny && is_free(g, i + g.nx)) acc += cy * (vi - v[i + g.nx]);
  return acc;
}

// The Clenshaw iterates are FP64 for both precisions: a high-degree
// recurrence cancels large intermediate terms in the far field, where the
// kernel's tail is many orders below its peak, and single precision there
// costs digits that the L separate solves keep; the stencil work is a small
// share of a launch at the grid sizes of this operator.

// First Clenshaw step: b_D = c_D v, b_{D+1} = 0 (v is 0 on the mask).
template <typename T>
__global__ void __launch_bounds__(HBX * HBY) heat_cl_init(const T* v, double* b1, double* b2,
                                                          HeatGeom g, double cD, Ctrl* ctrl,
                                                          const double* part, int nparts,
                                                          int decide) {
  __shared__ int s_it;
  if (stop_gate(ctrl, part, nparts, decide != 0, &s_it)) return;
  const int xx = blockIdx.x * HBX + threadIdx.x, yy = blockIdx.y * HBY + threadIdx.y;
  if (xx >= g.nx || yy >= g.ny) return;
  const int i = yy * g.nx + xx;
  b1[i] = is_free(g, i) ? cD * (double)v[i] : 0.0;
  b2[i] = 0.0;
}

// One Clenshaw step out = c_k v + s (B b1) - b2 with B = (A - theta Id) / delta:
// s = 2 inside the recurrence (O = double), s = 1 for the closing step (O = T).
// out may alias b2 (each thread reads its own b2 entry before writing it); b1
// is read at the 5-point stencil and is not written.
template <typename T, typename O>
__global__ void __launch_bounds__(HBX * HBY) heat_cl_step(const T* v, const double* b1,
                                                          const double* b2, O* out, HeatGeom g,
                                                          double ck, double s_over_delta,
                                                          double theta, Ctrl* ctrl) {
  __shared__ int s_it;
  if (stop_gate(ctrl, nullptr, 0, false, &s_it)) return;
  const int xx = blockIdx.x * HBX + threadIdx.x, yy = blockIdx.y * HBY + threadIdx.y;
  if (xx >= g.nx || yy >= g.ny) return;
  const int i = yy * g.nx + xx;
  if (!is_free(g, i)) {
    out[i] = O(0);
    return;
  }
  const double Ab = apply_A<double>(g, b1, xx, yy);
  out[i] = (O)(ck * (double)v[i] + s_over_delta * (Ab - theta * b1[i]) - b2[i]);
}

// b = q / Y (0 where q = 0 or Y is not a normal number), with the residual
// partial |b_old Y - q| of this block (Sec. 3.4), as the EPI_B epilogue.
template <typename T>
__global__ void __launch_bounds__(HBX * HBY) heat_bupdate(const T* Y, T* b, const T* q,
                                                          HeatGeom g, Ctrl* ctrl, double* part) {
  __shared__ int s_it;
  __shared__ double s_red[33];
  if (stop_gate(ctrl, nullptr, 0, false, &s_it)) return;
  const int xx = blockIdx.x * HBX + threadIdx.x, yy = blockIdx.y * HBY + threadIdx.y;
  T res = T(0);
  int bad = 0;
  if (xx < g.nx && yy < g.ny) {
    const int i = yy * g.nx + xx;
    const T Yi = Y[i], qi = q[i];
    if (s_it > 0) res = abs_residual<T>(b[i], Yi, qi);
    const T bn = b_update<T>(qi, Yi);
    bad = !dev_finite(bn);
    b[i] = bn;
  }
  const double tot = block_sum((double)res, s_red);
  if (threadIdx.x == 0 && threadIdx.y == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = tot;
  bad = warp_or(bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicOr(&ctrl->nonfinite, 1);
}

// a = Prox(s)/s, p = a s (Eq. update-formula-2), and the pair counter.
template <typename T, int EK>
__global__ void __launch_bounds__(HBX * HBY) heat_prox(const T* s, T* a, T* p, HeatGeom g,
                                                       ProxArgs<T> P, Ctrl* ctrl) {
  __shared__ int s_it;
  if (stop_gate(ctrl, nullptr, 0, false, &s_it)) return;
  const int xx = blockIdx.x * HBX + threadIdx.x, yy = blockIdx.y * HBY + threadIdx.y;
  int bad = 0;
  if (xx < g.nx && yy < g.ny) {
    const int i = yy * g.nx + xx;
    const T si = s[i];
    const T ai = prox_ratio<T, EK>(P, i, si);
    bad = !dev_finite(ai);
    a[i] = ai;
    p[i] = ai * si;
  }
  bad = warp_or(bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicOr(&ctrl->nonfinite, 1);
  if (threadIdx.x == 0 && threadIdx.y == 0 && blockIdx.x == 0 && blockIdx.y == 0)
    ctrl->it = s_it + 1;
}

dim3 heat_grid(int nx, int ny) { return dim3((nx + HBX - 1) / HBX, (ny + HBY - 1) / HBY); }

}  // namespace

int heat_blocks(int nx, int ny) {
  const dim3 g = heat_grid(nx, ny);
  return (int)(g.x * g.y);
}

// Chebyshev coefficients of f(lambda) = lambda^{-L} on [1, lmax], by
// interpolation at M Chebyshev points (compensated sums: the noise floor of
// the coefficients stays far below the FP64 target), and the degree D after
// which the next 8 coefficients sum below eps/2 (they decay geometrically:
// f is analytic on a Bernstein ellipse around the interval, its only pole
// at lambda = 0).  Degree above max_degree: D = -1.
HeatPlan heat_plan(int nx, int ny, double lx, double ly, double gamma, int L, bool fp64) {
  HeatPlan hp;
  hp.L = L;
  const double c = gamma / L;
  const double hx2 = (lx / nx) * (lx / nx), hy2 = (ly / ny) * (ly / ny);
  hp.cx = c / hx2;
  hp.cy = c / hy2;
  const double lmax = 1.0 + 4.0 * hp.cx + 4.0 * hp.cy;
  hp.theta = 0.5 * (lmax + 1.0);
  hp.delta = 0.5 * (lmax - 1.0);
  // FP32 handles run the recurrence in FP64 too: truncate well below their rounding
  const double eps = fp64 ? 1e-15 : 1e-10;
  constexpr int M = 4096, kWin = 8;
  const double pi = 3.14159265358979323846;
  std::vector<double> f(M), ang(M);
  for (int j = 0; j < M; ++j) {
    ang[j] = pi * (j + 0.5) / M;
    f[j] = std::pow(hp.theta + hp.delta * std::cos(ang[j]), -(double)L);
  }
  auto coef = [&](int k) {
    double sum = 0.0, comp = 0.0;   // Kahan summation
    for (int j = 0; j < M; ++j) {
      // cos(k pi (2j+1) / (2M)) with the angle reduced exactly modulo 2 pi
      const long long m = ((long long)k * (2 * j + 1)) % (4LL * M);
      const double y = f[j] * std::cos(pi * (double)m / (2.0 * M)) - comp;
      const double t = sum + y;
      comp = (t - sum) - y;
      sum = t;
    }
    return (k == 0 ? 1.0 : 2.0) * sum / M;
  };
  hp.D = -1;
  if (!(hp.delta > 0)) {   // lmax = 1: xi~ = Id
    hp.D = 1;
    hp.coef = {1.0, 0.0};
    return hp;
  }
  std::vector<double> cf;
  for (int k = 0; k <= kMaxHeatDegree + kWin; ++k) {
    cf.push_back(coef(k));
    const int D = k - kWin;
    if (D >= 1) {
      double win = 0.0;
      for (int j = D + 1; j <= k; ++j) win += std::fabs(cf[j]);
      if (win <= 0.5 * eps) {
        hp.D = D;
        cf.resize(D + 1);
        hp.coef = cf;
        return hp;
      }
    }
  }
  return hp;
}

// out_x = p(A) in with the Clenshaw recurrence of the expansion: D + 1 launches.
template <typename T>
cudaError_t heat_apply(const HeatPlan& hp, const HeatBuffers& B, const T* in, T* out_x,
                       int nx, int ny, const uint8_t* mask, Ctrl* ctrl, const double* part,
                       int nparts, int decide, cudaStream_t st) {
  HeatGeom g{nx, ny, hp.cx, hp.cy, mask};
  const dim3 grid = heat_grid(nx, ny), block(HBX, HBY);
  double* d[2] = {(double*)B.d[0], (double*)B.d[1]};
  const int D = hp.D;
  heat_cl_init<T><<<grid, block, 0, st>>>(in, d[0], d[1], g, hp.coef[D], ctrl, part, nparts,
                                          decide);
  // b_{k+1} in d[cur], b_{k+2} in d[cur ^ 1]; b_k overwrites b_{k+2}
  int cur = 0;
  const double inv_delta = hp.delta > 0 ? 1.0 / hp.delta : 0.0;   // delta = 0: p(A) = c_0 Id
  for (int k = D - 1; k >= 1; --k) {
    heat_cl_step<T, double><<<grid, block, 0, st>>>(in, d[cur], d[cur ^ 1], d[cur ^ 1], g,
                                                    hp.coef[k], 2.0 * inv_delta, hp.theta, ctrl);
    cur ^= 1;
  }
  heat_cl_step<T, T><<<grid, block, 0, st>>>(in, d[cur], d[cur ^ 1], out_x, g, hp.coef[0],
                                             inv_delta, hp.theta, ctrl);
  return cudaGetLastError();
}

template <typename T>
cudaError_t heat_bupdate_launch(const T* Y, T* b, const T* q, int nx, int ny, Ctrl* ctrl,
                                double* part, cudaStream_t st) {
  HeatGeom g{nx, ny, 0.0, 0.0, nullptr};
  heat_bupdate<T><<<heat_grid(nx, ny), dim3(HBX, HBY), 0, st>>>(Y, b, q, g, ctrl, part);
  return cudaGetLastError();
}

template <typename T>
cudaError_t heat_prox_launch(int ek, const T* s, T* a, T* p, int nx, int ny, const ProxArgs<T>& P,
                             Ctrl* ctrl, cudaStream_t st) {
  HeatGeom g{nx, ny, 0.0, 0.0, nullptr};
  const dim3 grid = heat_grid(nx, ny), block(HBX, HBY);
  if (ek == EK_CROWD) heat_prox<T, EK_CROWD><<<grid, block, 0, st>>>(s, a, p, g, P, ctrl);
  else if (ek == EK_ENTROPY) heat_prox<T, EK_ENTROPY><<<grid, block, 0, st>>>(s, a, p, g, P, ctrl);
  else heat_prox<T, EK_POWER><<<grid, block, 0, st>>>(s, a, p, g, P, ctrl);
  return cudaGetLastError();
}

#define JKO_HEAT_INST(T)                                                                      \
  template cudaError_t heat_apply<T>(const HeatPlan&, const HeatBuffers&, const T*, T*, int, \
                                     int, const uint8_t*, Ctrl*, const double*, int, int,     \
                                     cudaStream_t);                                           \
  template cudaError_t heat_bupdate_launch<T>(const T*, T*, const T*, int, int, Ctrl*,        \
                                              double*, cudaStream_t);                         \
  template cudaError_t heat_prox_launch<T>(int, const T*, T*, T*, int, int,                   \
                                           const ProxArgs<T>&, Ctrl*, cudaStream_t);
JKO_HEAT_INST(float)
JKO_HEAT_INST(double)
#undef JKO_HEAT_INST

}  // namespace jko
