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
// coefficients).  p(A) v is evaluated by Clenshaw's recurrence, two degrees
// per fused 5-point stencil kernel (the first on the tile and a one-cell halo
// in shared memory): 1 + ceil(D / 2) launches for the whole operator, against
// L separate solves.  p(A) stays symmetric, as xi~ is.
// The b-update (with the residual partials of the stop rule) and the prox
// (with the pair counter) are elementwise kernels around the two xi~
// applications of a pair; every kernel passes the stop gate first.
#include <cmath>
#include <vector>

#include "jko_internal.cuh"
#include "jko_kernels.h"

namespace jko {

namespace {

constexpr int HBX = 16, HBY = 8;   // small tiles: the work is FP64-bound per SM, so more blocks spread it

struct HeatGeom {
  int nx, ny;
  double cx, cy;          // c / hx^2, c / hy^2
  const uint8_t* mask;    // 1 = obstacle, or NULL
  double two_over_delta;  // 2 / delta (Clenshaw recurrence)
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

// The operator's output is clamped at 0: xi~ is positive, and the expansion's
// error is normwise (~1e-15 of the largest entry in FP64), so where the true
// kernel tail lies below it the sum can come out slightly negative; 0 there
// is the same underflow the Gaussian kernel meets far from its support (the
// b-update and the prox treat it so).  NaN passes through.
__device__ __forceinline__ double close_value(double r) { return r < 0.0 ? 0.0 : r; }

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
template <typename T, typename O, bool CLOSE>
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
  const double r = ck * (double)v[i] + s_over_delta * (Ab - theta * b1[i]) - b2[i];
  out[i] = (O)(CLOSE ? close_value(r) : r);
}

// Two Clenshaw steps in one launch: b_k on the block's tile plus a one-cell
// halo (shared memory), then b_{k-1} on the tile from it.  Reads b_{k+1} (at a
// two-cell halo) and b_{k+2}; writes b_k (o1) and b_{k-1} (o2), buffers that no
// block of this launch reads.  The second step is the closing one (s2 = 1 /
// delta, O = T, o2 = the operator's output) when k - 1 = 0.
template <typename T, typename O, bool CLOSE>
__global__ void __launch_bounds__(HBX * HBY) heat_cl_step2(const T* v, const double* b1,
                                                           const double* b2, double* o1, O* o2,
                                                           HeatGeom g, double ck, double ck1,
                                                           double s2, double theta, Ctrl* ctrl) {
  constexpr int RX = HBX + 2, RY = HBY + 2;
  __shared__ double sb[RY][RX];
  __shared__ int s_it;
  if (stop_gate(ctrl, nullptr, 0, false, &s_it)) return;
  const int x0 = blockIdx.x * HBX, y0 = blockIdx.y * HBY;
  const int tid = threadIdx.y * HBX + threadIdx.x;
  for (int idx = tid; idx < RX * RY; idx += HBX * HBY) {
    const int ry = idx / RX, rx = idx - ry * RX;
    const int x = x0 + rx - 1, y = y0 + ry - 1;
    double val = 0.0;
    if (x >= 0 && x < g.nx && y >= 0 && y < g.ny) {
      const int i = y * g.nx + x;
      if (is_free(g, i)) {
        const double Ab = apply_A<double>(g, b1, x, y);
        val = ck * (double)v[i] + g.two_over_delta * (Ab - theta * b1[i]) - b2[i];
      }
    }
    sb[ry][rx] = val;
  }
  __syncthreads();
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int i = y * g.nx + x;
  const int tx = threadIdx.x + 1, ty = threadIdx.y + 1;
  const double c = sb[ty][tx];
  o1[i] = c;
  if (!is_free(g, i)) {
    o2[i] = O(0);
    return;
  }
  // A b_k at (x, y) from the tile: the neighbour tests of apply_A
  double acc = c;
  if (x > 0 && is_free(g, i - 1)) acc += g.cx * (c - sb[ty][tx - 1]);
  if (x + 1 < g.nx && is_free(g, i + 1)) acc += g.cx * (c - sb[ty][tx + 1]);
  if (y > 0 && is_free(g, i - g.nx)) acc += g.cy * (c - sb[ty - 1][tx]);
  if (y + 1 < g.ny && is_free(g, i + g.nx)) acc += g.cy * (c - sb[ty + 1][tx]);
  const double r = ck1 * (double)v[i] + s2 * (acc - theta * c) - b1[i];
  o2[i] = (O)(CLOSE ? close_value(r) : r);
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
// which the next 8 coefficients sum below eps/2, or each lie at their
// rounding floor (they decay geometrically:
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
  // FP32 handles run the recurrence in FP64 too and truncate where FP64 does:
  // the scalings weigh the kernel's far tail by up to e^{sigma (max w - min w)},
  // so a normwise truncation error of 1e-10 became 2.5e-5 of relative L1 in p,
  // against 3e-8 with FP32 scalings around an exact kernel
  const double eps = 1e-15;
  (void)fp64;
  constexpr int M = 4096, kWin = 8;
  constexpr double kCoefFloor = 1.5e-16;
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
      double win = 0.0, wmax = 0.0;
      for (int j = D + 1; j <= k; ++j) {
        win += std::fabs(cf[j]);
        wmax = std::max(wmax, std::fabs(cf[j]));
      }
      // the coefficients carry a rounding floor of ~1e-16 (f <= 1 on the
      // interval): a window whose every entry is at that floor has ended the series
      if (win <= 0.5 * eps || wmax <= kCoefFloor) {
        hp.D = D;
        cf.resize(D + 1);
        hp.coef = cf;
        return hp;
      }
    }
  }
  return hp;
}

// out_x = p(A) in with the Clenshaw recurrence of the expansion: the first
// step b_D = c_D v, then the D remaining steps (k = D-1 .. 0, the last the
// closing one) two per launch, one single step first when D is odd:
// 1 + ceil(D / 2) launches.
template <typename T>
cudaError_t heat_apply(const HeatPlan& hp, const HeatBuffers& B, const T* in, T* out_x,
                       int nx, int ny, const uint8_t* mask, Ctrl* ctrl, const double* part,
                       int nparts, int decide, cudaStream_t st) {
  const double inv_delta = hp.delta > 0 ? 1.0 / hp.delta : 0.0;   // delta = 0: p(A) = c_0 Id
  HeatGeom g{nx, ny, hp.cx, hp.cy, mask, 2.0 * inv_delta};
  const dim3 grid = heat_grid(nx, ny), block(HBX, HBY);
  double* d[4] = {(double*)B.d[0], (double*)B.d[1], (double*)B.d[2], (double*)B.d[3]};
  const int D = hp.D;
  // b_{k+1} in d[r1], b_{k+2} in d[r2]; d[f1], d[f2] free
  int r1 = 0, r2 = 1, f1 = 2, f2 = 3;
  heat_cl_init<T><<<grid, block, 0, st>>>(in, d[r1], d[r2], g, hp.coef[D], ctrl, part, nparts,
                                          decide);
  int k = D - 1;
  if (D % 2 == 1) {   // one single step so that the rest pairs up
    if (k == 0) {
      heat_cl_step<T, T, true><<<grid, block, 0, st>>>(in, d[r1], d[r2], out_x, g, hp.coef[0],
                                                 inv_delta, hp.theta, ctrl);
      return cudaGetLastError();
    }
    heat_cl_step<T, double, false><<<grid, block, 0, st>>>(in, d[r1], d[r2], d[r2], g, hp.coef[k],
                                                    2.0 * inv_delta, hp.theta, ctrl);
    std::swap(r1, r2);
    --k;
  }
  for (; k >= 1; k -= 2) {
    if (k == 1) {   // steps 1 and the closing 0
      heat_cl_step2<T, T, true><<<grid, block, 0, st>>>(in, d[r1], d[r2], d[f1], out_x, g, hp.coef[1],
                                                  hp.coef[0], inv_delta, hp.theta, ctrl);
      break;
    }
    heat_cl_step2<T, double, false><<<grid, block, 0, st>>>(in, d[r1], d[r2], d[f1], d[f2], g,
                                                     hp.coef[k], hp.coef[k - 1],
                                                     2.0 * inv_delta, hp.theta, ctrl);
    // b_{k-1} (f2) and b_k (f1) are the next step's b_{k'+1}, b_{k'+2}
    const int o1 = r1, o2 = r2;
    r1 = f2;
    r2 = f1;
    f1 = o1;
    f2 = o2;
  }
  return cudaGetLastError();
}

int heat_launches(const HeatPlan& hp) { return 1 + (hp.D + 1) / 2; }

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
