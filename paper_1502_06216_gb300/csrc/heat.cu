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
#include <algorithm>
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
  bool linear;            // output not clamped at 0 (signed inputs: the adjoint)
};

__device__ __forceinline__ bool is_free(const HeatGeom& g, int i) {
  return g.mask == nullptr || g.mask[i] == 0;
}

// ---- the per-cell arithmetic of the recurrence ----
// Written with explicit roundings, so that every kernel below (per phase or
// persistent) performs the same operations whatever the compiler contracts.
// The iterates W are FP64 for both precisions: a high-degree recurrence
// cancels large intermediate terms in the far field, where the kernel's tail
// is many orders below its peak, so single precision there costs digits (the
// flows' error grew 16-fold with FP32 iterates).  Double-float iterates (two
// floats, ~48 significant bits, on the FP32 pipe) were measured slower than
// FP64 on GB300 (100^2: 4.8k against 5.3k pairs/s): the stencil is bound by
// the latency of its dependent chains, which double-float arithmetic
// lengthens, not by the FP64 pipe's throughput.
template <typename T> struct HeatIter { using W = double; };

// constants and inputs as iterates
template <typename W> __device__ __forceinline__ W wc(double d) { return d; }
__device__ __forceinline__ double wv(double v) { return v; }
template <typename W> __device__ __forceinline__ W wzero() { return 0.0; }
// c v (the first iterate b_D = c_D v)
__device__ __forceinline__ double wscale(double c, double v) { return __dmul_rn(c, v); }

// acc + c (vi - vj): one neighbour's term of A v
__device__ __forceinline__ double nb_term(double acc, double c, double vi, double vj) {
  return __fma_rn(c, __dsub_rn(vi, vj), acc);
}
// one Clenshaw step's value ck v + s (A b1 - theta b1) - b2
__device__ __forceinline__ double cl_value(double ck, double v, double s, double Ab, double theta,
                                          double b1, double b2) {
  return __dsub_rn(__fma_rn(ck, v, __dmul_rn(s, __fma_rn(-theta, b1, Ab))), b2);
}

// The operator's output is clamped at 0: xi~ is positive, and the expansion's
// error is normwise (~1e-15 of the largest entry), so where the true kernel
// tail lies below it the sum can come out slightly negative; 0 there is the
// same underflow the Gaussian kernel meets far from its support (the b-update
// and the prox treat it so).  NaN passes through.
template <typename T> __device__ __forceinline__ T close_out(double r) {
  return (T)(r < 0.0 ? 0.0 : r);
}

// (A v)_i = v_i + sum over free neighbours j of c_dir (v_i - v_j)
template <typename W>
__device__ __forceinline__ W apply_A(const HeatGeom& g, const W* v, int x, int y, W cx, W cy) {
  const int i = y * g.nx + x;
  const W vi = v[i];
  W acc = vi;
  if (x > 0 && is_free(g, i - 1)) acc = nb_term(acc, cx, vi, v[i - 1]);
  if (x + 1 < g.nx && is_free(g, i + 1)) acc = nb_term(acc, cx, vi, v[i + 1]);
  if (y > 0 && is_free(g, i - g.nx)) acc = nb_term(acc, cy, vi, v[i - g.nx]);
  if (y + 1 < g.ny && is_free(g, i + g.nx)) acc = nb_term(acc, cy, vi, v[i + g.nx]);
  return acc;
}

// First Clenshaw step: b_D = c_D v, b_{D+1} = 0 (v is 0 on the mask).
template <typename T>
__global__ void __launch_bounds__(HBX * HBY) heat_cl_init(const T* v, void* b1_, void* b2_,
                                                          HeatGeom g, double cD, Ctrl* ctrl,
                                                          const double* part, int nparts,
                                                          int decide) {
  using W = typename HeatIter<T>::W;
  W* b1 = (W*)b1_;
  W* b2 = (W*)b2_;
  __shared__ int s_it;
  if (stop_gate(ctrl, part, nparts, decide != 0, &s_it)) return;
  const int xx = blockIdx.x * HBX + threadIdx.x, yy = blockIdx.y * HBY + threadIdx.y;
  if (xx >= g.nx || yy >= g.ny) return;
  const int i = yy * g.nx + xx;
  b1[i] = is_free(g, i) ? wscale(wc<W>(cD), wv(v[i])) : wzero<W>();
  b2[i] = wzero<W>();
}

// One Clenshaw step c_k v + s (B b1) - b2 with B = (A - theta Id) / delta:
// s = 2 inside the recurrence (iterate out), s = 1 for the closing step
// (CLOSE: T out, the operator's output).  out may alias b2 (each thread reads
// its own b2 entry before writing it); b1 is read at the 5-point stencil and
// is not written.
template <typename T, bool CLOSE>
__global__ void __launch_bounds__(HBX * HBY) heat_cl_step(const T* v, const void* b1_,
                                                          const void* b2_, void* out_, HeatGeom g,
                                                          double ck_, double s_over_delta,
                                                          double theta_, Ctrl* ctrl) {
  using W = typename HeatIter<T>::W;
  const W* b1 = (const W*)b1_;
  const W* b2 = (const W*)b2_;
  __shared__ int s_it;
  if (stop_gate(ctrl, nullptr, 0, false, &s_it)) return;
  const int xx = blockIdx.x * HBX + threadIdx.x, yy = blockIdx.y * HBY + threadIdx.y;
  if (xx >= g.nx || yy >= g.ny) return;
  const int i = yy * g.nx + xx;
  if (!is_free(g, i)) {
    if (CLOSE) ((T*)out_)[i] = T(0);
    else ((W*)out_)[i] = wzero<W>();
    return;
  }
  const W cx = wc<W>(g.cx), cy = wc<W>(g.cy);
  const W Ab = apply_A<W>(g, b1, xx, yy, cx, cy);
  const W r = cl_value(wc<W>(ck_), wv(v[i]), wc<W>(s_over_delta), Ab, wc<W>(theta_), b1[i], b2[i]);
  if (CLOSE) ((T*)out_)[i] = g.linear ? (T)r : close_out<T>(r);
  else ((W*)out_)[i] = r;
}

// Two Clenshaw steps in one launch: b_k on the block's tile plus a one-cell
// halo (shared memory), then b_{k-1} on the tile from it.  Reads b_{k+1} (at a
// two-cell halo) and b_{k+2}; writes b_k (o1) and b_{k-1} (o2), buffers that no
// block of this launch reads.  The second step is the closing one (s2 = 1 /
// delta, CLOSE: o2 = the operator's output, of type T) when k - 1 = 0.
template <typename T, bool CLOSE>
__global__ void __launch_bounds__(HBX * HBY) heat_cl_step2(const T* v, const void* b1_,
                                                           const void* b2_, void* o1_, void* o2_,
                                                           HeatGeom g, double ck_, double ck1_,
                                                           double s2_, double theta_, Ctrl* ctrl) {
  using W = typename HeatIter<T>::W;
  const W* b1 = (const W*)b1_;
  const W* b2 = (const W*)b2_;
  W* o1 = (W*)o1_;
  constexpr int RX = HBX + 2, RY = HBY + 2;
  __shared__ W sb[RY][RX];
  __shared__ int s_it;
  if (stop_gate(ctrl, nullptr, 0, false, &s_it)) return;
  const W cx = wc<W>(g.cx), cy = wc<W>(g.cy), theta = wc<W>(theta_);
  const W two = wc<W>(g.two_over_delta), ck = wc<W>(ck_);
  const int x0 = blockIdx.x * HBX, y0 = blockIdx.y * HBY;
  const int tid = threadIdx.y * HBX + threadIdx.x;
  for (int idx = tid; idx < RX * RY; idx += HBX * HBY) {
    const int ry = idx / RX, rx = idx - ry * RX;
    const int x = x0 + rx - 1, y = y0 + ry - 1;
    W val = wzero<W>();
    if (x >= 0 && x < g.nx && y >= 0 && y < g.ny) {
      const int i = y * g.nx + x;
      if (is_free(g, i)) {
        const W Ab = apply_A<W>(g, b1, x, y, cx, cy);
        val = cl_value(ck, wv(v[i]), two, Ab, theta, b1[i], b2[i]);
      }
    }
    sb[ry][rx] = val;
  }
  __syncthreads();
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int i = y * g.nx + x;
  const int tx = threadIdx.x + 1, ty = threadIdx.y + 1;
  const W c = sb[ty][tx];
  o1[i] = c;
  if (!is_free(g, i)) {
    if (CLOSE) ((T*)o2_)[i] = T(0);
    else ((W*)o2_)[i] = wzero<W>();
    return;
  }
  // A b_k at (x, y) from the tile: the neighbour tests of apply_A
  W acc = c;
  if (x > 0 && is_free(g, i - 1)) acc = nb_term(acc, cx, c, sb[ty][tx - 1]);
  if (x + 1 < g.nx && is_free(g, i + 1)) acc = nb_term(acc, cx, c, sb[ty][tx + 1]);
  if (y > 0 && is_free(g, i - g.nx)) acc = nb_term(acc, cy, c, sb[ty - 1][tx]);
  if (y + 1 < g.ny && is_free(g, i + g.nx)) acc = nb_term(acc, cy, c, sb[ty + 1][tx]);
  const W r = cl_value(wc<W>(ck1_), wv(v[i]), wc<W>(s2_), acc, theta, c, b1[i]);
  if (CLOSE) ((T*)o2_)[i] = g.linear ? (T)r : close_out<T>(r);
  else ((W*)o2_)[i] = r;
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

// ------------------------------------------------------------ persistent form
// One cooperative launch runs up to `pairs` pairs: the Clenshaw phases of the
// two applications of xi~, the b-update and the prox, with a grid barrier
// (jko_internal.cuh) where the kernels above end one launch and start the next.
// Block b takes the 16x8 tiles b, b + G, ... of the grid (the same tiles in
// every phase), with the arithmetic of heat_cl_step / heat_cl_step2 per cell;
// a phase runs two or four Clenshaw steps between two grid barriers (four
// while every tile has a block of its own), on the tile and a halo one cell
// narrower per step (recomputed by neighbours):
//   * the first Clenshaw iterates b_D = c_D v, b_{D+1} = 0 are formed on the
//     fly from v where the kernels above store them (the same values);
//   * the closing step ends in the b-update (first application: b = q / Y
//     and the residual partial of the tile, as heat_bupdate) or the prox
//     (second application: a, p, as heat_prox);
//   * the stop rule (Sec. 3.4) adds the tiles' residual partials in the order
//     of stop_gate, in every block after the barrier that ends the b-update;
//     when it fires the second application and the prox are skipped, as the
//     kernels above return at their stop gate.
// So the two forms give the same bits and the same pair counts.  Reads of what
// other blocks wrote in an earlier phase are ordinary loads: the barrier's
// acquire, followed by the block barrier, orders them after those writes.
template <typename T>
struct HeatLoopArgs {
  HeatGeom g;
  const double* coef;      // c_0 .. c_D
  int D;
  double theta, inv_delta;
  void* d[4];              // Clenshaw iterates (HeatIter<T>::W, 8 bytes per cell)
  const T* q;
  T* a;
  T* b;
  T* p;
  ProxArgs<T> P;
  Ctrl* ctrl;
  double* part;            // residual partial of each tile (heat_bupdate's blocks)
  int ntiles, tiles_x;
  int pairs;
  int steps;               // Clenshaw steps per phase between grid barriers
};

template <typename T>
__device__ __forceinline__ T ld_plain(const T* p) { return *p; }

// A v at (x, y) where v is stored as c * v[j] (the first iterate b_D = c_D v):
// the neighbour terms of apply_A on those values.
// The closing step's output r at cell i of the grid, into the b-update (app 0)
// or the prox (app 1).
template <typename T, int EK>
__device__ __forceinline__ void heat_close_cell(const HeatLoopArgs<T>& A, int app, int i, T y,
                                                bool have_prev, T& res, int& bad) {
  if (app == 0) {
    const T qi = __ldg(A.q + i);
    if (have_prev) res = abs_residual<T>(ld_plain(A.b + i), y, qi);
    const T bn = b_update<T>(qi, y);
    bad |= !dev_finite(bn);
    A.b[i] = bn;
  } else {
    const T ai = prox_ratio<T, EK>(A.P, i, y);
    bad |= !dev_finite(ai);
    A.a[i] = ai;
    A.p[i] = ai * y;
  }
}

// Up to H Clenshaw steps of one phase on one tile: v, b_{k+1}, b_{k+2} and
// the free flags staged on the tile and an H-cell halo; step s (index
// k - s) on the tile and an (ns - 1 - s)-cell halo, in place over b_{k+2}'s
// array (a cell reads b_{k+2} only at itself), with the arithmetic of the
// kernels per phase cell by cell.  VIRT: the first iterates b_{k+1} = c1v v
// and b_{k+2} = 0 formed here.  The phase writes its newest iterate to o_new
// and the one before to o_prev on the tile, or, when its last step is step 0,
// closes into the epilogue.
constexpr int HMAX = 4;                      // Clenshaw steps per grid barrier
constexpr int HLT = HBX * HBY * 4;           // threads of a persistent block: four per tile
                                             // cell in the halo phases (the work is latency
                                             // bound; 2 or 8 per cell measured slower)
constexpr int HSX = HBX + 2 * HMAX, HSY = HBY + 2 * HMAX;
template <typename W>
struct HeatStageH {
  W v[HSY][HSX];
  W b1[HSY][HSX];
  W b2[HSY][HSX];
  unsigned char fr[HSY][HSX];
};

template <typename T, int EK, typename W>
__device__ __forceinline__ void heat_tile_steps(const HeatLoopArgs<T>& A, int app, int t, const T* v,
                                                const W* b1, const W* b2, W* o_new, W* o_prev,
                                                bool virt, W c1v, int k, int ns, bool have_prev,
                                                HeatStageH<W>& S, W cx, W cy, W theta, double* s_red,
                                                int& bad) {
  constexpr int H = HMAX;
  const HeatGeom& g = A.g;
  const int tyt = t / A.tiles_x;
  const int x0 = (t - tyt * A.tiles_x) * HBX, y0 = tyt * HBY;
  const int tid = threadIdx.y * HBX + threadIdx.x;
  // stage the tile and an ns-cell halo (at offset H - ns in the arrays)
  const int sx = HBX + 2 * ns, sy = HBY + 2 * ns;
  for (int idx = tid; idx < sx * sy; idx += HLT) {
    const int ey = H - ns + idx / sx, ex = H - ns + idx % sx;
    const int xx = x0 + ex - H, yy = y0 + ey - H;
    W vv = wzero<W>(), bb1 = wzero<W>(), bb2 = wzero<W>();
    unsigned char f = 0;
    if (xx >= 0 && xx < g.nx && yy >= 0 && yy < g.ny) {
      const int j = yy * g.nx + xx;
      vv = wv(ld_plain(v + j));
      if (!virt) {
        bb1 = ld_plain(b1 + j);
        bb2 = ld_plain(b2 + j);
      }
      f = g.mask == nullptr || g.mask[j] == 0;
    }
    S.v[ey][ex] = vv;
    S.b1[ey][ex] = virt ? wscale(c1v, vv) : bb1;
    S.b2[ey][ex] = bb2;
    S.fr[ey][ex] = f;
  }
  __syncthreads();
  W (*cur1)[HSX] = S.b1;
  W (*cur2)[HSX] = S.b2;
  T res = T(0);
  for (int st = 0; st < ns; ++st) {
    const int kk = k - st;
    const W ck = wc<W>(__ldg(A.coef + kk));
    const W sc = wc<W>(kk == 0 ? A.inv_delta : g.two_over_delta);
    if (st < ns - 1) {
      // b_kk on the tile and an (ns - 1 - st)-cell halo, into cur2's array
      const int h = ns - 1 - st;
      const int rx = HBX + 2 * h, ry = HBY + 2 * h;
      for (int idx = tid; idx < rx * ry; idx += HLT) {
        const int yy = idx / rx, xx = idx - yy * rx;
        const int ey = H - h + yy, ex = H - h + xx;
        W val = wzero<W>();
        if (S.fr[ey][ex]) {
          const W bc = cur1[ey][ex];
          W Ab = bc;
          if (S.fr[ey][ex - 1]) Ab = nb_term(Ab, cx, bc, cur1[ey][ex - 1]);
          if (S.fr[ey][ex + 1]) Ab = nb_term(Ab, cx, bc, cur1[ey][ex + 1]);
          if (S.fr[ey - 1][ex]) Ab = nb_term(Ab, cy, bc, cur1[ey - 1][ex]);
          if (S.fr[ey + 1][ex]) Ab = nb_term(Ab, cy, bc, cur1[ey + 1][ex]);
          val = cl_value(ck, S.v[ey][ex], sc, Ab, theta, bc, cur2[ey][ex]);
        }
        cur2[ey][ex] = val;
      }
      __syncthreads();
      W (*tmp)[HSX] = cur2;
      cur2 = cur1;
      cur1 = tmp;
    } else {
      // the last step, on the tile: written out, or closed into the epilogue
      const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
      if (threadIdx.y < HBY && x < g.nx && y < g.ny) {
        const int i = y * g.nx + x;
        const int ey = H + threadIdx.y, ex = H + threadIdx.x;
        W r = wzero<W>();
        if (S.fr[ey][ex]) {
          const W bc = cur1[ey][ex];
          W Ab = bc;
          if (S.fr[ey][ex - 1]) Ab = nb_term(Ab, cx, bc, cur1[ey][ex - 1]);
          if (S.fr[ey][ex + 1]) Ab = nb_term(Ab, cx, bc, cur1[ey][ex + 1]);
          if (S.fr[ey - 1][ex]) Ab = nb_term(Ab, cy, bc, cur1[ey - 1][ex]);
          if (S.fr[ey + 1][ex]) Ab = nb_term(Ab, cy, bc, cur1[ey + 1][ex]);
          r = cl_value(ck, S.v[ey][ex], sc, Ab, theta, bc, cur2[ey][ex]);
        }
        if (kk == 0) {
          heat_close_cell<T, EK>(A, app, i, close_out<T>(r), have_prev, res, bad);
        } else {
          o_new[i] = r;
          o_prev[i] = S.fr[ey][ex] ? cur1[ey][ex] : wzero<W>();
        }
      }
    }
  }
  if (k - ns + 1 == 0 && app == 0) {
    const double tot = block_sum((double)res, s_red);
    if (tid == 0) A.part[t] = tot;
  }
  __syncthreads();   // the staging is reused by the next tile
}

template <typename T, int EK>
__global__ void __launch_bounds__(HLT) heat_loop_kernel(HeatLoopArgs<T> A) {
  using W = typename HeatIter<T>::W;
  __shared__ HeatStageH<W> stg;
  __shared__ double s_red[33];
  __shared__ int s_stop, s_fault, s_it0, s_maxit;
  __shared__ unsigned s_base;
  __shared__ double s_tol;
  const int tid = threadIdx.y * HBX + threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const unsigned G = gridDim.x;
  Ctrl* ctrl = A.ctrl;
  if (tid == 0) {
    const int done = *(volatile int*)&ctrl->done;
    const int nonfinite = *(volatile int*)&ctrl->nonfinite;
    s_stop = (done != RUNNING || nonfinite) ? 1 : 0;
    if (done == RUNNING && nonfinite && blockIdx.x == 0) ctrl->done = NONFINITE;
    s_it0 = ctrl->it;
    s_maxit = ctrl->max_iter;
    s_tol = ctrl->tol;
    s_base = ctrl->bar_base;
    s_fault = 0;
  }
  __syncthreads();
  if (s_stop) return;
  unsigned nbar = 0;
  int bad = 0;
  int pairs_done = 0;
  // grid barrier of every thread of the block; false: the loop stops here
  // The flag slot of barrier b is final once b is complete; thread 0 loads it
  // then and acts on it at barrier b + 1 (the load stays off the path to the
  // next phase), so every block stops at the same barrier.
  unsigned flag_prev = 0;
  auto barrier = [&]() -> bool {
    bad = __syncthreads_or(bad);
    if (tid == 0) {
      if (bad) atomicOr(&ctrl->nonfinite, 1);
      const unsigned b = s_base + (++nbar);
      const bool ok = grid_barrier(ctrl, G, b, bad != 0 || s_fault != 0);
      if (!ok) {
        s_fault = 1;
        atomicOr(&ctrl->nonfinite, 2);
      }
      const int stop = flag_prev != 0 || !ok;
      if (stop && blockIdx.x == 0) ctrl->done = NONFINITE;
      s_stop = stop;
      flag_prev = *(volatile unsigned*)&ctrl->bar_flag[b % 3];
      if (blockIdx.x == 0) ctrl->bar_flag[(b + 2) % 3] = 0u;
    }
    bad = 0;
    __syncthreads();
    return s_stop == 0;
  };
  const int D = A.D;
  bool run = true;
  for (int pair = 0; pair < A.pairs && run; ++pair) {
    const int it = s_it0 + pair;
    for (int app = 0; app < 2 && run; ++app) {
      if (app == 1) {
        // stop rule from the b-update's partials, in stop_gate's order
        if (wid == 0) {
          double v = 0.0;
          for (int i = lane; i < A.ntiles; i += 32) v += ld_plain(A.part + i);
          v = warp_sum(v);
          const bool first = lane == 0 && blockIdx.x == 0;
          int d = RUNNING;
          if (it > 0 && !isfinite(v)) d = NONFINITE;
          else if (it > 0 && v <= s_tol) d = CONVERGED;
          else if (it >= s_maxit) d = MAX_ITER;
          else if (stall_rule(ctrl, it, v, first)) d = STALLED;
          if (first) {
            if (it > 0) ctrl->res_last = v;
            if (d != RUNNING) ctrl->done = d;
          }
          if (lane == 0) s_stop = d != RUNNING;
        }
        __syncthreads();
        if (s_stop) { run = false; break; }
      }
      const T* v = app == 0 ? A.a : A.b;
      const bool have_prev = app == 0 && it > 0;
      const W cD = wc<W>(__ldg(A.coef + D));
      const W cx = wc<W>(A.g.cx), cy = wc<W>(A.g.cy), theta = wc<W>(A.theta);
      W* dd[4] = {(W*)A.d[0], (W*)A.d[1], (W*)A.d[2], (W*)A.d[3]};
      // phases of up to HMAX steps from the first iterates (b_D = c_D v,
      // b_{D+1} = 0), the first one taking D mod HMAX steps; buffers: read
      // the newest / previous iterates from d[r1] / d[r2], write d[f1] / d[f2]
      int r1 = 0, r2 = 1, f1 = 2, f2 = 3;
      const int hm = A.steps;   // Clenshaw steps per phase (<= HMAX)
      int k = D - 1;
      int ns = D % hm == 0 ? hm : D % hm;
      bool virt = true;
      while (k >= 0) {
        for (int t = blockIdx.x; t < A.ntiles; t += G)
          heat_tile_steps<T, EK, W>(A, app, t, v, virt ? nullptr : dd[r1], virt ? nullptr : dd[r2],
                                    dd[f1], dd[f2], virt, cD, k, ns, have_prev, stg, cx, cy, theta,
                                    s_red, bad);
        if (!barrier()) { run = false; break; }
        k -= ns;
        ns = hm;
        virt = false;
        const int o1 = r1, o2 = r2;
        r1 = f1;
        r2 = f2;
        f1 = o1;
        f2 = o2;
      }
    }
    if (run) pairs_done = pair + 1;
  }
  if (tid == 0 && blockIdx.x == 0) {
    ctrl->it = s_it0 + pairs_done;
    ctrl->bar_base = s_base + nbar;   // every block crossed the same barriers
  }
}

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
// 1 + ceil(D / 2) launches.  `linear`: the output is not clamped at 0 (the
// adjoint applies xi~ to signed vectors).
template <typename T>
cudaError_t heat_apply(const HeatPlan& hp, const HeatBuffers& B, const T* in, T* out_x,
                       int nx, int ny, const uint8_t* mask, Ctrl* ctrl, const double* part,
                       int nparts, int decide, cudaStream_t st, bool linear) {
  const double inv_delta = hp.delta > 0 ? 1.0 / hp.delta : 0.0;   // delta = 0: p(A) = c_0 Id
  HeatGeom g{nx, ny, hp.cx, hp.cy, mask, 2.0 * inv_delta, linear};
  const dim3 grid = heat_grid(nx, ny), block(HBX, HBY);
  void* d[4] = {B.d[0], B.d[1], B.d[2], B.d[3]};   // iterates (8 bytes per cell)
  const int D = hp.D;
  // b_{k+1} in d[r1], b_{k+2} in d[r2]; d[f1], d[f2] free
  int r1 = 0, r2 = 1, f1 = 2, f2 = 3;
  heat_cl_init<T><<<grid, block, 0, st>>>(in, d[r1], d[r2], g, hp.coef[D], ctrl, part, nparts,
                                          decide);
  int k = D - 1;
  if (D % 2 == 1) {   // one single step so that the rest pairs up
    if (k == 0) {
      heat_cl_step<T, true><<<grid, block, 0, st>>>(in, d[r1], d[r2], out_x, g, hp.coef[0],
                                                    inv_delta, hp.theta, ctrl);
      return cudaGetLastError();
    }
    heat_cl_step<T, false><<<grid, block, 0, st>>>(in, d[r1], d[r2], d[r2], g, hp.coef[k],
                                                   2.0 * inv_delta, hp.theta, ctrl);
    std::swap(r1, r2);
    --k;
  }
  for (; k >= 1; k -= 2) {
    if (k == 1) {   // steps 1 and the closing 0
      heat_cl_step2<T, true><<<grid, block, 0, st>>>(in, d[r1], d[r2], d[f1], out_x, g, hp.coef[1],
                                                     hp.coef[0], inv_delta, hp.theta, ctrl);
      break;
    }
    heat_cl_step2<T, false><<<grid, block, 0, st>>>(in, d[r1], d[r2], d[f1], d[f2], g,
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

namespace {
template <typename T>
void* heat_loop_fn(int ek) {
  if (ek == EK_CROWD) return (void*)heat_loop_kernel<T, EK_CROWD>;
  if (ek == EK_ENTROPY) return (void*)heat_loop_kernel<T, EK_ENTROPY>;
  return (void*)heat_loop_kernel<T, EK_POWER>;
}
}  // namespace

// Blocks of the persistent form: one per 16x8 tile, at most 4 per SM and as
// many as can be co-resident (a cooperative launch); 0 where the device has
// no cooperative launch.
int heat_loop_grid(int nx, int ny, bool fp64, int ek) {
  int dev = 0, coop = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (!coop || sms <= 0) return 0;
  void* fn = fp64 ? heat_loop_fn<double>(ek) : heat_loop_fn<float>(ek);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, HLT, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const long long cap = (long long)std::min(per_sm, 4) * sms;
  const long long tiles = heat_blocks(nx, ny);
  return (int)std::min(cap, tiles);
}

template <typename T>
cudaError_t heat_loop_launch(const HeatPlan& hp, const HeatBuffers& B, int ek, const T* q, T* a,
                             T* b, T* p, int nx, int ny, const uint8_t* mask, const ProxArgs<T>& P,
                             Ctrl* ctrl, double* part, int G, int pairs, cudaStream_t st) {
  HeatLoopArgs<T> A{};
  const double inv_delta = hp.delta > 0 ? 1.0 / hp.delta : 0.0;
  A.g = HeatGeom{nx, ny, hp.cx, hp.cy, mask, 2.0 * inv_delta};
  A.coef = (const double*)B.coef;
  A.D = hp.D;
  A.theta = hp.theta;
  A.inv_delta = inv_delta;
  for (int i = 0; i < 4; ++i) A.d[i] = B.d[i];
  A.q = q;
  A.a = a;
  A.b = b;
  A.p = p;
  A.P = P;
  A.ctrl = ctrl;
  A.part = part;
  const dim3 tg = heat_grid(nx, ny);
  A.tiles_x = (int)tg.x;
  A.ntiles = (int)(tg.x * tg.y);
  A.pairs = pairs;
  // four steps per barrier while every tile has its own block (the barriers
  // dominate), two where blocks take several tiles (the recomputed halo's
  // FP64 work would)
  A.steps = A.ntiles <= G ? HMAX : 2;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)G);
  cfg.blockDim = dim3(HBX, HLT / HBX);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (ek == EK_CROWD) return cudaLaunchKernelEx(&cfg, heat_loop_kernel<T, EK_CROWD>, A);
  if (ek == EK_ENTROPY) return cudaLaunchKernelEx(&cfg, heat_loop_kernel<T, EK_ENTROPY>, A);
  return cudaLaunchKernelEx(&cfg, heat_loop_kernel<T, EK_POWER>, A);
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
                                     cudaStream_t, bool);                                     \
  template cudaError_t heat_bupdate_launch<T>(const T*, T*, const T*, int, int, Ctrl*,        \
                                              double*, cudaStream_t);                         \
  template cudaError_t heat_prox_launch<T>(int, const T*, T*, T*, int, int,                   \
                                           const ProxArgs<T>&, Ctrl*, cudaStream_t);           \
  template cudaError_t heat_loop_launch<T>(const HeatPlan&, const HeatBuffers&, int, const T*, \
                                           T*, T*, T*, int, int, const uint8_t*,               \
                                           const ProxArgs<T>&, Ctrl*, double*, int, int,       \
                                           cudaStream_t);
JKO_HEAT_INST(float)
JKO_HEAT_INST(double)
#undef JKO_HEAT_INST

}  // namespace jko
