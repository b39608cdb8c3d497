// jko_api.cu -- the C ABI of libjko (include/jko.h): handle set-up, the JKO
// step driver and the flow.
//
// One step (Eq. def-jko-operator) is the scaling loop of Prop. 3.3 in its
// 2-vector form.  Per (odd, even) pair the device runs four kernels:
//   pass y of xi a ; pass x of xi a fused with  b = q / xi a  and the residual
//   of the previous pair (stopping rule of Sec. 3.4) ;
//   pass y of xi b ; pass x of xi b fused with  p = Prox(s), a = p / s.
// A chunk of `check_every` pairs is captured once as a CUDA graph.  A step
// launches the number of chunks the last step needed with the finalisation
// behind the last one and waits once; only a longer step polls on, with one
// chunk in flight; kernels launched after the stop return at once.  In a flow
// the steps after the first run their chunks as a device-side loop (a graph
// WHILE node) and are enqueued without a wait between them.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "jko.h"
#include "jko_handle.h"
#include "jko_kernels.h"
#include "tc_gemm.h"

using jko::Ctrl;
using jko::PassArgs;
using jko::ProxArgs;

namespace {

thread_local std::string g_create_err;

jko_status set_err(jko_handle* h, jko_status st, const std::string& msg) {
  if (h) h->err = msg; else g_create_err = msg;
  return st;
}

jko_status cuda_err(jko_handle* h, cudaError_t e, const char* what) {
  std::string msg = std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                    cudaGetErrorString(e) + ")";
  return set_err(h, e == cudaErrorMemoryAllocation ? JKO_ERR_OOM : JKO_ERR_CUDA, msg);
}

#define CK(h, call)                                   \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_err(h, e_, #call); \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

// 1-D Gibbs factor along one axis (Sec. 4.1): k(d) = exp(-(d h)^2 / gamma),
// d = 0..n-1.  r = largest d whose tap is non-zero in the working precision, so
// dropping |d| > r changes nothing in that precision.  Returns the centred,
// zero-padded tap vector of length 2r + 1 + pad as doubles.
std::vector<double> gibbs_taps(int n, double length, double gamma, bool fp64, int pad, int* r_out) {
  const double h = length / n;
  std::vector<double> k(n);
  int r = 0;
  for (int d = 0; d < n; ++d) {
    k[d] = std::exp(-(d * h) * (d * h) / gamma);
    const bool nz = fp64 ? (k[d] != 0.0) : ((float)k[d] != 0.0f);
    if (nz) r = d;
  }
  std::vector<double> t(2 * r + 1 + pad, 0.0);
  for (int i = 0; i <= 2 * r; ++i) t[i] = k[std::abs(i - r)];
  *r_out = r;
  return t;
}

template <typename T>
cudaError_t upload(void** dst, const std::vector<double>& src) {
  std::vector<T> tmp(src.begin(), src.end());
  cudaError_t e = cudaMalloc(dst, sizeof(T) * tmp.size());
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, tmp.data(), sizeof(T) * tmp.size(), cudaMemcpyHostToDevice);
}


// The FFT tables of the pass along x (filtering lines of length nx) or y.
template <typename T>
jko::FftArgs<T> fft_args(const jko_handle* h, bool along_x) {
  jko::FftArgs<T> F;
  F.L = along_x ? h->fft_Lx : h->fft_Ly;
  F.log2L = along_x ? h->fft_lgx : h->fft_lgy;
  F.khat = (const T*)(along_x ? h->fft_khat_x : h->fft_khat_y);
  F.tw = (const T*)(along_x ? h->fft_tw_x : h->fft_tw_y);
  return F;
}

// Pass `which` of one (odd, even) pair in the SIMT form, on stream st:
//   0: pass along y of xi a          1: pass along x of xi a + b-update/residual
//   2: pass along y of xi b          3: pass along x of xi b + prox/a-update
template <typename T>
cudaError_t enqueue_pass_simt(jko_handle* h, int which, cudaStream_t st) {
  const int nx = h->grid.nx, ny = h->grid.ny;
  ProxArgs<T> P = jko::prox_args<T>(h);
  PassArgs<T> A{};
  A.ctrl = h->ctrl;
  A.part = h->part;
  A.nparts = h->nparts_simt;
  A.decide = which == 2 ? 1 : 0;  // the pass after the b-update takes the stop decision
  A.latency = h->simt_latency;
  const int half = which >> 1;
  if ((which & 1) == 0) {
    // pass along y: in [ny][nx] -> t1 [nx][ny]
    A.in = (const T*)(half == 0 ? h->a : h->b);
    A.out = (T*)h->t1;
    A.taps = (const T*)h->taps_y;
    A.n_i = ny; A.n_j = nx; A.r = h->ry;
    if (h->fft) return jko::fft_pass<T>(jko::EPI_STORE, h->ek, A, P, fft_args<T>(h, false), st);
    return jko::simt_pass<T>(jko::EPI_STORE, h->ek, A, P, st);
  }
  // pass along x with the epilogue: in [nx][ny] -> [ny][nx]
  A.in = (const T*)h->t1;
  A.out = (T*)(half == 0 ? h->b : h->a);
  A.p = (T*)h->p;
  A.q = (const T*)h->q;
  A.taps = (const T*)h->taps_x;
  A.n_i = nx; A.n_j = ny; A.r = h->rx;
  if (h->fft)
    return jko::fft_pass<T>(half == 0 ? jko::EPI_B : jko::EPI_A, h->ek, A, P, fft_args<T>(h, true), st);
  return jko::simt_pass<T>(half == 0 ? jko::EPI_B : jko::EPI_A, h->ek, A, P, st);
}

// One filter pass of the CUDA-core form with explicit buffers: along y
// ([ny][nx] -> [nx][ny]) or along x ([nx][ny] -> [ny][nx]).
template <typename T>
cudaError_t simt_pass_on(jko_handle* h, bool along_y, int epi, const void* in, void* out,
                         const void* q, double* part, int decide, int nparts, cudaStream_t st) {
  const int nx = h->grid.nx, ny = h->grid.ny;
  PassArgs<T> A{};
  A.ctrl = h->ctrl;
  A.part = part;
  A.nparts = nparts;
  A.decide = decide;
  A.latency = h->simt_latency;
  A.in = (const T*)in;
  A.out = (T*)out;
  A.q = (const T*)q;
  A.p = (T*)h->p;
  A.taps = (const T*)(along_y ? h->taps_y : h->taps_x);
  A.n_i = along_y ? ny : nx;
  A.n_j = along_y ? nx : ny;
  A.r = along_y ? h->ry : h->rx;
  if (h->fft) return jko::fft_pass<T>(epi, h->ek, A, jko::prox_args<T>(h), fft_args<T>(h, !along_y), st);
  return jko::simt_pass<T>(epi, h->ek, A, jko::prox_args<T>(h), st);
}

// One batched filter pass over n images of the grid (n <= 3): along y or x,
// in[m] -> out[m], one launch (blockIdx.z = m); the same arithmetic per block as
// n separate passes.  EPI_STORE, or EPI_B against q[m] with the partials of
// image m at part + m * (blocks per image).
template <typename T>
cudaError_t simt_pass_multi(jko_handle* h, bool along_y, int n, void* const* in, void* const* out,
                            int decide, int nparts, cudaStream_t st, int epi = jko::EPI_STORE,
                            const void* const* q = nullptr) {
  const int nx = h->grid.nx, ny = h->grid.ny;
  PassArgs<T> A{};
  A.ctrl = h->ctrl;
  A.part = h->part;
  A.nparts = nparts;
  A.decide = decide;
  A.latency = h->simt_latency;
  A.nz = n;
  for (int m = 0; m < n; ++m) {
    A.in_z[m] = (const T*)in[m];
    A.out_z[m] = (T*)out[m];
    A.q_z[m] = q ? (const T*)q[m] : nullptr;
  }
  A.in = A.in_z[0];
  A.out = A.out_z[0];
  A.q = A.q_z[0];
  A.p = (T*)h->p;
  A.taps = (const T*)(along_y ? h->taps_y : h->taps_x);
  A.n_i = along_y ? ny : nx;
  A.n_j = along_y ? nx : ny;
  A.r = along_y ? h->ry : h->rx;
  if (h->fft) {
    // the FFT form: one launch per image, the b-update partials of image m at
    // part + m * (blocks per image), the stop decision taken by image 0's launch
    // (the later launches find it recorded)
    const jko::FftArgs<T> F = fft_args<T>(h, !along_y);
    const int nb = jko::fft_pass_blocks(A.n_j);
    for (int m = 0; m < n; ++m) {
      PassArgs<T> Am = A;
      Am.nz = 1;
      Am.in = A.in_z[m];
      Am.out = A.out_z[m];
      Am.q = A.q_z[m];
      Am.part = epi == jko::EPI_B ? h->part + (size_t)m * nb : h->part;
      Am.decide = m == 0 ? decide : 0;
      cudaError_t e = jko::fft_pass<T>(epi, h->ek, Am, jko::prox_args<T>(h), F, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  return jko::simt_pass<T>(epi, h->ek, A, jko::prox_args<T>(h), st);
}

// One iteration of the Wasserstein attraction (Sec. 5.2, attraction.cu): the
// b-updates of both couplings with their residual partials (the next pass
// adds both sets for the stop rule), xi b_1 and xi b_2, then the joint prox.
template <typename T>
cudaError_t enqueue_pair_attraction(jko_handle* h, cudaStream_t st) {
  const int nb = h->nparts_simt;
  cudaError_t e;
  void* as[2] = {h->a, h->a2};
  void* bs[2] = {h->b, h->b2};
  void* ts[2] = {h->t1, h->t2};
  void* ss[2] = {h->s1, h->s2};
#define JKO_TRY(x) do { e = (x); if (e != cudaSuccess) return e; } while (0)
  const void* qs[2] = {h->q, h->tgt};
  JKO_TRY(simt_pass_multi<T>(h, true, 2, as, ts, 0, nb, st));
  JKO_TRY(simt_pass_multi<T>(h, false, 2, ts, bs, 0, nb, st, jko::EPI_B, qs));
  JKO_TRY(simt_pass_multi<T>(h, true, 2, bs, ts, 1, 2 * nb, st));
  JKO_TRY(simt_pass_multi<T>(h, false, 2, ts, ss, 0, nb, st));
#undef JKO_TRY
  return jko::launch_attraction_prox<T>(h->ek, (const T*)h->s1, (const T*)h->s2, (T*)h->a,
                                        (T*)h->a2, (T*)h->p, h->N, h->prm.tau,
                                        jko::prox_args<T>(h), h->ctrl, st);
}

// Start of an attraction step: b_1 = b_2 = 1, then the first joint prox from
// s_1 = s_2 = xi 1 (the generic scaling's first half-step, Prop.
// prop-implementation-generic, with a = b = 1).
template <typename T>
cudaError_t begin_attraction(jko_handle* h, cudaStream_t st) {
  const long long N = h->N;
  cudaError_t e = jko::launch_fill<T>((T*)h->b, T(1), N, st);
  if (e == cudaSuccess) e = jko::launch_fill<T>((T*)h->b2, T(1), N, st);
  if (e == cudaSuccess)
    e = simt_pass_on<T>(h, true, jko::EPI_STORE, h->b, h->t1, nullptr, h->part, 0, 1, st);
  if (e == cudaSuccess)
    e = simt_pass_on<T>(h, false, jko::EPI_STORE, h->t1, h->s1, nullptr, h->part, 0, 1, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->s2, h->s1, sizeof(T) * (size_t)N, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess)
    e = jko::launch_attraction_prox<T>(h->ek, (const T*)h->s1, (const T*)h->s2, (T*)h->a,
                                       (T*)h->a2, (T*)h->p, N, h->prm.tau,
                                       jko::prox_args<T>(h), h->ctrl, st);
  return e;
}

// Two species (Sec. 5.3): b_1 = q_1 / xi a_1, b_2 = q_2 / xi a_2 with their
// residual partials, xi b_1, xi b_2, then the joint prox on the sum.
template <typename T>
cudaError_t enqueue_pair_species(jko_handle* h, cudaStream_t st) {
  const int nb = h->nparts_simt;
  const T* q2 = (const T*)h->q + h->N;
  cudaError_t e;
  void* as[2] = {h->a, h->a2};
  void* bs[2] = {h->b, h->b2};
  void* ts[2] = {h->t1, h->t2};
  void* ss[2] = {h->s1, h->s2};
#define JKO_TRY(x) do { e = (x); if (e != cudaSuccess) return e; } while (0)
  const void* qs[2] = {h->q, q2};
  JKO_TRY(simt_pass_multi<T>(h, true, 2, as, ts, 0, nb, st));
  JKO_TRY(simt_pass_multi<T>(h, false, 2, ts, bs, 0, nb, st, jko::EPI_B, qs));
  JKO_TRY(simt_pass_multi<T>(h, true, 2, bs, ts, 1, 2 * nb, st));
  JKO_TRY(simt_pass_multi<T>(h, false, 2, ts, ss, 0, nb, st));
#undef JKO_TRY
  return jko::launch_species_prox<T>((const T*)h->s1, (const T*)h->s2, (const T*)h->E,
                                     (const T*)h->E2, (T*)h->a, (T*)h->a2, (T*)h->p, h->N,
                                     h->kappa_s, h->has_kappa, h->ctrl, st);
}

// Start of a two-species step: b_1 = b_2 = 1, the first joint prox from
// s_1 = s_2 = xi 1.
template <typename T>
cudaError_t begin_species(jko_handle* h, cudaStream_t st) {
  const long long N = h->N;
  cudaError_t e = jko::launch_fill<T>((T*)h->b, T(1), N, st);
  if (e == cudaSuccess) e = jko::launch_fill<T>((T*)h->b2, T(1), N, st);
  if (e == cudaSuccess)
    e = simt_pass_on<T>(h, true, jko::EPI_STORE, h->b, h->t1, nullptr, h->part, 0, 1, st);
  if (e == cudaSuccess)
    e = simt_pass_on<T>(h, false, jko::EPI_STORE, h->t1, h->s1, nullptr, h->part, 0, 1, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->s2, h->s1, sizeof(T) * (size_t)N, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess)
    e = jko::launch_species_prox<T>((const T*)h->s1, (const T*)h->s2, (const T*)h->E,
                                    (const T*)h->E2, (T*)h->a, (T*)h->a2, (T*)h->p, N,
                                    h->kappa_s, h->has_kappa, h->ctrl, st);
  return e;
}

// One iteration of the pairwise attraction of two densities (Sec. 5.3, 3
// couplings, attraction.cu): s_m = xi b_m for m = 1, 2, 3 (the first filter
// pass takes the stop decision on the partials of the previous column
// half-step), the row prox; y_m = xi a_m (xi is symmetric), the column prox
// with the residual partials, p_2 and the pair counter.
template <typename T>
cudaError_t enqueue_pair_pairwise(jko_handle* h, cudaStream_t st) {
  const int nb = h->nparts_pw;
  const long long N = h->N;
  const T* q1 = (const T*)h->q;
  T* p1 = (T*)h->p;
  const double t = h->prm.tau * h->pair_alpha;
  void* bs[3] = {h->b, h->b2, h->b3};
  void* as[3] = {h->a, h->a2, h->a3};
  void* ss[3] = {h->s1, h->s2, h->s3};
  cudaError_t e;
  void* ts[3] = {h->t1, h->t2, h->t3};
#define JKO_TRY(x) do { e = (x); if (e != cudaSuccess) return e; } while (0)
  JKO_TRY(simt_pass_multi<T>(h, true, 3, bs, ts, 1, nb, st));
  JKO_TRY(simt_pass_multi<T>(h, false, 3, ts, ss, 0, nb, st));
  JKO_TRY(jko::launch_pairwise_rows<T>((const T*)h->s1, (const T*)h->s2, (const T*)h->s3,
                                       (const T*)h->E, q1 + N, (T*)h->a, (T*)h->a2, (T*)h->a3,
                                       p1, N, t, h->kappa_s, h->has_kappa, h->ctrl, st));
  JKO_TRY(simt_pass_multi<T>(h, true, 3, as, ts, 0, nb, st));
  JKO_TRY(simt_pass_multi<T>(h, false, 3, ts, ss, 0, nb, st));
#undef JKO_TRY
  return jko::launch_pairwise_cols<T>((const T*)h->s1, (const T*)h->s2, (const T*)h->s3,
                                      (const T*)h->E2, q1, (T*)h->b, (T*)h->b2, (T*)h->b3,
                                      p1 + N, h->part, N, t, h->kappa_s, h->has_kappa, h->ctrl,
                                      st);
}

// Start of a pairwise-attraction step: b_m = 1 (Prop. prop-implementation-generic).
template <typename T>
cudaError_t begin_pairwise(jko_handle* h, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (void* b : {h->b, h->b2, h->b3})
    if (e == cudaSuccess) e = jko::launch_fill<T>((T*)b, T(1), h->N, st);
  return e;
}

// ---- the steps with several couplings on the tensor cores (tc_multi.cu) ----
// The same iterations as above with each filter pair replaced by the
// tensor-core passes over x then y (xi is separable and symmetric, so the
// order changes the rounding only).  TF32: the scalings that feed them are
// rounded to tf32 by the joint prox kernels.  BF16 / BF16x3: the scalings stay
// fp32 and each application of xi first splits its nz images into bf16 pairs
// (h->mpair); the intermediates are pairs.  xi b_m goes to the prox as fp32.

// rnd argument of the joint prox kernels for this handle's tensor-core form
int multi_rnd(const jko_handle* h) { return jko::tc_mode(h->tc) == 2 ? 1 : 0; }

// xi applied to nz images: in -> out, through the intermediates ts; the
// second pass's epilogue `epi` (EPI_B against q, or TC_EPI_RAW); the first
// pass takes the stop decision on `nparts` partials when decide = 1.
cudaError_t tc_xi_multi(jko_handle* h, int nz, void* const* in, void* const* out, int epi,
                        const void* const* q, int decide, int nparts, cudaStream_t st) {
  void* ts[3] = {h->t1, h->t2, h->t3};
  const void* ops[3] = {in[0], nz > 1 ? in[1] : in[0], nz > 2 ? in[2] : in[0]};
  if (h->mpair) {
    // BF16 / BF16x3: the operand pairs of the first pass, 4 bytes per cell each
    void* pairs[3];
    for (int z = 0; z < 3; ++z) pairs[z] = (unsigned char*)h->mpair + (size_t)z * 4 * h->N;
    cudaError_t e = jko::tc_split_pairs(nz, (const float* const*)in, pairs, h->N, st);
    if (e != cudaSuccess) return e;
    for (int z = 0; z < 3; ++z) ops[z] = pairs[z];
  }
  cudaError_t e = jko::tc_multi_pass(h->tc, 0, nz, ops, ts, jko::EPI_STORE, nullptr, h->part,
                                     nparts, decide, st);
  if (e != cudaSuccess) return e;
  return jko::tc_multi_pass(h->tc, 1, nz, (const void* const*)ts, out, epi,
                            (const float* const*)q, h->part, 0, 0, st);
}

cudaError_t enqueue_pair_attraction_tc(jko_handle* h, cudaStream_t st) {
  const int nb = jko::tc_multi_tiles(h->grid.nx, h->grid.ny, 1);
  void* as[2] = {h->a, h->a2};
  void* bs[2] = {h->b, h->b2};
  void* ss[2] = {h->s1, h->s2};
  const void* qs[2] = {h->q, h->tgt};
  cudaError_t e = tc_xi_multi(h, 2, as, bs, jko::EPI_B, qs, 0, 0, st);
  if (e == cudaSuccess) e = tc_xi_multi(h, 2, bs, ss, jko::TC_EPI_RAW, nullptr, 1, 2 * nb, st);
  if (e != cudaSuccess) return e;
  return jko::launch_attraction_prox<float>(h->ek, (const float*)h->s1, (const float*)h->s2,
                                            (float*)h->a, (float*)h->a2, (float*)h->p, h->N,
                                            h->prm.tau, jko::prox_args<float>(h), h->ctrl, st, multi_rnd(h));
}

cudaError_t enqueue_pair_species_tc(jko_handle* h, cudaStream_t st) {
  const int nb = jko::tc_multi_tiles(h->grid.nx, h->grid.ny, 1);
  void* as[2] = {h->a, h->a2};
  void* bs[2] = {h->b, h->b2};
  void* ss[2] = {h->s1, h->s2};
  const void* qs[2] = {h->q, (const float*)h->q + h->N};
  cudaError_t e = tc_xi_multi(h, 2, as, bs, jko::EPI_B, qs, 0, 0, st);
  if (e == cudaSuccess) e = tc_xi_multi(h, 2, bs, ss, jko::TC_EPI_RAW, nullptr, 1, 2 * nb, st);
  if (e != cudaSuccess) return e;
  return jko::launch_species_prox<float>((const float*)h->s1, (const float*)h->s2,
                                         (const float*)h->E, (const float*)h->E2, (float*)h->a,
                                         (float*)h->a2, (float*)h->p, h->N, h->kappa_s,
                                         h->has_kappa, h->ctrl, st, multi_rnd(h));
}

cudaError_t enqueue_pair_pairwise_tc(jko_handle* h, cudaStream_t st) {
  const long long N = h->N;
  const float* q1 = (const float*)h->q;
  float* p1 = (float*)h->p;
  const double t = h->prm.tau * h->pair_alpha;
  void* bs[3] = {h->b, h->b2, h->b3};
  void* as[3] = {h->a, h->a2, h->a3};
  void* ss[3] = {h->s1, h->s2, h->s3};
  cudaError_t e = tc_xi_multi(h, 3, bs, ss, jko::TC_EPI_RAW, nullptr, 1, h->nparts_pw, st);
  if (e == cudaSuccess)
    e = jko::launch_pairwise_rows<float>((const float*)h->s1, (const float*)h->s2,
                                         (const float*)h->s3, (const float*)h->E, q1 + N,
                                         (float*)h->a, (float*)h->a2, (float*)h->a3, p1, N, t,
                                         h->kappa_s, h->has_kappa, h->ctrl, st, multi_rnd(h));
  if (e == cudaSuccess) e = tc_xi_multi(h, 3, as, ss, jko::TC_EPI_RAW, nullptr, 0, 0, st);
  if (e != cudaSuccess) return e;
  return jko::launch_pairwise_cols<float>((const float*)h->s1, (const float*)h->s2,
                                          (const float*)h->s3, (const float*)h->E2, q1,
                                          (float*)h->b, (float*)h->b2, (float*)h->b3, p1 + N,
                                          h->part, N, t, h->kappa_s, h->has_kappa, h->ctrl, st, multi_rnd(h));
}

// Start of an attraction or two-species step on the tensor cores: b_m = 1,
// s_1 = s_2 = xi 1, then the first joint prox.
cudaError_t begin_multi_tc(jko_handle* h, cudaStream_t st) {
  const long long N = h->N;
  cudaError_t e = jko::launch_fill<float>((float*)h->b, 1.0f, N, st);
  if (e == cudaSuccess) e = jko::launch_fill<float>((float*)h->b2, 1.0f, N, st);
  void* bs[1] = {h->b};
  void* ss[1] = {h->s1};
  if (e == cudaSuccess) e = tc_xi_multi(h, 1, bs, ss, jko::TC_EPI_RAW, nullptr, 0, 0, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->s2, h->s1, sizeof(float) * (size_t)N, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  if (h->species == 2)
    return jko::launch_species_prox<float>((const float*)h->s1, (const float*)h->s2,
                                           (const float*)h->E, (const float*)h->E2, (float*)h->a,
                                           (float*)h->a2, (float*)h->p, N, h->kappa_s,
                                           h->has_kappa, h->ctrl, st, multi_rnd(h));
  return jko::launch_attraction_prox<float>(h->ek, (const float*)h->s1, (const float*)h->s2,
                                            (float*)h->a, (float*)h->a2, (float*)h->p, N,
                                            h->prm.tau, jko::prox_args<float>(h), h->ctrl, st, multi_rnd(h));
}

// One iteration with the heat-kernel Gibbs kernel (Sec. 4.1, heat.cu):
// Y = xi~ a, b = q / Y with the residual partials, s = xi~ b (its first kernel
// takes the stop decision), then a = Prox(s) / s.  xi~ is symmetric, so the
// same operator serves xi and xi^T.
template <typename T>
cudaError_t enqueue_pair_heat(jko_handle* h, cudaStream_t st) {
  const int nx = h->grid.nx, ny = h->grid.ny;
  const uint8_t* mask = (const uint8_t*)h->mask;
  const int nb = jko::heat_blocks(nx, ny);
  cudaError_t e;
#define JKO_TRY(x) do { e = (x); if (e != cudaSuccess) return e; } while (0)
  JKO_TRY(jko::heat_apply<T>(h->heat, h->hb, (const T*)h->a, (T*)h->t1, nx, ny, mask, h->ctrl,
                             h->part, nb, 0, st));
  JKO_TRY(jko::heat_bupdate_launch<T>((const T*)h->t1, (T*)h->b, (const T*)h->q, nx, ny, h->ctrl,
                                      h->part, st));
  JKO_TRY(jko::heat_apply<T>(h->heat, h->hb, (const T*)h->b, (T*)h->t1, nx, ny, mask, h->ctrl,
                             h->part, nb, 1, st));
#undef JKO_TRY
  return jko::heat_prox_launch<T>(h->ek, (const T*)h->t1, (T*)h->a, (T*)h->p, nx, ny,
                                  jko::prox_args<T>(h), h->ctrl, st);
}

// kernels one pair launches
long long pair_kernels(const jko_handle* h) {
  if (h->heat_L) return 2LL * jko::heat_launches(h->heat) + 2;
  const long long split = h->mpair ? 2 : 0;   // bf16 forms of several couplings: pair splits
  if (h->pair_alpha > 0) return 6 + split;
  return h->attract || h->species == 2 ? 5 + split : 4;
}

cudaError_t enqueue_pass(jko_handle* h, int which, cudaStream_t st) {
  if (h->tc) return jko::tc_enqueue_pass(h->tc, which, st);
  return h->fp64 ? enqueue_pass_simt<double>(h, which, st) : enqueue_pass_simt<float>(h, which, st);
}

cudaError_t enqueue_pair(jko_handle* h, cudaStream_t st) {
  if (h->heat_L)
    return h->fp64 ? enqueue_pair_heat<double>(h, st) : enqueue_pair_heat<float>(h, st);
  if (h->tc_multi) {
    if (h->pair_alpha > 0) return enqueue_pair_pairwise_tc(h, st);
    return h->species == 2 ? enqueue_pair_species_tc(h, st) : enqueue_pair_attraction_tc(h, st);
  }
  if (h->pair_alpha > 0)
    return h->fp64 ? enqueue_pair_pairwise<double>(h, st) : enqueue_pair_pairwise<float>(h, st);
  if (h->species == 2)
    return h->fp64 ? enqueue_pair_species<double>(h, st) : enqueue_pair_species<float>(h, st);
  if (h->attract)
    return h->fp64 ? enqueue_pair_attraction<double>(h, st) : enqueue_pair_attraction<float>(h, st);
  for (int k = 0; k < 4; ++k) {
    cudaError_t e = enqueue_pass(h, k, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Algorithmic flops of pass `which`: the band-limited separable filter does
// 2 (2r+1) flops per output (taps beyond r are zero in the working precision);
// the tensor-core form reports the multiply-adds of the tiles it executes.
double pass_flops(const jko_handle* h, int which) {
  if (h->tc) return jko::tc_pass_flops(h->tc, which);
  const int r = (which & 1) ? h->rx : h->ry;
  return 2.0 * (2.0 * r + 1.0) * (double)h->N;
}

// `pairs` pairs as one persistent launch: the tensor-core loop kernel, or the
// heat kernel's persistent form.
cudaError_t enqueue_loop(jko_handle* h, int pairs, cudaStream_t st) {
  if (h->tc) return jko::tc_enqueue_loop(h->tc, pairs, st);
  const int nx = h->grid.nx, ny = h->grid.ny;
  const uint8_t* mask = (const uint8_t*)h->mask;
  if (h->fp64)
    return jko::heat_loop_launch<double>(h->heat, h->hb, h->ek, (const double*)h->q, (double*)h->a,
                                         (double*)h->b, (double*)h->p, nx, ny, mask,
                                         jko::prox_args<double>(h), h->ctrl, h->part, h->heat_G,
                                         pairs, st);
  return jko::heat_loop_launch<float>(h->heat, h->hb, h->ek, (const float*)h->q, (float*)h->a,
                                      (float*)h->b, (float*)h->p, nx, ny, mask,
                                      jko::prox_args<float>(h), h->ctrl, h->part, h->heat_G, pairs,
                                      st);
}

jko_status capture_chunk(jko_handle* h) {
  cudaGraph_t g = nullptr;
  CK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  if (h->use_loop) e = enqueue_loop(h, h->chunk_iters, h->cap);
  else
    for (int i = 0; i < h->chunk_iters && e == cudaSuccess; ++i) e = enqueue_pair(h, h->cap);
  cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
  if (h->use_loop && (e != cudaSuccess || e2 != cudaSuccess)) {
    // a chunk is one launch: without a graph it is launched directly
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    h->chunk = nullptr;
    return JKO_OK;
  }
  if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_err(h, e, "capture of the iteration chunk"); }
  CK(h, e2);
  e = cudaGraphInstantiate(&h->chunk, g, 0);
  cudaGraphDestroy(g);
  if (h->use_loop && e != cudaSuccess) {
    cudaGetLastError();
    h->chunk = nullptr;
    return JKO_OK;
  }
  CK(h, e);
  return JKO_OK;
}

// One chunk of check_every pairs on stream st.
cudaError_t launch_chunk(jko_handle* h, cudaStream_t st) {
  if (h->chunk) return cudaGraphLaunch(h->chunk, st);
  return enqueue_loop(h, h->chunk_iters, st);
}

// The FP32 CUDA-core chunk that finishes a stalled tensor-core step: the four
// filter passes of kFinishChunk pairs on the handle's float images, captured
// once.  From the stalled scalings the FP32 form needs one or two pairs, so the
// chunk is short: its passes after the stop are launches that return at once.
constexpr int kFinishChunk = 2;
jko_status capture_finish_chunk(jko_handle* h) {
  cudaGraph_t g = nullptr;
  CK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < kFinishChunk && e == cudaSuccess; ++i)
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = enqueue_pass_simt<float>(h, k, h->cap);
  cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
  if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_err(h, e, "capture of the finish chunk"); }
  CK(h, e2);
  e = cudaGraphInstantiate(&h->chunk_fin, g, 0);
  cudaGraphDestroy(g);
  CK(h, e);
  return JKO_OK;
}

// ---- tile-shape autotuner (tensor-core handles) ----
// A candidate is how the scaling loop runs: the persistent loop kernel, or the
// per-pass kernels with 64- or 128-wide output tiles.
enum Cand : int { CAND_LOOP = 0, CAND_PP64 = 1, CAND_PP128 = 2 };

bool apply_cand(jko_handle* h, int cand) {
  if (cand == CAND_LOOP) {
    if (!jko::tc_loop_supported(h->tc)) return false;
    h->use_loop = 1;
    return jko::tc_set_tile(h->tc, 64) == 0;
  }
  h->use_loop = 0;
  return jko::tc_set_tile(h->tc, cand == CAND_PP128 ? 128 : 64) == 0;
}

// Puts a handle in a running state that never stops (it = 1, tol < 0, no
// budget) with q = 1/N and a = 1, so that timed launches do full work.
cudaError_t prime_for_timing(jko_handle* h, cudaStream_t st) {
  Ctrl c0;
  std::memcpy(&c0, h->ctrl_init, sizeof(Ctrl));
  c0.it = 1;
  c0.tol = -1.0;
  c0.max_iter = 0x7fffffff;
  cudaError_t e = cudaMemcpy(h->ctrl, &c0, sizeof(Ctrl), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = jko::launch_fill<float>((float*)h->q, 1.0f / (float)h->N, h->N, st);
  if (e == cudaSuccess) e = jko::tc_begin_step(h->tc, st);
  return e;
}

// Milliseconds of one replay of `g` (median of three after a warm-up), or a
// negative value on error.
float time_graph(cudaGraphExec_t g, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
  float best[3] = {0, 0, 0};
  if (cudaGraphLaunch(g, st) != cudaSuccess) return -1.f;
  for (int r = 0; r < 3; ++r) {
    if (cudaEventRecord(e0, st) != cudaSuccess || cudaGraphLaunch(g, st) != cudaSuccess ||
        cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&best[r], e0, e1) != cudaSuccess)
      return -1.f;
  }
  std::sort(best, best + 3);
  return best[1];
}

constexpr int kTunePairs = 16;

// Times `pairs` pairs of candidate `cand` on handle h as a captured graph.
float time_cand(jko_handle* h, int cand) {
  if (!apply_cand(h, cand)) return -1.f;
  if (prime_for_timing(h, h->cap) != cudaSuccess) return -1.f;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return -1.f;
  cudaError_t e = cudaSuccess;
  if (cand == CAND_LOOP) e = jko::tc_enqueue_loop(h->tc, kTunePairs, h->cap);
  else
    for (int i = 0; i < kTunePairs && e == cudaSuccess; ++i) e = enqueue_pair(h, h->cap);
  cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
  float ms = -1.f;
  if (e == cudaSuccess && e2 == cudaSuccess && cudaGraphInstantiate(&ge, g, 0) == cudaSuccess)
    ms = time_graph(ge, h->cap, h->ev0, h->ev1);
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  return ms;
}

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, double, double, double, int, int, int>, int> g_tune_cache;

// Picks the fastest candidate for h (cached per device, grid, lengths, gamma,
// precision, energy kind and absorption) and leaves it applied.
jko_status autotune(jko_handle* h, const jko_grid* g, const jko_params* p) {
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_tuple(dev, g->nx, g->ny, g->lx, g->ly, p->gamma, h->prec, h->ek,
                                   jko::tc_absorbed(h->tc));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      apply_cand(h, it->second);
      return JKO_OK;
    }
  }
  int best = -1;
  float best_ms = 0.f;
  for (int cand = CAND_LOOP; cand <= CAND_PP128; ++cand) {
    const float ms = time_cand(h, cand);
    if (ms > 0.f && (best < 0 || ms < best_ms)) { best = cand; best_ms = ms; }
  }
  CK(h, cudaMemcpy(h->ctrl, h->ctrl_init, sizeof(Ctrl), cudaMemcpyHostToDevice));
  if (best < 0) return set_err(h, JKO_ERR_CUDA, "autotuner: no candidate ran");
  apply_cand(h, best);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = best;
  return JKO_OK;
}

void free_handle(jko_handle* h) {
  if (!h) return;
  DeviceGuard dg(h->device);
  if (h->tc) jko::tc_destroy(h->tc);
  if (h->chunk) cudaGraphExecDestroy(h->chunk);
  if (h->chunk_fin) cudaGraphExecDestroy(h->chunk_fin);
  if (h->step_loop) cudaGraphExecDestroy(h->step_loop);
  for (cudaEvent_t ev : h->flow_ev) cudaEventDestroy(ev);
  if (h->flow_ctrl) cudaFreeHost(h->flow_ctrl);
  if (h->flow_ctrl_dev) cudaFree(h->flow_ctrl_dev);
  if (h->chunk_ctr) cudaFree(h->chunk_ctr);
  void* bufs[] = {h->a, h->b, h->t1, h->p, h->q, h->stage_in, h->stage_out, h->taps_x,
                  h->taps_y, h->E, h->sw, h->c, h->kap, h->m1f, h->mask, h->ctrl, h->part,
                  h->a2, h->b2, h->tgt, h->s1, h->s2, h->E2,
                  h->fft_khat_x, h->fft_tw_x, h->fft_khat_y, h->fft_tw_y,
                  h->tape, h->adj, h->adj2, h->adj_red, h->hb.d[0], h->hb.d[1], h->hb.d[2],
                  h->hb.d[3], h->hb.coef, h->a3, h->b3, h->s3, h->t2, h->t3, h->mpair};
  for (void* b : bufs) if (b) cudaFree(b);
  if (h->ctrl_init) cudaFreeHost(h->ctrl_init);
  if (h->poll) cudaFreeHost(h->poll);
  for (auto& e : h->ev_poll) if (e) cudaEventDestroy(e);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->cap) cudaStreamDestroy(h->cap);
  delete h;
}

jko_status validate_create(const jko_grid* g, const jko_params* p, const jko_energy* en) {
  const char* msg = "";
  const jko_status st = jko::check_create_args(g, p, en, &msg);
  return st == JKO_OK ? JKO_OK : set_err(nullptr, st, msg);
}

}  // namespace

namespace jko {
// The argument checks of jko_create, shared with jko_step_noalloc: no
// allocation, no device call; *msg receives a static description.
jko_status check_create_args(const jko_grid* g, const jko_params* p, const jko_energy* en,
                             const char** msg) {
  if (!g || !p || !en) return (*msg = "NULL grid, params or energy", JKO_ERR_INVALID_ARG);
  if (g->nx < 1 || g->ny < 1) return (*msg = "nx, ny must be >= 1", JKO_ERR_INVALID_ARG);
  if ((long long)g->nx * g->ny > (1LL << 30))
    return (*msg = "grid larger than 2^30 cells", JKO_ERR_INVALID_ARG);
  if (!(g->lx > 0) || !(g->ly > 0) || !std::isfinite(g->lx) || !std::isfinite(g->ly))
    return (*msg = "lx, ly must be finite and > 0", JKO_ERR_INVALID_ARG);
  if (!(p->gamma > 0) || !std::isfinite(p->gamma))
    return (*msg = "gamma must be finite and > 0", JKO_ERR_INVALID_ARG);
  if (!(p->tau > 0) || !std::isfinite(p->tau))
    return (*msg = "tau must be finite and > 0", JKO_ERR_INVALID_ARG);
  if (!(p->tol >= 0)) return (*msg = "tol must be >= 0", JKO_ERR_INVALID_ARG);
  if (p->max_iter < 1) return (*msg = "max_iter must be >= 1", JKO_ERR_INVALID_ARG);
  if (p->check_every < 0) return (*msg = "check_every must be >= 0", JKO_ERR_INVALID_ARG);
  if (p->precision < JKO_FP64 || p->precision > JKO_BF16X3)
    return (*msg = "unknown precision", JKO_ERR_INVALID_ARG);
  if (p->loop < 0 || p->loop > 3)
    return (*msg = "loop must be 0 (automatic), 1, 2 or 3", JKO_ERR_INVALID_ARG);
  if (p->tile != 0 && p->tile != 64 && p->tile != 128)
    return (*msg = "tile must be 0 (automatic), 64 or 128", JKO_ERR_INVALID_ARG);
  if (p->absorb < 0 || p->absorb > 3)
    return (*msg = "absorb must be 0 (automatic), 1, 2 or 3", JKO_ERR_INVALID_ARG);
  if (p->absorb == 3) {
    if (p->precision != JKO_TF32)
      return (*msg = "the log-domain form (absorb = 3) runs on JKO_TF32", JKO_ERR_UNSUPPORTED);
    if (en->m != 0.0 || en->m_field || en->binary || en->target || en->species == 2 ||
        g->heat_L || g->fft)
      return (*msg = "the log-domain form serves the congestion / potential energy of one "
                     "density on the Gaussian kernel", JKO_ERR_UNSUPPORTED);
    if (p->loop == 1 || p->loop == 3 || (p->tile != 0 && p->tile != 64) || p->finish)
      return (*msg = "the log-domain form runs its own per-pass kernels (loop 0 or 2, tile 0 "
                     "or 64, no finish)", JKO_ERR_UNSUPPORTED);
  }
  if (p->stall < 0) return (*msg = "stall must be >= 0", JKO_ERR_INVALID_ARG);
  if (p->finish != 0 && p->finish != 1) return (*msg = "finish must be 0 or 1", JKO_ERR_INVALID_ARG);
  if (p->finish && (p->precision == JKO_FP32 || p->precision == JKO_FP64))
    return (*msg = "finish continues a tensor-core step on the FP32 form: tensor-core precisions only",
            JKO_ERR_INVALID_ARG);
  if (p->finish && p->stall < 1)
    return (*msg = "finish takes over where the stall rule stops a step: it needs stall > 0",
            JKO_ERR_INVALID_ARG);
  if (!(en->kappa > 0)) return (*msg = "kappa must be > 0 (INFINITY = none)", JKO_ERR_INVALID_ARG);
  if (!(en->m == 0.0 || en->m >= 1.0) || !std::isfinite(en->m))
    return (*msg = "m must be 0 or >= 1", JKO_ERR_INVALID_ARG);
  if (en->target || en->species == 2) {
    // several couplings: the CUDA-core forms, or the tensor-core passes
    // (tc_multi.cu) on grids whose rows are whole 16-byte units
    if (p->precision == JKO_TF32 || p->precision == JKO_BF16 || p->precision == JKO_BF16X3) {
      const int unit = p->precision == JKO_TF32 ? 4 : 8;
      if (g->nx % unit != 0 || g->ny % unit != 0)
        return (*msg = p->precision == JKO_TF32
                           ? "several couplings on JKO_TF32 need nx and ny multiples of 4"
                           : "several couplings on JKO_BF16 / JKO_BF16X3 need nx and ny "
                             "multiples of 8",
                JKO_ERR_UNSUPPORTED);
      if (p->absorb == 1 || p->absorb == 3 || p->loop == 1 || p->loop == 3 || p->finish ||
          (p->tile != 0 && p->tile != 64))
        return (*msg = "several couplings on the tensor cores run their own passes: absorb 0 or "
                       "2, loop 0 or 2, tile 0 or 64, no finish", JKO_ERR_UNSUPPORTED);
    }
  }
  if (en->target) {
    double tot = 0.0;
    for (long long i = 0; i < (long long)g->nx * g->ny; ++i) {
      const double v = en->target[i];
      if (!(v >= 0) || !std::isfinite(v))
        return (*msg = "target must be finite and >= 0", JKO_ERR_INVALID_ARG);
      if (en->mask && en->mask[i] && v != 0)
        return (*msg = "target must vanish on the mask", JKO_ERR_INVALID_ARG);
      tot += v;
    }
    if (std::fabs(tot - 1.0) > 1e-3)
      return (*msg = "target must sum to 1", JKO_ERR_INVALID_ARG);
  }
  if (g->fft != 0 && g->fft != 1) return (*msg = "fft must be 0 or 1", JKO_ERR_INVALID_ARG);
  if (g->fft) {
    if (p->precision != JKO_FP32 && p->precision != JKO_FP64)
      return (*msg = "the FFT application of the Gaussian runs on JKO_FP32 / JKO_FP64 only",
              JKO_ERR_UNSUPPORTED);
    if (g->heat_L)
      return (*msg = "the FFT application serves the Gaussian kernel only", JKO_ERR_UNSUPPORTED);
    // the attraction's and the pairwise step's prox take a geometric mean of
    // two blurs, which needs each one entry by entry far from its support,
    // where the transforms are accurate only normwise (measured at 64^2 in
    // FP64: 0.71 and 0.06 relative L1 against the oracle, the loops never
    // meeting tol; two species, whose prox takes no such mean, match)
    if (en->target || en->pair_alpha > 0)
      return (*msg = "the FFT application does not serve the attraction steps (their geometric "
                     "mean reads small blurs entry by entry); use the band filter",
              JKO_ERR_UNSUPPORTED);
    // the transforms are accurate normwise: an output carries ~eps log2(L) of
    // its line's largest entry, and the potential spreads the scalings over
    // e^{sigma (max w - min w)}.  Measured (crowd flow, 64^2): FP32 5.5e-6 at a
    // range of 8, 5.4e-5 at 12; FP64 9.3e-11 at 24, 7.8e-9 at 32
    // (each density's potential: the second species has its own scalings)
    double range = 0.0;
    for (const double* wv : {en->w, en->species == 2 ? en->w2 : nullptr}) {
      if (!wv) continue;
      double lo = INFINITY, hi = -INFINITY;
      for (long long i = 0; i < (long long)g->nx * g->ny; ++i) {
        lo = std::min(lo, wv[i]);
        hi = std::max(hi, wv[i]);
      }
      range = std::max(range, p->tau / p->gamma * (hi - lo));
    }
    if (range > (p->precision == JKO_FP64 ? 24.0 : 8.0))
      return (*msg = "the FFT application needs the potential's scalings within e^8 (FP32) / "
                     "e^24 (FP64): tau/gamma (max w - min w) is larger; use the band filter",
              JKO_ERR_UNSUPPORTED);
  }
  if (g->heat_L < 0 || g->heat_L > 1000)
    return (*msg = "heat_L must be 0 (Gaussian) or in [1, 1000]", JKO_ERR_INVALID_ARG);
  if (g->heat_L > 0) {
    if (p->precision != JKO_FP32 && p->precision != JKO_FP64)
      return (*msg = "the heat kernel runs on JKO_FP32 / JKO_FP64 only", JKO_ERR_UNSUPPORTED);
    if (en->target || en->species == 2)
      return (*msg = "the heat kernel serves one density without attraction", JKO_ERR_UNSUPPORTED);
  }
  if (!(en->pair_alpha >= 0) || !std::isfinite(en->pair_alpha))
    return (*msg = "pair_alpha must be finite and >= 0", JKO_ERR_INVALID_ARG);
  if (en->pair_alpha > 0 && en->species != 2)
    return (*msg = "pair_alpha couples two species (species = 2)", JKO_ERR_INVALID_ARG);
  if (en->species < 0 || en->species > 2)
    return (*msg = "species must be 0, 1 or 2", JKO_ERR_INVALID_ARG);
  if (en->species == 2) {
    if (en->m != 0.0 || en->m_field || en->binary || en->target || en->kappa_field || en->mask)
      return (*msg = "two species take a scalar congestion bound and potentials only", JKO_ERR_UNSUPPORTED);
    if (en->w2)
      for (long long i = 0; i < (long long)g->nx * g->ny; ++i)
        if (!std::isfinite(en->w2[i])) return (*msg = "w2 must be finite", JKO_ERR_INVALID_ARG);
  }
  if (en->binary != 0 && en->binary != 1)
    return (*msg = "binary must be 0 or 1", JKO_ERR_INVALID_ARG);
  if (en->binary && (en->m != 0.0 || en->m_field))
    return (*msg = "binary congestion takes no entropy term (m = 0)", JKO_ERR_INVALID_ARG);
  if (en->binary && !en->kappa_field && !std::isfinite(en->kappa))
    return (*msg = "binary congestion needs a finite kappa", JKO_ERR_INVALID_ARG);
  if (en->binary && en->kappa_field)
    for (long long i = 0; i < (long long)g->nx * g->ny; ++i)
      if (!std::isfinite(en->kappa_field[i]))
        return (*msg = "binary congestion needs a finite kappa", JKO_ERR_INVALID_ARG);
  if (en->m_field)
    for (long long i = 0; i < (long long)g->nx * g->ny; ++i)
      if (!(en->m_field[i] >= 1.0) || !std::isfinite(en->m_field[i]))
        return (*msg = "m_field entries must be finite and >= 1", JKO_ERR_INVALID_ARG);
  const long long N = (long long)g->nx * g->ny;
  for (long long i = 0; i < N; ++i) {
    if (en->w && !std::isfinite(en->w[i]))
      return (*msg = "w must be finite", JKO_ERR_INVALID_ARG);
    if (en->kappa_field && !(en->kappa_field[i] > 0))
      return (*msg = "kappa_field must be > 0", JKO_ERR_INVALID_ARG);
    if (en->alpha && (!(en->alpha[i] > 0) || !std::isfinite(en->alpha[i])))
      return (*msg = "alpha must be finite and > 0", JKO_ERR_INVALID_ARG);
    if (en->mask && en->mask[i] > 1)
      return (*msg = "mask entries must be 0 or 1", JKO_ERR_INVALID_ARG);
  }
  return JKO_OK;
}
}  // namespace jko

namespace {

template <typename T>
jko_status build_energy(jko_handle* h, const jko_energy* en) {
  const int N = h->N;
  // the attraction's prox takes h with sigma / (1 + tau) (Eq. prox-psi-attraction)
  // and the pairwise attraction's h_i with sigma / (1 + tau alpha)
  const double sigma = h->prm.tau / h->prm.gamma / (en->target ? 1.0 + h->prm.tau : 1.0) /
                       (1.0 + h->prm.tau * en->pair_alpha);
  h->m = en->m;
  h->ek = en->m_field ? jko::EK_POWER
          : en->m == 0.0 ? jko::EK_CROWD : (en->m == 1.0 ? jko::EK_ENTROPY : jko::EK_POWER);
  std::vector<double> v(N);
  if (h->ek == jko::EK_CROWD) {
    for (int i = 0; i < N; ++i) v[i] = std::exp(-sigma * (en->w ? en->w[i] : 0.0));
    CK(h, upload<T>(&h->E, v));
    if (en->species == 2) {
      for (int i = 0; i < N; ++i) v[i] = std::exp(-sigma * (en->w2 ? en->w2[i] : 0.0));
      CK(h, upload<T>(&h->E2, v));
    }
  } else {
    if (en->w) {
      for (int i = 0; i < N; ++i) v[i] = sigma * en->w[i];
      CK(h, upload<T>(&h->sw, v));
    }
    const double m = en->m;
    for (int i = 0; i < N; ++i) {
      const double al = en->alpha ? en->alpha[i] : 1.0;
      // per-cell exponents: c = sigma alpha m_i of the paper's form of Eq. prox-psi
      v[i] = en->m_field ? sigma * al * en->m_field[i]
             : (h->ek == jko::EK_ENTROPY) ? sigma * al : sigma * al * m / (m - 1.0);
    }
    CK(h, upload<T>(&h->c, v));
    if (en->m_field) {
      for (int i = 0; i < N; ++i) v[i] = en->m_field[i] - 1.0;
      CK(h, upload<T>(&h->m1f, v));
    }
  }
  h->kappa_s = en->kappa;
  h->has_kappa = std::isfinite(en->kappa) ? 1 : 0;
  h->binary = en->binary;
  if (en->kappa_field) {
    bool any = false;
    for (int i = 0; i < N; ++i) { v[i] = en->kappa_field[i]; any |= std::isfinite(v[i]); }
    CK(h, upload<T>(&h->kap, v));
    h->has_kappa = any ? 1 : 0;
  }
  if (en->mask) {
    CK(h, cudaMalloc((void**)&h->mask, N));
    CK(h, cudaMemcpy(h->mask, en->mask, N, cudaMemcpyHostToDevice));
  }
  return JKO_OK;
}

template <typename T>
jko_status setup_simt(jko_handle* h) {
  const int pad = jko::simt_tap_padding();
  auto tx = gibbs_taps(h->grid.nx, h->grid.lx, h->prm.gamma, h->fp64, pad, &h->rx);
  auto ty = gibbs_taps(h->grid.ny, h->grid.ly, h->prm.gamma, h->fp64, pad, &h->ry);
  CK(h, upload<T>(&h->taps_x, tx));
  CK(h, upload<T>(&h->taps_y, ty));
  const size_t smem = sizeof(T) * (size_t)(2 * std::max(h->rx, h->ry) + 1 + pad);
  if (smem > 200 * 1024)
    return set_err(h, JKO_ERR_UNSUPPORTED, "kernel radius too large for the shared-memory taps");
  if (h->fft) {
    // spectra and twiddles of the FFT application, per axis, with the band radii of the taps
    std::vector<double> kh, tw;
    const int mx = jko::fft_max_length<T>();
    if (!jko::fft_axis_tables(h->grid.nx, h->rx, h->grid.lx, h->prm.gamma, mx, &h->fft_Lx,
                              &h->fft_lgx, &kh, &tw))
      return set_err(h, JKO_ERR_UNSUPPORTED, "FFT length along x above the limit of this precision");
    CK(h, upload<T>(&h->fft_khat_x, kh));
    CK(h, upload<T>(&h->fft_tw_x, tw));
    if (!jko::fft_axis_tables(h->grid.ny, h->ry, h->grid.ly, h->prm.gamma, mx, &h->fft_Ly,
                              &h->fft_lgy, &kh, &tw))
      return set_err(h, JKO_ERR_UNSUPPORTED, "FFT length along y above the limit of this precision");
    CK(h, upload<T>(&h->fft_khat_y, kh));
    CK(h, upload<T>(&h->fft_tw_y, tw));
  }
  return JKO_OK;
}

// ---- one step on device buffers of element type T ----
// The start of a step on stream st: the control block reset, q copied into
// the handle's image and the scalings' cold start (a = 1, Sec. 3.4) in one
// launch, or the coupled and tensor-core forms' set-up after it.
template <typename T>
jko_status enqueue_step_begin(jko_handle* h, const T* q_in, cudaStream_t st) {
  const bool plain = !h->tc_multi && !h->tc && !(h->pair_alpha > 0) && h->species != 2 &&
                     !h->attract;
  CK(h, jko::launch_step_begin<T>(*h->ctrl_init, h->ctrl, h->chunk_ctr,
                                  (const void*)q_in != h->q ? q_in : nullptr, (T*)h->q, h->ns,
                                  plain ? (T*)h->a : nullptr, plain ? (long long)h->N : 0, st));
  if (plain) return JKO_OK;
  if (h->tc_multi) {
    if (h->pair_alpha > 0) CK(h, begin_pairwise<float>(h, st));
    else CK(h, begin_multi_tc(h, st));
  } else if (h->tc) {
    jko_status s2 = jko::tc_begin_step(h->tc, st) == cudaSuccess ? JKO_OK : JKO_ERR_CUDA;
    if (s2 != JKO_OK) return set_err(h, s2, "tensor-core step set-up failed");
  } else if (h->pair_alpha > 0) {
    CK(h, begin_pairwise<T>(h, st));
  } else if (h->species == 2) {
    CK(h, begin_species<T>(h, st));
  } else if (h->attract) {
    CK(h, begin_attraction<T>(h, st));
  }
  return JKO_OK;
}

// The status a step's control block reports.
jko_status step_status(const Ctrl& c) {
  // nonfinite bit 1: NaN/Inf met by an epilogue; bit 2: a bounded device wait gave up
  if (c.nonfinite & 2) return JKO_ERR_TIMEOUT;
  if (c.done == jko::NONFINITE || c.nonfinite) return JKO_ERR_NUMERIC;
  if (c.done == jko::MAX_ITER || c.done == jko::STALLED) return JKO_NOT_CONVERGED;
  return JKO_OK;
}

// The chunk loop of a step as a graph: a WHILE node whose body is one chunk
// (the pairs of h->chunk, or one launch of the persistent loop kernel) and the
// loop condition, which ends it when the step has stopped or after the chunk
// budget of the host-driven loop.  Built once, at the first flow of more than
// one step; where the runtime refuses it (state -1) flows keep host-driven chunks.
void build_step_loop(jko_handle* h) {
  if (h->step_loop_state != 0) return;
  h->step_loop_state = -1;
  const int C = h->chunk_iters;
  const unsigned max_chunks = (unsigned)((h->prm.max_iter + 1 + C - 1) / C + 2);
  if (!h->chunk_ctr && cudaMalloc((void**)&h->chunk_ctr, sizeof(unsigned)) != cudaSuccess) {
    h->chunk_ctr = nullptr;
    cudaGetLastError();
    return;
  }
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) { cudaGetLastError(); return; }
  cudaGraphConditionalHandle hc{};
  cudaError_t e = cudaGraphConditionalHandleCreate(&hc, g, 1u, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hc;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
  if (e == cudaSuccess) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(h->cap, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = cudaSuccess;
      if (h->use_loop) e1 = enqueue_loop(h, C, h->cap);
      else
        for (int i = 0; i < C && e1 == cudaSuccess; ++i) e1 = enqueue_pair(h, h->cap);
      if (e1 == cudaSuccess)
        e1 = jko::launch_chunk_loop_cond(h->chunk_ctr, h->ctrl, hc, max_chunks, h->cap);
      cudaGraph_t captured = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(h->cap, &captured);
      e = e1 != cudaSuccess ? e1 : e2;
    }
  }
  cudaGraphExec_t ex = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  h->step_loop = ex;
  h->step_loop_state = 1;
}

template <typename T>
jko_status step_impl(jko_handle* h, const T* q_in, T* p_out, jko_step_info* info, bool validate) {
  cudaStream_t st = h->stream;
  const long long N = h->N;
  ProxArgs<T> P = jko::prox_args<T>(h);
  // The input checks count into the control block and are read back with the
  // step's result, so that a step waits on the device once: on a failed check
  // the step has run on q, but its output write was skipped (outputs
  // untouched) and the status is JKO_ERR_INVALID_ARG.
  auto q_check = [&](const Ctrl& c) -> jko_status {
    char buf[256];
    if (c.q_bad) { snprintf(buf, sizeof buf, "q has %llu non-finite entries", c.q_bad); return set_err(h, JKO_ERR_INVALID_ARG, buf); }
    if (c.q_neg) { snprintf(buf, sizeof buf, "q has %llu negative entries", c.q_neg); return set_err(h, JKO_ERR_INVALID_ARG, buf); }
    if (std::fabs(c.q_sum - 1.0) > 1e-3) { snprintf(buf, sizeof buf, "q sums to %.9g, not 1", c.q_sum); return set_err(h, JKO_ERR_INVALID_ARG, buf); }
    if (c.q_masked) { snprintf(buf, sizeof buf, "q has mass on %llu masked cells", c.q_masked); return set_err(h, JKO_ERR_INVALID_ARG, buf); }
    if (c.q_over) { snprintf(buf, sizeof buf, "q exceeds kappa on %llu cells", c.q_over); return set_err(h, JKO_ERR_INVALID_ARG, buf); }
    return JKO_OK;
  };
  // the checks of an input that also stopped the step with an error
  auto q_check_after_error = [&](jko_status s) -> jko_status {
    if (!validate || s == JKO_ERR_CUDA) return s;
    if (cudaMemcpyAsync(h->poll, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return s;
    const jko_status qs = q_check(h->poll[0]);
    return qs != JKO_OK ? qs : s;
  };
  CK(h, cudaEventRecord(h->ev0, st));
  {
    const jko_status sb = enqueue_step_begin<T>(h, q_in, st);   // resets the control block
    if (sb != JKO_OK) return sb;
  }
  if (validate) {
    CK(h, jko::launch_validate<T>(q_in, N, P, h->ctrl, st));
    if (h->species == 2) CK(h, jko::launch_validate<T>(q_in + N, N, P, h->ctrl, st));
  }

  // chunks: launch the number the last step needed at once, the last one with
  // the finalisation behind it, and wait once; only a step that runs longer
  // than that polls on, with one chunk in flight
  h->kernels = (validate ? 1 : 0) + 1 + (h->tc ? 0 : 1) + (p_out ? 2 : 1);
  // the finalisation: the FP64 mass and max p / kappa of the step's p, and p
  // written out (renormalised)
  auto finalize = [&]() -> cudaError_t {
    cudaError_t e = jko::launch_finalize_reduce<T>((const T*)h->p, h->ns, P, h->ctrl, h->part,
                                                    h->part_cap, st);
    if (e == cudaSuccess && p_out)
      e = jko::launch_finalize_write<T>((const T*)h->p, p_out, h->ns, h->prm.renormalize,
                                        h->ctrl, st, validate ? 1 : 0);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev1, st);
    return e;
  };
  // runs chunks until the step reports a stop; `fin`: the FP32 finish chunks.
  // Returns the stop state read back (h->poll slot) through *done and *it, and
  // through *final_slot the poll slot holding the whole control block after
  // the finalisation when the step stopped within the chunks launched first
  // (-1 otherwise: the caller finalises).
  auto run_chunks = [&](bool fin, int ahead_pairs, int* done, int* it,
                        int* final_slot) -> jko_status {
    const int C = fin ? kFinishChunk : h->chunk_iters;
    const int max_chunks = (h->prm.max_iter + 1 + C - 1) / C + 2;
    // the stop is decided in the pair after the last one completed
    int ahead = (ahead_pairs + 1 + C - 1) / C;
    int launched = 0, polled = 0;
    *final_slot = -1;
    auto launch = [&](bool with_final) -> cudaError_t {
      h->kernels += fin ? 4LL * C : (h->use_loop ? 1LL : pair_kernels(h) * C);
      cudaError_t e = fin ? cudaGraphLaunch(h->chunk_fin, st) : launch_chunk(h, st);
      if (e != cudaSuccess) return e;
      if (with_final) {
        e = finalize();
        if (e != cudaSuccess) return e;
      }
      const int slot = launched & 1;
      e = cudaMemcpyAsync(&h->poll[slot], h->ctrl, with_final ? sizeof(Ctrl) : 16,
                          cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) return e;
      e = cudaEventRecord(h->ev_poll[slot], st);
      ++launched;
      return e;
    };
    if (ahead < 1) ahead = 1;
    if (ahead > max_chunks) ahead = max_chunks;
    for (int i = 0; i < ahead; ++i) CK(h, launch(!fin && i == ahead - 1));
    {
      const int slot = (launched - 1) & 1;
      CK(h, cudaEventSynchronize(h->ev_poll[slot]));
      polled = launched;
      *done = h->poll[slot].done;
      *it = h->poll[slot].it;
      if (*done != jko::RUNNING) {
        if (!fin) *final_slot = slot;
        return JKO_OK;
      }
    }
    bool stopped = false;
    while (!stopped) {
      // keep one chunk in flight while waiting for the oldest poll we need
      if (launched - polled < 2 && launched < max_chunks) CK(h, launch(false));
      // wait for the newest-but-one launched chunk's poll (or the newest if only one)
      const int target = launched - 1 - ((launched - polled) >= 2 ? 1 : 0);
      const int slot = target & 1;
      CK(h, cudaEventSynchronize(h->ev_poll[slot]));
      polled = target + 1;
      *done = h->poll[slot].done;
      *it = h->poll[slot].it;
      stopped = *done != jko::RUNNING;
      if (!stopped && launched >= max_chunks && polled >= launched)
        return set_err(h, JKO_ERR_TIMEOUT, "scaling loop did not report a stop within its budget");
    }
    return JKO_OK;
  };
  int done = jko::RUNNING, it_tc = 0, it_end = 0, final_slot = -1, fin_slot = -1;
  jko_status sr = run_chunks(false, h->last_iters, &done, &it_tc, &final_slot);
  if (sr != JKO_OK) return q_check_after_error(sr);
  bool finished = false;
  if (done == jko::STALLED && h->prm.finish && h->tc) {
    // the tensor-core operands have reached their rounding floor: continue the
    // same step on the FP32 CUDA-core form from the current scalings (the
    // stopped step's pair counter came back with its stop state)
    if (!h->chunk_fin) {
      jko_status sc = capture_finish_chunk(h);
      if (sc != JKO_OK) return sc;
    }
    CK(h, jko::tc_export_scalings(h->tc, (float*)h->a, (float*)h->b, st));
    CK(h, jko::launch_resume(h->ctrl, st));
    h->kernels += 3;
    sr = run_chunks(true, h->last_fin, &done, &it_end, &fin_slot);
    if (sr != JKO_OK) return q_check_after_error(sr);
    finished = true;
    final_slot = -1;   // the finalisation launched with the first chunks is stale
  }

  if (final_slot < 0) {
    CK(h, finalize());
    CK(h, cudaMemcpyAsync(h->poll, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
    final_slot = 0;
  }
  const Ctrl& c = h->poll[final_slot];
  if (validate) {
    const jko_status qs = q_check(c);
    if (qs != JKO_OK) return qs;
  }
  jko_status st_out = JKO_OK;
  // nonfinite bit 1: NaN/Inf met by an epilogue; bit 2: a bounded device wait gave up
  if (c.nonfinite & 2) st_out = JKO_ERR_TIMEOUT;
  else if (c.done == jko::NONFINITE || c.nonfinite) st_out = JKO_ERR_NUMERIC;
  else if (c.done == jko::MAX_ITER || c.done == jko::STALLED) st_out = JKO_NOT_CONVERGED;
  const int fin_pairs = finished ? c.it - it_tc : 0;
  if (finished) h->last_fin = fin_pairs;
  h->last_iters = c.it - fin_pairs;
  if (info) {
    info->iters = c.it;
    info->status = st_out;
    info->residual_l1 = c.res_last;
    info->mass = c.mass;
    unsigned long long bits = c.maxpk_bits;
    double mx;
    std::memcpy(&mx, &bits, sizeof mx);
    info->max_p_over_kappa = h->has_kappa ? mx : 0.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    info->ms = ms;
    info->kernels = (int)h->kernels;
    info->iters_finish = fin_pairs;
  }
  if (st_out == JKO_ERR_TIMEOUT) set_err(h, st_out, "a bounded device-side wait gave up");
  else if (st_out == JKO_ERR_NUMERIC) set_err(h, st_out, "NaN or Inf in the scaling iterates");
  else if (st_out == JKO_NOT_CONVERGED)
    set_err(h, st_out, c.done == jko::STALLED ? "the residual stalled above tol (stall rule)"
                                              : "max_iter reached before tol");
  return st_out;
}

}  // namespace

jko_status jko::step_internal(jko_handle* h, const void* q_in, void* p_out, jko_step_info* info,
                              bool validate) {
  return h->fp64 ? step_impl<double>(h, (const double*)q_in, (double*)p_out, info, validate)
                 : step_impl<float>(h, (const float*)q_in, (float*)p_out, info, validate);
}

jko_status jko::handle_error(jko_handle* h, jko_status st, const std::string& msg) {
  return set_err(h, st, msg);
}

namespace {

int worse(int a, int b) {
  auto rank = [](int s) { return s == JKO_OK ? 0 : (s == JKO_NOT_CONVERGED ? 1 : 2); };
  return rank(b) > rank(a) ? b : a;
}

template <typename T>
jko_status flow_impl(jko_handle* h, const T* p0, int n_steps, T* traj, T* p_final,
                     jko_step_info* infos) {
  const long long N = h->ns;   // elements of a state image
  cudaStream_t st = h->stream;
  const T* q = p0;
  int worst = JKO_OK;
  // the output image of step t: its row of the trajectory, else a stage
  // buffer, never the step's own input
  auto out_for = [&](int t, T** out) -> jko_status {
    *out = traj ? traj + (size_t)t * N : (T*)h->stage_out;
    if (!traj && !h->stage_out) {
      CK(h, cudaMalloc(&h->stage_out, N * sizeof(T)));
      *out = (T*)h->stage_out;
    }
    if (!traj && (const void*)q == (const void*)*out) {
      if (!h->stage_in) CK(h, cudaMalloc(&h->stage_in, N * sizeof(T)));
      *out = (T*)h->stage_in;
    }
    return JKO_OK;
  };
  // The first step checks p0 and runs with host-driven chunks; the later ones
  // run their chunks as the device-side loop, all enqueued before one wait,
  // unless a step needs a host decision (the FP32 finish of a stalled
  // tensor-core step) or the runtime refused the loop graph.
  // The loop graph and the per-step reports are set up at the first flow of
  // any length (a one-step flow does it for the longer flows after it).
  if (!(h->prm.finish && h->tc)) {
    build_step_loop(h);
    if (h->step_loop_state == 1 && h->flow_cap < n_steps) {
      const int cap = std::max(n_steps, 64);
      if (h->flow_ctrl) cudaFreeHost(h->flow_ctrl);
      if (h->flow_ctrl_dev) cudaFree(h->flow_ctrl_dev);
      h->flow_ctrl = nullptr;
      h->flow_ctrl_dev = nullptr;
      h->flow_cap = 0;
      CK(h, cudaMallocHost((void**)&h->flow_ctrl, sizeof(Ctrl) * (size_t)cap));
      CK(h, cudaMalloc((void**)&h->flow_ctrl_dev, sizeof(Ctrl) * (size_t)cap));
      h->flow_cap = cap;
    }
    while (h->step_loop_state == 1 && (int)h->flow_ev.size() < 2 * h->flow_cap) {
      cudaEvent_t ev = nullptr;
      CK(h, cudaEventCreate(&ev));
      h->flow_ev.push_back(ev);
    }
  }
  const bool device_loop = n_steps > 1 && h->step_loop_state == 1 && !(h->prm.finish && h->tc);
  int t = 0;
  for (; t < (device_loop ? 1 : n_steps); ++t) {
    T* out = nullptr;
    jko_status so = out_for(t, &out);
    if (so != JKO_OK) return so;
    jko_step_info info{};
    jko_status s = step_impl<T>(h, q, out, &info, t == 0);
    if (s == JKO_ERR_INVALID_ARG || s == JKO_ERR_CUDA || s == JKO_ERR_OOM || s == JKO_ERR_TIMEOUT)
      return s;
    if (infos) infos[t] = info;
    worst = worse(worst, s);
    q = out;
  }
  if (device_loop && t < n_steps) {
    ProxArgs<T> P = jko::prox_args<T>(h);
    const int t0 = t;
    for (; t < n_steps; ++t) {
      T* out = nullptr;
      jko_status so = out_for(t, &out);
      if (so != JKO_OK) return so;
      // kernels only: the step's start, its chunk loop, the finalisation
      // (which also records the control block), no copy between them
      CK(h, cudaEventRecord(h->flow_ev[2 * t], st));
      jko_status sb = enqueue_step_begin<T>(h, q, st);
      if (sb != JKO_OK) return sb;
      CK(h, cudaGraphLaunch(h->step_loop, st));
      CK(h, jko::launch_finalize_reduce<T>((const T*)h->p, h->ns, P, h->ctrl, h->part,
                                           h->part_cap, st));
      CK(h, jko::launch_finalize_write<T>((const T*)h->p, out, h->ns, h->prm.renormalize,
                                          h->ctrl, st, 0, h->flow_ctrl_dev + t));
      CK(h, cudaEventRecord(h->flow_ev[2 * t + 1], st));
      q = out;
    }
    CK(h, cudaMemcpyAsync(h->flow_ctrl + t0, h->flow_ctrl_dev + t0,
                          sizeof(Ctrl) * (size_t)(n_steps - t0), cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
    const long long per_chunk = h->use_loop ? 1 : pair_kernels(h) * h->chunk_iters;
    for (int k = t0; k < n_steps; ++k) {
      const Ctrl& c = h->flow_ctrl[k];
      const jko_status sk = step_status(c);
      if (sk == JKO_ERR_TIMEOUT) return set_err(h, sk, "a bounded device-side wait gave up");
      h->last_iters = c.it;
      if (infos) {
        jko_step_info& info = infos[k];
        info = jko_step_info{};
        info.iters = c.it;
        info.status = sk;
        info.residual_l1 = c.res_last;
        info.mass = c.mass;
        unsigned long long bits = c.maxpk_bits;
        double mx;
        std::memcpy(&mx, &bits, sizeof mx);
        info.max_p_over_kappa = h->has_kappa ? mx : 0.0;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->flow_ev[2 * k], h->flow_ev[2 * k + 1]);
        info.ms = ms;
        // the step's start, the chunks (the stop is decided in the pair after
        // the last one completed) and their loop conditions, the finalisation
        const long long chunks =
            h->use_loop ? 1 : (c.it + 1 + h->chunk_iters - 1) / h->chunk_iters;
        info.kernels = (int)(1 + chunks * (per_chunk + 1) + 2);
        info.iters_finish = 0;
      }
      if (sk == JKO_ERR_NUMERIC) set_err(h, sk, "NaN or Inf in the scaling iterates");
      else if (sk == JKO_NOT_CONVERGED)
        set_err(h, sk, c.done == jko::STALLED ? "the residual stalled above tol (stall rule)"
                                              : "max_iter reached before tol");
      worst = worse(worst, sk);
    }
  }
  if (p_final && n_steps > 0)
    CK(h, cudaMemcpyAsync(p_final, q, N * sizeof(T), cudaMemcpyDeviceToDevice, st));
  if (p_final && n_steps == 0)
    CK(h, cudaMemcpyAsync(p_final, p0, N * sizeof(T), cudaMemcpyDeviceToDevice, st));
  CK(h, cudaStreamSynchronize(st));
  return (jko_status)worst;
}

}  // namespace

extern "C" {

jko_status jko_create(const jko_grid* grid, const jko_params* params, const jko_energy* energy,
                      void* stream, jko_handle** out) {
  if (!out) return set_err(nullptr, JKO_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  jko_status s = validate_create(grid, params, energy);
  if (s != JKO_OK) return s;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1)
    return set_err(nullptr, JKO_ERR_CUDA, "no CUDA device available");

  jko_handle* h = new jko_handle();
  h->grid = *grid;
  h->prm = *params;
  h->N = grid->nx * grid->ny;
  h->species = energy->species == 2 ? 2 : 1;
  h->ns = (long long)h->species * h->N;
  h->prec = params->precision;
  h->fp64 = params->precision == JKO_FP64;
  h->es = h->fp64 ? 8 : 4;
  h->stream = (cudaStream_t)stream;
  h->heat_L = grid->heat_L;
  // pairs per chunk: every pass after the stop is a launch that returns at once
  // (~1.5 us), so chunks stay short (a heat-kernel pair is 2 (1 + ceil(D / 2)) + 2
  // launches); the driver launches as many as the last step needed at once
  h->chunk_iters = params->check_every > 0 ? params->check_every : (h->heat_L ? 2 : 4);
  cudaGetDevice(&h->device);

  auto fail = [&](jko_status st) {
    g_create_err = h->err;
    free_handle(h);
    return st;
  };
  cudaError_t e;
  const size_t bytes = h->es * (size_t)h->N;
  void** imgs[] = {&h->a, &h->b, &h->t1, &h->p, &h->q};
  for (void** pp : imgs) {
    // p and q hold a state image: both species when there are two
    const size_t nb = (pp == &h->p || pp == &h->q) ? h->es * (size_t)h->ns : bytes;
    e = cudaMalloc(pp, nb);
    if (e != cudaSuccess) return fail(cuda_err(h, e, "cudaMalloc(image)"));
    e = cudaMemset(*pp, 0, nb);
    if (e != cudaSuccess) return fail(cuda_err(h, e, "cudaMemset(image)"));
  }
  e = cudaMalloc((void**)&h->ctrl, sizeof(Ctrl));
  if (e != cudaSuccess) return fail(cuda_err(h, e, "cudaMalloc(ctrl)"));
  h->fft = grid->fft;
  // the b-update pass runs along x: one residual partial per block
  h->nparts_simt = h->fft ? jko::fft_pass_blocks(grid->ny)
                           : jko::simt_pass_blocks(grid->nx, grid->ny, 1, h->fp64 ? 1 : 0);
  h->attract = energy->target ? 1 : 0;
  if (h->attract || h->species == 2) {
    void** more[] = {&h->a2, &h->b2, &h->s1, &h->s2, &h->t2};
    for (void** pp : more) {
      e = cudaMalloc(pp, bytes);
      if (e != cudaSuccess) return fail(cuda_err(h, e, "cudaMalloc(image)"));
      e = cudaMemset(*pp, 0, bytes);
      if (e != cudaSuccess) return fail(cuda_err(h, e, "cudaMemset(image)"));
    }
    h->pair_alpha = energy->species == 2 ? energy->pair_alpha : 0.0;
    if (h->pair_alpha > 0) {
      void* pw[] = {&h->a3, &h->b3, &h->s3, &h->t3};
      for (void* vp : pw) {
        void** pp = (void**)vp;
        e = cudaMalloc(pp, bytes);
        if (e != cudaSuccess) return fail(cuda_err(h, e, "cudaMalloc(image)"));
        e = cudaMemset(*pp, 0, bytes);
        if (e != cudaSuccess) return fail(cuda_err(h, e, "cudaMemset(image)"));
      }
      h->nparts_pw = jko::pairwise_blocks(h->N);
    }
    if (h->attract) {
      std::vector<double> r(energy->target, energy->target + h->N);
      e = h->fp64 ? upload<double>(&h->tgt, r) : upload<float>(&h->tgt, r);
      if (e != cudaSuccess) return fail(cuda_err(h, e, "upload of the target"));
    }
  }
  if (h->heat_L) {
    h->heat = jko::heat_plan(grid->nx, grid->ny, grid->lx, grid->ly, params->gamma, h->heat_L,
                             h->fp64);
    if (h->heat.D < 0)
      return fail(set_err(h, JKO_ERR_UNSUPPORTED,
                          "the heat kernel's expansion needs a degree above 1500 "
                          "(gamma / h^2 too large for this grid)"));
    void** hbufs[] = {&h->hb.d[0], &h->hb.d[1], &h->hb.d[2], &h->hb.d[3]};
    const size_t bytes64 = sizeof(double) * (size_t)h->N;   // FP64 Clenshaw iterates
    for (void** pp : hbufs) {
      e = cudaMalloc(pp, bytes64);
      if (e != cudaSuccess) return fail(cuda_err(h, e, "cudaMalloc(heat scratch)"));
      e = cudaMemset(*pp, 0, bytes64);
      if (e != cudaSuccess) return fail(cuda_err(h, e, "cudaMemset(heat scratch)"));
    }
    const size_t cbytes = sizeof(double) * h->heat.coef.size();
    e = cudaMalloc(&h->hb.coef, cbytes);
    if (e == cudaSuccess)
      e = cudaMemcpy(h->hb.coef, h->heat.coef.data(), cbytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(cuda_err(h, e, "upload of the heat kernel's coefficients"));
  }
  {
    int np = std::max((h->attract || h->species == 2 ? 2 : 1) * h->nparts_simt,
                      jko::tc_partials(grid->nx, grid->ny));
    if (h->heat_L) np = std::max(np, jko::heat_blocks(grid->nx, grid->ny));
    if (h->attract || h->species == 2)   // the tensor-core passes' b-update partials
      np = std::max(np, 3 * jko::tc_multi_tiles(grid->nx, grid->ny, 1));
    if (h->pair_alpha > 0) np = std::max(np, h->nparts_pw);
    e = cudaMalloc((void**)&h->part, sizeof(double) * np);
    h->part_cap = np;
    if (e != cudaSuccess) return fail(cuda_err(h, e, "cudaMalloc(partials)"));
    e = cudaMemset(h->part, 0, sizeof(double) * np);
    if (e != cudaSuccess) return fail(cuda_err(h, e, "cudaMemset(partials)"));
  }
  e = cudaMallocHost((void**)&h->ctrl_init, sizeof(Ctrl));
  if (e != cudaSuccess) return fail(cuda_err(h, e, "cudaMallocHost"));
  e = cudaMallocHost((void**)&h->poll, 2 * sizeof(Ctrl));
  if (e != cudaSuccess) return fail(cuda_err(h, e, "cudaMallocHost"));
  std::memset(h->ctrl_init, 0, sizeof(Ctrl));
  std::memset(h->poll, 0, 2 * sizeof(Ctrl));
  h->ctrl_init->tol = params->tol;
  h->ctrl_init->max_iter = params->max_iter;
  h->ctrl_init->stall = params->stall;
  for (auto& ev : h->ev_poll) {
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(cuda_err(h, e, "cudaEventCreate"));
  }
  if ((e = cudaEventCreate(&h->ev0)) != cudaSuccess || (e = cudaEventCreate(&h->ev1)) != cudaSuccess)
    return fail(cuda_err(h, e, "cudaEventCreate"));
  e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fail(cuda_err(h, e, "cudaStreamCreate"));

  s = h->fp64 ? build_energy<double>(h, energy) : build_energy<float>(h, energy);
  if (s == JKO_OK && h->heat_L && params->loop != 2) {
    // the heat kernel: one persistent cooperative kernel per step where the
    // device allows it (loop 0 or 1), else the kernels per Clenshaw phase (loop 2)
    h->heat_G = jko::heat_loop_grid(grid->nx, grid->ny, h->fp64, h->ek);
    if (h->heat_G <= 0 && (params->loop == 1 || params->loop == 3))
      s = set_err(h, JKO_ERR_UNSUPPORTED,
                  "the persistent heat-kernel loop cannot run here (no cooperative launch)");
    h->use_loop = h->heat_G > 0;
  }
  if (s != JKO_OK) return fail(s);
  if (h->prec == JKO_FP64 || h->prec == JKO_FP32) {
    // the heat kernel needs no Gaussian taps
    if (!h->heat_L) s = h->fp64 ? setup_simt<double>(h) : setup_simt<float>(h);
  } else {
    jko::TcConfig cfg{};
    cfg.nx = grid->nx; cfg.ny = grid->ny; cfg.lx = grid->lx; cfg.ly = grid->ly;
    cfg.gamma = params->gamma; cfg.precision = h->prec; cfg.ek = h->ek;
    cfg.a = (float*)h->a; cfg.b = (float*)h->b; cfg.p = (float*)h->p; cfg.q = (const float*)h->q;
    cfg.ctrl = h->ctrl;
    cfg.part = h->part;
    cfg.prox = jko::prox_args<float>(h);
    // separable log-domain absorption of the potential: on, off, or automatic
    // when the potential spans more than 120 e-folds (sigma (max w - min w)).
    // Below that the plain form is the more accurate one (its scalings stay in
    // range); beyond ~130 e-folds the plain form loses the far field.
    cfg.w_host = energy->w;
    cfg.sigma = params->tau / params->gamma;
    cfg.absorb = 0;
    const bool multi = h->attract || h->species == 2;   // several couplings: tc_multi.cu
    if (energy->w && params->absorb != 2 && params->absorb != 3 && !multi) {
      double lo = INFINITY, hi = -INFINITY;
      for (int i = 0; i < h->N; ++i) { lo = std::min(lo, energy->w[i]); hi = std::max(hi, energy->w[i]); }
      cfg.absorb = params->absorb == 1 || cfg.sigma * (hi - lo) > 120.0 ? 1 : 0;
    }
    std::string msg;
    int rc = jko::tc_create(cfg, &h->tc, &msg);
    if (rc == 1) s = set_err(h, JKO_ERR_UNSUPPORTED, msg);
    else if (rc != 0) s = set_err(h, JKO_ERR_CUDA, msg);
    if (s == JKO_OK && multi) {
      h->tc_multi = 1;
      h->use_loop = 0;
      if (params->precision == JKO_BF16 || params->precision == JKO_BF16X3) {
        // the bf16 pairs of the first pass's images (up to 3, 4 bytes per cell each)
        const size_t pb = (size_t)3 * 4 * h->N;
        cudaError_t me = cudaMalloc(&h->mpair, pb);
        if (me == cudaSuccess) me = cudaMemset(h->mpair, 0, pb);
        if (me != cudaSuccess) s = cuda_err(h, me, "cudaMalloc(operand pairs)");
      }
    } else if (s == JKO_OK) {
      const int ok = jko::tc_loop_supported(h->tc);
      if ((params->loop == 1 || params->loop == 3) && !ok)
        s = set_err(h, JKO_ERR_UNSUPPORTED,
                    "the persistent loop kernel cannot run here (nx % 4 != 0 or no cooperative launch)");
      else if (params->tile != 0 && jko::tc_set_tile(h->tc, params->tile) != 0)
        s = set_err(h, JKO_ERR_UNSUPPORTED, "tile width not available for this precision");
      h->use_loop = params->loop != 2 && ok;
    }
    if (s == JKO_OK && params->absorb == 3) {
      // the log-domain form: exponent images and its own per-pass kernels
      std::string lmsg;
      const int rc = jko::tc_log_setup(h->tc, energy->w, params->tau / params->gamma, &lmsg);
      if (rc == 1) s = set_err(h, JKO_ERR_UNSUPPORTED, lmsg);
      else if (rc != 0) s = set_err(h, JKO_ERR_CUDA, lmsg);
      h->use_loop = 0;
    }
    if (s == JKO_OK && params->finish) {
      // the FP32 CUDA-core form that finishes a stalled step: its taps
      if (jko::tc_absorbed(h->tc))
        s = set_err(h, JKO_ERR_UNSUPPORTED,
                    "finish needs scalings without log-domain absorption (absorb = 2)");
      else
        s = setup_simt<float>(h);
    }
  }
  if (s == JKO_OK && h->tc && !h->tc_multi && !jko::tc_logdomain(h->tc) && params->loop == 0 &&
      params->tile == 0 &&
      (long long)grid->nx * grid->ny >= 256LL * 256LL) {
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(cuda_err(h, e, "set-up"));
    s = autotune(h, grid, params);
  }
  if (s != JKO_OK) return fail(s);
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(cuda_err(h, e, "set-up"));
  // the loop kernel takes the stop decision itself: one launch runs the whole
  // pair budget (the decision at pair max_iter + 1 needs that many) and ends
  // where the rule fires, so the host waits once instead of polling chunks
  if (h->use_loop) h->chunk_iters = params->max_iter + 1;
  s = capture_chunk(h);
  if (s != JKO_OK) return fail(s);
  *out = h;
  return JKO_OK;
}

jko_status jko_step(jko_handle* h, const void* q_dev, void* p_out_dev, jko_step_info* info) {
  if (!h) return set_err(nullptr, JKO_ERR_INVALID_ARG, "NULL handle");
  if (!q_dev || !p_out_dev) return set_err(h, JKO_ERR_INVALID_ARG, "NULL q or p_out");
  DeviceGuard dg(h->device);
  h->err.clear();
  return h->fp64 ? step_impl<double>(h, (const double*)q_dev, (double*)p_out_dev, info, true)
                 : step_impl<float>(h, (const float*)q_dev, (float*)p_out_dev, info, true);
}

jko_status jko_flow(jko_handle* h, const void* p0_dev, int n_steps, void* traj_dev,
                    void* p_final_dev, jko_step_info* infos) {
  if (!h) return set_err(nullptr, JKO_ERR_INVALID_ARG, "NULL handle");
  if (!p0_dev || n_steps < 0) return set_err(h, JKO_ERR_INVALID_ARG, "NULL p0 or n_steps < 0");
  DeviceGuard dg(h->device);
  h->err.clear();
  return h->fp64 ? flow_impl<double>(h, (const double*)p0_dev, n_steps, (double*)traj_dev,
                                     (double*)p_final_dev, infos)
                 : flow_impl<float>(h, (const float*)p0_dev, n_steps, (float*)traj_dev,
                                    (float*)p_final_dev, infos);
}

jko_status jko_flow_host(jko_handle* h, const void* p0_host, int n_steps, void* traj_host,
                         void* p_final_host, jko_step_info* infos) {
  if (!h) return set_err(nullptr, JKO_ERR_INVALID_ARG, "NULL handle");
  if (!p0_host || n_steps < 0) return set_err(h, JKO_ERR_INVALID_ARG, "NULL p0 or n_steps < 0");
  DeviceGuard dg(h->device);
  h->err.clear();
  const size_t bytes = h->es * (size_t)h->ns;
  if (!h->stage_in) CK(h, cudaMalloc(&h->stage_in, bytes));
  if (!h->stage_out) CK(h, cudaMalloc(&h->stage_out, bytes));
  cudaStream_t st = h->stream;
  CK(h, cudaMemcpyAsync(h->stage_in, p0_host, bytes, cudaMemcpyHostToDevice, st));
  void* cur = h->stage_in;
  void* nxt = h->stage_out;
  int worst = JKO_OK;
  for (int t = 0; t < n_steps; ++t) {
    jko_step_info info{};
    jko_status s = h->fp64 ? step_impl<double>(h, (const double*)cur, (double*)nxt, &info, t == 0)
                           : step_impl<float>(h, (const float*)cur, (float*)nxt, &info, t == 0);
    if (s == JKO_ERR_INVALID_ARG || s == JKO_ERR_CUDA || s == JKO_ERR_OOM || s == JKO_ERR_TIMEOUT)
      return s;
    if (infos) infos[t] = info;
    worst = worse(worst, s);
    if (traj_host)
      CK(h, cudaMemcpyAsync((char*)traj_host + (size_t)t * bytes, nxt, bytes,
                            cudaMemcpyDeviceToHost, st));
    std::swap(cur, nxt);
  }
  if (p_final_host) CK(h, cudaMemcpyAsync(p_final_host, cur, bytes, cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  return (jko_status)worst;
}

jko_status jko_profile_passes(jko_handle* h, int reps, float* ms, double* flops) {
  if (!h) return set_err(nullptr, JKO_ERR_INVALID_ARG, "NULL handle");
  if (reps < 1 || !ms) return set_err(h, JKO_ERR_INVALID_ARG, "reps < 1 or NULL ms");
  if (h->heat_L)
    return set_err(h, JKO_ERR_UNSUPPORTED, "a heat-kernel handle has no separable passes to time");
  if (h->tc_multi)
    return set_err(h, JKO_ERR_UNSUPPORTED,
                   "the tensor-core passes of several couplings are timed through the steps");
  DeviceGuard dg(h->device);
  cudaStream_t st = h->stream;
  // A running control block that never stops: it = 1 (residuals computed),
  // tol < 0 and an unreachable budget.
  Ctrl c0;
  std::memcpy(&c0, h->ctrl_init, sizeof(Ctrl));
  c0.it = 1;
  c0.tol = -1.0;
  c0.max_iter = 0x7fffffff;
  CK(h, cudaMemcpy(h->ctrl, &c0, sizeof(Ctrl), cudaMemcpyHostToDevice));
  for (int k = 0; k < 4; ++k) {
    // the reps launches are captured in a graph, as the scaling loop runs them,
    // so that host launch latency does not enter the per-launch time
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    CK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = enqueue_pass(h, k, h->cap);
    cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
    if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_err(h, e, "profile capture"); }
    CK(h, e2);
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    CK(h, e);
    e = cudaGraphLaunch(ge, st);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(h->ev0, st);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, st);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(h->ev1);
    cudaGraphExecDestroy(ge);
    CK(h, e);
    float t = 0.f;
    CK(h, cudaEventElapsedTime(&t, h->ev0, h->ev1));
    ms[k] = t / reps;
    if (flops) flops[k] = pass_flops(h, k);
  }
  CK(h, cudaMemcpy(h->ctrl, h->ctrl_init, sizeof(Ctrl), cudaMemcpyHostToDevice));
  return JKO_OK;
}

jko_status jko_profile_loop(jko_handle* h, int pairs, int reps, float* ms, double* flops) {
  if (!h) return set_err(nullptr, JKO_ERR_INVALID_ARG, "NULL handle");
  if (pairs < 1 || reps < 1 || !ms) return set_err(h, JKO_ERR_INVALID_ARG, "pairs < 1, reps < 1 or NULL ms");
  if (!h->use_loop) return set_err(h, JKO_ERR_UNSUPPORTED, "the handle does not use the loop kernel");
  DeviceGuard dg(h->device);
  cudaStream_t st = h->stream;
  // a running control block that never stops (as in jko_profile_passes)
  Ctrl c0;
  std::memcpy(&c0, h->ctrl_init, sizeof(Ctrl));
  c0.it = 1;
  c0.tol = -1.0;
  c0.max_iter = 0x7fffffff;
  CK(h, cudaMemcpy(h->ctrl, &c0, sizeof(Ctrl), cudaMemcpyHostToDevice));
  cudaError_t e = enqueue_loop(h, pairs, st);   // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(h->ev0, st);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = enqueue_loop(h, pairs, st);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(h->ev1);
  CK(h, e);
  float t = 0.f;
  CK(h, cudaEventElapsedTime(&t, h->ev0, h->ev1));
  ms[0] = t / reps;
  if (flops) flops[0] = h->tc ? jko::tc_loop_flops(h->tc, pairs) : 0.0;
  CK(h, cudaMemcpy(h->poll, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
  const int nf = h->poll[0].nonfinite;
  CK(h, cudaMemcpy(h->ctrl, h->ctrl_init, sizeof(Ctrl), cudaMemcpyHostToDevice));
  if (nf & 2) return set_err(h, JKO_ERR_TIMEOUT, "a bounded device wait gave up");
  return JKO_OK;
}

jko_status jko_handle_info(const jko_handle* h, int* out) {
  if (!h || !out) return set_err(nullptr, JKO_ERR_INVALID_ARG, "NULL handle or out");
  out[0] = h->use_loop;
  out[1] = h->use_loop && h->tc ? jko::tc_loop_resident(h->tc) : 0;
  out[2] = h->chunk != nullptr;
  out[3] = h->chunk_iters;
  return JKO_OK;
}

jko_status jko_set_stream(jko_handle* h, void* stream) {
  if (!h) return set_err(nullptr, JKO_ERR_INVALID_ARG, "NULL handle");
  h->stream = (cudaStream_t)stream;
  return JKO_OK;
}

jko_status jko_destroy(jko_handle* h) {
  free_handle(h);
  return JKO_OK;
}

const char* jko_last_error(const jko_handle* h) {
  return h ? h->err.c_str() : g_create_err.c_str();
}

const char* jko_status_string(int s) {
  switch (s) {
    case JKO_OK: return "JKO_OK";
    case JKO_ERR_INVALID_ARG: return "JKO_ERR_INVALID_ARG";
    case JKO_ERR_CUDA: return "JKO_ERR_CUDA";
    case JKO_ERR_OOM: return "JKO_ERR_OOM";
    case JKO_ERR_NUMERIC: return "JKO_ERR_NUMERIC";
    case JKO_NOT_CONVERGED: return "JKO_NOT_CONVERGED";
    case JKO_ERR_TIMEOUT: return "JKO_ERR_TIMEOUT";
    case JKO_ERR_UNSUPPORTED: return "JKO_ERR_UNSUPPORTED";
    default: return "unknown jko_status";
  }
}

jko_status jko_heat_plan(int nx, int ny, double lx, double ly, double gamma, int L,
                         int precision, int* degree, double* coef, int cap, double* interval) {
  if (nx < 1 || ny < 1 || !(lx > 0) || !(ly > 0) || !std::isfinite(lx) || !std::isfinite(ly) ||
      !(gamma > 0) || !std::isfinite(gamma) || L < 1 || L > 1000 || !degree || cap < 0 ||
      (cap > 0 && !coef))
    return set_err(nullptr, JKO_ERR_INVALID_ARG, "jko_heat_plan: argument out of range");
  if (precision != JKO_FP32 && precision != JKO_FP64)
    return set_err(nullptr, JKO_ERR_UNSUPPORTED, "the heat kernel runs on JKO_FP32 / JKO_FP64 only");
  const jko::HeatPlan hp = jko::heat_plan(nx, ny, lx, ly, gamma, L, precision == JKO_FP64);
  *degree = hp.D;
  if (interval) {
    interval[0] = hp.theta - hp.delta;
    interval[1] = hp.theta + hp.delta;
  }
  if (hp.D < 0) return set_err(nullptr, JKO_ERR_UNSUPPORTED, "expansion degree above 1500");
  for (int k = 0; k < cap && k <= hp.D; ++k) coef[k] = hp.coef[k];
  return JKO_OK;
}

const char* jko_build_info(void) {
  return "libjko: sm_103a; precisions FP64 FP32 (CUDA cores), TF32 BF16 BF16X3 (tcgen05)";
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched flows: n independent flows (own grid, parameters, energy and
// precision each) advanced together.  Each JKO step runs three CUDA graphs
// whose branches are the flows (fork-join capture over worker streams): the
// prologue (control reset, cold start a = 1), a chunk of `check_every` pairs,
// and the finalisation (FP64 mass, renormalisation into the flow's input
// buffer for the next step).  Flows that have stopped turn their kernels into
// no-ops; one gather kernel and one small copy poll every flow at once.
// ---------------------------------------------------------------------------
struct jko_batch {
  int n = 0;
  std::vector<jko_handle*> h;
  cudaStream_t stream = nullptr;
  std::vector<cudaStream_t> cap;     // cap[0] is the capture root
  std::vector<cudaEvent_t> ev;       // fork / join events
  cudaGraphExec_t g_pro = nullptr, g_chunk = nullptr, g_fin = nullptr;
  int C = 16;
  int max_iter = 1;
  Ctrl** ctrl_ptrs = nullptr;        // device: control block of each flow
  Ctrl* ctrl_all = nullptr;          // device: gathered control blocks
  Ctrl* host_all = nullptr;          // pinned copy
  int* done_dev = nullptr;           // device: gathered stop states
  int* done_host = nullptr;          // pinned, 2 slots of n
  cudaEvent_t ev_poll[2] = {nullptr, nullptr};
  int last_iters = 0;
  bool per_pass = false;             // run every flow on per-pass kernels
  int tuned = -1;                    // candidate the batch autotuner chose
  std::vector<jko::TcGroup*> groups; // grouped launches (one per precision)
  std::vector<int> group_pairs;      // pairs one grouped launch may run
  std::vector<char> in_group;        // flow f runs in a grouped launch
  std::string err;
};

namespace {

jko_status batch_err(jko_batch* b, jko_status st, const std::string& msg) {
  if (b) b->err = msg; else g_create_err = msg;
  return st;
}

#define BCK(b, call)                                                        \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess)                                                  \
      return batch_err(b, e_ == cudaErrorMemoryAllocation ? JKO_ERR_OOM : JKO_ERR_CUDA, \
                       std::string(#call) + ": " + cudaGetErrorName(e_));   \
  } while (0)

void free_batch(jko_batch* b) {
  if (!b) return;
  for (auto* h : b->h) free_handle(h);
  for (auto* g : b->groups) jko::tc_group_destroy(g);
  if (b->g_pro) cudaGraphExecDestroy(b->g_pro);
  if (b->g_chunk) cudaGraphExecDestroy(b->g_chunk);
  if (b->g_fin) cudaGraphExecDestroy(b->g_fin);
  for (auto s : b->cap) if (s) cudaStreamDestroy(s);
  for (auto e : b->ev) if (e) cudaEventDestroy(e);
  for (auto e : b->ev_poll) if (e) cudaEventDestroy(e);
  if (b->ctrl_ptrs) cudaFree(b->ctrl_ptrs);
  if (b->ctrl_all) cudaFree(b->ctrl_all);
  if (b->done_dev) cudaFree(b->done_dev);
  if (b->host_all) cudaFreeHost(b->host_all);
  if (b->done_host) cudaFreeHost(b->done_host);
  delete b;
}

// The start of a flow's step inside the batch graphs: the control block reset
// and the cold start of its form (as enqueue_step_begin for a handle alone;
// the step input is already in h->q).
template <typename T>
cudaError_t flow_begin_t(jko_handle* h, cudaStream_t s) {
  if (h->pair_alpha > 0) return begin_pairwise<T>(h, s);
  if (h->species == 2) return begin_species<T>(h, s);
  if (h->attract) return begin_attraction<T>(h, s);
  return jko::launch_fill<T>((T*)h->a, T(1), h->N, s);
}

cudaError_t flow_prologue(jko_handle* h, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(h->ctrl, h->ctrl_init, sizeof(Ctrl), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  if (h->tc_multi) return h->pair_alpha > 0 ? begin_pairwise<float>(h, s) : begin_multi_tc(h, s);
  if (h->tc) return jko::tc_begin_step(h->tc, s);
  return h->fp64 ? flow_begin_t<double>(h, s) : flow_begin_t<float>(h, s);
}

cudaError_t flow_chunk(jko_handle* h, int C, bool per_pass, cudaStream_t s, int loop_pairs = 0) {
  // a flow on the loop kernel: one launch runs its whole pair budget and stops
  // itself; later chunks of the step find it stopped and return at once
  if (h->use_loop && h->tc && !per_pass)
    return jko::tc_enqueue_loop(h->tc, loop_pairs > 0 ? loop_pairs : h->chunk_iters, s);
  for (int i = 0; i < C; ++i) {
    cudaError_t e = enqueue_pair(h, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t flow_finalize_t(jko_handle* h, cudaStream_t s) {
  ProxArgs<T> P = jko::prox_args<T>(h);
  // h->ns: both densities of a two-species flow
  cudaError_t e = jko::launch_finalize_reduce<T>((const T*)h->p, h->ns, P, h->ctrl, h->part,
                                                 h->part_cap, s);
  if (e != cudaSuccess) return e;
  // the step output becomes the input of the next step
  return jko::launch_finalize_write<T>((const T*)h->p, (T*)h->q, h->ns, h->prm.renormalize,
                                       h->ctrl, s);
}

cudaError_t flow_finalize(jko_handle* h, cudaStream_t s) {
  return h->fp64 ? flow_finalize_t<double>(h, s) : flow_finalize_t<float>(h, s);
}

template <class H, class F, class G>
jko_status capture_batch(jko_batch* b, H head, F per_flow, G tail, cudaGraphExec_t* out,
                         bool skip_grouped = false);

cudaError_t no_op(cudaStream_t) { return cudaSuccess; }

void clear_groups(jko_batch* b) {
  for (auto* g : b->groups) jko::tc_group_destroy(g);
  b->groups.clear();
  b->group_pairs.clear();
  b->in_group.assign(b->n, 0);
}

// Puts the flows with sel[f] set that can run the loop kernel into grouped
// launches, one per precision and energy kind (and per 2048 flows); the
// others keep their own branch.
jko_status make_groups(jko_batch* b, const std::vector<char>& sel) {
  clear_groups(b);
  for (int key = 0; key < 9; ++key) {
    const int prec = key / 3 == 0 ? JKO_TF32 : key / 3 == 1 ? JKO_BF16 : JKO_BF16X3;
    const int ek = key % 3;
    std::vector<jko::TcPlan*> plans;
    std::vector<int> ids;
    for (int f = 0; f < b->n; ++f) {
      jko_handle* h = b->h[f];
      if (sel[f] && h->tc && h->prec == prec && h->ek == ek && jko::tc_loop_supported(h->tc)) {
        plans.push_back(h->tc);
        ids.push_back(f);
      }
    }
    for (size_t i0 = 0; i0 < plans.size(); i0 += 2048) {
      const int n = (int)std::min<size_t>(2048, plans.size() - i0);
      jko::TcGroup* g = nullptr;
      std::string msg;
      const int rc = jko::tc_group_create(plans.data() + i0, n, &g, &msg);
      if (rc == 2) return batch_err(b, JKO_ERR_CUDA, msg);
      if (rc != 0) continue;
      int pairs = 1;
      for (int k = 0; k < n; ++k) {
        jko_handle* h = b->h[ids[i0 + k]];
        apply_cand(h, CAND_LOOP);
        h->chunk_iters = h->prm.max_iter + 1;
        pairs = std::max(pairs, h->prm.max_iter + 1);
        b->in_group[ids[i0 + k]] = 1;
      }
      b->groups.push_back(g);
      b->group_pairs.push_back(pairs);
    }
  }
  return JKO_OK;
}

// Launches every grouped launch of the batch for up to `pairs` pairs (0: the
// flows' whole budgets) on stream st.
cudaError_t launch_groups(jko_batch* b, cudaStream_t st, int pairs = 0) {
  for (size_t i = 0; i < b->groups.size(); ++i) {
    cudaError_t e = jko::tc_group_enqueue(b->groups[i], pairs > 0 ? pairs : b->group_pairs[i], st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t begin_groups(jko_batch* b, cudaStream_t st) {
  for (auto* g : b->groups) {
    cudaError_t e = jko::tc_group_begin_step(g, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Batch autotuner: the configuration of every flow (loop kernel or per-pass
// kernels with 64- or 128-wide tiles) that runs the whole batch fastest.
// Candidates: each flow's own choice, all per-pass 64, all per-pass 128 (64
// where the precision has no 128), all on the loop kernel where it can run,
// and those flows in grouped launches (one cooperative launch per precision).
jko_status tune_batch(jko_batch* b) {
  const int n = b->n;
  std::vector<int> own(n);
  for (int f = 0; f < n; ++f)
    own[f] = b->h[f]->use_loop ? CAND_LOOP : (jko::tc_tile(b->h[f]->tc) == 128 ? CAND_PP128 : CAND_PP64);
  auto cand_of = [&](int c, int f) {
    jko_handle* h = b->h[f];
    if (c == 0) return own[f];
    if (c == 1) return (int)CAND_PP64;
    if (c == 2) return h->prec != JKO_TF32 ? (int)CAND_PP64 : (int)CAND_PP128;
    return jko::tc_loop_supported(h->tc) ? (int)CAND_LOOP : (int)CAND_PP64;
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BCK(b, cudaEventCreate(&e0));
  BCK(b, cudaEventCreate(&e1));
  int best = 0;
  float best_ms = -1.f;
  const std::vector<char> all(n, 1);
  for (int c = 0; c < 5; ++c) {
    bool ok = true;
    clear_groups(b);
    for (int f = 0; f < n && ok; ++f) ok = apply_cand(b->h[f], cand_of(c == 4 ? 3 : c, f));
    if (ok && c == 4) ok = make_groups(b, all) == JKO_OK && !b->groups.empty();
    for (int f = 0; f < n && ok; ++f) ok = prime_for_timing(b->h[f], b->stream) == cudaSuccess;
    if (!ok || cudaStreamSynchronize(b->stream) != cudaSuccess) { cudaGetLastError(); continue; }
    cudaGraphExec_t ge = nullptr;
    jko_status s = capture_batch(
        b, [b](cudaStream_t st) { return launch_groups(b, st, kTunePairs); },
        [](jko_handle* h, cudaStream_t st) { return flow_chunk(h, kTunePairs, false, st, kTunePairs); },
        no_op, &ge, true);
    if (s != JKO_OK) { cudaGetLastError(); continue; }
    const float ms = time_graph(ge, b->stream, e0, e1);
    cudaGraphExecDestroy(ge);
    if (ms > 0.f && (best_ms < 0.f || ms < best_ms)) { best = c; best_ms = ms; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  clear_groups(b);
  for (int f = 0; f < n; ++f) {
    apply_cand(b->h[f], cand_of(best == 4 ? 3 : best, f));
    BCK(b, cudaMemcpy(b->h[f]->ctrl, b->h[f]->ctrl_init, sizeof(Ctrl), cudaMemcpyHostToDevice));
  }
  if (best == 4) {
    jko_status s = make_groups(b, all);
    if (s != JKO_OK) return s;
  }
  b->tuned = best;
  b->err.clear();
  return JKO_OK;
}

// Captures one graph: `head` on the root stream, then branches running
// `per_flow` for every flow (but the grouped ones with skip_grouped), joined on
// the root, then `tail` on the root.
template <class H, class F, class G>
jko_status capture_batch(jko_batch* b, H head, F per_flow, G tail, cudaGraphExec_t* out,
                         bool skip_grouped) {
  cudaStream_t root = b->cap[0];
  const int nw = (int)b->cap.size() - 1;
  cudaGraph_t g = nullptr;
  BCK(b, cudaStreamBeginCapture(root, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = head(root);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev[0], root);
  std::vector<char> used(nw, 0);
  for (int f = 0; f < b->n && e == cudaSuccess; ++f) {
    if (skip_grouped && b->in_group[f]) continue;
    const int k = f % nw;
    cudaStream_t s = b->cap[1 + k];
    if (!used[k]) { e = cudaStreamWaitEvent(s, b->ev[0], 0); used[k] = 1; }
    if (e == cudaSuccess) e = per_flow(b->h[f], s);
  }
  for (int k = 0; k < nw && e == cudaSuccess; ++k) {
    if (!used[k]) continue;
    e = cudaEventRecord(b->ev[1 + k], b->cap[1 + k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(root, b->ev[1 + k], 0);
  }
  if (e == cudaSuccess) e = tail(root);
  cudaError_t e2 = cudaStreamEndCapture(root, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return batch_err(b, JKO_ERR_CUDA, std::string("batch graph capture: ") +
                                          cudaGetErrorName(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  BCK(b, e);
  return JKO_OK;
}

template <typename T>
jko_status check_input(jko_handle* h, const T* q, int flow, jko_batch* b) {
  cudaStream_t st = h->stream;
  ProxArgs<T> P = jko::prox_args<T>(h);
  BCK(b, cudaMemcpyAsync(h->ctrl, h->ctrl_init, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
  BCK(b, jko::launch_validate<T>(q, h->N, P, h->ctrl, st));
  if (h->species == 2) BCK(b, jko::launch_validate<T>(q + h->N, h->N, P, h->ctrl, st));
  BCK(b, cudaMemcpyAsync(h->poll, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
  BCK(b, cudaStreamSynchronize(st));
  const Ctrl& c = h->poll[0];
  if (c.q_bad || c.q_neg || std::fabs(c.q_sum - 1.0) > 1e-3 || c.q_masked || c.q_over) {
    char buf[200];
    snprintf(buf, sizeof buf, "flow %d: p0 must be finite, >= 0, sum to 1, vanish on the mask "
                              "and stay below kappa", flow);
    return batch_err(b, JKO_ERR_INVALID_ARG, buf);
  }
  return JKO_OK;
}

}  // namespace

extern "C" {

jko_status jko_batch_create(int n_flows, const jko_grid* grids, const jko_params* params,
                            const jko_energy* energies, void* stream, jko_batch** out) {
  if (!out) return batch_err(nullptr, JKO_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_flows < 1 || !grids || !params || !energies)
    return batch_err(nullptr, JKO_ERR_INVALID_ARG, "n_flows < 1 or NULL arrays");
  jko_batch* b = new jko_batch();
  b->n = n_flows;
  b->stream = (cudaStream_t)stream;
  b->C = params[0].check_every > 0 ? params[0].check_every : 16;
  auto fail = [&](jko_status st) {
    g_create_err = b->err;
    free_batch(b);
    return st;
  };
  for (int f = 0; f < n_flows; ++f) {
    if (params[f].check_every != params[0].check_every)
      return fail(batch_err(b, JKO_ERR_INVALID_ARG, "all flows must share check_every"));
    if (params[f].finish)
      return fail(batch_err(b, JKO_ERR_UNSUPPORTED,
                            "finish (the FP32 continuation of a stalled step) is for single handles"));
    if (params[f].absorb == 3)
      return fail(batch_err(b, JKO_ERR_UNSUPPORTED, "the log-domain form is for single handles"));
    jko_handle* h = nullptr;
    jko_status s = jko_create(&grids[f], &params[f], &energies[f], stream, &h);
    if (s != JKO_OK) {
      char buf[64];
      snprintf(buf, sizeof buf, "flow %d: ", f);
      return fail(batch_err(b, s, buf + g_create_err));
    }
    // other flows fill the GPU: the CUDA-core passes keep their throughput form,
    // and a heat-kernel flow runs its kernels per Clenshaw phase (its persistent
    // form is one cooperative launch over every SM)
    h->simt_latency = 0;
    h->nparts_simt = jko::simt_pass_blocks(grids[f].nx, grids[f].ny, 0);
    if (h->heat_L) h->use_loop = 0;
    b->h.push_back(h);
    b->max_iter = std::max(b->max_iter, params[f].max_iter);
  }
  const int nw = std::min(n_flows, 64);
  b->cap.assign(nw + 1, nullptr);
  b->ev.assign(nw + 1, nullptr);
  for (auto& s : b->cap)
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
      return fail(batch_err(b, JKO_ERR_CUDA, "cudaStreamCreate"));
  for (auto& e : b->ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return fail(batch_err(b, JKO_ERR_CUDA, "cudaEventCreate"));
  for (auto& e : b->ev_poll)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return fail(batch_err(b, JKO_ERR_CUDA, "cudaEventCreate"));
  std::vector<Ctrl*> ptrs(n_flows);
  for (int f = 0; f < n_flows; ++f) ptrs[f] = b->h[f]->ctrl;
  if (cudaMalloc((void**)&b->ctrl_ptrs, sizeof(Ctrl*) * n_flows) != cudaSuccess ||
      cudaMalloc((void**)&b->ctrl_all, sizeof(Ctrl) * n_flows) != cudaSuccess ||
      cudaMalloc((void**)&b->done_dev, sizeof(int) * n_flows) != cudaSuccess ||
      cudaMallocHost((void**)&b->host_all, sizeof(Ctrl) * n_flows) != cudaSuccess ||
      cudaMallocHost((void**)&b->done_host, 2 * sizeof(int) * n_flows) != cudaSuccess)
    return fail(batch_err(b, JKO_ERR_OOM, "batch allocation"));
  if (cudaMemcpy(b->ctrl_ptrs, ptrs.data(), sizeof(Ctrl*) * n_flows, cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return fail(batch_err(b, JKO_ERR_CUDA, "upload of control pointers"));
  const int C = b->C;
  // tile shapes for the batch as a whole: with every flow on automatic
  // kernels, time the candidates on the batch graph and keep the fastest
  bool tune = true;
  for (int f = 0; f < n_flows; ++f)
    tune = tune && params[f].loop == 0 && params[f].tile == 0 && b->h[f]->tc &&
           !b->h[f]->tc_multi;
  b->in_group.assign(n_flows, 0);
  if (tune) {
    jko_status st = tune_batch(b);
    if (st != JKO_OK) return fail(st);
  } else {
    // flows asking for the grouped kernel (loop = 3)
    std::vector<char> sel(n_flows, 0);
    bool any = false;
    for (int f = 0; f < n_flows; ++f) any |= (sel[f] = params[f].loop == 3 && b->h[f]->tc) != 0;
    if (any) {
      jko_status st = make_groups(b, sel);
      if (st != JKO_OK) return fail(st);
    }
  }
  for (auto* h : b->h)
    if (h->tc) h->chunk_iters = h->use_loop ? h->prm.max_iter + 1 : C;
  jko_status s = capture_batch(
      b, no_op, [](jko_handle* h, cudaStream_t st) { return flow_prologue(h, st); },
      [b](cudaStream_t root) { return begin_groups(b, root); }, &b->g_pro);
  if (s != JKO_OK) return fail(s);
  auto capture_chunks = [&]() {
    const bool pp = b->per_pass;
    return capture_batch(
        b, [b, pp](cudaStream_t root) { return pp ? cudaSuccess : launch_groups(b, root); },
        [C, pp](jko_handle* h, cudaStream_t st) { return flow_chunk(h, C, pp, st); },
        [b](cudaStream_t root) { return jko::launch_gather_done(b->ctrl_ptrs, b->done_dev, b->n, root); },
        &b->g_chunk, !pp);
  };
  s = capture_chunks();
  if (s != JKO_OK) {
    // cooperative launches that cannot be captured: per-pass kernels instead
    cudaGetLastError();
    b->per_pass = true;
    s = capture_chunks();
  }
  if (s != JKO_OK) return fail(s);
  // every flow on the loop kernel: one chunk launch covers the whole budget
  bool all_loop = !b->per_pass;
  for (auto* h : b->h) all_loop = all_loop && h->use_loop;
  if (all_loop) b->C = b->max_iter + 1;
  s = capture_batch(
      b, no_op, [](jko_handle* h, cudaStream_t st) { return flow_finalize(h, st); },
      [b](cudaStream_t root) { return jko::launch_gather_ctrl(b->ctrl_ptrs, b->ctrl_all, b->n, root); },
      &b->g_fin);
  if (s != JKO_OK) return fail(s);
  *out = b;
  return JKO_OK;
}

jko_status jko_batch_info(const jko_batch* b, int* out) {
  if (!b || !out) return batch_err(nullptr, JKO_ERR_INVALID_ARG, "NULL batch or out");
  int nl = 0, ng = 0;
  for (int f = 0; f < b->n; ++f) {
    const bool grouped = !b->per_pass && !b->in_group.empty() && b->in_group[f];
    nl += (b->h[f]->use_loop && !b->per_pass && !grouped) ? 1 : 0;
    ng += grouped ? 1 : 0;
  }
  out[0] = b->tuned;
  out[1] = nl;
  out[2] = b->per_pass ? 1 : 0;
  out[3] = ng;
  out[4] = b->per_pass ? 0 : (int)b->groups.size();
  return JKO_OK;
}

jko_status jko_batch_flow(jko_batch* b, const void* const* p0_dev, int n_steps,
                          void* const* p_final_dev, jko_step_info* infos) {
  if (!b) return batch_err(nullptr, JKO_ERR_INVALID_ARG, "NULL batch");
  if (!p0_dev || n_steps < 0) return batch_err(b, JKO_ERR_INVALID_ARG, "NULL p0 or n_steps < 0");
  b->err.clear();
  cudaStream_t st = b->stream;
  for (int f = 0; f < b->n; ++f) {
    jko_handle* h = b->h[f];
    h->stream = st;
    if (!p0_dev[f]) return batch_err(b, JKO_ERR_INVALID_ARG, "NULL p0 entry");
    jko_status s = h->fp64 ? check_input<double>(h, (const double*)p0_dev[f], f, b)
                           : check_input<float>(h, (const float*)p0_dev[f], f, b);
    if (s != JKO_OK) return s;
  }
  for (int f = 0; f < b->n; ++f)
    BCK(b, cudaMemcpyAsync(b->h[f]->q, p0_dev[f], b->h[f]->es * (size_t)b->h[f]->ns,
                           cudaMemcpyDeviceToDevice, st));
  const int n = b->n, C = b->C;
  const int max_chunks = (b->max_iter + 1 + C - 1) / C + 2;
  int worst = JKO_OK;
  for (int t = 0; t < n_steps; ++t) {
    BCK(b, cudaGraphLaunch(b->g_pro, st));
    int launched = 0, polled = 0;
    auto launch = [&]() -> cudaError_t {
      cudaError_t e = cudaGraphLaunch(b->g_chunk, st);
      if (e != cudaSuccess) return e;
      const int slot = launched & 1;
      e = cudaMemcpyAsync(b->done_host + slot * n, b->done_dev, sizeof(int) * n,
                          cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaEventRecord(b->ev_poll[slot], st);
      ++launched;
      return e;
    };
    int ahead = std::max(1, std::min(b->last_iters / C, max_chunks));
    for (int i = 0; i < ahead; ++i) BCK(b, launch());
    bool stopped = false;
    while (!stopped) {
      if (launched - polled < 2 && launched < max_chunks) BCK(b, launch());
      const int target = launched - 1 - ((launched - polled) >= 2 ? 1 : 0);
      const int slot = target & 1;
      BCK(b, cudaEventSynchronize(b->ev_poll[slot]));
      polled = target + 1;
      stopped = true;
      for (int f = 0; f < n && stopped; ++f) stopped = b->done_host[slot * n + f] != jko::RUNNING;
      if (!stopped && launched >= max_chunks && polled >= launched)
        return batch_err(b, JKO_ERR_TIMEOUT, "a flow did not report a stop within its budget");
    }
    BCK(b, cudaGraphLaunch(b->g_fin, st));
    BCK(b, cudaMemcpyAsync(b->host_all, b->ctrl_all, sizeof(Ctrl) * n, cudaMemcpyDeviceToHost, st));
    BCK(b, cudaStreamSynchronize(st));
    int max_it = 0;
    for (int f = 0; f < n; ++f) {
      const Ctrl& c = b->host_all[f];
      jko_status sf = JKO_OK;
      if (c.nonfinite & 2) sf = JKO_ERR_TIMEOUT;
      else if (c.done == jko::NONFINITE || c.nonfinite) sf = JKO_ERR_NUMERIC;
      else if (c.done == jko::MAX_ITER || c.done == jko::STALLED) sf = JKO_NOT_CONVERGED;
      worst = worse(worst, sf);
      max_it = std::max(max_it, c.it);
      if (infos) {
        jko_step_info& in = infos[(size_t)t * n + f];
        in.iters = c.it;
        in.status = sf;
        in.residual_l1 = c.res_last;
        in.mass = c.mass;
        double mx;
        std::memcpy(&mx, &c.maxpk_bits, sizeof mx);
        in.max_p_over_kappa = b->h[f]->has_kappa ? mx : 0.0;
        in.ms = 0.f;
        in.kernels = 0;
      }
    }
    b->last_iters = max_it;
  }
  if (p_final_dev)
    for (int f = 0; f < n; ++f)
      if (p_final_dev[f])
        BCK(b, cudaMemcpyAsync(p_final_dev[f], n_steps > 0 ? b->h[f]->q : p0_dev[f],
                               b->h[f]->es * (size_t)b->h[f]->ns, cudaMemcpyDeviceToDevice, st));
  BCK(b, cudaStreamSynchronize(st));
  return (jko_status)worst;
}

jko_status jko_batch_step(jko_batch* b, const void* const* q_dev, void* const* p_out_dev,
                          jko_step_info* infos) {
  if (!b) return batch_err(nullptr, JKO_ERR_INVALID_ARG, "NULL batch");
  if (!q_dev || !p_out_dev) return batch_err(b, JKO_ERR_INVALID_ARG, "NULL q or p_out array");
  for (int f = 0; f < b->n; ++f)
    if (!p_out_dev[f]) return batch_err(b, JKO_ERR_INVALID_ARG, "NULL p_out entry");
  return jko_batch_flow(b, q_dev, 1, p_out_dev, infos);
}

jko_status jko_batch_destroy(jko_batch* b) {
  free_batch(b);
  return JKO_OK;
}

const char* jko_batch_last_error(const jko_batch* b) {
  return b ? b->err.c_str() : g_create_err.c_str();
}

}  // extern "C"
