// jko_kernels.h -- host-side launch interface of the JKO kernels (internal).
#pragma once
#include <vector>

#include <cuda_runtime.h>
#include <stdint.h>

#include "jko_internal.cuh"

namespace jko {

// Epilogue kinds of a filter pass.
enum : int { EPI_STORE = 0, EPI_B = 1, EPI_A = 2 };

// One separable filter pass: out[j][i'] = sum_i k(|i'-i|) in[i][j] followed by
// the epilogue.  in is [n_i][n_j]; out (and p, q) are [n_j][n_i].
template <typename T>
struct PassArgs {
  const T* in;
  T* out;        // EPI_STORE: filtered image; EPI_B: b (read old, write new); EPI_A: a
  T* p;          // EPI_A: p = a s
  const T* q;    // EPI_B: target marginal q
  const T* taps; // k(d) for d = -r..r, then simt_tap_padding() zeros
  int n_i, n_j, r;
  Ctrl* ctrl;
  double* part;  // residual partials: one per block of the b-update pass
  int nparts;    // number of partials (read by the deciding pass)
  int decide;    // 1: this pass takes the stop decision (stop_gate)
  int latency;   // 1: small images take the 4-output, shared-memory-staged variant
                 // (a handle alone); 0: always 16 outputs per thread (flows of a
                 // batch, where other flows fill the GPU)
  // nz > 1 (EPI_STORE, EPI_B): one launch filters nz images of the same
  // shape, in_z[z] -> out_z[z] (EPI_B: against q_z[z], partials of image z at
  // part + z * blocks per image) at blockIdx.z; in, out and q are then unused
  int nz = 1;
  const T* in_z[3] = {nullptr, nullptr, nullptr};
  T* out_z[3] = {nullptr, nullptr, nullptr};
  const T* q_z[3] = {nullptr, nullptr, nullptr};
};

// FFT form of the pass (fft_filter.cu): the same out[j][i'] and epilogues by
// convolution through a transform of length L (a power of two >= n_i + r).
// khat: the real spectrum of the circulant embedding of the taps, with 1/L
// (L entries); tw: e^{-2 pi i j / L}, j < L/2, interleaved re, im.
template <typename T>
struct FftArgs {
  int L = 0, log2L = 0;
  const T* khat = nullptr;
  const T* tw = nullptr;
};
// Longest transform per element type (the block's 4 lines and twiddles in
// shared memory).
template <typename T> constexpr int fft_max_length() { return sizeof(T) == 4 ? 4096 : 2048; }
template <typename T>
cudaError_t fft_pass(int epi, int ek, const PassArgs<T>& A, const ProxArgs<T>& P,
                     const FftArgs<T>& F, cudaStream_t st);
// Blocks of an FFT pass over an [n_i][n_j] input (= its residual partials).
int fft_pass_blocks(int n_j);
// Host tables of one axis (n cells, band radius r): false if L > max_len.
bool fft_axis_tables(int n, int r, double length, double gamma, int max_len, int* L, int* log2L,
                     std::vector<double>* khat, std::vector<double>* tw);

int simt_tap_padding();
// Blocks of a filter pass over an [n_i][n_j] input (= residual partials of the
// b-update pass).
int simt_pass_blocks(int n_i, int n_j, int latency = 1, int fp64 = 0);

template <typename T>
cudaError_t simt_pass(int epi, int ek, const PassArgs<T>& A, const ProxArgs<T>& P,
                      cudaStream_t st);

// Step prologue / epilogue kernels (jko_step_kernels.cu).
template <typename T>
cudaError_t launch_fill(T* x, T v, long long n, cudaStream_t st);

// Counts invalid entries of q into ctrl (q_sum, q_neg, q_bad, q_over, q_masked).
template <typename T>
cudaError_t launch_validate(const T* q, long long n, const ProxArgs<T>& P, Ctrl* ctrl,
                            cudaStream_t st);

// ctrl->mass = sum p (FP64, fixed summation order: one partial per block in
// part[0 .. min(blocks, part_cap)), added by the last block), ctrl->maxpk_bits
// = max p/kappa, flags non-finite p.  part must not be in use by other work.
template <typename T>
cudaError_t launch_finalize_reduce(const T* p, long long n, const ProxArgs<T>& P, Ctrl* ctrl,
                                   double* part, int part_cap, cudaStream_t st);

// The condition of the device-side chunk loop (a graph WHILE node whose body
// is one chunk of pairs and then this kernel): counts the chunk in *chunks
// (reset by the step's start) and continues while the step runs and fewer
// than max_chunks chunks have run, so that the loop ends after max_chunks
// chunks at most.
cudaError_t launch_chunk_loop_cond(unsigned* chunks, const Ctrl* ctrl,
                                   cudaGraphConditionalHandle hc, unsigned max_chunks,
                                   cudaStream_t st);

// out = renorm ? p / ctrl->mass : p   (out may alias p); check = 1: nothing is
// written when the step's input checks (launch_validate into the same ctrl)
// found q invalid
// record (may be NULL): receives the step's final control block
template <typename T>
cudaError_t launch_finalize_write(const T* p, T* out, long long n, int renorm, const Ctrl* ctrl,
                                  cudaStream_t st, int check = 0, Ctrl* record = nullptr);

// The start of a step in one launch: *ctrl = init, *chunks = 0 (chunks may be
// NULL), q[0..nq) = q_in (q_in may be NULL: nothing copied), a[0..na) = 1 (a
// may be NULL).
template <typename T>
cudaError_t launch_step_begin(const Ctrl& init, Ctrl* ctrl, unsigned* chunks, const T* q_in,
                              T* q, long long nq, T* a, long long na, cudaStream_t st);

// Wasserstein attraction (attraction.cu): p = Prox(s1^{1/(1+tau)} s2^{tau/(1+tau)}),
// a_m = p / s_m, and the pair counter; returns at once once the step has stopped.
template <typename T>
cudaError_t launch_attraction_prox(int ek, const T* s1, const T* s2, T* a1, T* a2, T* p,
                                   long long n, double tau, const ProxArgs<T>& P, Ctrl* ctrl,
                                   cudaStream_t st, int rnd = 0);

// Two species (attraction.cu): p = [p_1, p_2] = a~_m min(1, kappa/(a~_1 + a~_2)),
// a~_m = s_m E_m (E_m = e^{-sigma w_m}, NULL = 1); a_m = E_m min(...).
template <typename T>
cudaError_t launch_species_prox(const T* s1, const T* s2, const T* E1, const T* E2, T* a1, T* a2,
                                T* p, long long n, double kappa, int has_kappa, Ctrl* ctrl,
                                cudaStream_t st, int rnd = 0);

// (rnd = 1: the scalings a_m, b_m written by these kernels are rounded to tf32,
// the operands of the tensor-core passes of tc_multi.cu.)
// Pairwise attraction of two densities (attraction.cu; Sec. 5.3, 3 couplings):
// the row half-step (psi_1) and the column half-step (psi_2, with the residual
// partials of the stop rule, p_2 and the pair counter).  E1, E2 = e^{-sigma' w_m}
// with sigma' = sigma / (1 + t), t = tau alpha.
int pairwise_blocks(long long n);
template <typename T>
cudaError_t launch_pairwise_rows(const T* s1, const T* s2, const T* s3, const T* E1, const T* q2,
                                 T* a1, T* a2, T* a3, T* p1, long long n, double t, double kappa,
                                 int has_kappa, Ctrl* ctrl, cudaStream_t st, int rnd = 0);
template <typename T>
cudaError_t launch_pairwise_cols(const T* y1, const T* y2, const T* y3, const T* E2, const T* q1,
                                 T* b1, T* b2, T* b3, T* p2, double* part, long long n, double t,
                                 double kappa, int has_kappa, Ctrl* ctrl, cudaStream_t st,
                                 int rnd = 0);

// Heat-kernel Gibbs kernel (heat.cu): xi~ = (Id - (gamma/L) Delta_M)^{-L} as
// the Chebyshev expansion of lambda^{-L} on the spectrum interval [1, lmax].
constexpr int kMaxHeatDegree = 1500;
struct HeatPlan {
  int L = 0;
  int D = 0;                    // degree of the expansion (-1: above kMaxHeatDegree)
  double cx = 0, cy = 0;        // (gamma / L) / hx^2, (gamma / L) / hy^2
  double theta = 0, delta = 0;  // centre and half-width of [1, lmax]
  std::vector<double> coef;     // Chebyshev coefficients c_0 .. c_D
};
struct HeatBuffers {
  void* d[4] = {nullptr, nullptr, nullptr, nullptr};   // Clenshaw iterates (FP64, N each)
  void* coef = nullptr;                                // c_0 .. c_D (FP64) for the persistent form
};
HeatPlan heat_plan(int nx, int ny, double lx, double ly, double gamma, int L, bool fp64);
int heat_blocks(int nx, int ny);   // blocks of heat_bupdate (= residual partials)
int heat_launches(const HeatPlan& hp);   // kernel launches of one heat_apply
// out_x = xi~ in (the first init takes the stop decision when decide = 1);
// linear = true leaves the output unclamped (signed inputs, the adjoint), else
// it is clamped at 0 (xi~ is positive; the expansion's normwise error can turn
// far tails slightly negative)
template <typename T>
cudaError_t heat_apply(const HeatPlan& hp, const HeatBuffers& B, const T* in, T* out_x,
                       int nx, int ny, const uint8_t* mask, Ctrl* ctrl, const double* part,
                       int nparts, int decide, cudaStream_t st, bool linear = false);
template <typename T>
cudaError_t heat_bupdate_launch(const T* Y, T* b, const T* q, int nx, int ny, Ctrl* ctrl,
                                double* part, cudaStream_t st);
template <typename T>
cudaError_t heat_prox_launch(int ek, const T* s, T* a, T* p, int nx, int ny, const ProxArgs<T>& P,
                             Ctrl* ctrl, cudaStream_t st);
// Persistent form: one cooperative launch of G blocks (heat_loop_grid; 0 =
// unavailable) runs up to `pairs` pairs with the stop rule inside, with the
// arithmetic and the pair counts of the kernels above.
int heat_loop_grid(int nx, int ny, bool fp64, int ek);
template <typename T>
cudaError_t heat_loop_launch(const HeatPlan& hp, const HeatBuffers& B, int ek, const T* q, T* a,
                             T* b, T* p, int nx, int ny, const uint8_t* mask, const ProxArgs<T>& P,
                             Ctrl* ctrl, double* part, int G, int pairs, cudaStream_t st);

// Batched flows: copy the stop state of n control blocks into a contiguous
// array (done flags only, or whole blocks).
// A stopped step runs on: done = RUNNING, the stall counters restart (the
// pair counter, the budget and the smallest residual carry over).
cudaError_t launch_resume(Ctrl* ctrl, cudaStream_t st);
cudaError_t launch_gather_done(Ctrl* const* ctrls, int* done, int n, cudaStream_t st);
cudaError_t launch_gather_ctrl(Ctrl* const* ctrls, Ctrl* out, int n, cudaStream_t st);

}  // namespace jko
