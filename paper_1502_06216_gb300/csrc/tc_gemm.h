// tc_gemm.h -- tensor-core (tcgen05 / TMA / TMEM) form of the Gibbs-kernel
// application with the fused scaling and proximal epilogues (internal).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "jko_internal.cuh"

namespace jko {

struct TcConfig {
  int nx, ny;
  double lx, ly, gamma;
  int precision;  // JKO_TF32 / JKO_BF16 / JKO_BF16X3
  int ek;         // energy kind of the proximal epilogue
  float* a;       // handle images (float, [ny][nx])
  float* b;
  float* p;
  const float* q;
  Ctrl* ctrl;
  double* part;   // residual partials (tc_partials(cfg) doubles)
  ProxArgs<float> prox;
  // separable log-domain absorption of the potential
  int absorb;             // 1: absorb (resolved by the caller)
  const double* w_host;   // potential (host, N doubles) or NULL
  double sigma;           // tau / gamma
};



// Number of residual partials (blocks of the b-update pass) for a grid.
int tc_partials(int nx, int ny);

struct TcPlan;

// 1 when the plan carries an absorbed potential (it then owns its energy images).
int tc_absorbed(const TcPlan* plan);

// 0 = ok, 1 = unsupported configuration (message set), 2 = CUDA error.
int tc_create(const TcConfig& cfg, TcPlan** out, std::string* msg);
// Log-domain form (tc_log.cu): every image carries base-2 exponents per row and
// group of 32 cells, the factor one per row and K-block; TF32 plans without
// separable absorption, per-pass kernels, the congestion/potential energy.
// 0 = ok, 1 = unsupported (message set), 2 = CUDA error.
int tc_log_setup(TcPlan* plan, const double* w_host, double sigma, std::string* msg);
int tc_logdomain(const TcPlan* plan);
// Passes of the steps with several couplings on a TF32, BF16 or BF16x3 plan
// (tc_multi.cu): one launch applies the pass over `axis` (0: x, in [ny][nx] ->
// out [nx][ny]; 1: y, in [nx][ny] -> out [ny][nx]) to nz <= 3 images (nx, ny
// multiples of 4 for TF32, of 8 for the bf16 forms).  Inputs are operand
// images: fp32 (TF32), or one buffer per image with the bf16 pair
// hi [rows][cols] then lo (BF16, BF16x3).  epi: EPI_STORE (out as operand image: rounded to tf32, or the
// pair), EPI_B (b = q / D as fp32, rounded to tf32 in the TF32 form; residual
// partials of image z at part + z * tiles), TC_EPI_RAW (out as fp32).  The
// pass takes the stop decision on `nparts` partials when decide = 1.
constexpr int TC_EPI_RAW = 3;
int tc_multi_tiles(int nx, int ny, int axis);
cudaError_t tc_multi_pass(TcPlan* plan, int axis, int nz, const void* const* in, void* const* out,
                          int epi, const float* const* q, double* part, int nparts, int decide,
                          cudaStream_t st);
// fp32 images x_z of n elements -> their bf16 pairs (hi at pairs[z], lo n
// elements after), the operands of the bf16 forms' first pass.
cudaError_t tc_split_pairs(int nz, const float* const* x, void* const* pairs, long long n,
                           cudaStream_t st);
int tc_mode(const TcPlan* plan);   // MODE_BF16 = 0, MODE_BF16X3 = 1, MODE_TF32 = 2
// Per-step reset of the scaling operands (a = 1).
cudaError_t tc_begin_step(TcPlan* plan, cudaStream_t st);
// The current scalings a, b as fp32 [ny][nx] images (the operand values the
// passes multiply with), for a step that continues on the CUDA-core form.
// Not for absorbed plans (their scalings carry the factor e^{beta}).
cudaError_t tc_export_scalings(const TcPlan* plan, float* a, float* b, cudaStream_t st);
// Pass `which` (0..3) of one (odd, even) pair, same numbering as the SIMT form.
cudaError_t tc_enqueue_pass(TcPlan* plan, int which, cudaStream_t st);
// Multiply-add flops (x2) of the tiles pass `which` executes.
double tc_pass_flops(const TcPlan* plan, int which);
// Output tile width of the per-pass kernels: 64, or 128 (not BF16X3).
// tc_set_tile returns 1 for a width the precision does not have.
int tc_tile(const TcPlan* plan);
int tc_set_tile(TcPlan* plan, int bn);
void tc_destroy(TcPlan* plan);

// Persistent pair-loop kernel (tc_loop.cu).  Set-up after the plan's images
// and maps exist: 0 = ok (tc_loop_supported tells whether it can run),
// 2 = CUDA error.
int tc_loop_setup(TcPlan* plan, std::string* msg);
int tc_loop_supported(const TcPlan* plan);
int tc_loop_resident(const TcPlan* plan);
// One cooperative launch running up to `pairs` pairs of the scaling loop with
// the stop protocol in the kernel (same Ctrl as the per-pass kernels).
cudaError_t tc_enqueue_loop(TcPlan* plan, int pairs, cudaStream_t st);
// Executed tensor-core flops of `pairs` pairs of the loop kernel.
double tc_loop_flops(const TcPlan* plan, int pairs);
// Grouped persistent kernel (tc_loop.cu): one cooperative launch runs the
// scaling loop of several flows of one precision and energy kind, each with
// its own stop rule in its own Ctrl.  Create: 0 = ok, 1 = not groupable (message set), 2 = CUDA
// error.  begin_step resets the launch's grid-barrier words (once per step).
struct TcGroup;
int tc_group_create(TcPlan* const* plans, int n, TcGroup** out, std::string* msg);
cudaError_t tc_group_begin_step(TcGroup* g, cudaStream_t st);
cudaError_t tc_group_enqueue(TcGroup* g, int pairs, cudaStream_t st);
int tc_group_flows(const TcGroup* g);
double tc_group_flops(const TcGroup* g, int pairs);
void tc_group_destroy(TcGroup* g);

}  // namespace jko
