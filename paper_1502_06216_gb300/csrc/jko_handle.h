// jko_handle.h -- the solver handle behind the C ABI (internal to libjko).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "jko.h"
#include "jko_internal.cuh"
#include "jko_kernels.h"
#include "tc_gemm.h"

using jko::Ctrl;
using jko::ProxArgs;

struct jko_handle {
  jko_grid grid{};
  jko_params prm{};
  int N = 0;
  int prec = JKO_FP32;
  int ek = jko::EK_CROWD;
  bool fp64 = false;
  size_t es = 4;  // element size of device images
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;  // private stream used for graph capture

  // working images (es bytes per element)
  void *a = nullptr, *b = nullptr, *t1 = nullptr, *p = nullptr, *q = nullptr;
  void *stage_in = nullptr, *stage_out = nullptr;  // for the host-buffer entry point
  // Gibbs factors (SIMT taps, centred and zero padded)
  void *taps_x = nullptr, *taps_y = nullptr;
  int rx = 0, ry = 0;
  // per-cell energy constants
  void *E = nullptr, *sw = nullptr, *c = nullptr, *kap = nullptr;
  void* m1f = nullptr;          // per-cell m - 1 of the generalised entropies, or NULL
  int binary = 0;               // congestion iota_{{0,kappa}} (Eq. dfn-congestion-noncvx)
  // Wasserstein attraction (Sec. 5.2): second coupling's scalings, the target
  // r and the two prox inputs xi b_m
  int attract = 0;
  int simt_latency = 1;         // small CUDA-core passes in their latency form (0 in batches)
  int species = 1;              // 2: two densities coupled through their sum (Sec. 5.3)
  void* E2 = nullptr;           // e^{-sigma w2} of the second species
  long long ns = 0;             // elements of a state image: N, or 2 N for two species
  int heat_L = 0;               // > 0: the heat-kernel Gibbs kernel (heat.cu)
  int fft = 0;                  // 1: the Gaussian applied by FFT convolution (fft_filter.cu)
  void *fft_khat_x = nullptr, *fft_tw_x = nullptr, *fft_khat_y = nullptr, *fft_tw_y = nullptr;
  int fft_Lx = 0, fft_lgx = 0, fft_Ly = 0, fft_lgy = 0;
  double pair_alpha = 0;        // > 0 (two species): pairwise attraction, 3 couplings
  void* t2 = nullptr;           // transposed intermediates of batched filter passes
  void* t3 = nullptr;
  void* a3 = nullptr;           // scalings and kernel image of the third coupling
  void* b3 = nullptr;
  void* s3 = nullptr;
  int nparts_pw = 0;            // residual partials of the pairwise column half-step
  jko::HeatPlan heat;
  jko::HeatBuffers hb;
  void *a2 = nullptr, *b2 = nullptr, *tgt = nullptr, *s1 = nullptr, *s2 = nullptr;
  uint8_t* mask = nullptr;
  double kappa_s = INFINITY;
  int has_kappa = 0;
  double m = 0.0;

  Ctrl* ctrl = nullptr;        // device control block
  double* part = nullptr;      // residual partials of the b-update pass (one per block)
  int nparts_simt = 0;
  int part_cap = 0;       // entries of part (residual and mass partials)
  int use_loop = 0;       // chunks run as one persistent kernel (tensor cores or heat kernel)
  int heat_G = 0;         // blocks of the heat kernel's persistent form
  int tc_multi = 0;       // several couplings on the tensor cores (tc_multi.cu)
  void* mpair = nullptr;  // bf16 forms of several couplings: pairs of the first pass's images
  Ctrl* ctrl_init = nullptr;   // pinned initial value
  Ctrl* poll = nullptr;        // pinned, 2 slots for pipelined polls
  cudaEvent_t ev_poll[2] = {nullptr, nullptr};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  cudaGraphExec_t chunk = nullptr;
  int chunk_iters = 16;
  int last_iters = 0;
  // a tensor-core step that stalled continues on the FP32 CUDA-core form
  // (jko_params.finish): its chunk of pairs, and the pairs it took last
  cudaGraphExec_t chunk_fin = nullptr;
  int last_fin = 0;
  // flows: a step's chunks as a graph WHILE node (one chunk, then the loop
  // condition on the device), so that the steps after the first are enqueued
  // without a host wait between them; the control block after each of them
  // (pinned) and two events per step
  cudaGraphExec_t step_loop = nullptr;
  int step_loop_state = 0;      // 0 not built, 1 built, -1 not available (host-driven chunks)
  unsigned* chunk_ctr = nullptr;  // device: chunks the loop has run in this step
  Ctrl* flow_ctrl = nullptr;       // pinned host copy
  Ctrl* flow_ctrl_dev = nullptr;   // device: written by each step's last kernel
  int flow_cap = 0;
  std::vector<cudaEvent_t> flow_ev;

  jko::TcPlan* tc = nullptr;   // tensor-core path state (JKO_TF32/BF16/BF16X3)
  long long kernels = 0;       // kernels enqueued by the running step

  // differentiation tape (jko_flow_record / jko_flow_backward)
  int tape_steps = 0;           // steps recorded
  int tape_cap = 0;             // steps the tape can hold
  void* tape = nullptr;         // per step: q_t and the final a_t (2 N elements)
  std::vector<double> tape_mass;  // sum of the unnormalised output per step
  void* adj = nullptr;          // adjoint work images (10 N elements)
  void* adj2 = nullptr;         // the attraction's adjoint work images (18 N elements)
  double* adj_red = nullptr;    // device reduction slots

  std::string err;
};


namespace jko {
template <typename T>
inline ProxArgs<T> prox_args(const jko_handle* h) {
  ProxArgs<T> P;
  P.E = (const T*)h->E;
  P.sw = (const T*)h->sw;
  P.c = (const T*)h->c;
  P.kappa = (const T*)h->kap;
  P.m1f = (const T*)h->m1f;
  P.kappa_s = (T)h->kappa_s;
  P.mask = h->mask;
  P.m1 = (T)(h->m - 1.0);
  P.newton = 40;
  P.has_kappa = h->has_kappa;
  P.binary = h->binary;
  P.sigma = (T)(h->prm.tau / h->prm.gamma);
  return P;
}

// One JKO step on device buffers (jko_api.cu); validate = check q first.
jko_status step_internal(jko_handle* h, const void* q_in, void* p_out, jko_step_info* info,
                         bool validate);
// Records an error message on the handle and returns the status.
jko_status handle_error(jko_handle* h, jko_status st, const std::string& msg);
// Argument checks of jko_create (sizes, parameters, energy fields): JKO_OK, or
// the error status with *msg set to a static description.  Allocates nothing
// and makes no device call, so jko_step_noalloc runs the same checks.
jko_status check_create_args(const jko_grid* g, const jko_params* p, const jko_energy* en,
                             const char** msg);

}  // namespace jko
