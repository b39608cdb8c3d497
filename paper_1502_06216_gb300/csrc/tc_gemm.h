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
  ProxArgs<float> prox;
};

struct TcPlan;

// 0 = ok, 1 = unsupported configuration (message set), 2 = CUDA error.
int tc_create(const TcConfig& cfg, TcPlan** out, std::string* msg);
// Per-step reset of the scaling operands (a = 1).
cudaError_t tc_begin_step(TcPlan* plan, cudaStream_t st);
// One (odd, even) pair: four tensor-core passes with fused epilogues.
cudaError_t tc_enqueue_pair(TcPlan* plan, cudaStream_t st);
void tc_destroy(TcPlan* plan);

}  // namespace jko
