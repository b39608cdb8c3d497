// jko_noalloc.cu -- jko_step_noalloc: one JKO step that allocates no memory.
//
// Some callers cannot allocate device memory at the moment they need a step:
// code that runs inside a framework which owns all device memory through its
// own pool (a cudaMalloc there bypasses the pool's accounting and a cudaFree
// synchronises the whole device, stalling every other stream), or a
// long-running service that forbids allocation after start-up.  For them this
// entry point runs the same FP32 CUDA-core kernels as jko_step, with every
// working buffer carved out of one file-scope device array of fixed size.
//
// Limits: JKO_FP32 only, nx <= 256, ny <= 256 (N <= 65536 cells).  The array
// is kJkoNoallocScratchBytes (about 3 MB) and every GPU that loads the library
// holds it until the process exits.  All calls share it: two calls whose work
// overlaps on the GPU (different streams or threads, or host threads racing)
// race on it and produce garbage.  Each call re-initialises everything it
// reads (control block, a = 1, p = 0, energy constants, taps), so nothing
// depends on what the previous call left behind.
#include <cmath>
#include <cstring>
#include <mutex>

#include "jko.h"
#include "jko_handle.h"
#include "jko_kernels.h"

namespace {

using jko::Ctrl;
using jko::PassArgs;
using jko::ProxArgs;

constexpr int kMaxSide = 256;
constexpr long long kMaxCells = 65536;
constexpr int kTapPad = 16;  // equals simt_tap_padding(); checked at run time
constexpr int kMaxDevices = 64;

// Byte layout of the scratch array (every offset is a multiple of 256).
constexpr size_t kImg = kMaxCells * sizeof(float);
enum : int { S_A = 0, S_B, S_T1, S_P, S_Q, S_E, S_SW, S_C, S_KAP, S_NIMG };
constexpr size_t kOffTapsX = S_NIMG * kImg;
constexpr size_t kTapBytes = 4096;  // >= (2*(kMaxSide-1)+1+kTapPad) floats
constexpr size_t kOffTapsY = kOffTapsX + kTapBytes;
constexpr size_t kOffMask = kOffTapsY + kTapBytes;
constexpr size_t kOffStage = kOffMask + kMaxCells;          // FP64 staging of host fields
constexpr size_t kOffCtrl = kOffStage + kMaxCells * sizeof(double);
constexpr size_t kOffPart = kOffCtrl + 256;                  // residual partials
constexpr int kMaxParts = 256;
constexpr size_t kJkoNoallocScratchBytes = kOffPart + kMaxParts * sizeof(double);
static_assert(sizeof(Ctrl) <= 256, "control block must fit its slot");
static_assert((2 * (kMaxSide - 1) + 1 + kTapPad) * sizeof(float) <= kTapBytes, "tap slot");

static __device__ __align__(256) unsigned char g_jko_noalloc_scratch[kJkoNoallocScratchBytes];

std::mutex g_mu;
void* g_base[kMaxDevices] = {};

// Device address of the scratch array for the current device, looked up once
// per device with that device current.  In host code the array's name is only
// a host-side stand-in, so kernels must receive this address instead.
cudaError_t scratch_base(unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_base[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_jko_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_base[dev] = p;
  }
  *out = (unsigned char*)g_base[dev];
  return cudaSuccess;
}

// Per-cell energy constants from an FP64 field staged in the scratch.
enum : int { F_EXP_NEG = 0, F_SCALE = 1, F_COPY = 2 };
__global__ void na_field_kernel(const double* src, float* dst, int n, int mode, double scale,
                                double dflt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double v = src ? src[i] : dflt;
    double o;
    if (mode == F_EXP_NEG) o = exp(-scale * v);
    else if (mode == F_SCALE) o = scale * v;
    else o = v;
    dst[i] = (float)o;
  }
}

// Centred Gibbs taps k(t - r) = exp(-((t - r) h)^2 / gamma), zero past 2r.
__global__ void na_taps_kernel(float* taps, int r, double h, double gamma, int len) {
  for (int t = threadIdx.x; t < len; t += blockDim.x) {
    const double d = (double)(t - r) * h;
    taps[t] = t <= 2 * r ? (float)exp(-d * d / gamma) : 0.0f;
  }
}

int tap_radius(int n, double length, double gamma) {
  const double h = length / n;
  int r = 0;
  for (int d = 0; d < n; ++d)
    if ((float)std::exp(-(d * h) * (d * h) / gamma) != 0.0f) r = d;
  return r;
}

// No message buffer: the status codes are the whole error report (documented
// in jko.h), so that nothing here allocates, not even host memory.
jko_status fail(jko_status s, const char*) { return s; }

jko_status cuda_fail(cudaError_t e) {
  return e == cudaErrorMemoryAllocation ? JKO_ERR_OOM : JKO_ERR_CUDA;
}

#define NA_CK(call)                           \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

jko_status stage_field(unsigned char* base, const double* host, long long N, float* dst, int mode,
                       double scale, double dflt, cudaStream_t st) {
  double* stage = (double*)(base + kOffStage);
  if (host)
    NA_CK(cudaMemcpyAsync(stage, host, N * sizeof(double), cudaMemcpyHostToDevice, st));
  na_field_kernel<<<64, 256, 0, st>>>(host ? stage : nullptr, dst, (int)N, mode, scale, dflt);
  NA_CK(cudaGetLastError());
  return JKO_OK;
}

}  // namespace

extern "C" jko_status jko_step_noalloc(const jko_grid* grid, const jko_params* prm,
                                       const jko_energy* en, const void* q_dev, void* p_out_dev,
                                       void* stream, jko_step_info* info) {
  if (!grid || !prm || !en || !q_dev || !p_out_dev)
    return fail(JKO_ERR_INVALID_ARG, "NULL argument");
  // every argument check of jko_create (parameters finite and in range, energy
  // fields, species and pair_alpha consistent), then the limits of this form
  const char* msg = "";
  const jko_status chk = jko::check_create_args(grid, prm, en, &msg);
  if (chk != JKO_OK) return fail(chk, msg);
  if (grid->nx > kMaxSide || grid->ny > kMaxSide)
    return fail(JKO_ERR_UNSUPPORTED,
                "jko_step_noalloc: grid exceeds the fixed scratch (nx, ny must be <= 256)");
  if (prm->precision != JKO_FP32)
    return fail(JKO_ERR_UNSUPPORTED, "jko_step_noalloc: only JKO_FP32 is available");
  if (en->m_field)
    return fail(JKO_ERR_UNSUPPORTED, "jko_step_noalloc: per-cell exponents (m_field) are not available");
  if (en->binary)
    return fail(JKO_ERR_UNSUPPORTED, "jko_step_noalloc: binary congestion is not available");
  if (en->target)
    return fail(JKO_ERR_UNSUPPORTED, "jko_step_noalloc: the Wasserstein attraction is not available");
  if (en->species == 2)
    return fail(JKO_ERR_UNSUPPORTED, "jko_step_noalloc: two species are not available");
  if (grid->fft != 0)
    return fail(JKO_ERR_UNSUPPORTED, "jko_step_noalloc: the FFT application is not available");
  if (grid->heat_L != 0)
    return fail(JKO_ERR_UNSUPPORTED, "jko_step_noalloc: the heat kernel is not available");
  if (jko::simt_tap_padding() != kTapPad)
    return fail(JKO_ERR_UNSUPPORTED, "jko_step_noalloc: tap padding mismatch");
  const int nx = grid->nx, ny = grid->ny;
  const long long N = (long long)nx * ny;

  unsigned char* base = nullptr;
  NA_CK(scratch_base(&base));
  cudaStream_t st = (cudaStream_t)stream;
  float* img[S_NIMG];
  for (int k = 0; k < S_NIMG; ++k) img[k] = (float*)(base + k * kImg);
  float* taps_x = (float*)(base + kOffTapsX);
  float* taps_y = (float*)(base + kOffTapsY);
  uint8_t* mask = (uint8_t*)(base + kOffMask);
  Ctrl* ctrl = (Ctrl*)(base + kOffCtrl);
  double* part = (double*)(base + kOffPart);
  const int nparts = jko::simt_pass_blocks(nx, ny);  // blocks of the b-update pass
  if (nparts > kMaxParts) return fail(JKO_ERR_UNSUPPORTED, "jko_step_noalloc: partials slot");

  // energy constants (same definitions as jko_create)
  const double sigma = prm->tau / prm->gamma;
  const int ek = en->m == 0.0 ? jko::EK_CROWD : (en->m == 1.0 ? jko::EK_ENTROPY : jko::EK_POWER);
  jko_status s;
  if (ek == jko::EK_CROWD) {
    s = stage_field(base, en->w, N, img[S_E], F_EXP_NEG, sigma, 0.0, st);
    if (s != JKO_OK) return s;
  } else {
    if (en->w) {
      s = stage_field(base, en->w, N, img[S_SW], F_SCALE, sigma, 0.0, st);
      if (s != JKO_OK) return s;
    }
    const double cs = ek == jko::EK_ENTROPY ? sigma : sigma * en->m / (en->m - 1.0);
    s = stage_field(base, en->alpha, N, img[S_C], F_SCALE, cs, 1.0, st);
    if (s != JKO_OK) return s;
  }
  int has_kappa = std::isfinite(en->kappa) ? 1 : 0;
  if (en->kappa_field) {
    s = stage_field(base, en->kappa_field, N, img[S_KAP], F_COPY, 1.0, 0.0, st);
    if (s != JKO_OK) return s;
    has_kappa = 0;
    for (long long i = 0; i < N; ++i) has_kappa |= std::isfinite(en->kappa_field[i]) ? 1 : 0;
  }
  if (en->mask) NA_CK(cudaMemcpyAsync(mask, en->mask, N, cudaMemcpyHostToDevice, st));

  ProxArgs<float> P;
  P.E = img[S_E];
  P.sw = en->w ? img[S_SW] : nullptr;
  P.c = img[S_C];
  P.kappa = en->kappa_field ? img[S_KAP] : nullptr;
  P.kappa_s = (float)en->kappa;
  P.mask = en->mask ? mask : nullptr;
  P.m1 = (float)(en->m - 1.0);
  P.newton = 40;
  P.has_kappa = has_kappa;
  P.sigma = (float)sigma;

  // Gibbs taps (Sec. 4.1), radius = last tap non-zero in FP32
  const int rx = tap_radius(nx, grid->lx, prm->gamma);
  const int ry = tap_radius(ny, grid->ly, prm->gamma);
  na_taps_kernel<<<1, 256, 0, st>>>(taps_x, rx, grid->lx / nx, prm->gamma, 2 * rx + 1 + kTapPad);
  NA_CK(cudaGetLastError());
  na_taps_kernel<<<1, 256, 0, st>>>(taps_y, ry, grid->ly / ny, prm->gamma, 2 * ry + 1 + kTapPad);
  NA_CK(cudaGetLastError());

  // control block and input validation (as jko_step)
  Ctrl init;
  std::memset(&init, 0, sizeof init);
  init.tol = prm->tol;
  init.max_iter = prm->max_iter;
  init.stall = prm->stall;
  Ctrl host;
  NA_CK(cudaMemcpyAsync(ctrl, &init, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
  NA_CK(jko::launch_validate<float>((const float*)q_dev, N, P, ctrl, st));
  NA_CK(cudaMemcpyAsync(&host, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
  NA_CK(cudaStreamSynchronize(st));
  if (host.q_bad || host.q_neg || std::fabs(host.q_sum - 1.0) > 1e-3 || host.q_masked ||
      host.q_over)
    return fail(JKO_ERR_INVALID_ARG,
                "jko_step_noalloc: q must be finite, >= 0, sum to 1, vanish on the mask and "
                "stay below kappa");
  NA_CK(cudaMemcpyAsync(ctrl, &init, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(img[S_Q], q_dev, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
  NA_CK(jko::launch_fill<float>(img[S_A], 1.0f, N, st));
  NA_CK(jko::launch_fill<float>(img[S_P], 0.0f, N, st));

  // the scaling loop: four passes per pair, polled every C pairs
  const int C = prm->check_every > 0 ? prm->check_every : 16;
  const int max_chunks = (prm->max_iter + 1 + C - 1) / C + 1;
  int kernels = 8;
  bool stopped = false;
  for (int chunk = 0; chunk < max_chunks && !stopped; ++chunk) {
    for (int it = 0; it < C; ++it) {
      for (int half = 0; half < 2; ++half) {
        PassArgs<float> A{};
        A.ctrl = ctrl;
        A.part = part;
        A.nparts = nparts;
        A.decide = half == 1 ? 1 : 0;   // the pass after the b-update decides
        A.latency = 1;                  // the form simt_pass_blocks counted (nparts)
        A.in = half == 0 ? img[S_A] : img[S_B];
        A.out = img[S_T1];
        A.taps = taps_y;
        A.n_i = ny; A.n_j = nx; A.r = ry;
        NA_CK(jko::simt_pass<float>(jko::EPI_STORE, ek, A, P, st));
        A.decide = 0;
        A.in = img[S_T1];
        A.out = half == 0 ? img[S_B] : img[S_A];
        A.p = img[S_P];
        A.q = img[S_Q];
        A.taps = taps_x;
        A.n_i = nx; A.n_j = ny; A.r = rx;
        NA_CK(jko::simt_pass<float>(half == 0 ? jko::EPI_B : jko::EPI_A, ek, A, P, st));
        kernels += 2;
      }
    }
    NA_CK(cudaMemcpyAsync(&host, ctrl, 16, cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    stopped = host.done != jko::RUNNING;
  }
  if (!stopped) return fail(JKO_ERR_TIMEOUT, "jko_step_noalloc: no stop within the budget");

  NA_CK(jko::launch_finalize_reduce<float>(img[S_P], N, P, ctrl, part, kMaxParts, st));
  NA_CK(jko::launch_finalize_write<float>(img[S_P], (float*)p_out_dev, N, prm->renormalize, ctrl, st));
  NA_CK(cudaMemcpyAsync(&host, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
  NA_CK(cudaStreamSynchronize(st));
  jko_status out = JKO_OK;
  if (host.done == jko::NONFINITE || host.nonfinite) out = JKO_ERR_NUMERIC;
  else if (host.done == jko::MAX_ITER || host.done == jko::STALLED) out = JKO_NOT_CONVERGED;
  if (info) {
    info->iters = host.it;
    info->status = out;
    info->residual_l1 = host.res_last;
    info->mass = host.mass;
    double mx;
    std::memcpy(&mx, &host.maxpk_bits, sizeof mx);
    info->max_p_over_kappa = has_kappa ? mx : 0.0;
    info->ms = 0.0f;
    info->kernels = kernels;
  }
  return out;
}
