// fft_filter.cu -- the Gibbs-kernel application by FFT convolution (CUDA
// cores, FP32 / FP64): the same pass as filter_pass (simt_filter.cu),
//     out[j][i'] = sum_i k(|i' - i|) in[i][j],   in: [n_i][n_j], out: [n_j][n_i],
// with the same epilogues, but each line is convolved through its discrete
// Fourier transform instead of the 2r+1 taps: O(n log n) per line against
// O(n r), the fast route to the separable Gaussian filtering of Sec. 4.1.
//
// The filter is the exact restriction of the Gaussian to the grid, a Toeplitz
// matrix of band radius r (r: the last offset whose tap is a normal number in
// the working precision, as for the taps).  Embedded in a circulant of length
// L >= n_i + r (a power of two), its product with a line zero-padded to L is
// the linear convolution on the line's n_i outputs: an input index wraps
// around only into the zero padding.  The circulant's first column c is
// symmetric (c[d] = c[L - d] = k(d), d <= r), so its spectrum
// K^[f] = sum_d c[d] e^{-2 pi i f d / L} is real; two real lines x, y packed as
// x + i y give k * x + i (k * y) in one transform.  Per block: 8 columns of
// the input as 4 complex lines in shared memory, a forward radix-2 transform
// (decimation in time from a bit-reversed load), the product with K^ (which
// carries 1/L), an inverse radix-2 transform (decimation in frequency with
// conjugate twiddles, its output in bit-reversed order), then the epilogue as
// in filter_pass.  Spectrum and twiddles are computed in FP64 on the host.
//
// Rounding: the transforms are accurate normwise: each output carries an
// error of about eps log2(L) times the largest entry of its input line,
// where the band filter's error is relative to each output's own terms.
#include <cmath>
#include <vector>

#include "jko_internal.cuh"
#include "jko_kernels.h"

namespace jko {

namespace {

constexpr int FNT = 256;   // threads per block
constexpr int FJ = 8;      // input columns per block (4 complex lines)
constexpr int FNL = FJ / 2;

template <typename T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };

template <typename V>
__device__ __forceinline__ V cmul(V a, V b) {
  V r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename V>
__device__ __forceinline__ V cmul_conj(V a, V b) {   // a * conj(b)
  V r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.y * b.x - a.x * b.y;
  return r;
}

template <typename T, int EPI, int EK>
__global__ void __launch_bounds__(FNT)
fft_pass_kernel(PassArgs<T> A, ProxArgs<T> P, FftArgs<T> F) {
  using V = typename C2<T>::t;
  Ctrl* ctrl = A.ctrl;
  __shared__ int s_it;
  if (stop_gate(ctrl, A.part, A.nparts, A.decide != 0, &s_it)) return;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = F.L, lg = F.log2L, half = L >> 1;
  V* s_z = reinterpret_cast<V*>(smem_raw);          // FNL lines of L
  V* s_w = s_z + (size_t)FNL * L;                     // twiddles e^{-2 pi i j / L}, j < L/2
  __shared__ double s_red[33];
  const int tid = threadIdx.x;
  for (int j = tid; j < half; j += FNT) s_w[j] = reinterpret_cast<const V*>(F.tw)[j];

  // load columns j0 .. j0+7 (zero beyond n_j and beyond row n_i) into the 4
  // lines at bit-reversed positions; columns 2m / 2m+1 are the real / imaginary
  // parts of line m
  const int j0 = blockIdx.x * FJ;
  for (int e = tid; e < FJ * L; e += FNT) {
    const int c = e % FJ, i = e / FJ;
    const int jj = j0 + c;
    const T v = (i < A.n_i && jj < A.n_j) ? __ldg(A.in + (size_t)i * A.n_j + jj) : T(0);
    const int pos = (int)(__brev((unsigned)i) >> (32 - lg));
    T* dst = reinterpret_cast<T*>(s_z + (size_t)(c >> 1) * L + pos) + (c & 1);
    *dst = v;
  }
  __syncthreads();

  // forward transform: decimation in time, natural-order output
  for (int s = 1; s <= lg; ++s) {
    const int m = 1 << s, hm = m >> 1, tstep = L >> s;
    for (int b = tid; b < FNL * half; b += FNT) {
      const int line = b / half, bb = b - line * half;
      const int grp = bb / hm, k = bb - grp * hm;
      V* z = s_z + (size_t)line * L;
      const int i1 = grp * m + k, i2 = i1 + hm;
      const V t = cmul(s_w[k * tstep], z[i2]);
      const V u = z[i1];
      z[i1] = V{u.x + t.x, u.y + t.y};
      z[i2] = V{u.x - t.x, u.y - t.y};
    }
    __syncthreads();
  }
  // times the real spectrum (with 1/L)
  for (int e = tid; e < FNL * L; e += FNT) {
    const T kh = F.khat[e % L];
    V z = s_z[e];
    z.x *= kh;
    z.y *= kh;
    s_z[e] = z;
  }
  __syncthreads();
  // inverse transform: decimation in frequency with conjugate twiddles,
  // bit-reversed output
  for (int s = lg; s >= 1; --s) {
    const int m = 1 << s, hm = m >> 1, tstep = L >> s;
    for (int b = tid; b < FNL * half; b += FNT) {
      const int line = b / half, bb = b - line * half;
      const int grp = bb / hm, k = bb - grp * hm;
      V* z = s_z + (size_t)line * L;
      const int i1 = grp * m + k, i2 = i1 + hm;
      const V u = z[i1], v = z[i2];
      z[i1] = V{u.x + v.x, u.y + v.y};
      z[i2] = cmul_conj(V{u.x - v.x, u.y - v.y}, s_w[k * tstep]);
    }
    __syncthreads();
  }

  // ---- epilogue: warp w owns output column j0 + w (out row), 32 outputs at a time ----
  const int warp = tid >> 5, lane = tid & 31;
  const int j = j0 + warp;
  T res_t = T(0);
  int bad = 0;
  if (j < A.n_j) {
    const size_t rowoff = (size_t)j * A.n_i;
    const T* zl = reinterpret_cast<const T*>(s_z + (size_t)(warp >> 1) * L) + (warp & 1);
    const bool have_prev = EPI == EPI_B && s_it > 0;
    for (int i = lane; i < A.n_i; i += 32) {
      const int pos = (int)(__brev((unsigned)i) >> (32 - lg));
      const T acc = zl[2 * (size_t)pos];
      const size_t idx = rowoff + i;
      if (EPI == EPI_STORE) {
        A.out[idx] = acc;
      } else if (EPI == EPI_B) {
        const T qv = A.q[idx];
        if (have_prev) res_t += abs_residual<T>(A.out[idx], acc, qv);
        const T bn = b_update<T>(qv, acc);
        bad |= !dev_finite(bn);
        A.out[idx] = bn;
      } else {
        // xi b >= 0 for b >= 0: an output below 0 is the transform's rounding
        // (of the line's largest entry) and is taken as 0, so that p >= 0
        const T sv = acc < T(0) ? T(0) : acc;
        const T a = prox_ratio<T, EK>(P, (int)idx, sv);
        bad |= !dev_finite(a);
        A.out[idx] = a;
        A.p[idx] = a * sv;
      }
    }
  }
  if (EPI == EPI_STORE) return;
  bad = warp_or(bad);
  if (EPI == EPI_B) {
    const double res = block_sum((double)res_t, s_red);
    if (tid == 0) A.part[blockIdx.x] = res;
  }
  if (lane == 0 && bad) atomicOr(&ctrl->nonfinite, 1);
  if (EPI == EPI_A && tid == 0 && blockIdx.x == 0) ctrl->it = s_it + 1;
}

template <typename T>
size_t fft_smem(int L) {
  return sizeof(typename C2<T>::t) * ((size_t)FNL * L + (size_t)(L / 2));
}

template <typename T, int EPI, int EK>
cudaError_t launch_fft(const PassArgs<T>& A, const ProxArgs<T>& P, const FftArgs<T>& F,
                       cudaStream_t st) {
  const size_t smem = fft_smem<T>(F.L);
  auto kern = fft_pass_kernel<T, EPI, EK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<fft_pass_blocks(A.n_j), FNT, smem, st>>>(A, P, F);
  return cudaGetLastError();
}

}  // namespace

int fft_pass_blocks(int n_j) { return (n_j + FJ - 1) / FJ; }

// Transform length and tables of one axis of n cells with band radius r.
bool fft_axis_tables(int n, int r, double length, double gamma, int max_len, int* L, int* log2L,
                     std::vector<double>* khat, std::vector<double>* tw) {
  int lg = 1;
  while ((1 << lg) < n + r) ++lg;
  const int Ln = 1 << lg;
  if (Ln > max_len) return false;
  *L = Ln;
  *log2L = lg;
  const double h = length / n;
  const double pi = 3.14159265358979323846;
  std::vector<double> c(r + 1);
  for (int d = 0; d <= r; ++d) c[d] = std::exp(-(d * h) * (d * h) / gamma);
  khat->assign(Ln, 0.0);
  for (int f = 0; f < Ln; ++f) {
    // K^[f] = c0 + 2 sum_{d=1}^{r} c_d cos(2 pi f d / L), the angle reduced
    // exactly modulo 2 pi; with the 1/L of the inverse transform
    double s = c[0];
    for (int d = 1; d <= r; ++d) {
      const long long m = ((long long)f * d) % Ln;
      s += 2.0 * c[d] * std::cos(2.0 * pi * (double)m / Ln);
    }
    (*khat)[f] = s / Ln;
  }
  tw->assign(Ln, 0.0);   // interleaved re, im of e^{-2 pi i j / L}, j < L/2
  for (int j = 0; j < Ln / 2; ++j) {
    (*tw)[2 * j] = std::cos(2.0 * pi * j / Ln);
    (*tw)[2 * j + 1] = -std::sin(2.0 * pi * j / Ln);
  }
  return true;
}

template <typename T>
size_t fft_pass_smem(int L) { return fft_smem<T>(L); }

template <typename T>
cudaError_t fft_pass(int epi, int ek, const PassArgs<T>& A, const ProxArgs<T>& P,
                     const FftArgs<T>& F, cudaStream_t st) {
  if (epi == EPI_STORE) return launch_fft<T, EPI_STORE, EK_CROWD>(A, P, F, st);
  if (epi == EPI_B) return launch_fft<T, EPI_B, EK_CROWD>(A, P, F, st);
  switch (ek) {
    case EK_CROWD: return launch_fft<T, EPI_A, EK_CROWD>(A, P, F, st);
    case EK_ENTROPY: return launch_fft<T, EPI_A, EK_ENTROPY>(A, P, F, st);
    default: return launch_fft<T, EPI_A, EK_POWER>(A, P, F, st);
  }
}

template cudaError_t fft_pass<float>(int, int, const PassArgs<float>&, const ProxArgs<float>&,
                                     const FftArgs<float>&, cudaStream_t);
template cudaError_t fft_pass<double>(int, int, const PassArgs<double>&, const ProxArgs<double>&,
                                      const FftArgs<double>&, cudaStream_t);
template size_t fft_pass_smem<float>(int);
template size_t fft_pass_smem<double>(int);

}  // namespace jko
