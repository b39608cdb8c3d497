/*
 * jko.h -- C ABI of the GB300 entropic JKO library (libjko.so).
 *
 * Computes discrete entropic Wasserstein gradient flows on a uniform 2-D grid
 * (Peyre 2015, "Entropic Wasserstein Gradient Flows"):
 *
 *   one step   p = Prox^{W_gamma}_{tau f}(q) = argmin_{p in Sigma_N} W_gamma(p,q) + tau f(p)
 *              (Eq. def-jko-operator), solved by the KL-proximal scaling
 *              iteration of Prop. 3.3, which with u, v identically 1 reads
 *                  b = q / xi^T a ;  s = xi b ;  p = Prox^{KL}_{sigma f}(s) ;  a = p / s
 *              with sigma = tau/gamma (Eq. defn-KL-prbm) and the Gibbs kernel
 *              xi = exp(-|x_i - x_j|^2 / gamma) applied as the separable product
 *              K_y X K_x^T (Sec. 4.1);
 *   the flow   p_{t+1} = Prox^{W_gamma}_{tau f}(p_t) (Eq. smooth-jko).
 *
 * Energy f (all terms optional, Sec. 4.2 and Sec. 4.4):
 *   f(p) = iota_{[0,kappa]}(p) + <w,p> + sum_i alpha_i e(p_i) + iota{p_i = 0 on mask}
 *   e(s) = s (log s - 1)            when m == 1   (Eq. defn-gen-entropies, m = 1)
 *   e(s) = s^m / (m - 1)            when m >  1   (power form; the paper's e_m equals it
 *                                                  plus the potential -m alpha/(m-1))
 *   no entropy term                 when m == 0.
 * Its pointwise KL proximal map is Prop. 4.1 (congestion + potential),
 * Eq. prox-entropy (m = 1) and the root of Eq. prox-psi (m > 1), clamped at
 * kappa, zero on the mask.
 *
 * Stopping rule (pseudo-code of Sec. 3.4): after each (odd, even) pair of
 * half-steps, stop when ||b (.) xi^T a - q||_1 <= tol; at most max_iter pairs.
 * Each step starts cold (a = b = 1).
 *
 * Memory and threading conventions (all entry points):
 *   - Images are row-major [ny][nx] (index y*nx + x), cell centres (i+1/2)h
 *     with h = lx/nx, ly/ny.
 *   - "_dev" pointers are CUDA device pointers owned by the caller; "_host"
 *     pointers are host memory owned by the caller.  Device images are double
 *     for JKO_FP64 and float for every other precision.
 *   - The handle owns every internal buffer; energy fields passed to
 *     jko_create are copied, so the caller may free them afterwards.
 *   - Work is enqueued on the handle's stream; jko_step / jko_flow return when
 *     their results are complete on that stream.
 *   - A handle may be used by one host thread at a time.  Distinct handles are
 *     independent.
 *   - Every entry point returns a jko_status; on an error the handle keeps a
 *     message readable with jko_last_error.  JKO_ERR_INVALID_ARG leaves all
 *     outputs untouched.  JKO_NOT_CONVERGED still writes the result.
 */
#ifndef JKO_H_
#define JKO_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum jko_status {
  JKO_OK = 0,
  JKO_ERR_INVALID_ARG = 1,  /* bad sizes, parameters or input data */
  JKO_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  JKO_ERR_OOM = 3,          /* device or pinned allocation failed */
  JKO_ERR_NUMERIC = 4,      /* a NaN or Inf appeared in the iterates */
  JKO_NOT_CONVERGED = 5,    /* max_iter pairs reached; result still written */
  JKO_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up */
  JKO_ERR_UNSUPPORTED = 7   /* configuration not supported by this build */
} jko_status;

/* Arithmetic of the Gibbs-kernel applications (the hot path). */
typedef enum jko_precision {
  JKO_FP64 = 0,    /* CUDA cores, double throughout */
  JKO_FP32 = 1,    /* CUDA cores, float throughout */
  JKO_TF32 = 2,    /* tensor cores (tcgen05 kind::tf32), fp32 accumulation */
  JKO_BF16 = 3,    /* tensor cores (tcgen05 kind::f16), fp32 accumulation: the Gibbs
                      factor in bf16, each scaling image as a bf16 pair hi + lo (two
                      products K * hi + K * lo, ~16 significant bits in the images) */
  JKO_BF16X3 = 4   /* tensor cores, the factor also as a pair: K_hi * (hi + lo) + K_lo * hi */
} jko_precision;

/* Uniform grid on [0,lx] x [0,ly] (Sec. 2, numerical grids of Sec. 4). */
typedef struct jko_grid {
  int nx, ny;      /* cells along x (contiguous) and y; each >= 1 */
  double lx, ly;   /* domain lengths; > 0 */
  /* Gibbs kernel: 0 = the separable Gaussian e^{-|x-y|^2/gamma} (Sec. 2.1);
   * L in [1, 1000] = the heat kernel (Id - (gamma/L) Delta_M)^{-L} of the
   * domain outside the obstacle mask (Sec. 4.1, Eq. heat-kernel), JKO_FP32 /
   * JKO_FP64 single-density handles only (JKO_ERR_UNSUPPORTED otherwise; in a
   * batch it runs its kernels per Clenshaw phase; no fixed-scratch step). */
  int heat_L;
  /* Application of the Gaussian (heat_L = 0): 0 = the band-limited separable
   * filter (CUDA cores) or tensor-core GEMMs; 1 = the same restricted Gaussian
   * by FFT convolution along each axis, O(N log N): each line zero-padded to a
   * power of two L >= n + r (r the band radius of the filter), transformed,
   * multiplied by the real spectrum of the kernel's circulant embedding and
   * transformed back.  Accurate normwise (each output within ~eps log2 L of its
   * line's largest entry), where the filter is accurate entry by entry.
   * The potential spreads the scalings over e^{tau/gamma (max w - min w)}, so
   * that range must stay <= 8 (FP32) / 24 (FP64) (measured errors 5.5e-6 /
   * 9.3e-11 there).  JKO_FP32 / JKO_FP64 handles of one density or of two
   * species (each potential within the rule; no target, pairwise attraction or
   * heat kernel: the attraction steps' geometric mean of two blurs reads small
   * entries the transform holds only normwise), L <= 4096 (FP32) / 2048 (FP64), else
   * JKO_ERR_UNSUPPORTED; no fixed-scratch step. */
  int fft;
} jko_grid;

typedef struct jko_params {
  double gamma;     /* entropic regularisation gamma > 0 (Sec. 2.1) */
  double tau;       /* JKO step size tau > 0 (Eq. def-jko-operator) */
  double tol;       /* L1 marginal residual tolerance >= 0 (Sec. 3.4) */
  int max_iter;     /* maximum (odd, even) pairs per step, >= 1 */
  int check_every;  /* iterations between host polls of the stop flag (0 = default 4);
                       handles on the persistent loop kernel run a step's whole budget
                       in one launch that stops itself, and ignore it */
  int precision;    /* a jko_precision value */
  int renormalize;  /* 1: divide each output p by its FP64 sum; 0: leave as computed */
  int absorb;       /* tensor-core precisions: separable log-domain absorption of the
                       potential (see jko_create); 0 = automatic, 1 = on, 2 = off;
                       3 = the log-domain form (JKO_TF32, congestion / potential energy of
                       one density, single handles, one kernel per pass): every scaling
                       image is held as a TF32 mantissa and a base-2 exponent per row and
                       group of 32 cells, the Gibbs factor with one per row and K-block of
                       32 cells; each pass accumulates every K-block of its band apart and
                       adds them with exact power-of-two scalings, so the scalings keep a
                       range beyond FP32 whatever the shape of the potential.  The band
                       ends where the Gaussian, against the largest growth of e^{-sigma w}
                       over the distance, falls below e^{-50}; JKO_ERR_UNSUPPORTED where
                       that band exceeds 16 K-blocks per 128 rows, or where sigma times the
                       largest step of w between neighbouring cells exceeds 70/32 e-folds
                       (a group could not hold its image's range) */
  int loop;         /* tensor-core precisions: 0 = automatic (one persistent kernel per
                       step, with the stop rule taken in the kernel, where the device
                       and the grid allow it, else one kernel per pass), 1 = persistent
                       kernel required (JKO_ERR_UNSUPPORTED if it cannot run), 2 = one
                       kernel per pass, 3 = as 1, and in a batch the flow joins the
                       grouped launch of its precision (jko_batch_create).  Heat-kernel
                       handles (jko_grid.heat_L > 0): 0 or 1 = one persistent cooperative
                       kernel per step where the device has cooperative launches (1:
                       JKO_ERR_UNSUPPORTED where not), 2 = kernels per Clenshaw phase;
                       both give the same bits.  Other CUDA-core handles ignore it */
  int tile;         /* tensor-core precisions: output tile width of the per-pass kernels,
                       64 or 128 (128: JKO_TF32 only), or 0 = automatic.  With loop = 0
                       and tile = 0 on grids of 256^2 cells or more, jko_create times the
                       loop kernel and the per-pass kernels at both widths on 16 pairs and
                       keeps the fastest; the choice is cached per grid, lengths, gamma,
                       precision and energy kind for the process, so handles created
                       alike run the same kernels (jko_handle_info reports them) */
  int stall;        /* > 0: a step also stops when its L1 residual has set no new minimum
                       for `stall` pairs in a row (the iterates have reached the rounding
                       floor of their arithmetic; a slowly converging step keeps setting
                       minima); the step reports JKO_NOT_CONVERGED unless `finish` takes
                       over.  0 = off (the stopping rule of Sec. 3.4 alone), >= 0 */
  int finish;       /* tensor-core precisions, 1: a step the stall rule stops continues
                       from its current scalings a, b on the JKO_FP32 CUDA-core form, within
                       the same max_iter budget and under the same rules, so it reaches tol
                       where the tensor-core operands cannot (the step's minimiser is unique,
                       Eq. def-jko-operator).  Needs stall > 0 and scalings without log-domain
                       absorption (absorb = 2, or automatic on a potential that does not turn
                       it on), else JKO_ERR_UNSUPPORTED; single handles only (jko_batch_create:
                       JKO_ERR_UNSUPPORTED).  0 = off */
} jko_params;

/* Energy f; every pointer is HOST memory of N = nx*ny entries, or NULL. */
typedef struct jko_energy {
  const double* w;            /* potential w (Eq. dfn-congestion); NULL = 0 */
  double kappa;               /* scalar congestion bound (> 0); +INFINITY = none */
  const double* kappa_field;  /* per-cell bound (Sec. 4.2 remark); overrides kappa */
  double m;                   /* 0: no entropy term, 1: entropy, > 1: power m */
  const double* alpha;        /* per-cell weights of the entropy term (> 0); NULL = 1 */
  const uint8_t* mask;        /* 1 = obstacle cell (f = +inf), 0 = free; NULL = none */
  const double* m_field;      /* per-cell exponents m_i >= 1 of the paper's generalised
                                 entropies sum_i alpha_i e_{m_i}(p_i), e_1(s) = s (log s - 1),
                                 e_m(s) = s (s^{m-1} - m)/(m-1) (Eq. defn-gen-entropies,
                                 Sec. 4.4); overrides m; NULL = the scalar m above */
  int binary;                 /* 1: the congestion is the non-convex iota_{{0,kappa}} + <w,p>
                                 (Eq. dfn-congestion-noncvx, Sec. 4.5): p_i in {0, kappa_i},
                                 kappa_i where s_i e^{-sigma w_i} > kappa_i / e (0 at the tie);
                                 needs m = 0, no m_field and a finite kappa; not for the
                                 adjoint (the prox has no derivative) */
  const double* target;       /* Wasserstein attraction with congestion (Sec. 5.2): f gains
                                 W_gamma(r, p) toward this target density r (N entries, >= 0,
                                 sum 1, 0 on the mask); the other terms form h of
                                 Eq. prox-psi-attraction.  The step runs the generic diagonal
                                 scaling with 2 couplings.  JKO_FP32 / JKO_FP64 (CUDA cores),
                                 or the tensor-core passes of every coupling: JKO_TF32 (nx, ny
                                 multiples of 4), JKO_BF16 / JKO_BF16X3 (multiples of 8), with
                                 absorb 0 or 2, loop 0 or 2, tile 0 or 64 and no finish; the
                                 adjoint on JKO_FP64 handles with the congestion / potential
                                 energy; not for jko_step_noalloc.  NULL = none */
  int species;                /* 2: two densities coupled through the congestion of their sum,
                                 f = iota_{[0,kappa]}(p_1 + p_2) + <p_1, w> + <p_2, w2>
                                 (Sec. 5.3, summation couplings): every state image (q, p,
                                 trajectories) holds [p_1, p_2], 2 N entries, of total mass 1;
                                 scalar kappa only (no kappa_field, mask, entropy, binary or
                                 target); the precisions of `target`; in a batch the flow's
                                 images hold 2 N entries too; the adjoint on JKO_FP32 /
                                 JKO_FP64 handles (dL/dw: the first species' potential, which
                                 jko_set_potential replaces); not for jko_step_noalloc.  0 or
                                 1: one density */
  const double* w2;           /* potential of the second species (N entries); NULL = 0 */
  double pair_alpha;          /* > 0 with species = 2: the Wasserstein pairwise attraction
                                 f = pair_alpha W_gamma(p_1, p_2) + h_1(p_1) + h_2(p_2),
                                 h_1 = iota_{[0,kappa]} + <w, .>, h_2 = iota_{[0,kappa]} +
                                 <w2, .> (Sec. 5.3, multiple densities), in place of the
                                 congestion of the sum; the step runs the generic diagonal
                                 scaling with 3 couplings; finite; 0 = none */
} jko_energy;

/* Per-step report. */
typedef struct jko_step_info {
  int iters;                 /* (odd, even) pairs performed */
  int status;                /* JKO_OK, JKO_NOT_CONVERGED or JKO_ERR_NUMERIC */
  double residual_l1;        /* ||b (.) xi^T a - q||_1 of the returned iterate */
  double mass;               /* sum of p before any renormalisation (FP64) */
  double max_p_over_kappa;   /* max_i p_i / kappa_i (0 without congestion) */
  float ms;                  /* device time of the step in milliseconds */
  int kernels;               /* kernels this library enqueued for the step */
  int iters_finish;          /* of `iters`, the pairs run on the FP32 CUDA-core form after
                                the tensor-core pairs stalled (jko_params.finish) */
} jko_step_info;

typedef struct jko_handle jko_handle;

/* Creates a solver for one grid, one set of step parameters and one energy.
 * Builds the 1-D Gibbs factors K_x, K_y (Sec. 4.1) and the per-cell energy
 * constants, allocates the working buffers and captures the iteration graph.
 * stream: a cudaStream_t (NULL = legacy default stream).
 * Log-domain absorption (tensor-core precisions): the scaling is carried as
 * a = e^{beta(x,y)} a~ with the separable log-scale beta = beta_x(x) + beta_y(y)
 * = -sigma times the additive separable fit of w, held in FP64 on the host and
 * absorbed into the 1-D Gibbs factors, K~[i][j] = K[i][j] e^{beta(j) - beta(i)}
 * for xi a and its transpose for xi b, and into the potential (sigma w + beta).
 * The iterates a~, b~ then stay O(1) however small gamma is (for separable w
 * entirely); p and the residual are unchanged and the step starts from a~ = 1.
 * Automatic mode turns it on when sigma (max w - min w) > 120 (below that
 * the plain form, whose scalings then stay in range, is the more accurate).
 * Returns JKO_ERR_INVALID_ARG on bad sizes or parameters (gamma, tau <= 0,
 * negative tol, max_iter < 1, kappa <= 0, alpha <= 0, m in (0, 1)),
 * JKO_ERR_UNSUPPORTED when the precision is not available for this grid,
 * JKO_ERR_OOM / JKO_ERR_CUDA on allocation or runtime failures.  *out is
 * NULL on failure. */
jko_status jko_create(const jko_grid* grid, const jko_params* params,
                      const jko_energy* energy, void* stream, jko_handle** out);

/* One JKO step p_out = Prox^{W_gamma}_{tau f}(q) (Eq. def-jko-operator).
 * q_dev, p_out_dev: device images of N elements (double for JKO_FP64, float
 * otherwise); they may alias.  q must be finite, >= 0, sum to 1 within 1e-3,
 * vanish on masked cells and satisfy q <= kappa (1 + 1e-2) (Sec. 4.2 asks
 * kappa >= max p_0), else JKO_ERR_INVALID_ARG.  info may be NULL. */
jko_status jko_step(jko_handle* h, const void* q_dev, void* p_out_dev, jko_step_info* info);

/* n_steps steps of the flow from p0 (Eq. smooth-jko).  traj_dev (may be NULL)
 * receives p_1 .. p_n as n_steps consecutive images; p_final_dev (may be NULL)
 * receives p_n.  infos (may be NULL) receives n_steps reports.  Only p0 is
 * validated.  Returns the worst status over the steps.  The steps after the
 * first are enqueued together and the host waits once: their chunks of pairs
 * run as a loop on the device (a CUDA graph with a conditional WHILE node that
 * ends when the step stops, or after the chunk budget of max_iter pairs), with
 * the same kernels, hence the same results, as jko_step.  Handles whose steps
 * need a host decision (jko_params.finish on a tensor-core form) run every
 * step with host-driven chunks.  The first call on a handle (of any length)
 * builds the loop graph and allocates pinned reports and events for
 * max(n_steps, 64) steps; a later longer flow allocates again. */
jko_status jko_flow(jko_handle* h, const void* p0_dev, int n_steps, void* traj_dev,
                    void* p_final_dev, jko_step_info* infos);

/* jko_flow on HOST buffers: copies p0 to the device, runs the flow, copies the
 * requested outputs back; returns once they are in host memory. */
jko_status jko_flow_host(jko_handle* h, const void* p0_host, int n_steps, void* traj_host,
                         void* p_final_host, jko_step_info* infos);

/* Times the four kernel passes of one (odd, even) pair in isolation on the
 * handle's stream (captured in a CUDA graph, as the scaling loop runs them): pass 0 / 2 apply the first 1-D factor of xi to a / b, pass
 * 1 / 3 the second factor fused with the b-update and residual / the KL prox
 * and a-update.  Each pass is launched `reps` times back to back after one
 * warm-up launch; ms[k] receives the mean milliseconds per launch (CUDA
 * events) and, if flops is not NULL, flops[k] the algorithmic floating-point
 * operations of one launch.  Overwrites the handle's scaling iterates: call it
 * between flows, not inside one.  Heat-kernel handles (jko_grid.heat_L > 0)
 * have no separable passes: JKO_ERR_UNSUPPORTED. */
jko_status jko_profile_passes(jko_handle* h, int reps, float* ms, double* flops);

/* Times the persistent pair-loop kernel of a tensor-core handle: `reps`
 * launches, each running `pairs` pairs with a stop rule that never fires.
 * ms[0] receives the mean milliseconds per launch (CUDA events on the handle's
 * stream) and flops[0] (may be NULL) the executed tensor-core flops of one
 * launch.  JKO_ERR_UNSUPPORTED when the handle does not use that kernel.
 * Overwrites the handle's scaling iterates, like jko_profile_passes. */
jko_status jko_profile_loop(jko_handle* h, int pairs, int reps, float* ms, double* flops);

/* How a handle runs its scaling loop (diagnostics; the paper has no
 * counterpart).  out[0] = 1 if it uses the persistent loop kernel, out[1] = 1
 * if that kernel keeps the Gibbs-factor band resident in shared memory,
 * out[2] = 1 if its launch (or chunk of per-pass launches) is replayed from a
 * CUDA graph, out[3] = pairs per launch or chunk.  out: 4 ints (host). */
jko_status jko_handle_info(const jko_handle* h, int* out);

/* One JKO step without any memory allocation (the paper has no counterpart;
 * this is a deployment variant of jko_step).
 *
 * For callers that cannot allocate device memory when they need a step: code
 * running inside a framework that owns all device memory through its own pool
 * (a cudaMalloc there escapes the pool's accounting, and a cudaFree
 * synchronises the whole device), or services that forbid allocation after
 * start-up.  It computes what jko_create + jko_step + jko_destroy compute for
 * JKO_FP32, with the same CUDA-core kernels, but every working buffer lives in
 * one fixed file-scope device array of about 3 MB that each GPU loading the
 * library holds until the process exits.  Nothing is allocated: no
 * cudaMalloc/cudaFree, no pinned memory, no graphs or events.
 *
 * Arguments are those of jko_create and jko_step (energy fields are HOST
 * arrays; q_dev / p_out_dev are float device images of N = nx*ny elements and
 * may alias); work is enqueued on `stream` (a cudaStream_t) and the call
 * returns when p_out is complete.  info->ms is always 0.
 *
 * Limits and errors: JKO_ERR_UNSUPPORTED when nx > 256 or ny > 256 (the fixed
 * array holds at most 256 x 256 cells) or precision != JKO_FP32;
 * JKO_ERR_INVALID_ARG for the argument and input checks of jko_create /
 * jko_step (outputs untouched); no message is recorded for jko_last_error.
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  All calls
 * share the array and re-initialise what they read, so consecutive calls are
 * independent, but calls whose GPU work overlaps (other streams or threads)
 * race on it. */
jko_status jko_step_noalloc(const jko_grid* grid, const jko_params* params,
                            const jko_energy* energy, const void* q_dev, void* p_out_dev,
                            void* stream, jko_step_info* info);

/* ---- differentiation of the flow (CUDA-core handles: JKO_FP32, JKO_FP64) ---- */

/* Replaces the potential w of the energy (HOST array of N doubles) without
 * recreating the handle; the handle must have been created with a potential
 * (or be of the congestion kind).  Used between gradient steps. */
jko_status jko_set_potential(jko_handle* h, const double* w_host);

/* jko_set_potential from a DEVICE image w_dev of N entries in the handle's
 * element type (double for JKO_FP64, float otherwise), stream-ordered on the
 * handle's stream: no host synchronisation, no allocation, no finiteness
 * check (a non-finite w makes the next step report JKO_ERR_NUMERIC).  The
 * caller keeps w_dev alive until the work queued on the stream has run. */
jko_status jko_set_potential_device(jko_handle* h, const void* w_dev);

/* jko_flow that also records, for every step t, its input q_t and the final
 * scaling a_t (the tape of jko_flow_backward).  p_final_dev receives p_n;
 * infos (may be NULL) n_steps reports.  Single-density JKO_FP32 / JKO_FP64
 * handles with the Gaussian (filter or FFT) or the heat kernel, JKO_FP32 /
 * JKO_FP64 two-species handles (tape and p_final of 2 N entries), and JKO_FP64
 * handles of the Wasserstein attraction with the congestion / potential
 * energy (its Jacobian a_m / s_m leaves the FP32 range).  JKO_ERR_UNSUPPORTED
 * for tensor-core and pairwise-attraction handles, other attraction handles
 * and the binary congestion (no derivative). */
jko_status jko_flow_record(jko_handle* h, const void* p0_dev, int n_steps, void* p_final_dev,
                           jko_step_info* infos);

/* Reverse-mode gradient of a scalar loss L(p_n) of the last recorded flow.
 * grad_final_dev = dL/dp_n (device image); grad_p0_dev (may be NULL) receives
 * dL/dp_0, grad_w_dev (may be NULL) dL/dw (device images, the handle's element
 * type).  Each step is differentiated implicitly at its fixed point (a = r(s),
 * s = xi(q / xi a), xi the handle's own symmetric Gibbs kernel: the Gaussian
 * or the heat kernel; the paper has no adjoint, this follows from Prop. 3.3's
 * fixed point by the implicit-function theorem), including the adjoint of the
 * mass renormalisation; the adjoint linear system is solved by the fixed-point
 * iteration of the transposed linearisation (tolerance params.tol relative,
 * at most 10 max_iter sweeps).  adj_iters (may be NULL) receives the sweeps
 * per step. */
jko_status jko_flow_backward(jko_handle* h, const void* grad_final_dev, void* grad_p0_dev,
                             void* grad_w_dev, int* adj_iters);

/* ---- batched flows (many independent problems advanced together) ---- */
typedef struct jko_batch jko_batch;

/* Creates n_flows independent flows, flow f with grids[f], params[f] and
 * energies[f] (the same rules as jko_create; each flow may have its own grid
 * size, gamma, tau, energy and precision; all share params[].check_every).
 * Each JKO step of the batch runs as three CUDA graphs whose parallel
 * branches are the flows, so small and large flows share the GPU; a flow that
 * has met its stopping rule (Sec. 3.4) turns its remaining kernels into
 * no-ops, and a flow on the persistent loop kernel is one launch per step in
 * its branch.  Grouped launch: the flows with loop = 3 (or all loop-capable
 * flows, when the autotuner picks it) that share a tensor-core precision run
 * their steps in ONE cooperative launch of a persistent kernel that walks
 * the tiles of all of them between grid barriers, each flow with its own
 * stop rule; such a flow gives the same bits as the flow alone on the loop
 * kernel.  When every flow is a tensor-core flow on automatic kernels
 * (loop = tile = 0), the batch times the candidate kernel configurations on
 * its own graph and keeps the fastest (jko_batch_info reports it).  Errors as jko_create, with the failing flow named in
 * jko_batch_last_error(NULL). */
jko_status jko_batch_create(int n_flows, const jko_grid* grids, const jko_params* params,
                            const jko_energy* energies, void* stream, jko_batch** out);

/* How a batch runs its flows (diagnostics).  out[0] = the configuration its
 * autotuner chose (-1: not tuned; 0: each flow's own choice, 1: per-pass
 * kernels with 64-wide tiles, 2: 128-wide tiles, 3: the loop kernel, 4: the
 * loop-capable flows in grouped launches), out[1] = number of flows on a loop
 * kernel launch of their own, out[2] = 1 if the per-pass fallback was taken
 * because loop launches could not be captured, out[3] = number of flows in
 * grouped launches, out[4] = number of grouped launches per chunk.  out: 5
 * ints. */
jko_status jko_batch_info(const jko_batch* b, int* out);

/* n_steps steps of every flow (Eq. smooth-jko) from p0_dev[f] (device image of
 * flow f, double for JKO_FP64 flows, float otherwise; validated as in
 * jko_step).  p_final_dev[f] (array and entries may be NULL) receives the last
 * iterate; infos (may be NULL) receives n_steps * n_flows reports, step-major
 * (infos[t * n_flows + f]).  Returns the worst status over flows and steps. */
jko_status jko_batch_flow(jko_batch* b, const void* const* p0_dev, int n_steps,
                          void* const* p_final_dev, jko_step_info* infos);

/* One JKO step (Eq. smooth-jko) of every flow: p_out_dev[f] = Prox step of
 * q_dev[f] (device images as in jko_batch_flow, validated the same way;
 * q_dev[f] and p_out_dev[f] may be the same buffer).  infos (may be NULL)
 * receives n_flows reports.  Returns the worst status over flows; the flows'
 * outputs are written for JKO_OK, JKO_NOT_CONVERGED and JKO_ERR_NUMERIC. */
jko_status jko_batch_step(jko_batch* b, const void* const* q_dev, void* const* p_out_dev,
                          jko_step_info* infos);

/* Frees the batch and its flows (NULL is accepted). */
jko_status jko_batch_destroy(jko_batch* b);

/* Message of the last error on b, or of the last failed jko_batch_create when
 * b is NULL (never NULL; "" when none). */
const char* jko_batch_last_error(const jko_batch* b);

/* Re-targets the handle to another stream (a cudaStream_t). */
jko_status jko_set_stream(jko_handle* h, void* stream);

/* Frees every resource of the handle (NULL is accepted). */
jko_status jko_destroy(jko_handle* h);

/* Message of the last error on h (never NULL; "" when none). */
const char* jko_last_error(const jko_handle* h);

/* Static name of a status code. */
const char* jko_status_string(int status);

/* Library description: precisions compiled in, device, version. */
const char* jko_build_info(void);

/* Host-only diagnostic (no device call): the expansion a heat-kernel handle
 * (jko_grid.heat_L = L > 0, Sec. 4.1, Eq. heat-kernel) applies.  xi~ =
 * (Id - (gamma/L) Delta)^{-L} is evaluated as p(A), p the Chebyshev series
 * sum_k coef[k] T_k((lambda - centre) / half-width) of lambda^{-L} on the
 * spectrum interval [1, lmax] of A = Id - (gamma/L) Delta, lmax = 1 + 4 (gamma/L)
 * (1/hx^2 + 1/hy^2), truncated for `precision` (JKO_FP64: dropped
 * coefficients below ~1e-15 or their rounding floor: the series within ~1e-14
 * of lambda^{-L}; JKO_FP32 handles truncate alike, since their recurrence
 * also runs in FP64).  Writes the degree D to
 * *degree, min(D + 1, cap) coefficients to coef (may be NULL when cap = 0) and,
 * if interval is not NULL, (1, lmax) to interval[0..1].  JKO_ERR_INVALID_ARG
 * for sizes, lengths, gamma or L out of range (as jko_create);
 * JKO_ERR_UNSUPPORTED when D would exceed 1500. */
jko_status jko_heat_plan(int nx, int ny, double lx, double ly, double gamma, int L,
                         int precision, int* degree, double* coef, int cap, double* interval);

#ifdef __cplusplus
}
#endif

#endif /* JKO_H_ */
