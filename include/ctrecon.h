/*
 * ctrecon -- GB300-native (sm_103a) preconditioned primal-dual TV-CT reconstruction
 * with inequality constraints.
 *
 * C ABI of libctrecon.so.  Plain pointers and sizes only.  Every device pointer is
 * owned by the caller and must hold the plan's element type (float for CTR_F32,
 * double for CTR_F64) unless stated otherwise; images are row-major u[i*n + j]
 * (first index i <-> x, second j <-> y), sinograms row-major g[l*M + k] (angle l,
 * detector bin k).  All calls are asynchronous on `stream` (a cudaStream_t, NULL =
 * the legacy default stream) except where a host output is returned, which
 * synchronises that stream.  No call throws, aborts or traps: every error is a
 * negative ctr_status with a message from ctr_last_error() (thread-local).
 * A plan is not thread-safe: calls on one plan must not overlap.
 *
 * The method: "TV-regularized CT Reconstruction and Metal Artifact Reduction
 * Using Inequality Constraints with Preconditioning" (C. Schiffer, 2018).
 * Section/equation/algorithm numbers below refer to it.
 */
#ifndef CTRECON_H
#define CTRECON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CTR_OK = 0,
    CTR_EINVAL = -1,        /* bad argument (null pointer, size, non-finite parameter) */
    CTR_ENOMEM = -2,        /* device or host allocation failed (only in ctr_plan_create) */
    CTR_ECUDA = -3,         /* a CUDA runtime call failed; message has the CUDA error string */
    CTR_ETIMEOUT = -4,      /* a bounded device wait ran out (reported through a status word) */
    CTR_ENUMERIC = -5,      /* NaN/Inf detected in diagnostics */
    CTR_EUNSUPPORTED = -6   /* geometry/dtype outside the implemented range */
} ctr_status;

typedef enum { CTR_F32 = 0, CTR_F64 = 1, CTR_BF16 = 2 } ctr_dtype;

/* Parallel-beam geometry of Sec. 3.1: n x n pixels of side h centred on the
 * rotation axis (x_i = h (i - (n-1)/2)); n_angles angles theta_l (radians, any
 * values); n_bins detector bins of width ds centred at s_k = (k - (n_bins-1)/2) ds.
 * angles_host is copied by ctr_plan_create. */
typedef struct {
    int n;
    int n_angles;
    int n_bins;
    double h;
    double ds;
    const double *angles_host;
} ctr_geometry;

typedef struct ctr_plan ctr_plan;   /* opaque: geometry tables + all device workspace */

/* Solver parameters of Alg. 4 (PDRQS1), and of Alg. 5 (PDRQS1 with u >= 0) when
 * nonneg = 1.  ctr_default_params fills the defaults. */
typedef struct {
    double sigma;        /* step sigma > 0 (default 1) */
    double tau;          /* gradient scaling tau > 0 (default 1/sqrt(8)) */
    double eps;          /* ||xi||_eps regulariser of the inverse-norm preconditioner (default pi/n) */
    double c;            /* preconditioner constant; <= 0: 1.05 x power iteration (Sec. 4.3.1) */
    double beta;         /* problem scaling ~ ||R_h||; <= 0: power iteration (Sec. 5.1) */
    int power_iters;     /* power-iteration steps for beta and c (default 50) */
    double c_margin;     /* c = c_margin * lambda_max estimate (default 1.05) */
    double trace_ratio;  /* metal-trace threshold C = trace_ratio * f (default 0.8, Sec. 5.2) */
    int check_every;     /* diagnostics cadence of Alg. 4, 5 and 3 solves (tv_pd_solve, tv_pd_run,
                          * tv_pd_solve_state, tv_pdrq2_solve, tv_mar_solve's second stage): k > 0
                          * computes the diagnostics of ctr_diag on the device after every k-th
                          * iteration (one extra R_h^* each, no host synchronisation unless
                          * stop_tol > 0) and keeps them as a history that ctr_plan_history
                          * returns -- the convergence record of Sec. 5 (objective against the
                          * iteration count).  At most 4096 checks per solve (iters / k > 4096:
                          * CTR_EINVAL).  0 (default): diagnostics only after the last
                          * iteration.  Alg. 1, ADMM and batches: CTR_EUNSUPPORTED for k > 0. */
    int graph_block;     /* iterations per captured CUDA graph; 0 = plain launches (default 10) */
    int nonneg;          /* 1: Alg. 5, the non-negativity constraint u >= 0 added to (C_h) (Sec.
                          * "Non-negativity constraints"): the preconditioner symbol gains the
                          * identity, ||xi|| / (||xi|| + sigma^2 c + (sigma tau)^2 L ||xi||), the
                          * first step adds bar u - u and bar u += max(2 u - bar u, 0) - u after
                          * each update.  0 (default): Alg. 4.  Also selects the symbol that
                          * precond_apply applies. */
    int precond;         /* 0 (default): inverse-norm preconditioner, S = F^{-1}(1/||xi||_eps)F
                          * (Sec. 4.3.1).  1: impulse response (Sec. "Impulse response
                          * preconditioners"): S = convolution with k = R_h^* R_h delta, the
                          * response to the impulse at (n/2, n/2) made point-symmetric, its DFT
                          * bounded below by 1e-3 of its maximum.  2: circulant (Sec.
                          * "Circulant matrix preconditioner"): the same response on the image
                          * flattened as t = i + n j, rolled to t = 0 and symmetrised, S its
                          * circulant matrix, inverted with the 1-D DFT of length n^2 (the
                          * Laplacian term likewise the circulant of -Delta_h).  3: Richardson
                          * (Sec. "Suitable Preconditioners"): S = id and the Laplacian term
                          * replaced by its bound 8/h^2, M = (sigma^2 c + 8 (sigma tau)^2/h^2) id.
                          * Kinds 1 and 2 build their kernel DFT on the plan's first use (a few
                          * kernel launches, no allocation).  In all kinds M = sigma^2 c S +
                          * (sigma tau)^2 Lap (+ id with nonneg) and c is from the power
                          * iteration on S^{-1/2} R^*R S^{-1/2}.  Batched solves take every kind. */
    double stop_tol;     /* > 0 (needs check_every > 0): stop at the first check whose rel_change
                          * ||u_k - u_{k-1}|| / ||u_k|| is <= stop_tol; diag_out->iters_done then
                          * tells how many iterations ran.  Each check synchronises the stream to
                          * read rel_change.  0 (default): run all iterations. */
} ctr_params;

/* Diagnostics after the solve (original, unscaled problem unless noted). */
typedef struct {
    double beta;           /* scaling used */
    double c;              /* preconditioner constant used */
    double objective;      /* sum_r w_r/2 (R u - a)_r^2 + alpha TV(u) */
    double data_fit;
    double tv;             /* ||grad_h u||_1, isotropic */
    double violation;      /* max_r max(lo_r - (R u)_r, (R u)_r - hi_r, 0) */
    double gap;            /* Fenchel-Young gap G(Ku)+G*(t)-<Ku,t> of the beta-scaled problem with the box
                            * indicators left out (they appear as `violation`): a certificate of
                            * optimality only at a feasible iterate (violation = 0); while the
                            * iterate violates a box the value can be negative */
    double dual_residual;  /* ||K^* t||_2 of the beta-scaled problem */
    double rel_change;     /* ||u_k - u_{k-1}|| / ||u_k|| */
    int iters_done;
} ctr_diag;

/* Iterate state of Alg. 4 for warm start / checkpoint-resume; device buffers of the
 * plan's dtype: u (n*n), Ru = R_h u / beta (N*M), v1b (N*M), v2b (2*n*n: x plane then
 * y plane), ub = bar u of Alg. 5 (n*n; needed with params->nonneg, ignored otherwise). */
typedef struct {
    void *u;
    void *Ru;
    void *v1b;
    void *v2b;
    void *ub;
} ctr_state;

/* Create a plan for `geo` computing in `dtype` (CTR_F32 or CTR_F64; CTR_BF16 stores
 * sinogram and image operands of R_h/R_h^* in bfloat16 with FP32 accumulation).
 * In a CTR_BF16 plan every buffer is float except the operands the projectors read:
 * u_dev (and uT_dev) of rh_forward / rh_forward_t and g_dev of rh_adjoint are
 * bfloat16 (uint16 storage); the solver keeps bfloat16 copies of its projector
 * operands internally and everything else (duals, preconditioner, power iterations,
 * diagnostics) in FP32/FP64.
 * Allocates all device workspace on the current device; nothing is allocated later.
 * Returns CTR_EINVAL for n < 1, n_angles < 1, n_bins < 1, h or ds <= 0 or a null
 * angles_host; CTR_EUNSUPPORTED for n > 4096 or an FFT length with a prime factor
 * other than 2 or 3, or ds/h > 2.5; CTR_ENOMEM if allocation fails. */
ctr_status ctr_plan_create(const ctr_geometry *geo, ctr_dtype dtype, ctr_plan **out);
void ctr_plan_destroy(ctr_plan *plan);
void ctr_default_params(ctr_params *p);
const char *ctr_last_error(void);
/* Bytes of device memory the plan holds. */
size_t ctr_plan_device_bytes(const ctr_plan *plan);
/* The diagnostics history of the plan's last solve (params->check_every > 0; Sec. 5's
 * convergence record): *count receives the number of checks it made, and the first
 * min(capacity, *count) records are copied to out_host in order (record r describes the
 * iterate after (r + 1) * check_every iterations; iters_done says which).  A solve with
 * check_every = 0 leaves 0 records.  Synchronises the plan's internal stream; out_host may
 * be NULL when capacity = 0.  CTR_EINVAL for a NULL plan or count or capacity < 0. */
ctr_status ctr_plan_history(ctr_plan *plan, ctr_diag *out_host, int capacity, int *count);
/* Number of this library's kernels the plan has launched so far (kernels replayed
 * inside CUDA graphs included). */
unsigned long long ctr_plan_launch_count(const ctr_plan *plan);
/* Number of jobs of the projectors' symmetric path, 0 when the plan projects angle by
 * angle.  The discrete geometry of Sec. 3.1 is exactly invariant under the symmetries
 * of the pixel grid: angles whose fixed-point (C, S) are (a, b), (-a, b), (b, a) and
 * (-b, a) (e.g. theta, pi - theta, pi/2 - theta, pi/2 + theta) share one job, one ray
 * march and one staged detector coordinate per pixel.  FP32 and BF16 plans with
 * ds >= h take the path when every angle is such an image of its canonical pair and the jobs hold
 * two angles or more on average, the unpaired angle 0 of an odd count aside (uniform angles
 * over [0, pi): an even count in jobs of up to four angles, an odd count in (N + 1) / 2 jobs
 * of theta and pi - theta, which the FP32 kernels run as two-channel "pair" jobs).
 * Results equal those of the per-angle path up to the order of FP32 summation. */
int ctr_plan_symmetric_jobs(const ctr_plan *plan);

/* g = R_h u, the discrete Radon transform of Sec. 3.1 (the adjoint of linear
 * backprojection): bin k of angle l gets sum_ij u_ij Lambda(p_ijl - k) with
 * p = (x_i cos theta_l + y_j sin theta_l)/ds + (M-1)/2 and the hat
 * Lambda(t) = max(0, 1 - |t|).  u_dev: n*n, g_dev: N*M (overwritten).
 * Ray-driven gather (no atomics); exact transpose of rh_adjoint. */
ctr_status rh_forward(ctr_plan *plan, const void *u_dev, void *g_dev, void *stream);

/* rh_forward for a caller that also holds the transposed image uT_dev[j*n + i] =
 * u[i*n + j] (the layout the solver keeps): one kernel launch, no workspace use.
 * Angles with |cos| >= |sin| read uT, the others read u. */
ctr_status rh_forward_t(ctr_plan *plan, const void *u_dev, const void *uT_dev, void *g_dev, void *stream);

/* u = R_h^* g, linear backprojection (Sec. 3.1, definition of R_h^*): pixel (i,j)
 * gets sum_l of g linearly interpolated at p_ijl.  g_dev: N*M, u_dev: n*n
 * (overwritten).  Pixel-driven gather. */
ctr_status rh_adjoint(ctr_plan *plan, const void *g_dev, void *u_dev, void *stream);

/* x = M^{-1} y, the inverse-norm Fourier preconditioner of Alg. 4 (Sec. 4.3.1, 4.4):
 * x = F^{-1}( F(y) ||xi||_eps / (sigma^2 c + (sigma tau)^2 L ||xi||_eps) ),
 * L_ij = 4 sin^2(pi i/n) + 4 sin^2(pi j/n), xi = 2 pi (i~, j~)/n wrapped.
 * Uses params->sigma, tau, eps, c (c must be > 0).  y_dev, x_dev: n*n (may alias). */
ctr_status precond_apply(ctr_plan *plan, const ctr_params *params, const void *y_dev,
                         void *x_dev, void *stream);

/* precond_apply for callers that cannot allocate device memory: no plan, no
 * cudaMalloc/cudaFree, no allocating library call.  Meant for code embedded in a
 * host application that owns all device memory (a fixed pool handed out at start-up)
 * and forbids allocation afterwards -- cudaMalloc/cudaFree may synchronise the
 * device and fragment that budget, which a real-time reconstruction loop cannot
 * accept.  The thesis has no counterpart: this is a packaging of precond_apply.
 * FP32 only; y_dev, x_dev: n*n floats owned by the caller (may alias); n must be
 * 2^a 3^b with n <= 1024 (larger n: CTR_EINVAL with a message).  sigma, tau, c,
 * eps as in precond_apply (all > 0).
 * Scratch: 12 MiB of static device arrays (the complex FFT buffer, the symbol, the
 * twiddles for n = 1024) that every GPU loading this library holds until the
 * process exits.  Each call overwrites all of the scratch it reads, so no state
 * carries over, but every call shares the same arrays: calls that overlap on the
 * GPU (concurrent streams or host threads) race and give wrong results.  The first
 * call on a device looks up the arrays' device addresses (cudaGetSymbolAddress) and
 * sets kernel attributes for that device; make that first call from one thread, on
 * the device it will run on, before any stream capture. */
ctr_status precond_apply_static(int n, double sigma, double tau, double c, double eps, const float *y_dev,
                                float *x_dev, void *stream);

/* Solve problem (C_h) (Sec. 3.2, with the data tolerance) by `iters` iterations of
 * Alg. 4 (PDRQS1) from u = 0:
 *   min_u  sum_{r off trace} 1/2 ((R_h u)_r - f_r)^2 + alpha ||grad_h u||_1
 *   s.t.   |(R_h u)_r - f_r| <= delta off the metal trace (delta < 0: no bound),
 *          (R_h u)_r >= trace_ratio * f_r on the trace (metal_mask_dev[r] != 0).
 * f_dev: N*M data; metal_mask_dev: N*M bytes or NULL (no trace); u_out_dev: n*n.
 * beta and c come from power iterations unless given in params (NULL = defaults).
 * diag_out (host, may be NULL) is filled after an internal sync of `stream`. */
ctr_status tv_pd_solve(ctr_plan *plan, const void *f_dev, const uint8_t *metal_mask_dev,
                       double alpha, double delta, int iters, const ctr_params *params,
                       void *u_out_dev, ctr_diag *diag_out, void *stream);

/* Detector-axis ramp filter F_1^{-1}|omega|F_1 of the filtered backprojection (Sec. 2),
 * the Ram-Lak kernel k(0) = 1/(4 ds^2), k(m) = -1/(pi^2 m^2 ds^2) (odd m), 0 (even m != 0)
 * applied per view as the linear convolution y(k) = ds sum_k' k(k - k') g(k') over the M
 * bins (an FFT of length L >= 2M - 1 along the bins, one CTA per view).  g_dev, y_dev:
 * N*M in the plan's real type (float for FP32 and BF16 plans).  The filter tables are
 * built on the first call (synchronous), later calls are asynchronous on `stream`.
 * CTR_EUNSUPPORTED when one padded view does not fit a CTA's shared memory (FP64 plans
 * with more than about 1600 bins, FP32 beyond about 4600). */
ctr_status ctr_ramp_filter(ctr_plan *plan, const void *g_dev, void *y_dev, void *stream);

/* Filtered backprojection u = (pi / N) R_h^*(ramp-filtered g) (Sec. 2, uniform angles over
 * [0, pi)), the classical reconstruction of the line integrals g_dev (N*M) into u_dev
 * (n*n).  BF16 plans backproject the filtered views stored in bfloat16.  Uses the
 * plan's sinogram scratch. */
ctr_status ctr_fbp(ctr_plan *plan, const void *g_dev, void *u_dev, void *stream);

/* Metal-trace estimation (Sec. "Real metal artifacts"): the pixels of u_dev (n*n, the
 * plan's real type: float for FP32 and BF16 plans, double for FP64) whose value exceeds
 * `threshold` (compared in FP64) are marked, the marks dilated by the disk
 * {di^2 + dj^2 <= radius^2} (0 <= radius <= 64; the thesis dilates by 5 px), and
 * trace_dev[r] (N*M bytes) = 1 where R_h of the 0/1 image of marks exceeds proj_tol >= 0,
 * else 0 (bins that no mark touches get exactly 0).  marked_dev (n*n bytes) receives the
 * dilated marks, or may be NULL.  The result is the metal_mask argument of tv_pd_solve.
 * Uses the plan's scratch (not reentrant per plan); asynchronous on `stream`. */
ctr_status ctr_metal_trace(ctr_plan *plan, const void *u_dev, double threshold, int radius, double proj_tol,
                           uint8_t *marked_dev, uint8_t *trace_dev, void *stream);

/* ADMM with PCG inner solves (Sec. "Alternating Direction Method of Multipliers") for the
 * unconstrained problem (U_h), from u = 0, on the beta-scaled problem: z = (w, v) = K u,
 * K = [R_h/beta; grad_h], weighting diag(I, tau I) (tau = params->tau), penalty mu > 0.
 * Per iteration: cg_iters (1..64) steps of preconditioned CG, warm-started, on
 * (Rt^* Rt - tau^2 Delta_h) u = Rt^*(w - eta_w) - tau^2 div_h(v - eta_v), preconditioned by
 * M = c S + tau^2 Lap of the kind params->precond selects (c, beta from power iterations
 * unless given); then w = (f/beta + mu (Rt u + eta_w))/(1 + mu), v = soft-threshold of
 * grad u + eta_v at lambda/(mu tau^2), eta -= z - K u.  Rt u is carried through the CG
 * updates (no extra projection).  Everything runs on the device (CG scalars in device
 * memory, no host round trip); graph_block iterations per CUDA graph.  diag_out's gap and
 * dual residual use t1 = Rt u - f/beta and t2 = mu tau eta_v.  FP32 and FP64 plans
 * (CTR_EUNSUPPORTED for BF16 or nonneg = 1); errors as tv_pd_solve. */
ctr_status tv_admm_solve(ctr_plan *plan, const void *f_dev, double alpha, int iters, double mu, int cg_iters,
                         const ctr_params *params, void *u_out_dev, ctr_diag *diag_out, void *stream);

/* The metal-artifact pipeline of Sec. "Real metal artifacts": iters_pre iterations of
 * Alg. 3 on the unconstrained problem give a first reconstruction (into u_out_dev),
 * ctr_metal_trace(threshold, radius, proj_tol) turns it into the trace (trace_out_dev,
 * N*M bytes), and tv_pd_solve(f, trace, alpha, delta, iters) solves (C_h) with it into
 * u_out_dev, reusing the first stage's beta and c.  params as for tv_pd_solve (nonneg
 * applies to the second stage only); diag_out describes the second stage. */
ctr_status tv_mar_solve(ctr_plan *plan, const void *f_dev, double alpha, double delta, double threshold,
                        int radius, double proj_tol, int iters_pre, int iters, const ctr_params *params,
                        uint8_t *trace_out_dev, void *u_out_dev, ctr_diag *diag_out, void *stream);

/* Alg. 3 (PDRQS2, Sec. "Suitable Preconditioners") for the unconstrained problem (U_h),
 *   min_u  1/2 ||R_h u - f||^2 + alpha ||grad_h u||_1,
 * from u = 0: the data term stays in the quadratic part (only the TV term is
 * dualised), so T = sigma Rt^* Rt + (sigma tau)^2 (-Delta_h) and M carries sigma c where
 * Alg. 4's carries sigma^2 c; c, beta and the preconditioner kind as in tv_pd_solve
 * (params->nonneg must be 0: CTR_EUNSUPPORTED).  Per iteration: one backprojection of
 * the residual R_h u/beta - f/beta (with the divergence and Laplacian terms in its
 * epilogue), the preconditioner, one forward projection writing the next residual,
 * and the TV dual step.  diag_out's gap and dual residual use t1 = R_h u/beta - f/beta,
 * the data term's gradient.  FP32, FP64 and BF16 plans; errors as tv_pd_solve. */
ctr_status tv_pdrq2_solve(ctr_plan *plan, const void *f_dev, double alpha, int iters, const ctr_params *params,
                          void *u_out_dev, ctr_diag *diag_out, void *stream);

/* Alg. 1 (Chambolle-Pock, Sec. 3.2) for the same problem as tv_pd_solve, from u = 0:
 * the unpreconditioned primal-dual baseline against which the thesis measures Alg. 4.
 * Runs on the beta-scaled problem (R_h / beta, so its norm is about 1) with primal step
 * sigma_p and dual step tau_d, sigma_p tau_d (1 + 8/h^2) < 1; sigma_p <= 0 or tau_d <= 0
 * selects 0.99 / sqrt(1.02 (1 + 8/h^2)) for both.  Per iteration: v = prox(v + tau_d R u_bar)
 * (in the forward projector's epilogue), w = P_lambda(w + tau_d grad u_bar), u_new = u +
 * sigma_p div w - sigma_p R^* v and u_bar = 2 u_new - u (in the backprojection's epilogue).
 * params: beta, power_iters, trace_ratio and graph_block are used (NULL = defaults);
 * params->tau only scales the reported dual (t2 = w / tau) so that diag_out's gap and
 * dual residual are those of tv_pd_solve's saddle problem.  FP32 and FP64 plans
 * (CTR_EUNSUPPORTED for BF16), any n (no FFT); errors as tv_pd_solve. */
ctr_status tv_cp_solve(ctr_plan *plan, const void *f_dev, const uint8_t *metal_mask_dev, double alpha,
                       double delta, int iters, double sigma_p, double tau_d, const ctr_params *params,
                       void *u_out_dev, ctr_diag *diag_out, void *stream);

/* General form: per-bin data term g_r(z) = w_r/2 (z - a_r)^2 + I_[lo_r, hi_r](z) given
 * by four device arrays of N*M (original scale, +-inf allowed in lo/hi), which covers
 * every resolvent variant of Sec. 3.3-3.5.  `state` (may be NULL) holds the start on
 * entry (NULL: zeros) and the final iterate on exit; u_out_dev (may be NULL if state
 * is given) receives u.  Iterations are counted from the state given. */
ctr_status tv_pd_run(ctr_plan *plan, const void *w_dev, const void *a_dev, const void *lo_dev,
                     const void *hi_dev, double alpha, int iters, const ctr_params *params,
                     ctr_state *state, void *u_out_dev, ctr_diag *diag_out, void *stream);

/* tv_pd_solve continuing from `state` (in/out, FP32/FP64 plans): runs `iters`
 * iterations of Alg. 4 from the given (u, Ru, v1b, v2b) and leaves the new state in
 * the same buffers (checkpoint / resume, and the forward replay of the reverse mode).
 * params->beta and ->c should be given so that every call uses the same scaling. */
ctr_status tv_pd_solve_state(ctr_plan *plan, const void *f_dev, const uint8_t *metal_mask_dev, double alpha,
                             double delta, int iters, const ctr_params *params, ctr_state *state,
                             ctr_diag *diag_out, void *stream);

/* Reverse mode of one iteration of Alg. 4 (vector-Jacobian product) for the
 * iteration that took state s0 to s1 (both as produced by tv_pd_solve_state with the
 * same f, mask, alpha, delta, params; params->beta, ->c > 0 required).
 * In: bu, b1, b2 = cotangents of s1's u (n*n), v1b (N*M), v2b (2*n*n).  Out (in
 * place): the cotangents of s0's u, v1b, v2b.  Accumulated: gf (N*M) += d/df,
 * *galpha_dev (device double) += d/dalpha.  beta and c are constants (they depend on
 * the geometry only).  Where clip or the TV projection has a kink the inside branch
 * is differentiated. */
ctr_status tv_pd_vjp_step(ctr_plan *plan, const void *f_dev, const uint8_t *metal_mask_dev, double alpha,
                          double delta, const ctr_params *params, const ctr_state *s0, const ctr_state *s1,
                          void *bu, void *b1, void *b2, void *gf, double *galpha_dev, void *stream);

/* Reverse mode of `length` (>= 1) consecutive iterations of Alg. 4 starting from the
 * checkpoint s_start: the iterations are replayed on the device (state k stored in
 * workspace_dev), then reversed newest first with the same kernels as tv_pd_vjp_step,
 * all on `stream` without host synchronisation.  workspace_dev: (length + 1) states of
 * n*n + 2*N*M + 2*n*n elements of the plan's real type, caller-owned (state k at offset
 * k * (3*n*n + 2*N*M): u, Ru, v1b, v2b).  bu, b1, b2, gf, galpha_dev as tv_pd_vjp_step
 * (the cotangents of the state after the last iteration in, of s_start out).  Equal to
 * replaying with tv_pd_solve_state and calling tv_pd_vjp_step per iteration. */
ctr_status tv_pd_vjp_segment(ctr_plan *plan, const void *f_dev, const uint8_t *metal_mask_dev, double alpha,
                             double delta, const ctr_params *params, const ctr_state *s_start, int length,
                             void *workspace_dev, void *bu, void *b1, void *b2, void *gf, double *galpha_dev,
                             void *stream);

/* Tuning hook: split the backprojection's angles (on the symmetric path: its jobs, see
 * ctr_plan_symmetric_jobs) into `groups` groups whose partial images are summed (more
 * CTAs for small images).  1 <= groups <= the capacity the plan allocated (up to 8 for
 * n <= 1024), else CTR_EINVAL.  No allocation.  ctr_plan_get_bp_groups returns the
 * split of the path the plan takes. */
ctr_status ctr_plan_set_bp_groups(ctr_plan *plan, int groups);
int ctr_plan_get_bp_groups(const ctr_plan *plan);

/* Tuning hook: the launch shape of the symmetric forward projector, one of the compiled
 * instances (jobs_per_cta, segments) = (1, 2), (1, 4) [default], (1, 8), (2, 2), (2, 4),
 * (4, 2), (4, 1).  A CTA takes jobs_per_cta adjacent jobs (nearly coincident rays: they
 * share the orbit image's lines in L1) and 31 bins; `segments` warps split the rows each
 * job's rays cross, and their sums are added in a fixed order.  (4, 1) is the staged form:
 * one warp per job, and for every block of 8 rows the union of the four jobs' bands of the
 * orbit image is copied into shared memory (cp.async, zero-filled outside the image) ahead
 * of the march, so each pixel comes from L2 once per four jobs.  The shape changes FP32
 * summation order only.  CTR_EINVAL for other shapes, CTR_EUNSUPPORTED off the symmetric path
 * and, for (4, 1), where the staged window would exceed one CTA's shared memory;
 * ctr_plan_get_fwd_shape reports (0, 0) off the symmetric path. */
ctr_status ctr_plan_set_fwd_shape(ctr_plan *plan, int jobs_per_cta, int segments);
ctr_status ctr_plan_get_fwd_shape(const ctr_plan *plan, int *jobs_per_cta, int *segments);

/* Tuning hook: the kernels of the Fourier preconditioner passes (Sec. 4.3.1, the 2-D DFT
 * diagonalisation of M).  form 0 [default]: on FP32 plans with n = 256, 512 or 1024 each
 * row pair and each column is one warp's transform (a four-step factorisation n = 32 x
 * n/32 in registers, no CTA barrier); other plans use form 1.  form 1: the CTA-level
 * mixed-radix Stockham passes through shared memory (every n = 2^a 3^b, FP64).  Both
 * compute the same DFT up to FP32 rounding.  CTR_EINVAL for other values.  No allocation;
 * ctr_plan_get_fft_form returns the form the plan's passes take (1 where 0 does not apply). */
ctr_status ctr_plan_set_fft_form(ctr_plan *plan, int form);
int ctr_plan_get_fft_form(const ctr_plan *plan);

/* Tuning hook: programmatic dependent launch of the kernels of one iteration on the
 * symmetric FP32 / BF16 path (the backprojection, the three preconditioner passes of form 0,
 * the orbit image with the TV step, the forward projector).  on = 1 [default]: each of them
 * is launched with the programmatic-serialization attribute and waits, before its first
 * global-memory access, for the kernel before it to complete, so its launch overlaps that
 * kernel's last wave; results are identical to on = 0 (plain stream order).  CTR_EINVAL
 * for values other than 0 and 1.  No allocation; ctr_plan_get_launch_overlap returns it. */
ctr_status ctr_plan_set_launch_overlap(ctr_plan *plan, int on);
int ctr_plan_get_launch_overlap(const ctr_plan *plan);


/* Batches: many independent slices (each its own geometry, image size and view
 * count), FP32, solved together.  Each stage of an iteration of Alg. 4 is ONE kernel
 * launch covering every slice (a block-offset table maps CTAs to slices), and the
 * iterations are captured as CUDA graphs.  Slices need n = 2^a 3^b and 1 <= ds/h <
 * sqrt(2).  The batch owns one plan per slice (ctr_batch_plan returns it; do not
 * destroy it separately). */
typedef struct ctr_batch ctr_batch;
ctr_status ctr_batch_create(const ctr_geometry *geos, int count, ctr_batch **out);
void ctr_batch_destroy(ctr_batch *batch);
ctr_plan *ctr_batch_plan(ctr_batch *batch, int index);
/* Rebuild the batch's launch tables after ctr_plan_set_bp_groups on its plans. */
ctr_status ctr_batch_retune(ctr_batch *batch);
unsigned long long ctr_batch_launch_count(const ctr_batch *batch);
/* How a batch runs an iteration of Alg. 4.  mode 0 (default): one kernel launch per stage
 * over all slices, iterations replayed from CUDA graphs.  mode 1: one persistent
 * cooperative launch per iteration that runs every stage for every slice (as many CTAs
 * as are resident at once, the stages separated by grid barriers); results are identical
 * to mode 0.  Each CTA polls a grid barrier at most spin_limit times (~100 ns per poll)
 * before it gives up; the launch then ends early and the solve returns CTR_ETIMEOUT
 * (spin_limit 0 makes every barrier give up at once, which tests that path).
 * CTR_EUNSUPPORTED for mode 1 when the persistent kernel cannot be resident with the
 * batch's shared memory.  ctr_batch_persistent_ctas returns the persistent grid size
 * (0: unavailable). */
ctr_status ctr_batch_set_mode(ctr_batch *batch, int mode, unsigned long long spin_limit);
int ctr_batch_get_mode(const ctr_batch *batch);
int ctr_batch_persistent_ctas(const ctr_batch *batch);
/* tv_pd_solve for every slice i: f_devs[i] (N_i*M_i floats), masks[i] (bytes or NULL;
 * masks may be NULL), alphas[i], deltas[i], shared iters and params (every
 * preconditioner kind; nonneg = 1 runs Alg. 5 on all slices); betas/cs (may be NULL,
 * or entries <= 0) select power iterations per slice; u_outs[i] (n_i^2 floats); diags
 * (NULL or count entries, host) filled after an internal sync. */
ctr_status tv_pd_solve_batched(ctr_batch *batch, const void *const *f_devs, const uint8_t *const *masks,
                               const double *alphas, const double *deltas, int iters, const ctr_params *params,
                               const double *betas, const double *cs, void *const *u_outs, ctr_diag *diags,
                               void *stream);

/* Power iterations of Sec. 4.3 / 5.1 from the fixed R2 start pattern
 * x_ij = frac(1/2 + i/g + j/g^2) - 1/2 (g the plastic number): beta ~ ||R_h||
 * (iters steps on R_h^* R_h) and lambda_max(Mt^{-1} Rt^* Rt) with Rt = R_h/beta,
 * Mt = F^{-1}(1/||xi||_eps) F.  Host outputs; synchronises `stream`. */
ctr_status ctr_power_beta(ctr_plan *plan, int iters, double *beta_out, void *stream);
ctr_status ctr_power_lambda(ctr_plan *plan, double beta, double eps, int iters,
                            double *lambda_out, void *stream);

/* Measured FP32 FMA ceiling of the current device (FMA/s): independent FMA chains in
 * registers, scalar and paired (.f32x2) forms, 8 CTAs of 256 threads per SM; the faster
 * form after a warm-up launch.  The denominator of the projectors' roofline (they do two
 * FMAs per (pixel, angle) sample, Sec. 3.1, on operands staged on chip).  No counterpart
 * in the thesis: a measurement utility.  Synchronises `stream`; no allocation. */
ctr_status ctr_fp32_fma_rate(double *fma_per_s, void *stream);

/* grad_h (forward differences, Neumann; Sec. 3.1): u (n*n) -> p (2*n*n, x then y). */
ctr_status ctr_grad(ctr_plan *plan, const void *u_dev, void *p_dev, void *stream);
/* div_h = -grad_h^* (backward differences, Dirichlet; Sec. 3.1): p (2*n*n) -> d (n*n). */
ctr_status ctr_div(ctr_plan *plan, const void *p_dev, void *d_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* CTRECON_H */
