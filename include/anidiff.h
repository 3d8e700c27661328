/*
 * anidiff.h -- C ABI of the GB300 (sm_103a) exponential-integrator library for
 * the 2-D anisotropic diffusion-advection equation with sources
 *
 *     du/dt = div(D grad u) + div(a u) + S(x, y, t)              (Eq. anidiff)
 *
 * of Deka, Kissmann & Einkemmer, "Efficient numerical methods for Anisotropic
 * Diffusion of Galactic Cosmic Rays" (ICRC 2023).  The matrix functions
 * phi_l(dt A) are applied by Newton interpolation at Leja points on [-2, 2]
 * (Section 2), inside exponential quadrature steps (Eqs. exp_quad,
 * exp_midpoint, exp_quad_Gauss); Crank-Nicolson is the comparison solver.
 *
 * Conventions shared by every call
 *   - Grid: nx x ny cells on [x0, x1] x [y0, y1], cell centred.  Every field and
 *     vector is row-major [ny][nx] (x fastest), contiguous, no padding.
 *   - Coefficient fields passed to ad_create_operator are float64 DEVICE
 *     pointers; they are read during the call only (the library packs its own
 *     copy).  Vectors (u, v, out) have the operator's storage type: float64
 *     for AD_FP64, float32 for AD_FP32_STORAGE.  A vector argument may be a
 *     device pointer or a host pointer; host data is staged through
 *     library-owned device buffers with copies on the operator's stream.
 *   - Ownership: the caller owns every buffer it passes.  The library owns the
 *     operator (packed coefficients, workspace, host-pointer staging buffers,
 *     CUDA graphs), allocated in ad_create_operator and released by
 *     ad_destroy_operator.  No step allocates device memory: the GMRES basis
 *     of ad_cn_step is allocated by ad_reserve_gmres beforehand, and the
 *     first step of each kind instantiates its CUDA graph once (graph
 *     instantiation is the driver's, not a cudaMalloc).
 *   - Streams: all work is enqueued on the CUDA stream given at creation.
 *     Calls that report statistics or a convergence status synchronise that
 *     stream before returning.
 *   - Errors: every call returns an ad_status; ad_last_error() gives a
 *     thread-local message for the last failure.  No C++ exception crosses
 *     the ABI.  A CUDA error is reported as AD_ERR_CUDA.
 */
#ifndef ANIDIFF_H
#define ANIDIFF_H

#if defined(__GNUC__)
#define AD_API __attribute__((visibility("default")))
#else
#define AD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AD_OK = 0,
  AD_ERR_INVALID = 1,        /* bad argument (sizes, pointers, s, c, tolerances) */
  AD_ERR_CUDA = 2,           /* a CUDA runtime call or kernel launch failed */
  AD_ERR_NOT_CONVERGED = 3,  /* Leja series or GMRES hit its iteration cap */
  AD_ERR_TIMEOUT = 4,        /* a bounded device-side wait gave up */
  AD_ERR_NOMEM = 5           /* device allocation failed */
} ad_status;

typedef enum { AD_BC_PERIODIC = 0, AD_BC_DIRICHLET0 = 1 } ad_bc;
typedef enum { AD_FP64 = 0, AD_FP32_STORAGE = 1 } ad_precision;
typedef enum { AD_BOUND_GERSHGORIN = 0, AD_BOUND_POWER = 1, AD_BOUND_LEARNED = 2 } ad_bound_method;

typedef struct {
  int nx, ny;                /* cells; nx, ny >= 1 */
  double x0, x1, y0, y1;     /* domain; x1 > x0, y1 > y0 */
  int bc;                    /* ad_bc */
} ad_grid;

typedef struct {
  int iters;                 /* Leja (or GMRES) iterations, summed over substeps (and
                                rejected adaptive attempts) */
  int matvecs;               /* all applications of A, including A u and substep couplings */
  int substeps;              /* K: the step was split into K (accepted) substeps */
  int converged;             /* 1 if every series met its stopping rule */
  double err_est;            /* largest |d_{m+1}| ||y_{m+1}|| / ||p_{m+1}|| (GMRES: relative residual) */
  double alpha;              /* spectral bound used */
  int kernel_launches;       /* device kernels this call enqueued (graph-loop bodies included) */
  int rejected;              /* substeps rejected by adaptive substep control */
} ad_stats;

/* Time profile h_k(t) of a separable source S(x, y, t) = sum_k h_k(t) g_k(x, y).
 * Called on the host, from the calling thread, during the step call. */
typedef double (*ad_time_profile)(int k, double t, void* ctx);

typedef struct {
  int nterms;                /* 0 <= nterms <= 16 */
  const void* const* g;      /* host array of nterms DEVICE pointers, storage type, [ny][nx] */
  ad_time_profile h;         /* NULL: every h_k(t) = 1 (time-independent source) */
  void* ctx;
} ad_source;

typedef struct ad_operator ad_operator;

/* Build the discretised operator A = div(D grad .) + div(a .) of Eq. anidiff
 * (A is defined below Eq. exp_quad; the tensor D = [[Dxx, Dxy], [Dxy, Dyy]] in
 * Section 1).  The paper gives no spatial scheme: the library uses the
 * conservative 9-point flux form on the cell-centred grid (face coefficients
 * are means of the two adjacent cells; centred advective flux; periodic
 * wrap or zero Dirichlet by odd-reflection ghosts).
 *   Dxx, Dxy, Dyy : float64 device fields [ny][nx] (required).
 *   ax, ay        : float64 device fields, or NULL to use the constants ax_c, ay_c.
 *   precision     : AD_FP64 (9 packed float64 weights per cell) or
 *                   AD_FP32_STORAGE (float32 fields, float32 stencil arithmetic,
 *                   float64 Leja scalars and norm accumulation).
 *   cuda_stream   : cudaStream_t (NULL = legacy default stream) for all work.
 *   out           : receives the handle.
 * Errors: AD_ERR_INVALID for null pointers or a bad grid, AD_ERR_NOMEM,
 * AD_ERR_CUDA.  The spectral bound is computed here by Gershgorin (Section 2);
 * override it with ad_spectral_bound or ad_set_spectral_bound. */
AD_API int ad_create_operator(const ad_grid* grid, const double* Dxx, const double* Dxy,
                       const double* Dyy, const double* ax, const double* ay,
                       double ax_c, double ay_c, int precision, void* cuda_stream,
                       ad_operator** out);

/* Release the operator and everything it owns.  NULL is accepted. */
AD_API int ad_destroy_operator(ad_operator* op);

/* Leja series options: rho_max is the largest gamma*dt per substep (a step
 * with rho = gamma dt > rho_max is split into ceil(rho / rho_max) substeps);
 * max_iters caps the number of Leja iterations per series (<= 500).
 * Values <= 0 keep the current setting.  Defaults: rho_max 200, max_iters 500. */
AD_API int ad_set_options(ad_operator* op, double rho_max, int max_iters);

/* Substep control of the Leja series (the paper fixes none).
 * adaptive = 0 (default): ceil(gamma dt / rho_max) equal substeps; a series
 * that reaches max_iters still contributes and the call returns
 * AD_ERR_NOT_CONVERGED.  adaptive = 1: start from that substep; a substep
 * whose series reaches max_iters without meeting the stopping rule is
 * rejected and retried at half the size; after an accepted substep of m
 * iterations the next one doubles when 4 m <= max_iters (not right after a
 * rejection); the last substep is the remainder of the step.  Substeps may
 * then differ in size (phi_1: w_{k+1} = w_k + h_k phi_1(h_k A)(A w_k + v);
 * augmented exponential: exp(h_k Atilde) applied in turn).  More than 40
 * rejections or 4096 accepted substeps give up: AD_ERR_NOT_CONVERGED with u
 * (ad_expquad_step) or out (ad_leja_phi1) not written.  Forced iteration
 * counts (force_iters >= 0) always use the fixed rule.  Stats: substeps =
 * accepted, rejected = rejected attempts; iters and matvecs include rejected
 * work.  Applies to ad_leja_phi1 and ad_expquad_step; ad_batch_midpoint_step
 * and the no-allocation entry point keep one substep. */
AD_API int ad_set_substep_control(ad_operator* op, int adaptive);

/* Estimate alpha, the largest-magnitude (negative) eigenvalue of A (Section 2:
 * Gershgorin's disc theorem, smallest eigenvalue taken as 0), store it in the
 * operator and return it in *alpha.
 *   method AD_BOUND_GERSHGORIN: alpha = min_i (a_ii - sum_{j!=i} |a_ij|).
 *   method AD_BOUND_POWER: power iteration, x <- A x / ||A x|| for power_iters
 *     steps from x0 (device vector of the storage type) or, with x0 == NULL,
 *     from the counter-based SplitMix64 sequence with the given seed mapped to
 *     [-0.5, 0.5); alpha = -safety * ||A x_last||.
 *   method AD_BOUND_LEARNED: the bound model attached by ad_set_bound_model
 *     (ad_learned_bounds on this one operator with the attached margin and
 *     dt; x0, seed, power_iters and safety are ignored).  AD_ERR_INVALID when
 *     no model is attached. */
AD_API int ad_spectral_bound(ad_operator* op, int method, const void* x0, unsigned long long seed,
                      int power_iters, double safety, double* alpha);

/* Set alpha directly (alpha < 0); c = alpha/2 and gamma = -alpha/4 follow. */
AD_API int ad_set_spectral_bound(ad_operator* op, double alpha);
AD_API int ad_get_spectral_bound(const ad_operator* op, double* alpha);

/* Au = A u (one matrix-free 9-point stencil pass).  u and Au: storage type. */
AD_API int ad_apply(ad_operator* op, const void* u, void* Au);

/* out = phi_1(dt A) v by Leja interpolation (Section 2): Leja points on
 * [-2, 2] with xi_0 = 2, divided differences of xi -> phi_1((c + gamma xi) dt),
 * and the recurrence y_{m+1} = ((A - c)/gamma - xi_m) y_m,
 * p_{m+1} = p_m + d_{m+1} y_{m+1}, each iteration one fused device pass.
 * Stopping rule: after term m+1 >= 2, stop when |d_{m+1}| ||y_{m+1}|| <=
 * tol ||p_{m+1}||.  force_iters > 0 runs exactly that many iterations per
 * substep (no test); force_iters == 0 returns d_0 v.  tol > 0 unless forced.
 * v and out may alias.  Returns AD_ERR_NOT_CONVERGED when a series reaches
 * max_iters (out then holds the partial sum).  stats may be NULL. */
AD_API int ad_leja_phi1(ad_operator* op, const void* v, void* out, double dt, double tol,
                 int force_iters, ad_stats* stats);

/* One exponential quadrature step, Eq. exp_quad, in place on u (t -> t + dt):
 *   s = 1: u += dt phi_1(dt A)(A u + S(t + c[0] dt))   (Eq. exp_midpoint for c = 1/2);
 *   s = 2: weights b_1, b_2 of Section 2, collected as
 *          u += dt phi_1(dt A) w1 + dt^2 phi_2(dt A) w2,
 *          w1 = A u + (c2 S1 - c1 S2)/(c2 - c1), w2 = (S2 - S1)/((c2 - c1) dt),
 *          evaluated as the exponential of the augmented matrix (Section 2)
 *          by one Leja series (Eq. exp_quad_Gauss for c = (1 -+ 1/sqrt 3)/2).
 * c: host array of s nodes with c[0] != c[1] for s = 2.  src may be NULL (S = 0).
 * force_iters as in ad_leja_phi1.  stats may be NULL. */
AD_API int ad_expquad_step(ad_operator* op, void* u, double t, double dt, int s, const double* c,
                    const ad_source* src, double tol, int force_iters, ad_stats* stats);

/* ad_expquad_step without the synchronisation, for running many steps with no
 * host round trip between them.  When u is a device pointer, the substep
 * control is the fixed rule and the step takes one substep (gamma dt <=
 * rho_max), the call only enqueues the step on the operator's stream and
 * returns; its iteration count and convergence status are accumulated on the
 * device.  Otherwise it runs ad_expquad_step (synchronously) and adds that
 * step to the same totals.  u must stay valid until the stream has run the
 * step.  Returns AD_OK, or AD_ERR_INVALID / AD_ERR_CUDA / AD_ERR_TIMEOUT when
 * enqueueing (or the synchronous run) fails; a series that misses the
 * tolerance is reported by ad_async_totals, not here.  Same arguments as
 * ad_expquad_step with force_iters = -1. */
AD_API int ad_expquad_step_async(ad_operator* op, void* u, double t, double dt, int s,
                                 const double* c, const ad_source* src, double tol);

/* Synchronises the operator's stream and returns the totals of the
 * ad_expquad_step_async calls since the previous ad_async_totals call, then
 * resets them: iters, matvecs, substeps, rejected and kernel_launches summed;
 * err_est the largest; converged 0 if any series missed the tolerance; alpha
 * the current bound.  stats may be NULL.  Returns the worst status among those
 * steps: AD_OK, AD_ERR_NOT_CONVERGED (a series reached max_iters; its step was
 * still applied, as in ad_expquad_step) or AD_ERR_TIMEOUT. */
AD_API int ad_async_totals(ad_operator* op, ad_stats* stats);

/* Allocate the Krylov basis of ad_cn_step for restarts up to max_restart
 * (1..200): (max_restart + 1) float64 vectors of the grid's size, kept until
 * the operator is destroyed or a larger reservation replaces it.  AD_FP64
 * operators only.  Synchronises the operator's stream when it reallocates. */
AD_API int ad_reserve_gmres(ad_operator* op, int max_restart);

/* One Crank-Nicolson step (the paper's comparison solver; its linear solver
 * is unspecified): (I - dt/2 A) u+ = (I + dt/2 A) u + dt (S(t) + S(t+dt))/2,
 * solved by restarted GMRES(restart) from x0 = u to relative residual
 * gmres_tol.  force_iters > 0 runs exactly that many Arnoldi steps in one
 * cycle (force_iters <= restart <= 200).  AD_FP64 operators only.  The basis
 * must have been reserved for at least max(restart, force_iters) by
 * ad_reserve_gmres (AD_ERR_INVALID otherwise); the step allocates nothing. */
AD_API int ad_cn_step(ad_operator* op, void* u, double t, double dt, const ad_source* src,
               double gmres_tol, int restart, int force_iters, ad_stats* stats);

/* ---------------------------------------------------------------- batched form
 * Many independent problems of uneven size (for example the momentum slices
 * of a cosmic-ray grid: with the momentum terms of the full transport
 * equation dropped, each momentum only sets its own coefficients) advanced by
 * one exponential-midpoint step each (Eq. exp_midpoint) in ONE CUDA graph
 * launch: the series start of every slice in one pass, the Newton series of
 * every slice in ONE persistent cooperative kernel (two iterations per pass
 * over warp tiles; a slice's next pass waits only for its own previous pass,
 * so slices at different passes overlap; converged slices drop out), and the
 * update in one pass.  Each slice keeps its own spectral bound, Leja scalars
 * and stopping rule.  Where the persistent kernel does not apply (slices with
 * nx % 4 != 0 or an advection field, unaligned vectors, more than two source
 * terms, AD_BATCH_PERSIST=0) the series runs as a graph loop of iteration
 * launches instead. */
typedef struct ad_batch ad_batch;

/* Group nslices AD_FP32_STORAGE operators (same advection mode, same stream;
 * sizes may differ).  The operators must outlive the batch and their
 * workspaces are used by it.  autotune != 0: time tile heights {8,16,32,64} x
 * {2,3,4} resident blocks per SM on this batch and keep the fastest; the
 * choice is cached in a JSON file (AD_AUTOTUNE_CACHE, default
 * autotune_cache.json beside the library) keyed by the slice-size mix. */
AD_API int ad_create_batch(ad_operator* const* ops, int nslices, int autotune, ad_batch** out);
AD_API int ad_destroy_batch(ad_batch* b);

/* One exponential-midpoint step of every slice, in place on u[s] (float32
 * device vectors).  src: NULL or an array of nslices sources (at most 4 terms
 * each, evaluated at t + dt/2).  Every slice needs gamma_s dt <= rho_max (one
 * substep).  force_iters > 0 runs exactly that many iterations per slice.
 * per_slice: NULL or nslices stats (kernel_launches holds the whole step's
 * count in every entry).  AD_ERR_NOT_CONVERGED if any slice hit max_iters
 * (or produced a non-finite norm); such a slice keeps its input state, so the
 * caller can repeat it alone with a safer bound, while every converged slice
 * has been advanced.  AD_ERR_TIMEOUT if a bounded wait of the persistent
 * kernel gave up (the context stays usable). */
AD_API int ad_batch_midpoint_step(ad_batch* b, void* const* u, double t, double dt,
                                  const ad_source* src, double tol, int force_iters,
                                  ad_stats* per_slice);

/* Binds the batch to state vectors and sources held by the caller, for
 * repeated steps with ad_batch_step (no per-call arrays to pass or check):
 * u and src as for ad_batch_midpoint_step.  The pointers to the vectors and
 * to the source fields are copied (the arrays u, src and src[s].g need not
 * outlive the call); the vectors, the fields and any h context must stay
 * valid until the batch is rebound or destroyed.  AD_ERR_INVALID as
 * ad_batch_midpoint_step. */
AD_API int ad_batch_bind(ad_batch* b, void* const* u, const ad_source* src);

/* One exponential-midpoint step of the bound vectors: ad_batch_midpoint_step
 * with the arguments of the last ad_batch_bind (AD_ERR_INVALID if none). */
AD_API int ad_batch_step(ad_batch* b, double t, double dt, double tol, int force_iters,
                         ad_stats* per_slice);

/* Queue order of the slices' warp tiles.  In every pass of the batched
 * series the tiles of the slices expected to iterate longest are handed out
 * first, so that the longest series, which bound the step, do not wait behind
 * slices that stop earlier.  iters: nslices expected Leja iteration counts
 * (e.g. the learned model's predictions from ad_learned_bounds), or NULL for
 * slice order.  After every step the batch re-queues the slices by the counts
 * that step took (AD_BATCH_ORDER=0 keeps the order set here).  The order
 * changes no result: each slice's tile sums keep their order.  Takes effect
 * at the next ad_batch_midpoint_step; AD_ERR_INVALID for a non-finite count. */
AD_API int ad_batch_iteration_hint(ad_batch* b, const double* iters);

/* The current queue order: order[q] is the slice queued q-th (nslices ints,
 * caller memory). */
AD_API int ad_batch_order(const ad_batch* b, int* order);

/* Chosen tile height, launch blocks, tile count, the autotuned kernel time
 * and the marching of the two-iteration kernels (0 plain, 1 one row of
 * lookahead in registers, 2 the same with packed FP32 pair arithmetic; the
 * autotuner times 1 and 2 on the persistent kernel).  Any pointer may be
 * NULL. */
AD_API int ad_batch_info(const ad_batch* b, int* tile_rows, int* blocks, int* ntiles,
                         double* tuned_ms, int* marching);

/* ---------------------------------------------------------------- learned bound
 * A small network predicting, from per-field features, the spectral bound
 * that Section 2 estimates with Gershgorin discs (here: the dimensionless
 * log(|alpha| dx^2 / D_par)) and the Leja iteration count, trained on spectra
 * the method itself computes.  h1 = tanh(x W1 + b1), h2 = tanh(h1 W2 + b2),
 * y = h2 W3 + b3; inputs standardised, outputs de-standardised.  FP32
 * training (forward, MSE backward, Adam), BF16 inference with FP32
 * accumulation.  X: float32 DEVICE [B][n_in]; Y: float32 DEVICE [B][n_out]. */
typedef struct ad_mlp ad_mlp;
/* Glorot-uniform weights from SplitMix64(seed), zero biases, identity normalisation. */
AD_API int ad_mlp_create(int n_in, int n_hidden, int n_out, unsigned long long seed,
                         void* cuda_stream, ad_mlp** out);
AD_API int ad_mlp_destroy(ad_mlp* m);
AD_API int ad_mlp_num_params(const ad_mlp* m, int* n);
/* set != 0: host -> model (resets Adam state); set == 0: model -> host.
 * Flat order W1 [n_in][h], b1, W2 [h][h], b2, W3 [h][n_out], b3. */
AD_API int ad_mlp_params(ad_mlp* m, float* host, int n, int set);
AD_API int ad_mlp_normalization(ad_mlp* m, float* x_mean, float* x_std, float* y_mean,
                                float* y_std, int set);
/* Loss 1/(2B) sum (y - t)^2 on standardised data and its gradient (host, flat order). */
AD_API int ad_mlp_loss_grad(ad_mlp* m, const float* X, const float* Y, int B, float* loss,
                            float* host_grad);
/* Full-batch Adam for `epochs` steps (fit_normalization: first compute the
 * column statistics of X and Y on the GPU).  final_loss may be NULL. */
AD_API int ad_mlp_train(ad_mlp* m, const float* X, const float* Y, int B, int epochs, float lr,
                        int fit_normalization, float* final_loss);
/* Y = model(X), de-standardised; bf16 != 0 runs the BF16 inference kernels. */
AD_API int ad_mlp_predict(ad_mlp* m, const float* X, int B, int bf16, float* Y);
/* The learned spectral bound through the library (replaces the bound pass
 * of Section 2 for operators whose fields resemble the training fields):
 * ad_create_operator records the 21 input features of its fields (as
 * ad_field_features, with max |a| over the advection fields or the constant
 * advection).  For each of nops operators, the model m (21 inputs, 2
 * outputs, as trained by ad_mlp_train on ad_bound_training_sample data)
 * predicts t0 = log(|alpha| dx^2 / D_par) and t1 = log(iterations) from those
 * features and log dt[k] (host array); the library sets
 *   alpha_k = -margin * exp(t0) * D_par / dx^2   (dx = min(dx, dy), margin >= 1)
 * as the operator's bound (c and gamma follow) and returns alpha_k in
 * alpha_out and exp(t1) in iters_out (host arrays of nops, either may be
 * NULL).  One batched inference for all operators, BF16 kernels when
 * bf16 != 0.  AD_ERR_INVALID when a prediction is not a finite negative
 * bound (no operator is changed then).  The model's activation workspace
 * grows to the largest batch it has seen (an allocation on first use). */
AD_API int ad_learned_bounds(ad_mlp* m, ad_operator* const* ops, int nops, const double* dt,
                             double margin, int bf16, double* alpha_out, double* iters_out);
/* Attach a bound model (or detach with m == NULL) for ad_spectral_bound's
 * AD_BOUND_LEARNED method, with its margin (>= 1) and the step dt it predicts
 * for.  The model must outlive the attachment. */
AD_API int ad_set_bound_model(ad_operator* op, ad_mlp* m, double margin, double dt);
/* One training sample of the bound model from an AD_FP64 operator: the 21
 * inputs (its recorded features and log dt) into x21, and the targets into
 * t2: t0 = log(est dx^2 / D_par) with est the power-iteration estimate of
 * |lambda|max (power_iters steps from the SplitMix64 vector of seed + 1),
 * t1 = log(max(1, m)) with m the Leja iterations of phi_1(dt A) v at tol
 * for the SplitMix64 vector v of seed, with alpha = -safety * est (the
 * operator keeps that bound).  *power_estimate (may be NULL) receives est. */
AD_API int ad_bound_training_sample(ad_operator* op, double dt, unsigned long long seed,
                                    int power_iters, double safety, double tol, float* x21,
                                    float* t2, double* power_estimate);

/* The 21 input features of one field: log max lambda_1(D), log min lambda_2(D),
 * log(max|a| + 1e-6), log min(dx, dy), log dt, and the anisotropy-weighted
 * 16-bin histogram of the principal direction of D over (-pi/2, pi/2]
 * (normalised).  Dxx, Dxy, Dyy: float64 device fields; out21: host. */
AD_API int ad_field_features(const ad_grid* grid, const double* Dxx, const double* Dxy,
                             const double* Dyy, double max_a, double dt, void* cuda_stream,
                             float* out21);

/* Penalised IMEX step: the alternative to the exponential method that
 * Section 4 names (penalise the anisotropic diffusion by an isotropic
 * operator treated implicitly, the rest explicitly).  The paper gives no
 * formula; this is the first-order IMEX Euler step
 *   (I - dt beta L)(u+ - u) = dt (A u + S(t)),
 * L = the operator of Eq. anidiff for D = I, a = 0 (the 5-point Laplacian of
 * the same flux form and boundary rule), solved by conjugate gradients to a
 * relative residual cg_tol (at most max_cg iterations; the CG scalars stay on
 * the device, the host reads the residual every 8 iterations).  The scheme is
 * stable for beta >= lambda_max(D) / 2; ad_penalty_beta gives max lambda_max(D).
 * beta = 0 is the explicit Euler step.  AD_FP64 operators only.  On
 * AD_ERR_NOT_CONVERGED u is left unchanged.  Stats: iters = CG iterations,
 * err_est = final relative residual. */
AD_API int ad_penalised_step(ad_operator* op, void* u, double t, double dt, const ad_source* src,
                             double beta, double cg_tol, int max_cg, ad_stats* stats);
/* max over cells of the largest eigenvalue of D (device float64 fields). */
AD_API int ad_penalty_beta(const ad_grid* grid, const double* Dxx, const double* Dxy,
                           const double* Dyy, void* cuda_stream, double* beta);

/* ---------------------------------------------------------------------
 * Momentum coupling (Eq. cr_full, Section 1).  The paper integrates only the
 * two-dimensional Eq. anidiff and names the momentum terms of Eq. cr_full,
 *   d/dp(p^2 D_pp d/dp(u/p^2)) - d/dp((pdot - (p/3) div v) u) - (1/tau_f + 1/tau_r) u,
 * as future work.  This operator adds them on np momentum cells:
 *   - faces P[0] < ... < P[np] (> 0), centres p_k = sqrt(P[k] P[k+1]);
 *   - D(x, y, p_k) = beta[k] D(x, y); the constant advection (ax, ay) does not
 *     depend on p;
 *   - dpp[f], b[f] = D_pp and pdot - (p/3) div v at face f (f = 0..np; the
 *     two outer values are unused: no flux leaves the momentum range);
 *     loss[k] = 1/tau_f + 1/tau_r of cell k;
 *   - finite volumes in p: the diffusion flux
 *     P_f^2 D_pp (u_{k+1}/p_{k+1}^2 - u_k/p_k^2)/(p_{k+1} - p_k), the advective
 *     flux b u taken from the upwind cell.
 * Vectors are float64, device memory, slice-major: u[k * nx * ny + j * nx + i]
 * (each momentum slice is one field in the layout of ad_create_operator).
 * All arrays of ad_momentum are host memory. */
typedef struct {
  int np;                    /* momentum cells, 1..1024 */
  const double* P;           /* np + 1 increasing positive faces */
  const double* beta;        /* np scales of the spatial diffusion (>= 0) */
  const double* dpp;         /* np + 1 face values of D_pp (>= 0) */
  const double* b;           /* np + 1 face values of pdot - (p/3) div v */
  const double* loss;        /* np loss rates */
} ad_momentum;

typedef struct ad_momentum_operator ad_momentum_operator;

/* Build the coupled operator (FP64).  Dxx, Dxy, Dyy: device float64 fields
 * [ny][nx] of the spatial tensor (scaled by beta[k] in slice k).  The
 * Gershgorin bound of the coupled matrix is computed here (Section 2).
 * Errors: AD_ERR_INVALID (NULL, bad sizes, non-increasing faces, negative
 * D_pp or beta, nx * ny * np >= 2^31), AD_ERR_NOMEM, AD_ERR_CUDA. */
AD_API int ad_create_momentum_operator(const ad_grid* grid, const ad_momentum* mom,
                                       const double* Dxx, const double* Dxy, const double* Dyy,
                                       double ax, double ay, void* cuda_stream,
                                       ad_momentum_operator** out);
AD_API int ad_destroy_momentum_operator(ad_momentum_operator* op);
/* The spectral bound alpha in use (Gershgorin unless set). */
AD_API int ad_momentum_spectral_bound(const ad_momentum_operator* op, double* alpha);
AD_API int ad_momentum_set_spectral_bound(ad_momentum_operator* op, double alpha);
/* rho_max and max_iters as in ad_set_options (fixed substep rule). */
AD_API int ad_momentum_set_options(ad_momentum_operator* op, double rho_max, int max_iters);
/* Au = A u (device, non-aliasing). */
AD_API int ad_momentum_apply(ad_momentum_operator* op, const double* u, double* Au);
/* out = phi_1(dt A) v by the Leja series of Section 2, with the stopping
 * rule, cap and substeps of ad_leja_phi1.  v, out: device (may alias). */
AD_API int ad_momentum_leja_phi1(ad_momentum_operator* op, const double* v, double* out,
                                 double dt, double tol, int force_iters, ad_stats* stats);
/* u += dt phi_1(dt A)(A u + S): the exponential midpoint rule (Eq. exp_midpoint)
 * for a time-independent source S (device, or NULL), exact in time for it. */
AD_API int ad_momentum_step(ad_momentum_operator* op, double* u, double dt, const double* S,
                            double tol, int force_iters, ad_stats* stats);

/* Measurement helper (no counterpart in the paper): time the fused Leja
 * iteration kernel alone.  Runs a forced series of `reps` iterations (aug =
 * 0: phi_1 form, 1: augmented form) on the operator's stream and returns the
 * mean device time of one iteration in *ms_per_launch: on the persistent FP64
 * path (one cooperative launch per series) the launch time / reps; on the
 * FP32 two-iteration kernel (phi_1 form, nx % 4 == 0, ny >= 2, no varying
 * advection) the mean of CUDA event pairs around each launch / 2 (an odd
 * reps runs one more iteration); otherwise the mean of CUDA event pairs
 * around each iteration kernel.  Overwrites the
 * operator's series workspace; results of earlier calls are unaffected.
 * 1 <= reps <= 500. */
AD_API int ad_profile_leja_iteration(ad_operator* op, int aug, int reps, double* ms_per_launch);

/* Measurement helper (no counterpart in the paper): device time of the Newton
 * series inside real calls.  enable != 0 resets the totals and from then on
 * records a CUDA event pair on the operator's stream around the iteration
 * kernels of every series the operator runs (the cooperative launch, the
 * graph launch or the host-driven launches; substeps and both series of a
 * step count separately); enable == 0 stops recording.  ad_series_timing
 * returns the totals since the last enable: milliseconds, number of series
 * and their total Leja iterations, and (kernel may be NULL) the path of the
 * last timed series: 1 persistent kernel with a grid barrier per iteration,
 * 2 persistent kernel with neighbour synchronisation (row ranges), 7 the same
 * on 2-D tiles, 3 graph loop of
 * per-iteration kernels, 4 host-driven per-iteration launches, 5 and 6 the
 * same with the FP32 two-iteration kernel, 8 and 9 the same with its rows
 * brought in by TMA, 10 the FP64 series of a small grid in one thread-block
 * cluster, 0 none yet.
 * Recording adds two event records and no synchronisation (each series
 * already ends with one). */
AD_API int ad_time_series(ad_operator* op, int enable);
AD_API int ad_series_timing(const ad_operator* op, double* ms, int* series, long long* iters,
                            int* kernel);

/* out = phi_1(dt A) v without allocating any device memory.  The paper has
 * no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc (code inside a host framework that owns the device heap, code
 * under a no-allocation-after-start-up rule, or paths where an allocation's
 * implicit synchronisation is not acceptable) and therefore cannot create an
 * operator.  It runs the same kernels as ad_create_operator + ad_leja_phi1,
 * with all scratch (packed weights, Newton vectors, partial sum, Leja
 * scalars, control block, norm partials) in one fixed file-scope device array
 * of about 6.4 MB that every GPU loading the library holds until exit.
 *   grid, Dxx, Dxy, Dyy : as in ad_create_operator (device fields, FP64);
 *   ax_c, ay_c          : constant advection;
 *   alpha               : spectral bound (< 0), or 0 to compute it by Gershgorin
 *                         (AD_ERR_INVALID if that bound is not negative, as in
 *                         ad_spectral_bound);
 *   v, out              : float64 DEVICE vectors [ny][nx] (may alias);
 *   dt, tol, force_iters: as in ad_leja_phi1; one substep only.
 * Limits: at most 65536 cells and gamma*dt <= 200 (AD_ERR_INVALID with a
 * message otherwise).  Every call shares the scratch and it keeps the last
 * call's contents; calls that overlap on the GPU race and must be serialised
 * by the caller.  Every call looks up the scratch's device address on the
 * current device (no saved address can go stale); the first call on a device
 * may load the module, so make it before any stream capture.  Synchronises the
 * stream before returning. */
AD_API int ad_leja_phi1_noalloc(const ad_grid* grid, const double* Dxx, const double* Dxy,
                                const double* Dyy, double ax_c, double ay_c, double alpha,
                                const double* v, double* out, double dt, double tol,
                                int force_iters, void* cuda_stream, ad_stats* stats);

/* Measurement helper (no counterpart in the paper): the FP64 FMA rate this
 * device sustains, in TFLOP/s (2 flops per FMA), from one timed launch (after
 * one untimed) of blocks_per_sm (1..8) blocks of 256 threads per SM, each
 * thread running four independent fused multiply-add chains of iters steps
 * (1024..2^24).  The FP64 kernels of this library are bound by this rate;
 * it is reported beside the nominal peak of their roofline. */
AD_API int ad_fp64_fma_rate(int blocks_per_sm, int iters, void* cuda_stream, double* tflops);

/* Failure-detection check (no counterpart in the paper): one block waits on a
 * device barrier that nothing releases, with the library's bounded-wait
 * machinery and a bound of timeout_ms (0 < timeout_ms <= 1000).  Returns
 * AD_ERR_TIMEOUT when the wait gives up as designed; the CUDA context stays
 * usable.  Any other status means the bounded-wait path is broken. */
AD_API int ad_check_wait_timeout(double timeout_ms, void* cuda_stream);

/* Thread-local message for the last error of this thread ("" if none). */
AD_API const char* ad_last_error(void);

/* Library ABI version (major * 10000 + minor * 100 + patch). */
AD_API int ad_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ANIDIFF_H */
