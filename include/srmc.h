/*
 * srmc.h -- C ABI of libsrmc, a GB300 (sm_103a) implementation of the
 * stratified regression Monte Carlo scheme (SRMDP) for discrete-time BSDEs
 * and semilinear parabolic PDEs (Gobet, Lopez-Salas, Turkedjiev, Vazquez).
 *
 * Problem solved (Sec. 1, eqs. fbsde/eds/pde; Sec. 2, eq. MDP): the
 * multistep-forward dynamic programming equation on the grid t_i = i T/N,
 *     Y_i    = E_i[ g(X_N) + sum_{j=i}^{N-1} f_j(X_j, Y_{j+1}, Z_j) dt ],
 *     dt Z_i = E_i[ (g(X_N) + sum_{j=i+1}^{N-1} f_j(X_j, Y_{j+1}, Z_j) dt) dW_i ],
 * with X the Euler chain X_{j+1} = X_j + b(X_j) dt + sigma dW_j (Alg. 2) or the
 * SDE itself (Alg. 1, affine drift), approximated by Alg. SRMDP: for every time
 * step i = N-1..0 and every hypercube stratum H_k, draw M fresh paths started
 * from the restricted logistic law nu_k (assumption A_nu, Alg. 3), simulate
 * them to t_N, and fit the Z-response then the Y-response by least squares on
 * LP0 (constants), LP1 (affine functions) or LP2 (quadratics) local to H_k
 * (eq. PsiM; Sec. 4.1), truncating the fitted values (eq. TL).
 *
 * Conventions for every call:
 *   - Host arrays passed in are read during the call and copied; the caller
 *     keeps ownership.
 *   - "dev" pointers are device memory of the current CUDA device, owned by
 *     the caller; the library never frees them and never keeps them after
 *     the call returns (work on them is enqueued on the given stream).
 *   - "stream" is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Compute calls are asynchronous on that stream.
 *   - Errors come back as an srmc_status; srmc_last_error() gives a message
 *     for the calling thread.  No C++ exception crosses this ABI.
 *   - Random numbers: Philox-4x32-10 (Salmon et al., SC'11) with
 *     key = (seed_lo ^ instance, seed_hi) and counter = (n/4, m, k, i) for word
 *     n of path m of cloud C_{i,k}; words 0..d-1 draw the start point,
 *     words d + (j-i) q + l the normal of component l of dW_j (the exact
 *     dynamics draw two blocks per step, see srmc_problem).  Uniforms are
 *     U = (w + 1/2) 2^-32 and normals Phi^{-1}(U).  Nothing is stored: a path
 *     is regenerated from its counter whenever it is needed.
 */
#ifndef SRMC_H
#define SRMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SRMC_DMAX 19    /* largest dimension d supported                    */
#define SRMC_PMAX 24    /* length of the model parameter array             */

typedef enum {
    SRMC_OK = 0,
    SRMC_ERR_INVALID_ARG = 1,   /* a size, pointer or parameter is out of range */
    SRMC_ERR_CUDA = 2,          /* a CUDA runtime call failed                   */
    SRMC_ERR_OOM = 3,           /* device allocation failed                     */
    SRMC_ERR_UNSUPPORTED = 4,   /* valid input outside what this build supports */
    SRMC_ERR_STATE = 5          /* call out of order (e.g. step i before i+1)   */
} srmc_status;

/* Local polynomials (Sec. 2, assumption HS examples; Sec. 4.1): LP0 constants,
 * LP1 affine functions, LP2 quadratics [1, u_l, u_a u_b (a <= b)] in the
 * centred coordinates u (higher order than the paper's experiments, which it
 * notes is possible; built for d <= 3, equal-size strata and Euler dynamics). */
typedef enum { SRMC_LP0 = 0, SRMC_LP1 = 1, SRMC_LP2 = 2 } srmc_basis;
typedef enum { SRMC_FP32 = 0, SRMC_FP64 = 1 } srmc_precision;

/* Built-in driver/terminal families.  params[] layouts:
 *   SRMC_MODEL_COS:      {lam, kap, kapz, s0};  g(x) = cos(s), s = sum_l x_l / sqrt(d),
 *                        f_j(x,y,z) = (lam + s0^2/2) y + kap (y^2 - u(t_j,x)^2)
 *                                     + kapz (|z|^2 - s0^2 e^{2 lam (T-t_j)} sin^2 s),
 *                                     - (1/s0) sum_l b_l(x) z_l,
 *                        u(t,x) = e^{lam (T-t)} cos(s) solves the PDE when sigma = s0 I
 *                        (the last term cancels the drift b(x).grad u; it vanishes
 *                        without drift).
 *   SRMC_MODEL_LOGISTIC: {} ; the test BSDE of Sec. 5.1: w = exp(t + sum x),
 *                        g = w(T,x)/(1+w(T,x)), f = (sum_l z_l)(y - (2+q)/(2q)).
 *   SRMC_MODEL_AFFINE:   {g0, g_1..g_d, f0, f_1..f_d, a}; g = g0 + g.x,
 *                        f_j(x,y,z) = f0 + f.x + a y.
 *   SRMC_MODEL_USER:     g and f given as source (srmc_problem.user_source),
 *                        params passed to them; compiled at srmc_create for the
 *                        solver's device by NVRTC (see srmc_problem). */
typedef enum { SRMC_MODEL_COS = 0, SRMC_MODEL_LOGISTIC = 1, SRMC_MODEL_AFFINE = 2,
               SRMC_MODEL_USER = 3 } srmc_model;

/* Forward SDE, driver, terminal condition and time grid (Sec. 1-2).
 * Drift b_l(x) = b_l - theta_l x_l (theta = 0: constant drift; theta > 0:
 * Ornstein-Uhlenbeck, mean reverting to b_l/theta_l).  b: [d] (host).
 * theta: [d] (host) or NULL for 0.  sigma: [d*q] row-major constant diffusion
 * (host, finite), q the number of Brownian components (1 <= q <= 19).  A
 * diagonal d x d sigma moves each coordinate by its own increment; any other
 * (an off-diagonal sigma_lr != 0: correlated coordinates, or q != d: the general
 * constant diffusion of Sec. 1) is built for d <= 8 (d, q <= 4 when q != d) with
 * Euler dynamics, equal-size strata, LP0/LP1 and the built-in models, without a
 * drift in the cos model when q != d (else SRMC_ERR_UNSUPPORTED), and takes
 * X_{j+1,l} = X_{j,l} + b_l(X_j) dt + sum_r sigma_lr dW_{j,r}; z and the Z fits
 * then have q components.  The closed-form error metrics, the batched form and
 * (for q != d) the network tabulation do not take it.
 * params: [n_params <= SRMC_PMAX] (host).
 * dynamics: how X moves between grid times (assumption HX):
 *   SRMC_DYN_EULER (Alg. 2): X_{j+1} = X_j + b(X_j) dt + sigma dW_j;
 *   SRMC_DYN_EXACT (Alg. 1): the SDE itself, X_{j+1,l} = X_{j,l} e^{-theta_l dt}
 *     + b_l B_l + sigma_l I_l with B_l = (1 - e^{-theta_l dt})/theta_l and
 *     I_l = int e^{-theta_l (t_{j+1} - s)} dW_s, drawn jointly with dW_j: given
 *     dW_j, I_l = (B_l/dt) dW_{j,l} + r_l xi_l with r_l^2 = Var I_l - B_l^2/dt,
 *     xi a second standard normal per coordinate and step (draws d + 2(j-i)q + q
 *     + l; dW_j takes d + 2(j-i)q + l).  Equal-size strata only; identical to
 *     Euler when theta = 0 up to the draw layout.
 * user_source (SRMC_MODEL_USER only, else ignored): C source defining
 *     SRMC_USER srmc_real srmc_user_g(const srmc_real *x, int d, const double *prm);
 *     SRMC_USER srmc_real srmc_user_f(srmc_real t, const srmc_real *x, srmc_real y,
 *                                     const srmc_real *z, int d, const double *prm);
 *   (g(x) and f(t_j, x, y, z) of eq. MDP; prm = params); with user_dynamics
 *   != 0 also
 *     SRMC_USER srmc_real srmc_user_b(srmc_real t, const srmc_real *x, int l, int d,
 *                                     const double *prm);
 *     SRMC_USER srmc_real srmc_user_sigma(srmc_real t, const srmc_real *x, int l, int d,
 *                                         const double *prm);
 *   the drift b_l(t, x) and diagonal diffusion sigma_l(t, x) (assumption HX), taken
 *   by the Euler step X_{j+1,l} = X_{j,l} + b_l(t_j, X_j) dt + sigma_l(t_j, X_j) dW_{j,l}
 *   (Alg. 2; b, theta and sigma of the problem are then unused).  The library
 *   prepends the typedef of srmc_real (float for the FP32 form, double for
 *   FP64) and the SRMC_USER qualifiers, compiles it with its step kernel
 *   (NVRTC, the toolkit headers from SRMC_CUDA_INCLUDE or the build's CUDA
 *   include directory) and reports compiler messages through
 *   srmc_last_error (SRMC_ERR_INVALID_ARG).  The source is copied.  User
 *   models: LP0/LP1, equal-size strata, Euler dynamics; no closed-form
 *   metrics, no srmc_eval at i == N, no batched form. */
typedef enum { SRMC_DYN_EULER = 0, SRMC_DYN_EXACT = 1 } srmc_dynamics;
typedef struct {
    int d, q;
    int N;
    double T;
    const double *b;
    const double *sigma;
    srmc_model model;
    const double *params;
    int n_params;
    const double *theta;
    int dynamics;              /* srmc_dynamics */
    const char *user_source;
    int user_dynamics;         /* user model also supplies b and sigma (see above) */
} srmc_problem;

/* Strata (assumption HS): cells[l] half-open cells per dimension, stratum
 * index k = sum_l c_l prod_{l'<l} cells[l'] (dimension 0 fastest).
 *   kind SRMC_STRATA_EQUAL_SIZE (HS, example i): the box [lo_l, hi_l) cut
 *     into equal cells, the first and last cell of every dimension extended
 *     to -inf / +inf; x is in cell c_l = clamp(floor((x_l - lo_l) / h_l), 0,
 *     cells[l]-1), h_l = (hi_l - lo_l)/cells[l], in FP64 (single-precision
 *     paths take the same decision as floor((x_l - lo_l) * r_l), r_l =
 *     cells[l] / (hi_l - lo_l) rounded to float).  Basis centre: the centre of
 *     the nominal cell; basis unit h_l / 2.
 *   kind SRMC_STRATA_EQUAL_PROB (HS, example ii): nu(H_k) = 1/K; the axis is
 *     cut at the logistic quantiles e_c = log(c / (C - c)) / mu, c = 1..C-1
 *     (C = cells[l]), x is in the cell c with e_c <= x < e_{c+1} (the edges
 *     held in double, or rounded to float for single-precision paths).  Basis
 *     centre: the median of nu restricted to the cell, F^{-1}((c + 1/2)/C);
 *     basis unit: F^{-1}((c + 3/4)/C) - F^{-1}((c + 1/4)/C).  lo, hi unused
 *     (may be NULL).
 * The centred LP1 basis of a stratum is phi = [1, (x_l - centre_l) / unit_l].
 * mu: scale of the logistic law nu (eq. logistic).  Arrays host, [d]. */
typedef enum { SRMC_STRATA_EQUAL_SIZE = 0, SRMC_STRATA_EQUAL_PROB = 1 } srmc_strata_kind;
typedef struct {
    const int *cells;
    const double *lo, *hi;
    double mu;
    int kind;                  /* srmc_strata_kind */
} srmc_strata;

/* Scheme configuration.  M: paths per stratum and step, M >= dim of the basis
 * (Def. of the clouds).  M_strata: NULL, or a host array [K] of per-stratum
 * path counts M_k (each >= dim of the basis and < 2^32; copied) that
 * replaces M -- the paper fixes M for all strata to balance the work and
 * notes that the analysis adapts to M_k (Sec. 3, after Alg. SRMDP).  Cy, Cz:
 * truncation levels of y and of each component of z (eq. TL, Prop. a.s.
 * bounds); a value <= 0 disables that truncation.  block_threads: threads per
 * stratum block, a multiple of 32 in [32, 256], or 0 for the library's
 * choice. */
typedef struct {
    srmc_basis basis;
    srmc_precision prec;
    long long M;
    unsigned long long seed;
    unsigned instance;
    double Cy, Cz;
    int block_threads;
    const long long *M_strata;
} srmc_config;

typedef struct srmc_solver srmc_solver;   /* opaque, library-owned */

/* Validate the problem and allocate the solver's device tables on the
 * current device: coefficient rows of every (i, k), i < N, in FP64 (and FP32
 * for the FP32 form), zero-filled.  1 <= d <= SRMC_DMAX (19, the largest
 * dimension of the paper's Sec. 5.2); d = 9..19 is built for equal-size
 * strata, Euler dynamics and the FP32 form, without controls, and user
 * models for d <= 11 (SRMC_ERR_UNSUPPORTED otherwise).  Errors: SRMC_ERR_INVALID_ARG, SRMC_ERR_UNSUPPORTED,
 * SRMC_ERR_OOM, SRMC_ERR_CUDA; *out is NULL on error. */
srmc_status srmc_create(const srmc_problem *problem, const srmc_strata *strata,
                        const srmc_config *config, srmc_solver **out);

/* Release everything the solver owns.  NULL is accepted. */
void srmc_destroy(srmc_solver *s);

/* The whole backward recursion of Alg. SRMDP, i = N-1 .. 0, enqueued on
 * stream: per step one launch over all strata (Z fit, then Y fit).  The N
 * launches are captured once into a CUDA graph (on a private stream, at the
 * first call) and replayed on `stream` by every call.  Asynchronous; results
 * are valid once the stream has reached this point. */
srmc_status srmc_solve(srmc_solver *s, void *stream);

/* One step i of Alg. SRMDP for all strata.  Requires the rows of steps
 * i+1..N-1 (enqueued earlier on the same stream); SRMC_ERR_STATE otherwise. */
srmc_status srmc_solve_step(srmc_solver *s, int i, void *stream);

/* Truncated y_i(x) and z_i(x) (Alg. SRMDP, the fitted functions restricted to
 * the stratum holding x) at n points.  dev_x: [n][d] double; dev_y: [n]
 * double; dev_z: [n][q] double (may be NULL).  i == N gives y = g, z = 0.
 * n == 0 is a no-op. */
srmc_status srmc_eval(const srmc_solver *s, int i, const double *dev_x, long long n,
                      double *dev_y, double *dev_z, void *stream);

/* The K stratum basis centres (the centre of the nominal finite cell, or
 * the median of nu restricted to the cell, in every dimension), written to
 * dev_x: [K][d] double. */
srmc_status srmc_centres(const srmc_solver *s, double *dev_x, void *stream);

/* Layout of the FP64 coefficient table: row (i,k) holds alpha[p] then
 * beta[q][p] in the centred basis phi(x) = [1, (x - c_k)/s_k], p = 1 (LP0)
 * or d+1 (LP1), c_k and s_k the basis centre and unit of the stratum (see
 * srmc_strata: h/2 and the nominal cell centre for equal-size cells);
 * y_i(x) = T_Cy(alpha . phi(x)).
 * *dev_y64 / *dev_z64 are borrowed pointers to [N][K][ry] and [N][K][rz]
 * doubles, valid until srmc_destroy. */
srmc_status srmc_table(const srmc_solver *s, const double **dev_y64, const double **dev_z64,
                       int *p, int *ry, int *rz, long long *K);

/* Copy the FP64 coefficient tables (layout of srmc_table, all N*K rows) into
 * caller memory: dst_y [N][K][ry] and dst_z [N][K][rz] doubles, host (pinned
 * or pageable) or device; either may be NULL.  Asynchronous on stream for
 * device or pinned destinations; the caller synchronises before reading. */
srmc_status srmc_read_table(const srmc_solver *s, double *dst_y, double *dst_z, void *stream);

/* Install the fitted rows of step i of every stratum (Alg. SRMDP: the
 * functions y_i, z_i that the fits of the steps before i read), in place of
 * the solver's own: src_y [K][ry] and src_z [K][rz] doubles in the layout of
 * srmc_table (centred basis; e.g. the step-i slice of another solver's tables
 * on the same strata and basis), caller-owned, device or host (pinned or
 * pageable).  The FP32 form's copies of the rows are refreshed (round to
 * nearest).  Steps count as present from the last one down: installing step i
 * when steps i+1..N-1 are present (solved or installed; none for i = N-1)
 * makes steps i..N-1 present, after which srmc_solve_step(i - 1) may follow
 * and fits step i-1 from the given functions (teacher forcing).  Asynchronous
 * on stream; SRMC_ERR_INVALID_ARG for a NULL argument or i outside [0, N). */
srmc_status srmc_set_rows(srmc_solver *s, int i, const double *src_y, const double *src_z, void *stream);

/* Martingale control variate (an extension of Alg. SRMDP, not in the
 * paper): with rows beta_{j,k} installed, every response of cloud C_{i,k}
 * loses the control built from zc_j(x) = T_Cz(beta_{j,k} . phi(x)), x in H_k:
 * the Y response loses sum_{j>=i} zc_j(X_j).dW_j and the Z response
 * sum_{j>i} zc_j(X_j).dW_j.  Both terms have zero conditional mean given
 * x_i (dW_j is independent of everything known at t_j), so the fitted
 * functions keep their expectation while the response variance drops when
 * zc approximates the true z = sigma^T grad u.  rows: [N][K][q][p] doubles,
 * host or device memory, centred basis phi = [1, (x - c_k)/s_k]; copied
 * (synchronously).  LP1 solvers only (SRMC_ERR_UNSUPPORTED otherwise).
 * The FP64 form uses the rows as given.  The FP32 form keeps them in
 * binary16 (round to nearest even, magnitudes above 65504 saturated, below
 * 2^-14 with reduced relative precision) and evaluates zc in FP32: its
 * control is the function of the rounded rows, still free of dW_j, so the
 * expectation argument above holds unchanged; only the variance reduction
 * depends on the rounding (relative 2^-11 in the coefficients).
 * srmc_read_control returns the rows as given (FP64). */
srmc_status srmc_set_control(srmc_solver *s, const double *rows);

/* The run's own martingale control (an extension of Alg. SRMDP, not in the
 * paper): both responses of cloud C_{i,k} lose sum_{j>i} z_j(X_j).dW_j, z_j
 * the truncated z fit of step j in the stratum holding X_j -- the function
 * the path already looks up when the driver depends on z.  Each z_j is fitted
 * from clouds drawn independently of C_{i,k} before step i is solved, so the
 * term has zero conditional mean given x_i (independence of the clouds, the
 * definition of the simulations in Sec. 4) and the fitted functions keep their
 * expectation.  There is no step-i term (z_i is fitted from the same cloud).
 * No rows are stored: the control costs one z-row gather per path-step where
 * the driver does not already need it.  Replaces any installed rows;
 * srmc_read_control then fails with SRMC_ERR_STATE.  LP1 solvers, not the
 * affine model (SRMC_ERR_UNSUPPORTED otherwise). */
srmc_status srmc_set_own_control(srmc_solver *s);

/* Remove the control variate (the plain scheme again). */
srmc_status srmc_clear_control(srmc_solver *s);

/* Copy the installed control rows ([N][K][q][p] doubles) into caller memory
 * (host or device); SRMC_ERR_STATE if no control is installed. */
srmc_status srmc_read_control(const srmc_solver *s, double *rows);

/* ---- learned control variate: a small MLP u_theta(t, x) -------------------
 * (an extension of the paper's scheme).  Architecture: a = (t, x_1..x_d)
 * (n_in = d + 1 <= 15) -> 64 -> 64 -> 1 with SiLU activations.  Parameters
 * (FP32 master copy, float vector): W1 [64][n_in], b1 [64], W2 [64][64],
 * b2 [64], w3 [64], b3.  The kernels run the two 64-wide layers on BF16
 * tensor-core tiles with FP32 accumulation: inputs, W1, h1, W2 (and in the
 * backward passes g_z2, g_z1) are rounded to bfloat16, everything else is
 * FP32.  Training: mean squared error, Adam (beta1 0.9, beta2 0.999). */
typedef struct srmc_mlp srmc_mlp;   /* opaque, library-owned */

/* Create on the current device with seeded initial weights (uniform
 * +-sqrt(6/fan_in), biases 0).  hidden must be 64. */
srmc_status srmc_mlp_create(int n_in, int hidden, unsigned long long seed, srmc_mlp **out);
void srmc_mlp_destroy(srmc_mlp *m);
int srmc_mlp_nparams(const srmc_mlp *m);
/* Parameter vector in/out (host or device pointer, float[nparams]); copied. */
srmc_status srmc_mlp_set_params(srmc_mlp *m, const float *params);
srmc_status srmc_mlp_get_params(const srmc_mlp *m, float *params);
/* u(a) and the input gradient du/da at n points: dev_a [n][n_in] float,
 * dev_u [n], dev_grad [n][n_in] (may be NULL). */
srmc_status srmc_mlp_eval(const srmc_mlp *m, const float *dev_a, long long n, float *dev_u,
                          float *dev_grad, void *stream);
/* Gradient of the loss (1/n) sum (u(a_s) - y_s)^2 with respect to the
 * parameters into dev_grad [nparams] and the loss into dev_loss [1]. */
srmc_status srmc_mlp_loss_grad(srmc_mlp *m, const float *dev_a, const float *dev_y, long long n,
                               float *dev_grad, float *dev_loss, void *stream);
/* Train on n_data points drawn from a finished (coarse) solve: steps i and
 * strata k uniform, x ~ nu_k, a = (t_i, x), target y_i(x) from its FP64 table.
 * iters Adam steps on consecutive batches (lr decays geometrically to lr/10).
 * dev_loss_curve [iters] (may be NULL) receives the batch losses.
 * n_data must be a multiple of batch and at most 2^40. */
srmc_status srmc_mlp_fit(srmc_mlp *m, const srmc_solver *coarse, long long n_data, int iters,
                         int batch, float lr, unsigned long long seed, float *dev_loss_curve,
                         void *stream);
/* Allocation-free twin of srmc_mlp_fit (no counterpart in the paper; an
 * engineering entry point).  Some callers cannot allocate device memory
 * while they train: code that runs under a fixed, pre-reserved memory
 * budget, code whose device memory is owned by another allocator (a
 * framework's caching pool), and latency-critical loops that must not pay
 * the implicit device synchronisation of cudaFree.  This call does the same
 * work as srmc_mlp_fit with the same arguments, but keeps the training
 * points, their targets and the gradient accumulator in one scratch array
 * compiled into the library (static device memory: every GPU that loads the
 * library holds it until the process exits) instead of allocating them:
 *   - limit: n_data * (n_in + 1) + nparams + 64 <= 2^21 floats (8 MiB);
 *     larger requests fail with SRMC_ERR_INVALID_ARG and a message;
 *   - the network's device must be the current device (else
 *     SRMC_ERR_INVALID_ARG); the first call on a device looks the array up
 *     on that device and keeps its address for the life of the process, so
 *     make that first call before any stream capture; a cudaDeviceReset (or
 *     anything else that tears down the device's primary context) leaves the
 *     kept address stale: do not call this entry point after one;
 *   - every call on a device shares the one array, so calls whose work
 *     overlaps on the GPU (different streams or threads) race; serialise
 *     them.  The parts that must start at zero are cleared by each call.
 * It calls no cudaMalloc, cudaFree or allocating library routine.  Unlike
 * srmc_mlp_fit it does not synchronise: the work is enqueued on stream. */
srmc_status srmc_mlp_fit_noalloc(srmc_mlp *m, const srmc_solver *coarse, long long n_data,
                                 int iters, int batch, float lr, unsigned long long seed,
                                 float *dev_loss_curve, void *stream);

/* Tabulate zc = sigma^T grad_x u_theta(t_j, .) as the control rows of s for
 * every (j, k): value at the stratum's basis centre and central differences
 * at +- half a basis unit along each axis (h/4 for equal-size cells; LP1 rows
 * in the centred basis), then install them as by srmc_set_control.  LP1
 * solvers with d <= 7, n_in == d + 1. */
srmc_status srmc_cv_tabulate(const srmc_mlp *m, srmc_solver *s, void *stream);

/* ---- batched form: many independent instances in one launch sequence -------
 * (an engineering extension; the paper solves one problem at a time).  The
 * instances may differ in d, strata, N, M and model parameters.  Their
 * backward loops are aligned at the end: in round s every instance with
 * N_r > s solves its step i = N_r - 1 - s, and all (instance, stratum) work
 * items of a round that share a kernel variant go to one launch over a
 * persistent grid (blocks stride through the items).  The rounds are captured
 * once into a CUDA graph and replayed.  FP32 solvers with equal-size strata
 * only (SRMC_ERR_UNSUPPORTED otherwise). */
typedef struct srmc_batch srmc_batch;   /* opaque, library-owned */

/* Plan a batch over n solvers (borrowed: they must outlive the batch and stay
 * on the current device). */
srmc_status srmc_batch_create(srmc_solver *const *solvers, int n, srmc_batch **out);
void srmc_batch_destroy(srmc_batch *b);
/* Pick, for every kernel variant of the batch, the threads per stratum block
 * (64, 128 or 256: 2, 4 or 8 warps per stratum) and the blocks per SM of the
 * persistent grid by timing candidate launches of its first rounds on stream,
 * give every solver of the group that block size, then time the three strategies
 * (see srmc_batch_mode) on the whole batch and keep the fastest (the tables of
 * the solvers are overwritten; solve afterwards).  Optional: an untuned batch
 * uses 256 threads, the occupancy limit and the rounds strategy.  out_threads
 * (may be NULL) receives the chosen threads per variant group, in group order,
 * up to max_out entries; returns the number of groups in *n_groups. */
srmc_status srmc_batch_tune(srmc_batch *b, void *stream, int *out_threads, int max_out, int *n_groups);
/* All instances' backward loops, enqueued on stream (graph replay). */
srmc_status srmc_batch_solve(srmc_batch *b, void *stream);

/* Strategy in use: 0 = rounds of multi-instance launches, 1 = one graph
 * branch per instance (concurrent single-instance launches), 2 = one
 * persistent launch per kernel variant over all rounds: blocks take
 * (instance, step, stratum) items in round order from a device counter and
 * each item waits only for the previous step of its own instance (bounded
 * waits; see srmc_batch_stats).  An untuned batch uses 0; srmc_batch_tune
 * keeps the fastest. */
int srmc_batch_mode(const srmc_batch *b);

/* Force a strategy (0, 1 or 2; SRMC_ERR_INVALID_ARG otherwise). */
srmc_status srmc_batch_set_mode(srmc_batch *b, int mode);

/* The device time in ms of one whole-batch solve by each strategy (0, 1, 2)
 * as measured by the last srmc_batch_tune (-1 before any tuning). */
srmc_status srmc_batch_strategy_ms(const srmc_batch *b, float out_ms[3]);

/* Synchronise the device and report in *timeouts whether a wait of the
 * persistent strategy (2) ran past its iteration limit (about a second)
 * since the batch was created: then the tables of that solve are not valid.
 * 0 in normal operation. */
srmc_status srmc_batch_stats(srmc_batch *b, unsigned long long *timeouts);

/* Error of the fitted functions against the closed-form solution of the
 * model at the K stratum centres, for every step i = 0..N-1 (the metric of
 * the benchmark plan; Sec. 5.1 uses the same comparison at nu-distributed
 * points).  dev_out: [N][4] doubles: max_k |y_i - u|, mean_k (y_i - u)^2,
 * max_k max_l |z_i,l - z*_l|, mean_k |z_i - z*|^2.  Cos model: u = e^{lam(T-t)}
 * cos(s), z* = -s0 e^{lam(T-t)} sin(s) / sqrt(d) (sigma = s0 I); logistic model
 * (Sec. 5.1): u = w/(1+w), z*_l = w/(1+w)^2.  SRMC_ERR_UNSUPPORTED for the
 * affine model.  Requires a finished solve. */
srmc_status srmc_closed_form_error(const srmc_solver *s, double *dev_out, void *stream);

/* The same restricted to the inner strata (no cell of the stratum is a
 * semi-infinite outer cell), where the nominal centre lies in the stratum's
 * bulk; K_inner = prod_l (cells[l] - 2) must be > 0. */
srmc_status srmc_closed_form_error_inner(const srmc_solver *s, double *dev_out, void *stream);

/* Squared errors against the closed form at caller-given points, the
 * ingredients of the error indicators of Sec. 5.1 (eq. mse): dev_x
 * [N][n][d] doubles (device), n points per step i = 0..N-1 (in Sec. 5.1
 * drawn i.i.d. from nu, independently of the clouds); dev_out [N][2]
 * doubles (device): sum_a (y_i(x) - u(t_i, x))^2 and sum_a |z_i(x) - z*(t_i, x)|^2
 * over the n points of step i, with y_i, z_i the truncated fitted functions
 * of the stratum holding x and the closed forms of srmc_closed_form_error.
 * dev_out is overwritten (cleared on stream first).  Summation order across
 * blocks is not fixed (double atomics).  SRMC_ERR_UNSUPPORTED for the affine
 * model; requires a finished solve.  Asynchronous on stream. */
srmc_status srmc_point_error(const srmc_solver *s, const double *dev_x, long long n, double *dev_out,
                             void *stream);

/* Counters since creation: [0] strata fits that fell back from LP1 to LP0
 * because the Gram matrix was numerically singular (Cholesky pivot below
 * 1e-12 of its trace); [1] non-finite coefficients written; [2] stratum-path
 * steps simulated.  Synchronises the device. */
srmc_status srmc_stats(const srmc_solver *s, unsigned long long out[3]);

/* ---- the method's primitives, exposed for testing and reuse --------------- */

/* Philox-4x32-10 of n counters: dev_ctr [n][4] uint32, key[2] host, dev_out
 * [n][4]. */
srmc_status srmc_philox(const uint32_t *dev_ctr, const uint32_t key[2], long long n,
                        uint32_t *dev_out, void *stream);

/* Standard normals xi = Phi^{-1}((w + 1/2) 2^-32) of n words; FP64 into
 * dev_out64 and/or the single-precision form into dev_out32 (either NULL).
 * The single-precision form takes words 2t and 2t + 1 as a pair, as the FP32
 * step kernels do for the increments of a step, and an unpaired last word
 * alone; both ways give the same values. */
srmc_status srmc_normals(const uint32_t *dev_words, long long n, double *dev_out64,
                         float *dev_out32, void *stream);

/* Stratum index of n points: dev_x64 [n][d] double decided in FP64, or
 * dev_x32 [n][d] float decided in FP32 (exactly one non-NULL). */
srmc_status srmc_locate(const srmc_solver *s, const double *dev_x64, const float *dev_x32,
                        long long n, long long *dev_k, void *stream);

/* Start points (Alg. 3) of paths m0..m0+n-1 of cloud C_{i,k} in the solver's
 * precision, widened to double: dev_x [n][d]. */
srmc_status srmc_start_points(const srmc_solver *s, int i, long long k, long long m0,
                              long long n, double *dev_x, void *stream);

/* ---- measurement aid (not part of the method) ------------------------------ */

/* FP32 FMA throughput probe for the roofline of the path kernels: grid blocks
 * of `threads` threads each run iters rounds of 16 independent fused
 * multiply-adds, as 8 packed two-wide FFMA2 (packed != 0) or 16 scalar FFMA,
 * i.e. grid * threads * iters * 32 FLOP; dev_out [grid * threads] float
 * receives one value per thread.  threads a multiple of 32 in [32, 1024].
 * Asynchronous on stream; the caller times it. */
srmc_status srmc_fp32_fma_probe(int grid, int threads, int iters, int packed, float *dev_out,
                                void *stream);

/* Message of the last error on this thread ("" if none). */
const char *srmc_last_error(void);

/* ABI version of this header. */
int srmc_version(void);

#ifdef __cplusplus
}
#endif
#endif
