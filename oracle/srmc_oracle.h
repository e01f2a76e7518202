/*
 * srmc_oracle.h -- plain FP64 CPU oracle of the stratified regression Monte
 * Carlo scheme (SRMDP) for discrete BSDEs.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this code.  It
 * shares no header, helper, table or constant generator with the CUDA path
 * (paper_2407_21085_gb300/csrc); the two meet only through plain numbers
 * handed to both by the seeded workload definitions.
 *
 * What it computes, with the passage it follows:
 *   - time grid t_i = i*dt, dt = T/N                               (Sec. 2, eq. MDP)
 *   - Euler Markov chain X_{j+1} = X_j + b(X_j) dt + sigma dW_j     (Alg. 2, "Euler dynamics")
 *     with the affine drift b(x) = b - theta x, or the exact
 *     transition of that SDE (Ornstein-Uhlenbeck)                   (Alg. 1, "SDE dynamics")
 *   - equal-size hypercube strata, exterior cells infinite, or
 *     strata of equal nu-probability                                (assumption HS, i and ii)
 *   - logistic law nu, restricted law nu_k, inverse-CDF sampler     (assumption A_nu, Alg. 3)
 *   - fresh, independent clouds C_{i,k} of M paths                  (Def. "Simulations and empirical measures")
 *   - backward SRMDP recursion: Z-OLS then Y-OLS, truncation T_L    (Alg. SRMDP, eq. PsiM; eq. TL)
 *   - LP0 as the mean, LP1 by Householder QR of A=[1, x_i]          (Sec. 4.1, eqs. lp0/lp1 explicit)
 *     (LP2: A = [1, x_i, x_i,a x_i,b], the same QR)                  (Sec. 4, footnote on higher orders)
 *   - Philox-4x32-10 counter RNG from its published definition      (Salmon, Moraes, Dror, Shaw, SC'11)
 *   - standard normal by inversion, Phi^{-1}(U), one uniform each
 *   - martingale controls subtracted from the responses (tabulated rows or
 *     the run's own fitted z) and a small MLP with bf16 emulation: extensions
 *     of the method, not in the paper
 *
 * Parity pins of every function live in tests/test_oracle_*.py.
 */
#ifndef SRMC_ORACLE_H
#define SRMC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_DMAX 19
#define ORC_PMAX 24

enum { ORC_MODEL_COS = 0, ORC_MODEL_LOGISTIC = 1, ORC_MODEL_AFFINE = 2, ORC_MODEL_USER = 3 };
/* Local polynomials: constants, affine functions (Sec. 4.1) and quadratics
 * (LP2: 1, x_l, x_a x_b for a <= b; the higher order the paper mentions as
 * possible, Sec. 4 footnote).  ORC_PBMAX = the largest basis dimension. */
enum { ORC_LP0 = 0, ORC_LP1 = 1, ORC_LP2 = 2 };
#define ORC_PBMAX (1 + ORC_DMAX + ORC_DMAX * (ORC_DMAX + 1) / 2)
/* Strata (assumption HS): equal size on the box [lo, hi) (example i), or equal
 * probability under nu, nu(H_k) = 1/K (example ii; lo and hi unused). */
enum { ORC_STRATA_SIZE = 0, ORC_STRATA_PROB = 1 };
/* Markov chain between grid times (Sec. 2, assumption HX): the Euler scheme
 * (Alg. 2) or the SDE itself (Alg. 1, exact for the affine drift below). */
enum { ORC_EULER = 0, ORC_EXACT = 1 };

/* One SRMC problem: forward SDE, driver/terminal model, grid, strata, basis. */
typedef struct {
    int d, q;                       /* dim of X and of W                     */
    int N;                          /* number of time steps                  */
    double T;                       /* horizon                               */
    double b[ORC_DMAX];             /* drift b_l - theta_l x_l (constant part) */
    double sigma[ORC_DMAX * ORC_DMAX]; /* constant diffusion, row-major d x q */
    int model;                      /* ORC_MODEL_*                           */
    double params[ORC_PMAX];        /* model parameters (see srmc_oracle.c)  */
    int cells[ORC_DMAX];            /* cells per dimension                   */
    double lo[ORC_DMAX], hi[ORC_DMAX]; /* box; outer cells extend to +-inf   */
    double mu;                      /* logistic scale                        */
    int basis;                      /* ORC_LP0 / ORC_LP1                     */
    int64_t M;                      /* paths per stratum                     */
    uint64_t seed;                  /* Philox seed                           */
    uint32_t instance;              /* instance id folded into the key       */
    double Cy, Cz;                  /* truncation levels; <= 0 disables      */
    int strata;                     /* ORC_STRATA_SIZE / ORC_STRATA_PROB     */
    const int64_t *M_strata;        /* [K] paths of each stratum, or NULL: M */
    double theta[ORC_DMAX];         /* mean reversion of the drift (0: constant) */
    int dynamics;                   /* ORC_EULER / ORC_EXACT (diagonal sigma)  */
    /* ORC_MODEL_USER: g(x) and f(t, x, y, z) supplied as functions (params = prm) */
    double (*user_g)(const double *x, int d, const double *prm);
    double (*user_f)(double t, const double *x, double y, const double *z, int d, const double *prm);
    /* optional: drift b_l(t, x) and diagonal diffusion sigma_l(t, x) for the
     * Euler step (both NULL: b - theta x and sigma above) */
    double (*user_b)(double t, const double *x, int l, int d, const double *prm);
    double (*user_sigma)(double t, const double *x, int l, int d, const double *prm);
} orc_problem;

/* ---- primitives ---------------------------------------------------------- */
void     orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double   orc_uniform(uint32_t w);                 /* (w + 1/2) 2^-32            */
double   orc_norminv(double u);                   /* Phi^{-1}(u), u in (0,1)    */
double   orc_normal_from_word(uint32_t w);        /* Phi^{-1}((w+1/2) 2^-32)    */
uint32_t orc_draw_word(const orc_problem *P, int i, int64_t k, int64_t m, int64_t n);
double   orc_logistic_cdf(double x, double mu);
double   orc_sample_restricted(double U, double xlo, double xhi, double mu);
int      orc_locate_dim(const orc_problem *P, int l, double x);
int64_t  orc_locate(const orc_problem *P, const double *x);
int      orc_locate_dim_f32(float x, float lo, float r, int C);
void     orc_cell_edges(const orc_problem *P, int l, int c, double *xlo, double *xhi);
void     orc_stratum_cells(const orc_problem *P, int64_t k, int *cells);
void     orc_stratum_centre(const orc_problem *P, int64_t k, double *x);
/* Unit of the centred basis coordinate of cell c in dimension l: h/2 for
 * equal-size cells; for equal-probability cells the width between the
 * quantiles (c + 1/4)/C and (c + 3/4)/C of nu (finite for the outer cells). */
double   orc_cell_scale(const orc_problem *P, int l, int c);
void     orc_start_point(const orc_problem *P, int i, int64_t k, int64_t m, double *x);
double   orc_g(const orc_problem *P, const double *x);
double   orc_f(const orc_problem *P, int j, const double *x, double y, const double *z);

/* ---- least squares ------------------------------------------------------- */
/* Householder QR least squares: A (n x p, row-major), B (n x r) -> X (p x r).
 * Returns 0 on success, 1 if R is numerically singular.  A and B are
 * overwritten. */
int orc_lstsq_householder(int n, int p, int r, double *A, double *B, double *X);

/* ---- the scheme ---------------------------------------------------------- */
typedef struct orc_ctx orc_ctx;
orc_ctx *orc_create(const orc_problem *P);
void     orc_destroy(orc_ctx *C);
int      orc_row_len(const orc_ctx *C);           /* (1+q)*(dim of basis)        */
/* Full backward solve, OpenMP over strata with nthreads threads (0 = default). */
int      orc_solve_full(orc_ctx *C, int nthreads);
/* Lazy, memoised fit of one (i,k): computes every row it depends on first. */
int      orc_fit_lazy(orc_ctx *C, int i, int64_t k);
/* Fit of one (i,k) given that every row of steps > i it visits exists.
 * Returns the number of rows it was missing (0 on success). */
int64_t  orc_fit_one(orc_ctx *C, int i, int64_t k);
/* Raw-basis row (alpha[dimb], beta[q*dimb]) of (i,k); NULL if not computed. */
const double *orc_row(const orc_ctx *C, int i, int64_t k);
/* Truncated y_i(x), z_i(x) at n points (row-major n x d); rows must exist.
 * Returns the number of points whose row is missing. */
int64_t  orc_eval(orc_ctx *C, int i, int64_t n, const double *x, double *y, double *z);
/* Control variate (a martingale control subtracted from the responses):
 * rows [N][K][q][p] in the centred basis phi = [1, (x - c_k)/s] (c_k and s
 * from orc_stratum_centre and orc_cell_scale) give zc_j(x) = T_Cz(beta . phi(x))
 * for x in stratum k; the Y response loses sum_{j>=i} zc_j(X_j).dW_j and the
 * Z response sum_{j>i} zc_j(X_j).dW_j.
 * Both have zero conditional mean given x_i, so the fitted functions keep
 * their expectation.  The rows are copied; NULL removes the control. */
int      orc_set_control(orc_ctx *C, const double *rows);
/* The run's own control: with on != 0 both responses of cloud C_{i,k} lose
 * sum_{j>i} z_j(X_j).dW_j, z_j the truncated fit of the stratum holding X_j
 * at step j (fitted from other, independent clouds before step i, so
 * E[z_j(X_j).dW_j | X_j] = 0; no step-i term).  Replaces any control rows;
 * orc_set_control(C, NULL) or on = 0 removes it. */
void     orc_set_own_control(orc_ctx *C, int on);

/* ---- teacher forcing: a step fitted from given later rows ----------------
 * Install the rows of step i of every stratum from a table in the monomials
 * of the centred coordinate u_l = (x_l - c_{k,l}) / s_{k,l} (c_k and s from
 * orc_stratum_centre and orc_cell_scale; the basis of the control rows):
 * yrows[k * ystride + c] = alpha_c, zrows[k * zstride + l * dimb + c] =
 * beta_{l,c}.  Each row is expanded into the raw monomials of x, in which the
 * oracle fits and evaluates (the same function on H_k), and marked fitted, so
 * that fits of steps i' < i read it.  A fit of step i' reads rows of steps
 * > i' only, so fits taken in increasing i' never see a row of their own step
 * that they wrote.  Returns 0, or 1 for an invalid step. */
int      orc_set_rows_centred(orc_ctx *C, int i, const double *yrows, int64_t ystride,
                              const double *zrows, int64_t zstride);
/* Fit the n strata ks[] of step i (OpenMP over the list with nthreads
 * threads, 0 = default), each as orc_fit_one; returns the number of rows of
 * later steps they were missing (0 on success). */
int64_t  orc_fit_many(orc_ctx *C, int i, int64_t n, const int64_t *ks, int nthreads);
/* Timing aid: with on != 0 a missing row of a later step reads as the zero
 * function (y = 0, z = 0) instead of being counted as missing, so that a fit
 * of any (i, k) runs all of its arithmetic without the rows it depends on.
 * Fits made so are stored like others; not for results. */
void     orc_set_missing_zero(orc_ctx *C, int on);

/* Number of (i,k) fits that fell back to LP0 because R was singular. */
int64_t  orc_fallbacks(const orc_ctx *C);
/* Path-steps simulated so far (diagnostic; one unit = one Euler step). */
int64_t  orc_path_steps(const orc_ctx *C);

/* ---- small MLP u(a), a = (t, x_1..x_d): nin -> H -> H -> 1, SiLU ----------
 * Parameter vector (float): W1 [H][nin], b1 [H], W2 [H][H], b2 [H], w3 [H], b3.
 * bf16 != 0 rounds to bfloat16 (nearest even) exactly where the GPU kernels
 * feed tensor-core operands: the inputs, W1, h1, W2, and in the backward pass
 * g_z2 and g_z1; everything else is FP64. */
int    orc_mlp_nparams(int nin, int H);
float  orc_bf16(double v);
void   orc_mlp_eval(const float *prm, int nin, int H, int bf16, const double *a, double *u,
                    double *grad_a);
/* Mean squared error (1/n) sum (u(a_s) - y_s)^2 and its gradient (nparams). */
double orc_mlp_loss_grad(const float *prm, int nin, int H, int bf16, int64_t n, const double *a,
                         const double *y, double *grad);

#ifdef __cplusplus
}
#endif
#endif
