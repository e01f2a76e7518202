/*
 * srmc_oracle.c -- plain FP64 CPU oracle of the SRMDP scheme.
 *
 * TEST INFRASTRUCTURE ONLY (see srmc_oracle.h).  Written for clarity, not
 * speed: straight loops over (i, k, m, j), no blocking, no fusion, the raw
 * basis [1, x] of the paper and Householder QR, exactly the route of
 * Sec. 4.1.  Compiled with -ffp-contract=off so that x86 and Arm hosts give
 * the same bits.
 *
 * Model parameter layouts (params[]):
 *   ORC_MODEL_COS       u(t,x) = e^{lam(T-t)} cos(s), s = sum_l x_l / sqrt(d),
 *                       g(x) = cos(s),
 *                       f_j(x,y,z) = (lam + s0^2/2) y + kap (y^2 - u(t_j,x)^2)
 *                                    + kapz (|z|^2 - s0^2 e^{2 lam (T-t_j)} sin^2 s)
 *                       params = {lam, kap, kapz, s0}
 *   ORC_MODEL_LOGISTIC  the test BSDE of Sec. 5.1: w(t,x) = exp(t + sum x),
 *                       g = w(T,x)/(1+w(T,x)), f = (sum_l z_l)(y - (2+q)/(2q))
 *   ORC_MODEL_AFFINE    g(x) = p0 + sum_l p_{1+l} x_l,
 *                       f_j(x,y,z) = p_{1+d} + sum_l p_{2+d+l} x_l + p_{2+2d} y
 */
#include "srmc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10 (Salmon et al., SC'11): ten rounds of the Philox S-box     */
/* with multipliers 0xD2511F53, 0xCD9E8D57 and Weyl key increments           */
/* 0x9E3779B9, 0xBB67AE85 between rounds.                                    */
/* ------------------------------------------------------------------------ */
static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
        philox_round(c, k);
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Word n of the stream of path m of cloud C_{i,k}: key = (seed_lo ^ instance,
 * seed_hi), counter = (n / 4, m, k, i), word n mod 4.  Every (i,k,m) owns its
 * own counter range, so the clouds are independent across (i,k) as the
 * definition of C_{i,k} requires. */
uint32_t orc_draw_word(const orc_problem *P, int i, int64_t k, int64_t m, int64_t n)
{
    uint32_t key[2] = {(uint32_t)(P->seed & 0xFFFFFFFFu) ^ P->instance,
                       (uint32_t)(P->seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)(n / 4), (uint32_t)m, (uint32_t)k, (uint32_t)i};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[n % 4];
}

double orc_uniform(uint32_t w) { return ((double)w + 0.5) * 0x1p-32; }

/* Standard normal CDF through the complementary error function. */
static double Phi(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

/* Phi^{-1}(u) for u in (0,1).  For p = min(u, 1-u) <= 1/2 solve
 * log Phi(x) = log p by Newton's method from x0 = -sqrt(-2 log p).  Since
 * Phi(x) <= exp(-x^2/2)/2 for x <= 0, x0 lies left of the root, and log Phi is
 * increasing and concave, so the iterates rise monotonically to the root. */
double orc_norminv(double u)
{
    if (!(u > 0.0 && u < 1.0)) return NAN;
    if (u == 0.5) return 0.0;
    double p = u < 0.5 ? u : 1.0 - u;
    double lp = log(p);
    double x = -sqrt(-2.0 * lp);
    for (int it = 0; it < 200; ++it) {
        double P = Phi(x);
        double h = log(P) - lp;
        double dens = exp(-0.5 * x * x) / sqrt(2.0 * M_PI);
        double step = h * P / dens;         /* h / (d/dx log Phi) */
        double xn = x - step;
        if (xn > 0.0) xn = 0.0;
        if (fabs(xn - x) <= 1e-16 * fmax(1.0, fabs(x))) { x = xn; break; }
        x = xn;
    }
    return u < 0.5 ? x : -x;
}

/* The normal of one word: xi = Phi^{-1}(U), U = (w+1/2) 2^-32.  1-U is exact
 * in double, so the upper half is computed from its own tail. */
double orc_normal_from_word(uint32_t w)
{
    if (w < 0x80000000u) return orc_norminv(orc_uniform(w));
    return -orc_norminv(orc_uniform(0xFFFFFFFFu - w));
}

/* ------------------------------------------------------------------------ */
/* Logistic law and its restriction to one cell (assumption A_nu, Alg. 3)   */
/* ------------------------------------------------------------------------ */
double orc_logistic_cdf(double x, double mu)
{
    if (x == -INFINITY) return 0.0;
    if (x == INFINITY) return 1.0;
    return 1.0 / (1.0 + exp(-mu * x));
}

/* F^{-1} restricted to [xlo, xhi) applied to U: x with F(x) = F(xlo) +
 * U (F(xhi) - F(xlo)).  Written as x = log(p/qc)/mu with p = F(xlo) + U w,
 * qc = 1 - F(xhi) + (1-U) w, w = F(xhi) - F(xlo): p + qc = 1, so
 * F(x) = p/(p+qc) = p, the same map as Alg. 3 without the cancellation of
 * 1/p - 1 in the upper tail.  U and 1-U are both exact lattice values. */
static double sample_from_masses(double U, double Uc, double Flo, double Fchi, double w, double mu)
{
    double p = Flo + U * w;
    double qc = Fchi + Uc * w;
    return log(p / qc) / mu;
}

static double sample_restricted_uc(double U, double Uc, double xlo, double xhi, double mu)
{
    double Flo = orc_logistic_cdf(xlo, mu);
    double Fchi = orc_logistic_cdf(-xhi, mu);             /* 1 - F(xhi) */
    double w;
    if (xlo > 0.0) w = orc_logistic_cdf(-xlo, mu) - Fchi;  /* both in the upper tail */
    else w = orc_logistic_cdf(xhi, mu) - Flo;
    return sample_from_masses(U, Uc, Flo, Fchi, w, mu);
}

double orc_sample_restricted(double U, double xlo, double xhi, double mu)
{
    return sample_restricted_uc(U, 1.0 - U, xlo, xhi, mu);
}

/* ------------------------------------------------------------------------ */
/* Strata (assumption A_Strat): the box [lo, hi) cut into cells[l] equal    */
/* cells per dimension; the first and last cell of every dimension extend   */
/* to -inf / +inf so that the strata cover R^d.  Half-open cells: a point on */
/* an inner edge belongs to the upper cell.                                  */
/* ------------------------------------------------------------------------ */
static double cell_width(const orc_problem *P, int l)
{
    return (P->hi[l] - P->lo[l]) / (double)P->cells[l];
}

/* Equal-probability cells (assumption HS, example ii): nu is the product of
 * one-dimensional logistic laws, so cutting every axis at the quantiles
 * F^{-1}(c/C) = log(c/(C-c))/mu, c = 1..C-1, gives nu(H_k) = 1/K. */
static double prob_quantile(double num, double den, double mu)    /* F^{-1}(num/(num+den)) */
{
    return log(num / den) / mu;
}

static double prob_edge(const orc_problem *P, int l, int c)
{
    int C = P->cells[l];
    if (c <= 0) return -INFINITY;
    if (c >= C) return INFINITY;
    return prob_quantile((double)c, (double)(C - c), P->mu);
}

int orc_locate_dim(const orc_problem *P, int l, double x)
{
    if (P->strata == ORC_STRATA_PROB) {
        /* the cell [e_c, e_{c+1}) holding x, by scanning the edges upwards
         * (NaN compares false everywhere and lands in cell 0) */
        int c = 0;
        while (c < P->cells[l] - 1 && x >= prob_edge(P, l, c + 1)) ++c;
        return c;
    }
    double t = (x - P->lo[l]) / cell_width(P, l);
    int C = P->cells[l];
    if (!(t >= 0.0)) return 0;                 /* below the box, or NaN */
    if (t >= (double)C) return C - 1;
    int c = (int)floor(t);
    return c > C - 1 ? C - 1 : c;
}

/* The same decision taken in IEEE single precision, for single-precision
 * paths: c = floor((x - lo) * r) with r = cells / (hi - lo) rounded to float. */
int orc_locate_dim_f32(float x, float lo, float r, int C)
{
    volatile float diff = x - lo;
    volatile float t = diff * r;
    if (!(t >= 0.0f)) return 0;
    if (t >= (float)C) return C - 1;
    int c = (int)floorf(t);
    return c > C - 1 ? C - 1 : c;
}

int64_t orc_locate(const orc_problem *P, const double *x)
{
    int64_t k = 0, stride = 1;
    for (int l = 0; l < P->d; ++l) {
        k += (int64_t)orc_locate_dim(P, l, x[l]) * stride;
        stride *= P->cells[l];
    }
    return k;
}

void orc_stratum_cells(const orc_problem *P, int64_t k, int *cells)
{
    for (int l = 0; l < P->d; ++l) {
        cells[l] = (int)(k % P->cells[l]);
        k /= P->cells[l];
    }
}

void orc_cell_edges(const orc_problem *P, int l, int c, double *xlo, double *xhi)
{
    if (P->strata == ORC_STRATA_PROB) {
        *xlo = prob_edge(P, l, c);
        *xhi = prob_edge(P, l, c + 1);
        return;
    }
    double h = cell_width(P, l);
    *xlo = (c == 0) ? -INFINITY : P->lo[l] + (double)c * h;
    *xhi = (c == P->cells[l] - 1) ? INFINITY : P->lo[l] + (double)(c + 1) * h;
}

void orc_stratum_centre(const orc_problem *P, int64_t k, double *x)
{
    int cells[ORC_DMAX];
    orc_stratum_cells(P, k, cells);
    for (int l = 0; l < P->d; ++l) {
        if (P->strata == ORC_STRATA_PROB) {
            /* the median of nu restricted to the cell: F^{-1}((c + 1/2)/C) */
            const int C = P->cells[l], c = cells[l];
            x[l] = prob_quantile(c + 0.5, C - c - 0.5, P->mu);
        } else {
            x[l] = P->lo[l] + ((double)cells[l] + 0.5) * cell_width(P, l);
        }
    }
}

double orc_cell_scale(const orc_problem *P, int l, int c)
{
    if (P->strata == ORC_STRATA_PROB) {
        const int C = P->cells[l];
        return prob_quantile(c + 0.75, C - c - 0.75, P->mu) - prob_quantile(c + 0.25, C - c - 0.25, P->mu);
    }
    return 0.5 * cell_width(P, l);
}

/* Exact transition of one coordinate of dX = (b - theta X) dt + s dW over dt
 * (Alg. 1): X' = X A + b B + s I with A = e^{-theta dt}, where the Ito integral
 * I = int_0^dt e^{-theta (dt - u)} dW_u is Gaussian with Var I =
 * (1 - e^{-2 theta dt})/(2 theta) and Cov(I, dW) = B = (1 - e^{-theta dt})/theta.
 * Given dW, I = (B/dt) dW + r xi2 with r^2 = Var I - B^2/dt and xi2 ~ N(0,1)
 * independent of dW.  theta = 0 gives A = 1, B = dt, I = dW (Brownian). */
static void ou_coeffs(double theta, double dt, double *A, double *B, double *r)
{
    if (theta == 0.0) { *A = 1.0; *B = dt; *r = 0.0; return; }
    const double a = theta * dt;
    *A = exp(-a);
    *B = -expm1(-a) / theta;
    double r2;
    if (fabs(a) < 1e-4) r2 = dt * a * a / 12.0 * (1.0 - a);   /* series; the difference cancels */
    else r2 = -expm1(-2.0 * a) / (2.0 * theta) - (*B) * (*B) / dt;
    *r = sqrt(r2 > 0.0 ? r2 : 0.0);
}

/* Start point of path m of cloud C_{i,k}: draws 0..d-1, one per coordinate
 * (Alg. 3). */
void orc_start_point(const orc_problem *P, int i, int64_t k, int64_t m, double *x)
{
    int cells[ORC_DMAX];
    orc_stratum_cells(P, k, cells);
    for (int l = 0; l < P->d; ++l) {
        uint32_t w = orc_draw_word(P, i, k, m, l);
        if (P->strata == ORC_STRATA_PROB) {
            /* F(e_c) = c/C and 1 - F(e_{c+1}) = (C-c-1)/C by the choice of the edges */
            const double C = (double)P->cells[l], c = (double)cells[l];
            x[l] = sample_from_masses(orc_uniform(w), orc_uniform(0xFFFFFFFFu - w),
                                      c / C, (C - c - 1.0) / C, 1.0 / C, P->mu);
            continue;
        }
        double xlo, xhi;
        orc_cell_edges(P, l, cells[l], &xlo, &xhi);
        x[l] = sample_restricted_uc(orc_uniform(w), orc_uniform(0xFFFFFFFFu - w),
                                    xlo, xhi, P->mu);
    }
}

/* ------------------------------------------------------------------------ */
/* Model: terminal g and driver f_j                                          */
/* ------------------------------------------------------------------------ */
static double sum_over_sqrt_d(const orc_problem *P, const double *x)
{
    double s = 0.0;
    for (int l = 0; l < P->d; ++l) s += x[l];
    return s / sqrt((double)P->d);
}

double orc_g(const orc_problem *P, const double *x)
{
    if (P->model == ORC_MODEL_USER) return P->user_g(x, P->d, P->params);
    switch (P->model) {
    case ORC_MODEL_COS:
        return cos(sum_over_sqrt_d(P, x));
    case ORC_MODEL_LOGISTIC: {
        double s = P->T;
        for (int l = 0; l < P->d; ++l) s += x[l];
        double w = exp(s);
        return w / (1.0 + w);
    }
    case ORC_MODEL_AFFINE: {
        double v = P->params[0];
        for (int l = 0; l < P->d; ++l) v += P->params[1 + l] * x[l];
        return v;
    }
    }
    return NAN;
}

double orc_f(const orc_problem *P, int j, const double *x, double y, const double *z)
{
    double dt = P->T / (double)P->N;
    double tj = (double)j * dt;
    switch (P->model) {
    case ORC_MODEL_COS: {
        double lam = P->params[0], kap = P->params[1], kapz = P->params[2], s0 = P->params[3];
        double s = sum_over_sqrt_d(P, x);
        double e = exp(lam * (P->T - tj));
        double u = e * cos(s);
        double v = (lam + 0.5 * s0 * s0) * y + kap * (y * y - u * u);
        /* with a drift b(x) = b - theta x the generator adds b(x).grad u =
         * b(x).z / s0 (z = s0 grad u), which the driver cancels */
        double bz = 0.0;
        int drift = 0;
        for (int l = 0; l < P->d; ++l) {
            if (P->b[l] != 0.0 || P->theta[l] != 0.0) drift = 1;
            bz += (P->b[l] - P->theta[l] * x[l]) * z[l];
        }
        if (drift) v -= bz / s0;
        if (kapz != 0.0) {
            double zz = 0.0;
            for (int l = 0; l < P->q; ++l) zz += z[l] * z[l];
            double sn = sin(s);
            v += kapz * (zz - s0 * s0 * e * e * sn * sn);
        }
        return v;
    }
    case ORC_MODEL_LOGISTIC: {
        double sz = 0.0;
        for (int l = 0; l < P->q; ++l) sz += z[l];
        return sz * (y - (2.0 + P->q) / (2.0 * P->q));
    }
    case ORC_MODEL_USER:
        return P->user_f(tj, x, y, z, P->d, P->params);
    case ORC_MODEL_AFFINE: {
        int d = P->d;
        double v = P->params[1 + d];
        for (int l = 0; l < d; ++l) v += P->params[2 + d + l] * x[l];
        return v + P->params[2 + 2 * d] * y;
    }
    }
    return NAN;
}

/* Truncation T_L, eq. TL; L <= 0 means no truncation. */
static double trunc_L(double v, double L)
{
    if (L <= 0.0) return v;
    return v < -L ? -L : (v > L ? L : v);
}

/* ------------------------------------------------------------------------ */
/* Householder QR least squares (Golub & Van Loan, Sec. 5.3)                 */
/* ------------------------------------------------------------------------ */
int orc_lstsq_householder(int n, int p, int r, double *A, double *B, double *X)
{
    double colnorm_max = 0.0;
    for (int c = 0; c < p; ++c) {
        double s = 0.0;
        for (int m = 0; m < n; ++m) s += A[m * p + c] * A[m * p + c];
        if (sqrt(s) > colnorm_max) colnorm_max = sqrt(s);
    }
    int singular = (n < p);
    for (int c = 0; c < p && !singular; ++c) {
        /* Reflector H = I - 2 v v^T / (v^T v) mapping A[c:, c] onto -sign * ||.|| e_1. */
        double nrm = 0.0;
        for (int m = c; m < n; ++m) nrm += A[m * p + c] * A[m * p + c];
        nrm = sqrt(nrm);
        if (nrm <= 1e-12 * colnorm_max) { singular = 1; break; }
        double alpha = A[c * p + c] >= 0.0 ? -nrm : nrm;
        /* v = A[c:, c] - alpha e_1, stored in place in column c. */
        A[c * p + c] -= alpha;
        double vtv = 0.0;
        for (int m = c; m < n; ++m) vtv += A[m * p + c] * A[m * p + c];
        for (int cc = c + 1; cc < p; ++cc) {
            double dot = 0.0;
            for (int m = c; m < n; ++m) dot += A[m * p + c] * A[m * p + cc];
            double fac = 2.0 * dot / vtv;
            for (int m = c; m < n; ++m) A[m * p + cc] -= fac * A[m * p + c];
        }
        for (int rr = 0; rr < r; ++rr) {
            double dot = 0.0;
            for (int m = c; m < n; ++m) dot += A[m * p + c] * B[m * r + rr];
            double fac = 2.0 * dot / vtv;
            for (int m = c; m < n; ++m) B[m * r + rr] -= fac * A[m * p + c];
        }
        /* R[c][c] = alpha; the rest of column c below the diagonal is v. */
        A[c * p + c] = alpha;
    }
    if (singular) return 1;
    /* Back substitution R X = (Q^T B)[0:p]. */
    for (int rr = 0; rr < r; ++rr) {
        for (int c = p - 1; c >= 0; --c) {
            double s = B[c * r + rr];
            for (int cc = c + 1; cc < p; ++cc) s -= A[c * p + cc] * X[cc * r + rr];
            X[c * r + rr] = s / A[c * p + c];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The scheme: Alg. SRMDP                                                    */
/* ------------------------------------------------------------------------ */
struct orc_ctx {
    orc_problem P;
    double *control;    /* [N][K][q][dimb] centred-basis control rows, or NULL */
    int own_control;    /* control from the fitted z of later steps        */
    int64_t K;          /* number of strata                                 */
    int dimb;           /* basis dimension: 1 (LP0), d+1 (LP1), 1+d+d(d+1)/2 (LP2) */
    int R;              /* row length (1+q)*dimb                            */
    double *rows;       /* [N][K][R], raw basis                             */
    unsigned char *done;/* [N][K]                                           */
    int64_t fallbacks;
    int64_t path_steps;
    int missing_zero;   /* timing aid: a missing row reads as zero        */
};

orc_ctx *orc_create(const orc_problem *P)
{
    if (P->d < 1 || P->d > ORC_DMAX || P->q < 1 || P->q > ORC_DMAX || P->N < 1) return NULL;
    orc_ctx *C = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    if (!C) return NULL;
    C->P = *P;
    C->K = 1;
    for (int l = 0; l < P->d; ++l) C->K *= P->cells[l];
    C->dimb = P->basis == ORC_LP0 ? 1 : P->basis == ORC_LP1 ? P->d + 1 : 1 + P->d + P->d * (P->d + 1) / 2;
    C->R = (1 + P->q) * C->dimb;
    C->rows = (double *)calloc((size_t)P->N * (size_t)C->K * (size_t)C->R, sizeof(double));
    C->done = (unsigned char *)calloc((size_t)P->N * (size_t)C->K, 1);
    if (!C->rows || !C->done) { orc_destroy(C); return NULL; }
    return C;
}

void orc_destroy(orc_ctx *C)
{
    if (!C) return;
    free(C->control);
    free(C->rows);
    free(C->done);
    free(C);
}

int orc_row_len(const orc_ctx *C) { return C->R; }

int orc_set_control(orc_ctx *C, const double *rows)
{
    free(C->control);
    C->control = NULL;
    C->own_control = 0;
    if (!rows) return 0;
    size_t n = (size_t)C->P.N * (size_t)C->K * (size_t)C->P.q * (size_t)C->dimb;
    C->control = (double *)malloc(sizeof(double) * n);
    if (!C->control) return 1;
    memcpy(C->control, rows, sizeof(double) * n);
    return 0;
}

void orc_set_own_control(orc_ctx *C, int on)
{
    free(C->control);
    C->control = NULL;
    C->own_control = on != 0;
}

/* The monomials of the basis at the coordinates u: [1] (LP0), [1, u] (LP1),
 * [1, u, u_a u_b for a <= b in row order] (LP2). */
static void monomials(const orc_ctx *C, const double *u, double *phi)
{
    const int d = C->P.d;
    phi[0] = 1.0;
    if (C->dimb > 1)
        for (int l = 0; l < d; ++l) phi[1 + l] = u[l];
    if (C->dimb > d + 1) {
        int e = 1 + d;
        for (int a = 0; a < d; ++a)
            for (int b = a; b < d; ++b) phi[e++] = u[a] * u[b];
    }
}

/* zc_j(x) . dw for a point x of stratum k (control rows in the monomials of
 * the centred coordinate u = (x - c_k)/s_k, values truncated at C_z). */
static double control_dot(const orc_ctx *C, int j, int64_t k, const double *x, const double *dw)
{
    const orc_problem *P = &C->P;
    const int p = C->dimb;
    double phi[ORC_PBMAX], ctr[ORC_DMAX], u[ORC_DMAX];
    int cells[ORC_DMAX];
    orc_stratum_centre(P, k, ctr);
    orc_stratum_cells(P, k, cells);
    for (int l = 0; l < P->d; ++l) u[l] = (x[l] - ctr[l]) / orc_cell_scale(P, l, cells[l]);
    monomials(C, u, phi);
    const double *row = C->control + ((size_t)j * (size_t)C->K + (size_t)k) * (size_t)(P->q * p);
    double s = 0.0;
    for (int l = 0; l < P->q; ++l) {
        double v = 0.0;
        for (int c = 0; c < p; ++c) v += row[l * p + c] * phi[c];
        s += trunc_L(v, P->Cz) * dw[l];
    }
    return s;
}
int64_t orc_fallbacks(const orc_ctx *C) { return C->fallbacks; }
int64_t orc_path_steps(const orc_ctx *C) { return C->path_steps; }

const double *orc_row(const orc_ctx *C, int i, int64_t k)
{
    if (i < 0 || i >= C->P.N || k < 0 || k >= C->K) return NULL;
    size_t idx = (size_t)i * (size_t)C->K + (size_t)k;
    return C->done[idx] ? C->rows + idx * (size_t)C->R : NULL;
}

/* Raw basis: the monomials of x itself (the fits are made in it, Sec. 4.1). */
static void basis(const orc_ctx *C, const double *x, double *phi)
{
    monomials(C, x, phi);
}

/* y_j(x) and z_j(x) from the fitted row of the stratum holding x, both
 * truncated (Alg. SRMDP); y_N = g. */
static void eval_row(const orc_ctx *C, const double *row, const double *x, double *y, double *z)
{
    double phi[ORC_PBMAX];
    basis(C, x, phi);
    double v = 0.0;
    for (int c = 0; c < C->dimb; ++c) v += row[c] * phi[c];
    *y = trunc_L(v, C->P.Cy);
    if (z) {
        for (int l = 0; l < C->P.q; ++l) {
            const double *bl = row + C->dimb * (1 + l);
            double w = 0.0;
            for (int c = 0; c < C->dimb; ++c) w += bl[c] * phi[c];
            z[l] = trunc_L(w, C->P.Cz);
        }
    }
}

/* Row (j, k) for a lookup; in lazy mode a missing row is fitted first.
 * Returns NULL (and counts) when the row is missing and lazy is off. */
static const double zero_row[(1 + ORC_DMAX) * ORC_PBMAX];

static const double *need_row(orc_ctx *C, int j, int64_t k, int lazy, int64_t *missing)
{
    const double *row = orc_row(C, j, k);
    if (row) return row;
    if (C->missing_zero) return zero_row;
    if (lazy) {
        orc_fit_lazy(C, j, k);
        row = orc_row(C, j, k);
        if (row) return row;
    }
    (*missing)++;
    return NULL;
}

static int64_t fit_impl(orc_ctx *C, int i, int64_t k, int lazy)
{
    const orc_problem *P = &C->P;
    const int d = P->d, q = P->q, N = P->N, p = C->dimb;
    /* M may vary with the stratum (Sec. 3: the analysis adapts to M_k) */
    const int64_t M = P->M_strata ? P->M_strata[k] : P->M;
    const double dt = P->T / (double)N, sdt = sqrt(dt);
    int64_t missing = 0;

    double *X0 = (double *)malloc(sizeof(double) * (size_t)(M * d));   /* x_i       */
    double *DW = (double *)malloc(sizeof(double) * (size_t)(M * q));   /* Delta W_i */
    double *S1 = (double *)malloc(sizeof(double) * (size_t)M);         /* S_{Y,i+1} */
    double *Y1 = (double *)malloc(sizeof(double) * (size_t)M);         /* y_{i+1}(x_{i+1}) */
    double *CZ = (double *)calloc((size_t)M, sizeof(double));          /* sum_{j>i} zc_j.dW_j */
    double *CI = (double *)calloc((size_t)M, sizeof(double));          /* zc_i(x_i).dW_i */
    double *A = (double *)malloc(sizeof(double) * (size_t)(M * p));
    double *B = (double *)malloc(sizeof(double) * (size_t)(M * (q > 1 ? q : 1)));
    double *coef = (double *)malloc(sizeof(double) * (size_t)(p * (q > 1 ? q : 1)));
    double row[(1 + ORC_DMAX) * ORC_PBMAX];
    int64_t steps = 0;
    const int nw = P->dynamics == ORC_EXACT ? 2 : 1;   /* normal blocks per step */

    for (int64_t m = 0; m < M; ++m) {
        double x[ORC_DMAX], xn[ORC_DMAX], dw[ORC_DMAX], zj[ORC_DMAX], zn[ORC_DMAX];
        double yn = 0.0;
        orc_start_point(P, i, k, m, x);
        for (int l = 0; l < d; ++l) X0[m * d + l] = x[l];
        double S = 0.0;
        for (int j = i; j < N; ++j) {
            /* Delta W_j = sqrt(dt) xi, xi ~ N(0, I_q): draws d + (j-i) nw q + l;
             * the exact dynamics takes q more normals per step (xi2, next q draws). */
            const int64_t base = d + (int64_t)(j - i) * nw * q;
            for (int l = 0; l < q; ++l)
                dw[l] = sdt * orc_normal_from_word(orc_draw_word(P, i, k, m, base + l));
            if (P->dynamics == ORC_EXACT) {
                /* Alg. 1, per coordinate (diagonal sigma) */
                for (int l = 0; l < d; ++l) {
                    const double xi2 = orc_normal_from_word(orc_draw_word(P, i, k, m, base + q + l));
                    double A, B, r;
                    ou_coeffs(P->theta[l], dt, &A, &B, &r);
                    const double I = (B / dt) * dw[l] + r * xi2;
                    xn[l] = x[l] * A + P->b[l] * B + P->sigma[l * q + l] * I;
                }
            } else if (P->user_b) {
                /* Euler step with the user's b(t, x) and diagonal sigma(t, x) at (t_j, X_j) */
                const double tj = (double)j * dt;
                for (int l = 0; l < d; ++l)
                    xn[l] = x[l] + P->user_b(tj, x, l, d, P->params) * dt
                            + P->user_sigma(tj, x, l, d, P->params) * dw[l];
            } else {
                /* Euler step, Alg. 2, read with the coefficients at (t_j, X_j). */
                for (int l = 0; l < d; ++l) {
                    double v = x[l] + (P->b[l] - P->theta[l] * x[l]) * dt;
                    for (int r = 0; r < q; ++r) v += P->sigma[l * q + r] * dw[r];
                    xn[l] = v;
                }
            }
            steps++;
            if (C->control) {
                const double cd = control_dot(C, j, j == i ? k : orc_locate(P, x), x, dw);
                if (j == i) CI[m] = cd; else CZ[m] += cd;
            } else if (C->own_control && j > i) {
                /* z_j(x_j) of the fitted row, as looked up for the driver */
                for (int l = 0; l < q; ++l) CZ[m] += zj[l] * dw[l];
            }
            if (j + 1 == N) {
                yn = orc_g(P, xn);
            } else {
                const double *rw = need_row(C, j + 1, orc_locate(P, xn), lazy, &missing);
                if (!rw) { yn = 0.0; for (int l = 0; l < q; ++l) zn[l] = 0.0; }
                else eval_row(C, rw, xn, &yn, zn);
            }
            if (j == i) {
                for (int l = 0; l < q; ++l) DW[m * q + l] = dw[l];
                Y1[m] = yn;
            } else {
                /* f_j(x_j, y_{j+1}(x_{j+1}), z_j(x_j)) dt, j >= i+1 (eq. PsiM) */
                S += orc_f(P, j, x, yn, zj) * dt;
            }
            for (int l = 0; l < d; ++l) x[l] = xn[l];
            for (int l = 0; l < q; ++l) zj[l] = zn[l];
        }
        S += orc_g(P, x);                   /* g(x_N) */
        S1[m] = S;
    }

    if (missing == 0) {
        int fell_back = 0;
        /* Z: OLS of S_{Y,i+1} Delta W_i / dt on L_{Z,k}. */
        for (int64_t m = 0; m < M; ++m) {
            basis(C, X0 + m * d, A + m * p);
            for (int l = 0; l < q; ++l) B[m * q + l] = (S1[m] - CZ[m]) * DW[m * q + l] / dt;
        }
        if (p == 1 || orc_lstsq_householder((int)M, p, q, A, B, coef)) {
            /* LP0, eq. lp0 explicit: the mean (also the fallback). */
            if (p > 1) fell_back = 1;
            for (int l = 0; l < q; ++l) {
                double s = 0.0;
                for (int64_t m = 0; m < M; ++m) s += (S1[m] - CZ[m]) * DW[m * q + l] / dt;
                for (int c = 0; c < p; ++c) coef[c * q + l] = (c == 0) ? s / (double)M : 0.0;
            }
        }
        for (int l = 0; l < q; ++l)
            for (int c = 0; c < p; ++c) row[p * (1 + l) + c] = coef[c * q + l];

        /* Y: OLS of S_{Y,i} = S_{Y,i+1} + f_i(x_i, y_{i+1}(x_{i+1}), z_i(x_i)) dt,
         * where z_i is the truncated fit just made (Z before Y). */
        for (int64_t m = 0; m < M; ++m) {
            double phi[ORC_PBMAX], zi[ORC_DMAX];
            basis(C, X0 + m * d, phi);
            for (int l = 0; l < q; ++l) {
                double w = 0.0;
                for (int c = 0; c < p; ++c) w += row[p * (1 + l) + c] * phi[c];
                zi[l] = trunc_L(w, P->Cz);
            }
            for (int c = 0; c < p; ++c) A[m * p + c] = phi[c];
            B[m] = S1[m] + orc_f(P, i, X0 + m * d, Y1[m], zi) * dt - CZ[m] - CI[m];
        }
        double ysum = 0.0;
        for (int64_t m = 0; m < M; ++m) ysum += B[m];
        if (p == 1 || fell_back || orc_lstsq_householder((int)M, p, 1, A, B, coef)) {
            if (p > 1) fell_back = 1;
            for (int c = 0; c < p; ++c) coef[c] = (c == 0) ? ysum / (double)M : 0.0;
        }
        for (int c = 0; c < p; ++c) row[c] = coef[c];

        size_t idx = (size_t)i * (size_t)C->K + (size_t)k;
        memcpy(C->rows + idx * (size_t)C->R, row, sizeof(double) * (size_t)C->R);
        C->done[idx] = 1;
#pragma omp atomic
        C->fallbacks += fell_back;
    }
#pragma omp atomic
    C->path_steps += steps;

    free(X0); free(DW); free(S1); free(Y1); free(CZ); free(CI); free(A); free(B); free(coef);
    return missing;
}

int64_t orc_fit_one(orc_ctx *C, int i, int64_t k)
{
    if (i < 0 || i >= C->P.N || k < 0 || k >= C->K) return -1;
    return fit_impl(C, i, k, 0);
}

int orc_fit_lazy(orc_ctx *C, int i, int64_t k)
{
    if (i < 0 || i >= C->P.N || k < 0 || k >= C->K) return -1;
    if (orc_row(C, i, k)) return 0;
    return fit_impl(C, i, k, 1) == 0 ? 0 : 1;
}

void orc_set_missing_zero(orc_ctx *C, int on) { C->missing_zero = on != 0; }

/* A row given in the monomials of u = (x - c)/s, written out in the monomials
 * of x: 1 stays 1; u_l = x_l / s_l - c_l / s_l; u_a u_b = (x_a x_b - c_b x_a
 * - c_a x_b + c_a c_b) / (s_a s_b).  cen and raw hold dimb coefficients. */
static void centred_to_raw(const orc_ctx *C, int64_t k, const double *cen, double *raw)
{
    const orc_problem *P = &C->P;
    const int d = P->d, p = C->dimb;
    double ctr[ORC_DMAX], sc[ORC_DMAX];
    int cells[ORC_DMAX];
    orc_stratum_centre(P, k, ctr);
    orc_stratum_cells(P, k, cells);
    for (int l = 0; l < d; ++l) sc[l] = orc_cell_scale(P, l, cells[l]);
    for (int c = 0; c < p; ++c) raw[c] = 0.0;
    raw[0] = cen[0];
    if (p > 1) {
        for (int l = 0; l < d; ++l) {
            raw[1 + l] += cen[1 + l] / sc[l];
            raw[0] -= cen[1 + l] * ctr[l] / sc[l];
        }
    }
    if (p > d + 1) {
        int e = 1 + d;
        for (int a = 0; a < d; ++a)
            for (int b = a; b < d; ++b, ++e) {
                const double w = cen[e] / (sc[a] * sc[b]);
                raw[e] += w;
                raw[1 + a] -= w * ctr[b];
                raw[1 + b] -= w * ctr[a];
                raw[0] += w * ctr[a] * ctr[b];
            }
    }
}

int orc_set_rows_centred(orc_ctx *C, int i, const double *yrows, int64_t ystride,
                         const double *zrows, int64_t zstride)
{
    if (i < 0 || i >= C->P.N) return 1;
    const int p = C->dimb, q = C->P.q;
    for (int64_t k = 0; k < C->K; ++k) {
        const size_t idx = (size_t)i * (size_t)C->K + (size_t)k;
        double *row = C->rows + idx * (size_t)C->R;
        centred_to_raw(C, k, yrows + k * ystride, row);
        for (int l = 0; l < q; ++l)
            centred_to_raw(C, k, zrows + k * zstride + (int64_t)l * p, row + p * (1 + l));
        C->done[idx] = 1;
    }
    return 0;
}

int64_t orc_fit_many(orc_ctx *C, int i, int64_t n, const int64_t *ks, int nthreads)
{
    if (i < 0 || i >= C->P.N) return -1;
    for (int64_t a = 0; a < n; ++a)
        if (ks[a] < 0 || ks[a] >= C->K) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int64_t missing = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : missing)
    for (int64_t a = 0; a < n; ++a) missing += fit_impl(C, i, ks[a], 0);
    return missing;
}

int orc_solve_full(orc_ctx *C, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int64_t bad = 0;
    for (int i = C->P.N - 1; i >= 0; --i) {
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad)
        for (int64_t k = 0; k < C->K; ++k) bad += fit_impl(C, i, k, 0) != 0;
        if (bad) return 1;
    }
    return 0;
}

int64_t orc_eval(orc_ctx *C, int i, int64_t n, const double *x, double *y, double *z)
{
    const orc_problem *P = &C->P;
    int64_t missing = 0;
    for (int64_t a = 0; a < n; ++a) {
        const double *xa = x + a * P->d;
        if (i == P->N) {
            y[a] = orc_g(P, xa);
            for (int l = 0; l < P->q; ++l) z[a * P->q + l] = 0.0;
            continue;
        }
        const double *row = orc_row(C, i, orc_locate(P, xa));
        if (!row) { missing++; y[a] = NAN; for (int l = 0; l < P->q; ++l) z[a * P->q + l] = NAN; continue; }
        eval_row(C, row, xa, y + a, z + a * P->q);
    }
    return missing;
}

/* ------------------------------------------------------------------------ */
/* Small MLP u(a) with SiLU activations, forward, input gradient and the    */
/* gradient of the mean squared error (plain backpropagation).              */
/* ------------------------------------------------------------------------ */
int orc_mlp_nparams(int nin, int H) { return H * nin + H + H * H + H + H + 1; }

float orc_bf16(double v)
{
    float f = (float)v;
    uint32_t b;
    memcpy(&b, &f, 4);
    b += 0x7FFFu + ((b >> 16) & 1u);        /* round to nearest, ties to even */
    b &= 0xFFFF0000u;
    memcpy(&f, &b, 4);
    return f;
}

static double rnd(double v, int bf16) { return bf16 ? (double)orc_bf16(v) : v; }
static double sigm(double z) { return 1.0 / (1.0 + exp(-z)); }

typedef struct {
    const float *W1, *b1, *W2, *b2, *w3, *b3;
} mlp_view;

static mlp_view mlp_split(const float *prm, int nin, int H)
{
    mlp_view v;
    v.W1 = prm; v.b1 = v.W1 + H * nin; v.W2 = v.b1 + H; v.b2 = v.W2 + H * H; v.w3 = v.b2 + H;
    v.b3 = v.w3 + H;
    return v;
}

/* Forward pass keeping what the backward passes need. */
static double mlp_forward(const mlp_view *m, int nin, int H, int bf16, const double *a, double *ar,
                          double *z1, double *h1r, double *z2, double *h2)
{
    for (int c = 0; c < nin; ++c) ar[c] = rnd(a[c], bf16);
    for (int o = 0; o < H; ++o) {
        double s = 0.0;
        for (int c = 0; c < nin; ++c) s += rnd(m->W1[o * nin + c], bf16) * ar[c];
        z1[o] = s + m->b1[o];
        h1r[o] = rnd(z1[o] * sigm(z1[o]), bf16);
    }
    double u = m->b3[0];
    for (int o = 0; o < H; ++o) {
        double s = 0.0;
        for (int c = 0; c < H; ++c) s += rnd(m->W2[o * H + c], bf16) * h1r[c];
        z2[o] = s + m->b2[o];
        h2[o] = z2[o] * sigm(z2[o]);
        u += (double)m->w3[o] * h2[o];
    }
    return u;
}

static double dsilu(double z) { double sg = sigm(z); return sg * (1.0 + z * (1.0 - sg)); }

void orc_mlp_eval(const float *prm, int nin, int H, int bf16, const double *a, double *u,
                  double *grad_a)
{
    mlp_view m = mlp_split(prm, nin, H);
    double ar[64], z1[256], h1r[256], z2[256], h2[256], gz2[256], gz1[256];
    *u = mlp_forward(&m, nin, H, bf16, a, ar, z1, h1r, z2, h2);
    if (!grad_a) return;
    for (int o = 0; o < H; ++o) gz2[o] = rnd((double)m.w3[o] * dsilu(z2[o]), bf16);
    for (int c = 0; c < H; ++c) {
        double s = 0.0;
        for (int o = 0; o < H; ++o) s += gz2[o] * rnd(m.W2[o * H + c], bf16);
        gz1[c] = rnd(s * dsilu(z1[c]), bf16);
    }
    for (int c = 0; c < nin; ++c) {
        double s = 0.0;
        for (int o = 0; o < H; ++o) s += gz1[o] * rnd(m.W1[o * nin + c], bf16);
        grad_a[c] = s;
    }
}

double orc_mlp_loss_grad(const float *prm, int nin, int H, int bf16, int64_t n, const double *a,
                         const double *y, double *grad)
{
    mlp_view m = mlp_split(prm, nin, H);
    const int P = orc_mlp_nparams(nin, H);
    double *gW1 = grad, *gb1 = gW1 + H * nin, *gW2 = gb1 + H, *gb2 = gW2 + H * H, *gw3 = gb2 + H;
    double *gb3 = gw3 + H;
    for (int q = 0; q < P; ++q) grad[q] = 0.0;
    double loss = 0.0;
    double ar[64], z1[256], h1r[256], z2[256], h2[256], gz2[256], gz1[256];
    for (int64_t s = 0; s < n; ++s) {
        double u = mlp_forward(&m, nin, H, bf16, a + s * nin, ar, z1, h1r, z2, h2);
        double r = u - y[s];
        loss += r * r;
        double du = 2.0 * r / (double)n;
        gb3[0] += du;
        for (int o = 0; o < H; ++o) {
            gw3[o] += du * h2[o];
            gz2[o] = rnd(du * (double)m.w3[o] * dsilu(z2[o]), bf16);
            gb2[o] += gz2[o];
        }
        for (int o = 0; o < H; ++o)
            for (int c = 0; c < H; ++c) gW2[o * H + c] += gz2[o] * h1r[c];
        for (int c = 0; c < H; ++c) {
            double t = 0.0;
            for (int o = 0; o < H; ++o) t += gz2[o] * rnd(m.W2[o * H + c], bf16);
            gz1[c] = rnd(t * dsilu(z1[c]), bf16);
            gb1[c] += gz1[c];
        }
        for (int o = 0; o < H; ++o)
            for (int c = 0; c < nin; ++c) gW1[o * nin + c] += gz1[o] * ar[c];
    }
    return loss / (double)n;
}
