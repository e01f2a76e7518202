// srmc_capi.cu -- the C ABI of libsrmc (include/srmc.h): solver set-up, the
// backward time loop, evaluation of the fitted functions, and kernels for the
// method's primitives.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <utility>
#include <vector>

#include "../../include/srmc.h"
#include "srmc_internal.h"

using srmc::Params;


namespace {

thread_local std::string g_last_error;

srmc_status fail(srmc_status st, const std::string &msg)
{
    g_last_error = msg;
    return st;
}
}  // namespace

void srmc::set_last_error(const std::string &msg) { g_last_error = msg; }

namespace {

srmc_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(e == cudaErrorMemoryAllocation ? SRMC_ERR_OOM : SRMC_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define SRMC_CUDA(call, what)                                   \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);      \
    } while (0)

double logistic_cdf(double x, double mu)
{
    if (x == -INFINITY) return 0.0;
    if (x == INFINITY) return 1.0;
    return 1.0 / (1.0 + std::exp(-mu * x));
}

int pad_to(int v, int m) { return (v + m - 1) / m * m; }

// Exact step over dt of dX = (b - theta X) dt + s dW (Alg. 1): X' = A X + b B
// + s I, where the stochastic integral I = int_0^dt e^{-theta (dt - u)} dW_u has
// Var I = (1 - e^{-2 theta dt}) / (2 theta) and Cov(I, dW) = B =
// (1 - e^{-theta dt}) / theta; given dW, I = (B/dt) dW + r xi with
// r^2 = Var I - B^2/dt (a second-order series where the two nearly cancel).
void ou_transition(double theta, double dt, double &A, double &B, double &r)
{
    if (theta == 0.0) { A = 1.0; B = dt; r = 0.0; return; }
    const double a = theta * dt;
    A = std::exp(-a);
    B = -std::expm1(-a) / theta;
    const double r2 = std::fabs(a) < 1e-4 ? dt * a * a / 12.0 * (1.0 - a)
                                          : -std::expm1(-2.0 * a) / (2.0 * theta) - B * B / dt;
    r = std::sqrt(r2 > 0.0 ? r2 : 0.0);
}

// Basis dimension: 1 (LP0), d + 1 (LP1), 1 + d + d(d+1)/2 (LP2).
int basis_dim(int basis, int d)
{
    return basis == SRMC_LP0 ? 1 : basis == SRMC_LP1 ? d + 1 : 1 + d + d * (d + 1) / 2;
}

// F^{-1}(num / (num + den)) of the logistic law with scale mu.
double logistic_quantile(double num, double den, double mu) { return std::log(num / den) / mu; }

// Halves per component of a binary16 control row: 4 (one 8-byte load) for
// p <= 4, else p rounded up to 8 (16-byte loads).

// Stratum locality order: the strata sorted by the Morton code of their
// cell coordinates (coordinate bits interleaved from the most significant
// level down; a dimension of 2^b cells contributes b bits, at most 39 bits in
// all since K < 2^31).  Work item t of a step launch solves stratum order[t],
// so the blocks resident at one time cover a compact box of cells and the
// rows their paths gather at later steps overlap in L1/L2.  The order only
// assigns strata to blocks: every stratum is solved by exactly one block and
// its result does not depend on the order.
std::vector<unsigned> morton_order(const int *cells, int d, long long K)
{
    int bits[SRMC_DMAX], maxb = 0;
    for (int l = 0; l < d; ++l) {
        bits[l] = 0;
        while ((1LL << bits[l]) < cells[l]) ++bits[l];
        maxb = std::max(maxb, bits[l]);
    }
    std::vector<std::pair<unsigned long long, unsigned>> key((size_t)K);
    for (long long k = 0; k < K; ++k) {
        long long rem = k;
        int c[SRMC_DMAX];
        for (int l = 0; l < d; ++l) { c[l] = (int)(rem % cells[l]); rem /= cells[l]; }
        unsigned long long m = 0;
        for (int t = maxb - 1; t >= 0; --t)
            for (int l = d - 1; l >= 0; --l)
                if (t < bits[l]) m = (m << 1) | (unsigned long long)((c[l] >> t) & 1);
        key[(size_t)k] = {m, (unsigned)k};
    }
    std::sort(key.begin(), key.end());
    std::vector<unsigned> order((size_t)K);
    for (size_t t = 0; t < order.size(); ++t) order[t] = key[t].second;
    return order;
}

void free_all(srmc_solver *s)
{
    if (s->graph) cudaGraphExecDestroy(s->graph);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    cudaFree(s->cellF); cudaFree(s->cellF_f); cudaFree(s->cellB); cudaFree(s->cellB_f);
    cudaFree(s->stepc); cudaFree(s->stepc_f);
    cudaFree(s->Y32); cudaFree(s->Z32); cudaFree(s->Y64); cudaFree(s->Z64); cudaFree(s->stats);
    cudaFree(s->C16); cudaFree(s->C64); cudaFree(s->order); cudaFree(s->Mk);
    srmc::rtc_release(s->rtc[0]);
    srmc::rtc_release(s->rtc[1]);
}

}  // namespace

int srmc_prepare_user_control(srmc_solver *s)
{
    if (s->P.model != srmc::MODEL_USER || s->rtc[1].kernel) return SRMC_OK;
    std::string log;
    if (!srmc::rtc_compile(s->user_source, s->P.d, s->fp64, s->lp1, true, s->user_dynamics, s->rtc[1], log))
        return fail(SRMC_ERR_INVALID_ARG, "user model, control-variate kernel: " + log);
    return SRMC_OK;
}

namespace {
cudaError_t launch_step(const srmc_solver *s, int i, cudaStream_t st)
{
    Params P = s->P;
    const bool rows = s->cv && !s->cv_own;
    P.C16 = rows ? s->C16 : nullptr;
    P.C64 = rows ? s->C64 : nullptr;
    P.cv_own = s->cv && s->cv_own ? 1 : 0;
    const int mv = srmc::kernel_mv(s);
    const int grid = (int)(P.K < 2147483647LL ? P.K : 2147483647LL);
    if (P.model == srmc::MODEL_USER) {
        const srmc::RtcKernel &k = s->rtc[s->cv ? 1 : 0];
        if (!k.kernel) return cudaErrorInvalidValue;
        return srmc::rtc_launch(k, P, i, grid, s->threads, st);
    }
    if (s->lp2) {
        switch (P.d) {
        case 1: return srmc::launch_step_quad_d1(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 2: return srmc::launch_step_quad_d2(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 3: return srmc::launch_step_quad_d3(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        }
        return cudaErrorInvalidValue;
    }
    if (s->dense && P.q != P.d) {
        switch (P.d * 8 + P.q) {
        case 1 * 8 + 2: return srmc::launch_step_dense_d1_q2(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 1 * 8 + 3: return srmc::launch_step_dense_d1_q3(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 1 * 8 + 4: return srmc::launch_step_dense_d1_q4(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 2 * 8 + 1: return srmc::launch_step_dense_d2_q1(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 2 * 8 + 3: return srmc::launch_step_dense_d2_q3(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 2 * 8 + 4: return srmc::launch_step_dense_d2_q4(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 3 * 8 + 1: return srmc::launch_step_dense_d3_q1(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 3 * 8 + 2: return srmc::launch_step_dense_d3_q2(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 3 * 8 + 4: return srmc::launch_step_dense_d3_q4(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 4 * 8 + 1: return srmc::launch_step_dense_d4_q1(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 4 * 8 + 2: return srmc::launch_step_dense_d4_q2(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 4 * 8 + 3: return srmc::launch_step_dense_d4_q3(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        }
        return cudaErrorInvalidValue;
    }
    if (s->dense) {
        switch (P.d) {
        case 1: return srmc::launch_step_dense_d1(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 2: return srmc::launch_step_dense_d2(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 3: return srmc::launch_step_dense_d3(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 4: return srmc::launch_step_dense_d4(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 5: return srmc::launch_step_dense_d5(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 6: return srmc::launch_step_dense_d6(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 7: return srmc::launch_step_dense_d7(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 8: return srmc::launch_step_dense_d8(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        }
        return cudaErrorInvalidValue;
    }
    if (s->exact) {
        switch (P.d) {
        case 1: return srmc::launch_step_exact_d1(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 2: return srmc::launch_step_exact_d2(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 3: return srmc::launch_step_exact_d3(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 4: return srmc::launch_step_exact_d4(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 5: return srmc::launch_step_exact_d5(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 6: return srmc::launch_step_exact_d6(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 7: return srmc::launch_step_exact_d7(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 8: return srmc::launch_step_exact_d8(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        }
        return cudaErrorInvalidValue;
    }
    if (P.kind != 0) {
        switch (P.d) {
        case 1: return srmc::launch_step_prob_d1(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 2: return srmc::launch_step_prob_d2(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 3: return srmc::launch_step_prob_d3(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 4: return srmc::launch_step_prob_d4(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 5: return srmc::launch_step_prob_d5(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 6: return srmc::launch_step_prob_d6(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 7: return srmc::launch_step_prob_d7(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        case 8: return srmc::launch_step_prob_d8(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
        }
        return cudaErrorInvalidValue;
    }
    switch (P.d) {
    case 1: return srmc::launch_step_d1(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
    case 2: return srmc::launch_step_d2(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
    case 3: return srmc::launch_step_d3(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
    case 4: return srmc::launch_step_d4(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
    case 5: return srmc::launch_step_d5(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
    case 6: return srmc::launch_step_d6(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
    case 7: return srmc::launch_step_d7(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
    case 8: return srmc::launch_step_d8(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
    case 9: return srmc::launch_step_d9(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
    case 10: return srmc::launch_step_d10(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
    case 11: return srmc::launch_step_d11(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
    case 12: return srmc::launch_step_d12(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
    case 13: return srmc::launch_step_d13(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
    case 14: return srmc::launch_step_d14(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
    case 15: return srmc::launch_step_d15(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
    case 16: return srmc::launch_step_d16(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
    case 17: return srmc::launch_step_d17(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
    case 18: return srmc::launch_step_d18(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
    case 19: return srmc::launch_step_d19(P, i, s->fp64, s->lp1, mv, grid, s->threads, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t srmc_launch_solver_step(const srmc_solver *s, int i, cudaStream_t st)
{
    return launch_step(s, i, st);
}

namespace {

// ---- kernels of the primitives and of the evaluation ----------------------

__global__ void philox_kernel(const uint32_t *ctr, uint32_t k0, uint32_t k1, long long n,
                              uint32_t *out)
{
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        unsigned c0 = ctr[4 * a], c1 = ctr[4 * a + 1], c2 = ctr[4 * a + 2], c3 = ctr[4 * a + 3];
        srmc::philox10(c0, c1, c2, c3, k0, k1);
        out[4 * a] = c0; out[4 * a + 1] = c1; out[4 * a + 2] = c2; out[4 * a + 3] = c3;
    }
}

// FP64: one word per item.  FP32: words (2t, 2t + 1) taken as a pair by the
// packed form the step kernels use for the increments of a step; a last word
// without a partner takes the scalar form (the same values).
__global__ void normals_kernel(const uint32_t *w, long long n, double *o64, float *o32)
{
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        if (o64) o64[a] = srmc::normal_of(w[a], 0.0);
    }
    if (!o32) return;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; 2 * t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const long long a = 2 * t;
#if SRMC_NORMAL_PAIRS
        if (a + 1 < n) {
            const float2 v = srmc::normal_pair(w[a], w[a + 1]);
            o32[a] = v.x;
            o32[a + 1] = v.y;
            continue;
        }
#else
        if (a + 1 < n) o32[a + 1] = srmc::normal_of(w[a + 1], 0.0f);
#endif
        o32[a] = srmc::normal_of(w[a], 0.0f);
    }
}

__global__ void locate_kernel(const Params P, const double *x64, const float *x32, long long n,
                              long long *kout)
{
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        long long k = 0;
        for (int l = 0; l < P.d; ++l) {
            int c;
            if (x64) {
                double u;
                c = srmc::cell_of(P, l, x64[a * P.d + l], u);
            } else {
                float u;
                c = srmc::cell_of(P, l, x32[a * P.d + l], u);
            }
            k += (long long)c * P.stride[l];
        }
        kout[a] = k;
    }
}

__global__ void start_points_kernel(const Params P, bool fp64, int i, long long k, long long m0,
                                    long long n, double *xout)
{
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        srmc::Words W;
        W.init(P, (unsigned)(m0 + a), (unsigned)k, (unsigned)i);
        long long rem = k;
        int pos = 0;
        for (int l = 0; l < P.d; ++l) {
            const int c = (int)(rem % P.cells[l]);
            rem /= P.cells[l];
            const int o = 3 * (P.cell_off[l] + c);
            const unsigned w = W.next_dynamic(P, pos);
            if (fp64)
                xout[a * P.d + l] = srmc::sample_cell(w, P.cellF[o], P.cellF[o + 1], P.cellF[o + 2], P.mu);
            else
                xout[a * P.d + l] = (double)srmc::sample_cell(w, P.cellF_f[o], P.cellF_f[o + 1],
                                                              P.cellF_f[o + 2], P.inv_mu_f);
        }
    }
}

__global__ void centres_kernel(const Params P, double *x)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < P.K;
         k += (long long)gridDim.x * blockDim.x) {
        long long rem = k;
        for (int l = 0; l < P.d; ++l) {
            const int c = (int)(rem % P.cells[l]);
            rem /= P.cells[l];
            x[k * P.d + l] = srmc::cell_centre(P, l, c);
        }
    }
}

__device__ double g_eval(const Params &P, const double *x)
{
    double s = 0.0;
    for (int l = 0; l < P.d; ++l) s += x[l];
    if (P.model == srmc::MODEL_COS) return cos(s / P.sqrt_d);
    if (P.model == srmc::MODEL_LOGISTIC) {
        const double w = exp(P.T + s);
        return w / (1.0 + w);
    }
    double v = P.prm[0];
    for (int l = 0; l < P.d; ++l) v += P.prm[1 + l] * x[l];
    return v;
}

// Truncated y_i, z_i from the FP64 rows, in the centred basis.
__global__ void eval_kernel(const Params P, int i, const double *x, long long n, double *y,
                            double *z)
{
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        const double *xa = x + a * P.d;
        if (i == P.N) {
            y[a] = g_eval(P, xa);
            if (z)
                for (int l = 0; l < P.q; ++l) z[a * P.q + l] = 0.0;
            continue;
        }
        double phi[srmc::PBMAX];
        phi[0] = 1.0;
        long long k = 0;
        for (int l = 0; l < P.d; ++l) {
            const int c = srmc::cell_of(P, l, xa[l], phi[1 + l]);
            k += (long long)c * P.stride[l];
        }
        srmc::add_quadratic_rt(phi, P.d, P.p);
        const long long row = (long long)i * P.K + k;
        const double *al = P.Y64 + row * P.ry64;
        double v = al[0];
        for (int c = 1; c < P.p; ++c) v += al[c] * phi[c];
        y[a] = fmin(fmax(v, -P.Cy), P.Cy);
        if (z) {
            const double *be = P.Z64 + row * P.rz64;
            for (int l = 0; l < P.q; ++l) {
                double w = be[l * P.p];
                for (int c = 1; c < P.p; ++c) w += be[l * P.p + c] * phi[c];
                z[a * P.q + l] = fmin(fmax(w, -P.Cz), P.Cz);
            }
        }
    }
}

int grid_for(long long n, int threads)
{
    long long g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 65535LL * 32) g = 65535LL * 32;
    return (int)g;
}

}  // namespace

extern "C" {

const char *srmc_last_error(void) { return g_last_error.c_str(); }

int srmc_version(void) { return 1; }

srmc_status srmc_create(const srmc_problem *pr, const srmc_strata *sa, const srmc_config *cf,
                        srmc_solver **out)
{
    if (!out) return fail(SRMC_ERR_INVALID_ARG, "srmc_create: out is NULL");
    *out = nullptr;
    if (!pr || !sa || !cf) return fail(SRMC_ERR_INVALID_ARG, "srmc_create: NULL argument");
    const int d = pr->d, q = pr->q;
    if (d < 1 || d > SRMC_DMAX) return fail(SRMC_ERR_INVALID_ARG, "d must be in [1, 19]");
    if (q < 1 || q > SRMC_DMAX) return fail(SRMC_ERR_INVALID_ARG, "q must be in [1, 19]");
    if (pr->N < 1 || pr->N > 1000000) return fail(SRMC_ERR_INVALID_ARG, "N must be in [1, 1e6]");
    if (!(pr->T > 0.0) || !std::isfinite(pr->T)) return fail(SRMC_ERR_INVALID_ARG, "T must be > 0");
    if (!pr->b || !pr->sigma) return fail(SRMC_ERR_INVALID_ARG, "b and sigma are required");
    bool dense = q != d;                 // sigma is not a diagonal d x d matrix
    for (int l = 0; l < d; ++l)
        for (int r = 0; r < q; ++r) {
            if (!std::isfinite(pr->sigma[l * q + r])) return fail(SRMC_ERR_INVALID_ARG, "sigma must be finite");
            if (l != r && pr->sigma[l * q + r] != 0.0) dense = true;
        }
    if (dense && (d > srmc::SD_DMAX || pr->dynamics != SRMC_DYN_EULER || pr->model == SRMC_MODEL_USER ||
                  cf->basis == SRMC_LP2 || sa->kind != SRMC_STRATA_EQUAL_SIZE))
        return fail(SRMC_ERR_UNSUPPORTED, "a non-diagonal sigma is built for d <= 8, Euler dynamics, "
                                          "equal-size strata, LP0/LP1 and the built-in models");
    if (q != d && (d > SRMC_DENSEQ_MAX || q > SRMC_DENSEQ_MAX))
        return fail(SRMC_ERR_UNSUPPORTED, "q != d is built for d, q <= 4");
    if (pr->model < SRMC_MODEL_COS || pr->model > SRMC_MODEL_USER)
        return fail(SRMC_ERR_INVALID_ARG, "unknown model");
    if (pr->model == SRMC_MODEL_USER && (!pr->user_source || !pr->user_source[0]))
        return fail(SRMC_ERR_INVALID_ARG, "a user model needs its source");
    if (pr->user_dynamics && pr->model != SRMC_MODEL_USER)
        return fail(SRMC_ERR_INVALID_ARG, "user_dynamics needs a user model");
    if (pr->dynamics != SRMC_DYN_EULER && pr->dynamics != SRMC_DYN_EXACT)
        return fail(SRMC_ERR_INVALID_ARG, "unknown dynamics");
    bool has_drift = false;
    for (int l = 0; l < d; ++l) {
        const double th = pr->theta ? pr->theta[l] : 0.0;
        if (!std::isfinite(th) || !std::isfinite(pr->b[l])) return fail(SRMC_ERR_INVALID_ARG, "b and theta must be finite");
        has_drift = has_drift || th != 0.0 || pr->b[l] != 0.0;
    }
    if (q != d && has_drift && pr->model == SRMC_MODEL_COS)
        return fail(SRMC_ERR_UNSUPPORTED, "the cos model's drift term needs q == d");
    if (pr->n_params < 0 || pr->n_params > SRMC_PMAX || (pr->n_params > 0 && !pr->params))
        return fail(SRMC_ERR_INVALID_ARG, "params: n_params must be in [0, 24]");
    const int need = pr->model == SRMC_MODEL_COS ? 4 : pr->model == SRMC_MODEL_AFFINE ? 3 + 2 * d : 0;
    if (pr->n_params < need) return fail(SRMC_ERR_INVALID_ARG, "too few model parameters");
    if (sa->kind != SRMC_STRATA_EQUAL_SIZE && sa->kind != SRMC_STRATA_EQUAL_PROB)
        return fail(SRMC_ERR_INVALID_ARG, "unknown strata kind");
    const bool prob = sa->kind == SRMC_STRATA_EQUAL_PROB;
    if (prob && pr->dynamics == SRMC_DYN_EXACT)
        return fail(SRMC_ERR_UNSUPPORTED, "exact dynamics are built for equal-size strata only");
    if (!sa->cells || (!prob && (!sa->lo || !sa->hi)))
        return fail(SRMC_ERR_INVALID_ARG, "strata arrays are required");
    if (!(sa->mu > 0.0) || !std::isfinite(sa->mu)) return fail(SRMC_ERR_INVALID_ARG, "mu must be > 0");
    long long K = 1, cells_total = 0;
    for (int l = 0; l < d; ++l) {
        if (sa->cells[l] < 1) return fail(SRMC_ERR_INVALID_ARG, "cells must be >= 1");
        if (!prob && (!(sa->lo[l] < sa->hi[l]) || !std::isfinite(sa->lo[l]) || !std::isfinite(sa->hi[l])))
            return fail(SRMC_ERR_INVALID_ARG, "need finite lo < hi");
        K *= sa->cells[l];
        cells_total += sa->cells[l];
        if (K > 2147483647LL) return fail(SRMC_ERR_INVALID_ARG, "too many strata (K > 2^31-1)");
    }
    {
        const int p_ = basis_dim(cf->basis, d);
        const long long rmax = std::max((long long)q * pad_to(p_, 4), (long long)pad_to(p_ * ((q + 1) / 2 * 2), 8));
        if ((long long)pr->N * K * rmax >= 4294967296LL)
            return fail(SRMC_ERR_UNSUPPORTED, "table too large: N K row-length must be < 2^32");
    }
    if (cf->basis != SRMC_LP0 && cf->basis != SRMC_LP1 && cf->basis != SRMC_LP2)
        return fail(SRMC_ERR_INVALID_ARG, "basis");
    const int p = basis_dim(cf->basis, d);
    if (cf->basis == SRMC_LP2 && (d > SRMC_LP2_DMAX || prob || pr->dynamics != SRMC_DYN_EULER))
        return fail(SRMC_ERR_UNSUPPORTED, "LP2 is built for d <= 3, equal-size strata and Euler dynamics");
    if (cf->prec != SRMC_FP32 && cf->prec != SRMC_FP64) return fail(SRMC_ERR_INVALID_ARG, "precision");
    if (d >= srmc::SRMC_WIDE_DMIN_V && (prob || pr->dynamics != SRMC_DYN_EULER || cf->prec != SRMC_FP32))
        return fail(SRMC_ERR_UNSUPPORTED,
                    "d >= 9 is built for equal-size strata, Euler dynamics and the FP32 form");
    if (d >= 12 && pr->model == SRMC_MODEL_USER)
        return fail(SRMC_ERR_UNSUPPORTED, "user models are built for d <= 11");
    if (cf->M < p) return fail(SRMC_ERR_INVALID_ARG, "M must be >= the basis dimension");
    if (cf->M > 4294967295LL) return fail(SRMC_ERR_INVALID_ARG, "M must be < 2^32");
    long long M_max = cf->M, M_sum = cf->M * K;
    if (cf->M_strata) {
        M_max = 0; M_sum = 0;
        for (long long k = 0; k < K; ++k) {
            const long long mk = cf->M_strata[k];
            if (mk < p) return fail(SRMC_ERR_INVALID_ARG, "M_strata: every M_k must be >= the basis dimension");
            if (mk > 4294967295LL) return fail(SRMC_ERR_INVALID_ARG, "M_strata: every M_k must be < 2^32");
            M_max = std::max(M_max, mk);
            M_sum += mk;
        }
    }
    int threads = cf->block_threads;
    if (threads == 0) threads = M_max >= 256 ? 256 : (int)((M_max + 31) / 32 * 32);
    if (threads < 32 || threads > srmc::MAX_THREADS || threads % 32)
        return fail(SRMC_ERR_INVALID_ARG, "block_threads must be a multiple of 32 in [32, 256]");

    if (d >= 12) {
        // the kernels of d >= 12 keep their shared memory dynamically: allow it
        // (per device, before any launch, outside stream capture)
        cudaError_t pe = cudaSuccess;
        switch (d) {
        case 12: pe = srmc::prepare_step_d12(); break;
        case 13: pe = srmc::prepare_step_d13(); break;
        case 14: pe = srmc::prepare_step_d14(); break;
        case 15: pe = srmc::prepare_step_d15(); break;
        case 16: pe = srmc::prepare_step_d16(); break;
        case 17: pe = srmc::prepare_step_d17(); break;
        case 18: pe = srmc::prepare_step_d18(); break;
        case 19: pe = srmc::prepare_step_d19(); break;
        }
        if (pe != cudaSuccess) return cuda_fail(pe, "srmc_create: shared memory of the d >= 12 kernels");
    }
    srmc_solver *s = new srmc_solver();
    Params &P = s->P;
    std::memset(&P, 0, sizeof(P));
    cudaGetDevice(&s->device);
    s->fp64 = cf->prec == SRMC_FP64;
    s->lp1 = cf->basis != SRMC_LP0;              // the kernels' affine part (LP1 and LP2)
    s->lp2 = cf->basis == SRMC_LP2;
    s->threads = threads;
    s->done_from = pr->N;
    P.d = d; P.q = q; P.N = pr->N; P.p = p;
    P.K = K; P.M = cf->M;
    s->M_sum = M_sum;
    P.model = pr->model;
    const double kapz = pr->model == SRMC_MODEL_COS ? pr->params[2] : 0.0;
    // the cos model's driver reads z when kapz != 0 or when it cancels a drift
    s->mv = pr->model == SRMC_MODEL_COS ? (kapz != 0.0 || has_drift ? srmc::MV_COS_Z : srmc::MV_COS)
          : pr->model == SRMC_MODEL_LOGISTIC ? srmc::MV_LOGISTIC : srmc::MV_AFFINE;
    s->exact = pr->dynamics == SRMC_DYN_EXACT;
    s->dense = dense;
    if (pr->model == SRMC_MODEL_USER) {
        // user model: the run-time compiled kernels read z at every path point
        s->mv = srmc::MV_COS_Z;
        s->user_source = pr->user_source;
        s->user_dynamics = pr->user_dynamics != 0;
        if (s->lp2 || prob || s->exact) {
            delete s;
            return fail(SRMC_ERR_UNSUPPORTED, "user models: LP0/LP1, equal-size strata, Euler dynamics");
        }
        std::string log;
        if (!srmc::rtc_compile(s->user_source, d, s->fp64, s->lp1, false, s->user_dynamics, s->rtc[0], log)) {
            delete s;
            return fail(SRMC_ERR_INVALID_ARG, "user model: " + log);
        }
    }
    P.drift = pr->model == SRMC_MODEL_COS && has_drift ? 1 : 0;
    // The step kernels take these paddings as constants of their basis dimension (row_pad).
    P.ry32 = pad_to(p, 4); P.rz32 = pad_to(q * p, 4);
    P.ry64 = pad_to(p, 2); P.rz64 = pad_to(q * p, 2);
    P.ph = (q + 1) / 2 * 2; P.rc16 = pad_to(p * P.ph, 8);
    int stride = 1;
    int off = 0;
    P.kind = prob ? 1 : 0;
    for (int l = 0; l < d; ++l) {
        P.cells[l] = sa->cells[l];
        P.stride[l] = stride;
        P.kbias += 0x4B000000u * (unsigned)stride;     // wraps mod 2^32 (see locate_point)
        stride *= sa->cells[l];
        P.cell_off[l] = off; off += sa->cells[l];
        // (equal-probability strata use the per-cell table; lo = 0, h = 1 unused)
        const double lo = prob ? 0.0 : sa->lo[l], hi = prob ? (double)sa->cells[l] : sa->hi[l];
        P.lo[l] = lo;
        P.h[l] = (hi - lo) / (double)sa->cells[l];
        P.b[l] = pr->b[l];
        P.sig[l] = l < q ? pr->sigma[l * q + l] : 0.0;
        P.lo_f[l] = (float)lo;
        P.r_f[l] = (float)((double)sa->cells[l] / (hi - lo));
        P.b_f[l] = (float)pr->b[l];
        P.sig_f[l] = (float)P.sig[l];
    }
    P.T = pr->T;
    P.dt = pr->T / (double)pr->N;
    for (int l = 0; l < d; ++l) {
        const double th = pr->theta ? pr->theta[l] : 0.0;
        P.theta[l] = th;
        if (s->exact) {
            double A, B, r;
            ou_transition(th, P.dt, A, B, r);
            P.A[l] = A; P.c[l] = pr->b[l] * B; P.s1[l] = P.sig[l] * B / P.dt; P.s2[l] = P.sig[l] * r;
        } else {
            P.A[l] = 1.0 - th * P.dt; P.c[l] = pr->b[l] * P.dt; P.s1[l] = P.sig[l]; P.s2[l] = 0.0;
        }
        P.A_f[l] = (float)P.A[l]; P.c_f[l] = (float)P.c[l];
        P.s1_f[l] = (float)P.s1[l]; P.s2_f[l] = (float)P.s2[l]; P.theta_f[l] = (float)th;
    }
    if (dense) {                         // row-major d x q, read at l q + r
        P.dense = 1;
        for (int l = 0; l < d; ++l)
            for (int r = 0; r < q; ++r) {
                P.sd[l * q + r] = pr->sigma[l * q + r];
                P.sd_f[l * q + r] = (float)pr->sigma[l * q + r];
            }
    }
    P.unit_drift = 1;
    for (int l = 0; l < d; ++l) P.unit_drift &= (P.A_f[l] == 1.0f && P.c_f[l] == 0.0f) ? 1 : 0;
    if (P.drift) {
        if (!(pr->params[3] != 0.0)) {
            delete s;
            return fail(SRMC_ERR_INVALID_ARG, "the cos model with a drift needs s0 != 0");
        }
        P.inv_s0 = 1.0 / pr->params[3];
        P.inv_s0_f = (float)P.inv_s0;
    }
    P.sdt = std::sqrt(P.dt);
    P.mu = sa->mu;
    P.sqrt_d = std::sqrt((double)d);
    P.dt_f = (float)P.dt; P.sdt_f = (float)P.sdt;
    P.inv_mu_f = (float)(1.0 / sa->mu);
    P.mu_f = (float)sa->mu;
    P.inv_sqrt_d_f = (float)(1.0 / std::sqrt((double)d));
    const double inf = std::numeric_limits<double>::infinity();
    P.Cy = cf->Cy > 0.0 ? cf->Cy : inf;
    P.Cz = cf->Cz > 0.0 ? cf->Cz : inf;
    P.Cy_f = (float)P.Cy; P.Cz_f = (float)P.Cz;
    P.key0 = (unsigned)(cf->seed & 0xFFFFFFFFull) ^ cf->instance;
    P.key1 = (unsigned)(cf->seed >> 32);
    for (int r = 0; r < 10; ++r) {
        P.rk0[r] = P.key0 + (unsigned)r * 0x9E3779B9u;
        P.rk1[r] = P.key1 + (unsigned)r * 0xBB67AE85u;
    }
    for (int a = 0; a < pr->n_params; ++a) { P.prm[a] = pr->params[a]; P.prm_f[a] = (float)pr->params[a]; }
    if (pr->model == SRMC_MODEL_COS) {
        P.lin = pr->params[0] + 0.5 * pr->params[3] * pr->params[3];
        P.lin_f = (float)P.lin;
    }

    // Sampler constants of every cell side (Alg. 3): F(x-), 1 - F(x+), F(x+) - F(x-);
    // per-cell edges, basis centre and 1/unit (the centred LP1 coordinate).
    std::vector<double> cellF(3 * cells_total), cellB(4 * cells_total);
    std::vector<float> cellF_f(3 * cells_total), cellB_f(4 * cells_total);
    for (int l = 0; l < d; ++l) {
        const int C = sa->cells[l];
        for (int c = 0; c < C; ++c) {
            double xlo, xhi, Flo, Fchi, w, ctr, unit;
            if (prob) {
                // equal nu-probability cells: edges at the logistic quantiles c/C,
                // so F(x-) = c/C and 1 - F(x+) = (C-c-1)/C exactly
                xlo = c == 0 ? -inf : logistic_quantile((double)c, (double)(C - c), sa->mu);
                xhi = c == C - 1 ? inf : logistic_quantile((double)(c + 1), (double)(C - c - 1), sa->mu);
                Flo = (double)c / (double)C;
                Fchi = (double)(C - c - 1) / (double)C;
                w = 1.0 / (double)C;
                ctr = logistic_quantile(c + 0.5, C - c - 0.5, sa->mu);
                unit = logistic_quantile(c + 0.75, C - c - 0.75, sa->mu) -
                       logistic_quantile(c + 0.25, C - c - 0.25, sa->mu);
            } else {
                const double h = P.h[l];
                xlo = c == 0 ? -inf : sa->lo[l] + (double)c * h;
                xhi = c == C - 1 ? inf : sa->lo[l] + (double)(c + 1) * h;
                Flo = logistic_cdf(xlo, sa->mu);
                Fchi = logistic_cdf(-xhi, sa->mu);
                w = xlo > 0.0 ? logistic_cdf(-xlo, sa->mu) - Fchi : logistic_cdf(xhi, sa->mu) - Flo;
                ctr = sa->lo[l] + ((double)c + 0.5) * h;
                unit = 0.5 * h;
            }
            const int o = 3 * (P.cell_off[l] + c);
            cellF[o] = Flo; cellF[o + 1] = Fchi; cellF[o + 2] = w;
            cellF_f[o] = (float)Flo; cellF_f[o + 1] = (float)Fchi; cellF_f[o + 2] = (float)w;
            const int b = 4 * (P.cell_off[l] + c);
            cellB[b] = xlo; cellB[b + 1] = xhi; cellB[b + 2] = ctr; cellB[b + 3] = 1.0 / unit;
            for (int a = 0; a < 4; ++a) cellB_f[b + a] = (float)cellB[b + a];
        }
    }
    // Per-step driver constants of the cos model: kap e_j^2, kapz s0^2 e_j^2.
    std::vector<double> stepc(2 * (pr->N + 1), 0.0);
    std::vector<float> stepc_f(2 * (pr->N + 1), 0.0f);
    if (pr->model == SRMC_MODEL_COS) {
        const double lam = pr->params[0], kap = pr->params[1], s0 = pr->params[3];
        for (int j = 0; j <= pr->N; ++j) {
            const double tj = (double)j * P.dt;
            const double e = std::exp(lam * (pr->T - tj));
            stepc[2 * j] = kap * e * e;
            stepc[2 * j + 1] = kapz * s0 * s0 * e * e;
            stepc_f[2 * j] = (float)stepc[2 * j];
            stepc_f[2 * j + 1] = (float)stepc[2 * j + 1];
        }
    }

    auto bail = [&](cudaError_t e, const char *what) {
        free_all(s);
        delete s;
        return cuda_fail(e, what);
    };
    cudaError_t e;
    const size_t rows = (size_t)pr->N * (size_t)K;
    if ((e = cudaMalloc(&s->cellF, sizeof(double) * cellF.size())) != cudaSuccess) return bail(e, "cudaMalloc");
    if ((e = cudaMalloc(&s->cellF_f, sizeof(float) * cellF_f.size())) != cudaSuccess) return bail(e, "cudaMalloc");
    if ((e = cudaMalloc(&s->cellB, sizeof(double) * cellB.size())) != cudaSuccess) return bail(e, "cudaMalloc");
    if ((e = cudaMalloc(&s->cellB_f, sizeof(float) * cellB_f.size())) != cudaSuccess) return bail(e, "cudaMalloc");
    if ((e = cudaMalloc(&s->stepc, sizeof(double) * stepc.size())) != cudaSuccess) return bail(e, "cudaMalloc");
    if ((e = cudaMalloc(&s->stepc_f, sizeof(float) * stepc_f.size())) != cudaSuccess) return bail(e, "cudaMalloc");
    if ((e = cudaMalloc(&s->Y64, sizeof(double) * rows * P.ry64)) != cudaSuccess) return bail(e, "cudaMalloc Y64");
    if ((e = cudaMalloc(&s->Z64, sizeof(double) * rows * P.rz64)) != cudaSuccess) return bail(e, "cudaMalloc Z64");
    if (!s->fp64) {
        if ((e = cudaMalloc(&s->Y32, sizeof(float) * rows * P.ry32)) != cudaSuccess) return bail(e, "cudaMalloc Y32");
        if ((e = cudaMalloc(&s->Z32, sizeof(float) * rows * P.rz32)) != cudaSuccess) return bail(e, "cudaMalloc Z32");
    }
    if ((e = cudaMalloc(&s->stats, sizeof(unsigned long long) * 4)) != cudaSuccess) return bail(e, "cudaMalloc");
    if ((e = cudaMemcpy(s->cellF, cellF.data(), sizeof(double) * cellF.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return bail(e, "cudaMemcpy");
    if ((e = cudaMemcpy(s->cellF_f, cellF_f.data(), sizeof(float) * cellF_f.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return bail(e, "cudaMemcpy");
    if ((e = cudaMemcpy(s->cellB, cellB.data(), sizeof(double) * cellB.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return bail(e, "cudaMemcpy");
    if ((e = cudaMemcpy(s->cellB_f, cellB_f.data(), sizeof(float) * cellB_f.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return bail(e, "cudaMemcpy");
    if ((e = cudaMemcpy(s->stepc, stepc.data(), sizeof(double) * stepc.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return bail(e, "cudaMemcpy");
    if ((e = cudaMemcpy(s->stepc_f, stepc_f.data(), sizeof(float) * stepc_f.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return bail(e, "cudaMemcpy");
    if ((e = cudaMemset(s->Y64, 0, sizeof(double) * rows * P.ry64)) != cudaSuccess) return bail(e, "cudaMemset");
    if ((e = cudaMemset(s->Z64, 0, sizeof(double) * rows * P.rz64)) != cudaSuccess) return bail(e, "cudaMemset");
    if (s->Y32 && (e = cudaMemset(s->Y32, 0, sizeof(float) * rows * P.ry32)) != cudaSuccess) return bail(e, "cudaMemset");
    if (s->Z32 && (e = cudaMemset(s->Z32, 0, sizeof(float) * rows * P.rz32)) != cudaSuccess) return bail(e, "cudaMemset");
    if ((e = cudaMemset(s->stats, 0, sizeof(unsigned long long) * 4)) != cudaSuccess) return bail(e, "cudaMemset");
    P.cellF = s->cellF; P.cellF_f = s->cellF_f; P.stepc = s->stepc; P.stepc_f = s->stepc_f;
    P.cellB = s->cellB; P.cellB_f = s->cellB_f;
    P.Y32 = s->Y32; P.Z32 = s->Z32; P.Y64 = s->Y64; P.Z64 = s->Z64; P.stats = s->stats;
    if (cf->M_strata) {
        std::vector<unsigned> mk((size_t)K);
        for (long long k = 0; k < K; ++k) mk[(size_t)k] = (unsigned)cf->M_strata[k];
        if ((e = cudaMalloc(&s->Mk, sizeof(unsigned) * mk.size())) != cudaSuccess) return bail(e, "cudaMalloc M_strata");
        if ((e = cudaMemcpy(s->Mk, mk.data(), sizeof(unsigned) * mk.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(e, "cudaMemcpy M_strata");
        P.Mk = s->Mk;
    }
    if (d >= SRMC_ORDER_MIN_D && K > 1 && K <= SRMC_ORDER_MAX_K) {
        const std::vector<unsigned> order = morton_order(sa->cells, d, K);
        if ((e = cudaMalloc(&s->order, sizeof(unsigned) * order.size())) != cudaSuccess) return bail(e, "cudaMalloc order");
        if ((e = cudaMemcpy(s->order, order.data(), sizeof(unsigned) * order.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(e, "cudaMemcpy order");
        P.order = s->order;
    }
    *out = s;
    g_last_error.clear();
    return SRMC_OK;
}

void srmc_destroy(srmc_solver *s)
{
    if (!s) return;
    free_all(s);
    delete s;
}

srmc_status srmc_solve_step(srmc_solver *s, int i, void *stream)
{
    if (!s) return fail(SRMC_ERR_INVALID_ARG, "srmc_solve_step: NULL solver");
    if (i < 0 || i >= s->P.N) return fail(SRMC_ERR_INVALID_ARG, "srmc_solve_step: i out of range");
    if (s->done_from > i + 1) return fail(SRMC_ERR_STATE, "srmc_solve_step: steps > i not solved yet");
    SRMC_CUDA(launch_step(s, i, (cudaStream_t)stream), "step kernel launch");
    if (i < s->done_from) s->done_from = i;
    return SRMC_OK;
}

srmc_status srmc_solve(srmc_solver *s, void *stream)
{
    if (!s) return fail(SRMC_ERR_INVALID_ARG, "srmc_solve: NULL solver");
    if (!s->graph) {
        if (!s->cap_stream)
            SRMC_CUDA(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking), "graph stream");
        cudaGraph_t g = nullptr;
        SRMC_CUDA(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t le = cudaSuccess;
        for (int i = s->P.N - 1; i >= 0 && le == cudaSuccess; --i) le = launch_step(s, i, s->cap_stream);
        cudaError_t ce = cudaStreamEndCapture(s->cap_stream, &g);
        if (le != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(le, "step kernel capture"); }
        if (ce != cudaSuccess) return cuda_fail(ce, "end capture");
        cudaError_t ie = cudaGraphInstantiate(&s->graph, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) { s->graph = nullptr; return cuda_fail(ie, "graph instantiate"); }
    }
    SRMC_CUDA(cudaGraphLaunch(s->graph, (cudaStream_t)stream), "graph launch");
    s->done_from = 0;
    return SRMC_OK;
}

namespace {
__device__ void closed_form(const Params &P, int i, const double *x, double &u, double *zs)
{
    const double t = (double)i * P.dt;
    double sx = 0.0;
    for (int l = 0; l < P.d; ++l) sx += x[l];
    if (P.model == srmc::MODEL_COS) {
        const double e = exp(P.prm[0] * (P.T - t));
        const double s = sx / P.sqrt_d;
        u = e * cos(s);
        for (int l = 0; l < P.q; ++l) zs[l] = -P.prm[3] * e * sin(s) / P.sqrt_d;
    } else {
        // w = exp(a), a = t + sum x: u = w/(1+w), z_l = w/(1+w)^2, written with
        // e = exp(-|a|) <= 1 so that no intermediate overflows
        const double a = t + sx;
        const double e = exp(-fabs(a));
        u = a >= 0.0 ? 1.0 / (1.0 + e) : e / (1.0 + e);
        for (int l = 0; l < P.q; ++l) zs[l] = e / ((1.0 + e) * (1.0 + e));
    }
}

// Squared errors of y_i, z_i against the closed form at the points
// x[i][a][d], a < n, summed per step into out[2 i] (y) and out[2 i + 1]
// (|z|^2 over the q components); grid (blocks per step, steps), out cleared.
__global__ void point_error_kernel(const Params P, const double *x, long long n, double *out)
{
    __shared__ double red[2][32];
    for (int i = blockIdx.y; i < P.N; i += gridDim.y) {
        double ysq = 0.0, zsq = 0.0;
        for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
             a += (long long)gridDim.x * blockDim.x) {
            const double *xa = x + ((long long)i * n + a) * P.d;
            double phi[srmc::PBMAX], zs[srmc::DMAX], u;
            phi[0] = 1.0;
            long long k = 0;
            for (int l = 0; l < P.d; ++l) {
                const int c = srmc::cell_of(P, l, xa[l], phi[1 + l]);
                k += (long long)c * P.stride[l];
            }
            srmc::add_quadratic_rt(phi, P.d, P.p);
            closed_form(P, i, xa, u, zs);
            const long long row = (long long)i * P.K + k;
            const double *al = P.Y64 + row * P.ry64;
            double v = al[0];
            for (int c = 1; c < P.p; ++c) v += al[c] * phi[c];
            const double dy = fmin(fmax(v, -P.Cy), P.Cy) - u;
            ysq += dy * dy;
            const double *be = P.Z64 + row * P.rz64;
            for (int l = 0; l < P.q; ++l) {
                double w = be[l * P.p];
                for (int c = 1; c < P.p; ++c) w += be[l * P.p + c] * phi[c];
                const double dz = fmin(fmax(w, -P.Cz), P.Cz) - zs[l];
                zsq += dz * dz;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            ysq += __shfl_xor_sync(0xffffffffu, ysq, o);
            zsq += __shfl_xor_sync(0xffffffffu, zsq, o);
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) { red[0][warp] = ysq; red[1][warp] = zsq; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, b = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += red[0][w]; b += red[1][w]; }
            atomicAdd(out + 2 * i, a);
            atomicAdd(out + 2 * i + 1, b);
        }
        __syncthreads();                               // red is reused for the next step
    }
}

// One block per step: errors of y_i, z_i at every stratum centre.
__global__ void closed_form_error_kernel(const Params P, bool inner, double *out)
{
    const int i = blockIdx.x;
    double ymax = 0.0, ysq = 0.0, zmax = 0.0, zsq = 0.0;
    long long cnt = 0;
    for (long long k = threadIdx.x; k < P.K; k += blockDim.x) {
        double x[srmc::DMAX], phi[srmc::PBMAX], zs[srmc::DMAX], u;
        long long rem = k;
        phi[0] = 1.0;
        bool outer = false;
        for (int l = 0; l < P.d; ++l) {
            const int c = (int)(rem % P.cells[l]);
            rem /= P.cells[l];
            outer = outer || c == 0 || c == P.cells[l] - 1;
            x[l] = srmc::cell_centre(P, l, c);
            phi[1 + l] = 0.0;                    // the basis centre of the cell
        }
        srmc::add_quadratic_rt(phi, P.d, P.p);
        if (inner && outer) continue;
        ++cnt;
        closed_form(P, i, x, u, zs);
        const long long row = (long long)i * P.K + k;
        const double *al = P.Y64 + row * P.ry64;
        double v = al[0];
        for (int c = 1; c < P.p; ++c) v += al[c] * phi[c];
        const double dy = fmin(fmax(v, -P.Cy), P.Cy) - u;
        ymax = fmax(ymax, fabs(dy));
        ysq += dy * dy;
        const double *be = P.Z64 + row * P.rz64;
        for (int l = 0; l < P.q; ++l) {
            double w = be[l * P.p];
            for (int c = 1; c < P.p; ++c) w += be[l * P.p + c] * phi[c];
            const double dz = fmin(fmax(w, -P.Cz), P.Cz) - zs[l];
            zmax = fmax(zmax, fabs(dz));
            zsq += dz * dz;
        }
    }
    __shared__ double red[5][32];
    double cntd = (double)cnt;
    for (int o = 16; o > 0; o >>= 1) {
        ymax = fmax(ymax, __shfl_xor_sync(0xffffffffu, ymax, o));
        ysq += __shfl_xor_sync(0xffffffffu, ysq, o);
        zmax = fmax(zmax, __shfl_xor_sync(0xffffffffu, zmax, o));
        zsq += __shfl_xor_sync(0xffffffffu, zsq, o);
        cntd += __shfl_xor_sync(0xffffffffu, cntd, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][warp] = ymax; red[1][warp] = ysq; red[2][warp] = zmax; red[3][warp] = zsq;
        red[4][warp] = cntd;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, c = 0, e = 0, n = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a = fmax(a, red[0][w]); b += red[1][w]; c = fmax(c, red[2][w]); e += red[3][w]; n += red[4][w];
        }
        out[4 * i + 0] = a;
        out[4 * i + 1] = b / n;
        out[4 * i + 2] = c;
        out[4 * i + 3] = e / n;
    }
}
}  // namespace

srmc_status srmc_closed_form_error(const srmc_solver *s, double *out, void *stream)
{
    if (!s || !out) return fail(SRMC_ERR_INVALID_ARG, "srmc_closed_form_error: NULL argument");
    if (s->P.model == srmc::MODEL_AFFINE || s->P.model == srmc::MODEL_USER)
        return fail(SRMC_ERR_UNSUPPORTED, "srmc_closed_form_error: no closed form for the affine and user models");
    if (s->dense) return fail(SRMC_ERR_UNSUPPORTED, "srmc_closed_form_error: no closed form with a non-diagonal sigma");
    if (s->done_from > 0) return fail(SRMC_ERR_STATE, "srmc_closed_form_error: solve not finished");
    closed_form_error_kernel<<<s->P.N, 256, 0, (cudaStream_t)stream>>>(s->P, false, out);
    SRMC_CUDA(cudaGetLastError(), "closed form error kernel launch");
    return SRMC_OK;
}

srmc_status srmc_point_error(const srmc_solver *s, const double *x, long long n, double *out, void *stream)
{
    if (!s || !out) return fail(SRMC_ERR_INVALID_ARG, "srmc_point_error: NULL argument");
    if (n < 0) return fail(SRMC_ERR_INVALID_ARG, "srmc_point_error: n < 0");
    if (n > 0 && !x) return fail(SRMC_ERR_INVALID_ARG, "srmc_point_error: NULL points");
    if (s->P.model == srmc::MODEL_AFFINE || s->P.model == srmc::MODEL_USER)
        return fail(SRMC_ERR_UNSUPPORTED, "srmc_point_error: no closed form for the affine and user models");
    if (s->dense) return fail(SRMC_ERR_UNSUPPORTED, "srmc_point_error: no closed form with a non-diagonal sigma");
    if (s->done_from > 0) return fail(SRMC_ERR_STATE, "srmc_point_error: solve not finished");
    SRMC_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * 2 * (size_t)s->P.N, (cudaStream_t)stream),
              "srmc_point_error: clear");
    if (n == 0) return SRMC_OK;
    long long bx = (n + 255) / 256;
    if (bx > 64) bx = 64;
    const unsigned by = (unsigned)(s->P.N < 65535 ? s->P.N : 65535);
    point_error_kernel<<<dim3((unsigned)bx, by), 256, 0, (cudaStream_t)stream>>>(s->P, x, n, out);
    SRMC_CUDA(cudaGetLastError(), "point error kernel launch");
    return SRMC_OK;
}

srmc_status srmc_closed_form_error_inner(const srmc_solver *s, double *out, void *stream)
{
    if (!s || !out) return fail(SRMC_ERR_INVALID_ARG, "srmc_closed_form_error_inner: NULL argument");
    if (s->P.model == srmc::MODEL_AFFINE || s->P.model == srmc::MODEL_USER)
        return fail(SRMC_ERR_UNSUPPORTED, "srmc_closed_form_error_inner: no closed form for the affine and user models");
    if (s->dense) return fail(SRMC_ERR_UNSUPPORTED, "srmc_closed_form_error_inner: no closed form with a non-diagonal sigma");
    for (int l = 0; l < s->P.d; ++l)
        if (s->P.cells[l] < 3) return fail(SRMC_ERR_INVALID_ARG, "srmc_closed_form_error_inner: no inner strata");
    if (s->done_from > 0) return fail(SRMC_ERR_STATE, "srmc_closed_form_error_inner: solve not finished");
    closed_form_error_kernel<<<s->P.N, 256, 0, (cudaStream_t)stream>>>(s->P, true, out);
    SRMC_CUDA(cudaGetLastError(), "closed form error kernel launch");
    return SRMC_OK;
}

srmc_status srmc_eval(const srmc_solver *s, int i, const double *x, long long n, double *y,
                      double *z, void *stream)
{
    if (!s) return fail(SRMC_ERR_INVALID_ARG, "srmc_eval: NULL solver");
    if (i < 0 || i > s->P.N) return fail(SRMC_ERR_INVALID_ARG, "srmc_eval: i out of range");
    if (n < 0) return fail(SRMC_ERR_INVALID_ARG, "srmc_eval: n < 0");
    if (n == 0) return SRMC_OK;
    if (!x || !y) return fail(SRMC_ERR_INVALID_ARG, "srmc_eval: NULL buffer");
    if (i < s->P.N && s->done_from > i) return fail(SRMC_ERR_STATE, "srmc_eval: step i not solved");
    if (i == s->P.N && s->P.model == srmc::MODEL_USER)
        return fail(SRMC_ERR_UNSUPPORTED, "srmc_eval: g of a user model is not evaluated here (i == N)");
    eval_kernel<<<grid_for(n, 128), 128, 0, (cudaStream_t)stream>>>(s->P, i, x, n, y, z);
    SRMC_CUDA(cudaGetLastError(), "eval kernel launch");
    return SRMC_OK;
}

srmc_status srmc_centres(const srmc_solver *s, double *x, void *stream)
{
    if (!s || !x) return fail(SRMC_ERR_INVALID_ARG, "srmc_centres: NULL argument");
    centres_kernel<<<grid_for(s->P.K, 128), 128, 0, (cudaStream_t)stream>>>(s->P, x);
    SRMC_CUDA(cudaGetLastError(), "centres kernel launch");
    return SRMC_OK;
}

srmc_status srmc_table(const srmc_solver *s, const double **y64, const double **z64, int *p,
                       int *ry, int *rz, long long *K)
{
    if (!s) return fail(SRMC_ERR_INVALID_ARG, "srmc_table: NULL solver");
    if (y64) *y64 = s->Y64;
    if (z64) *z64 = s->Z64;
    if (p) *p = s->P.p;
    if (ry) *ry = s->P.ry64;
    if (rz) *rz = s->P.rz64;
    if (K) *K = s->P.K;
    return SRMC_OK;
}

srmc_status srmc_read_table(const srmc_solver *s, double *dst_y, double *dst_z, void *stream)
{
    if (!s) return fail(SRMC_ERR_INVALID_ARG, "srmc_read_table: NULL solver");
    const size_t rows = (size_t)s->P.N * (size_t)s->P.K;
    if (dst_y)
        SRMC_CUDA(cudaMemcpyAsync(dst_y, s->Y64, sizeof(double) * rows * s->P.ry64, cudaMemcpyDefault,
                                  (cudaStream_t)stream), "srmc_read_table: copy y");
    if (dst_z)
        SRMC_CUDA(cudaMemcpyAsync(dst_z, s->Z64, sizeof(double) * rows * s->P.rz64, cudaMemcpyDefault,
                                  (cudaStream_t)stream), "srmc_read_table: copy z");
    return SRMC_OK;
}

namespace {
// FP32 copies (round to nearest) of the K rows of one step of the FP64 tables.
__global__ void rows_to_fp32_kernel(const Params P, long long off)
{
    const int qp = P.q * P.p;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < P.K;
         r += (long long)gridDim.x * blockDim.x) {
        const long long row = off + r;
        for (int a = 0; a < P.p; ++a) P.Y32[row * P.ry32 + a] = (float)P.Y64[row * P.ry64 + a];
        for (int a = 0; a < qp; ++a) P.Z32[row * P.rz32 + a] = (float)P.Z64[row * P.rz64 + a];
    }
}
}  // namespace

srmc_status srmc_set_rows(srmc_solver *s, int i, const double *src_y, const double *src_z, void *stream)
{
    if (!s || !src_y || !src_z) return fail(SRMC_ERR_INVALID_ARG, "srmc_set_rows: NULL argument");
    if (i < 0 || i >= s->P.N) return fail(SRMC_ERR_INVALID_ARG, "srmc_set_rows: i out of range");
    const cudaStream_t st = (cudaStream_t)stream;
    const size_t K = (size_t)s->P.K, off = (size_t)i * K;
    SRMC_CUDA(cudaMemcpyAsync(s->Y64 + off * s->P.ry64, src_y, sizeof(double) * K * s->P.ry64, cudaMemcpyDefault,
                              st), "srmc_set_rows: copy y");
    SRMC_CUDA(cudaMemcpyAsync(s->Z64 + off * s->P.rz64, src_z, sizeof(double) * K * s->P.rz64, cudaMemcpyDefault,
                              st), "srmc_set_rows: copy z");
    if (s->P.Y32) {
        const int grid = (int)std::min<size_t>((K + 255) / 256, 65535);
        rows_to_fp32_kernel<<<grid, 256, 0, st>>>(s->P, (long long)off);
        SRMC_CUDA(cudaGetLastError(), "srmc_set_rows: FP32 copies");
    }
    if (i + 1 == s->done_from) s->done_from = i;      // steps i..N-1 are present
    return SRMC_OK;
}

namespace {
// [N][K][q][p] -> padded rows of the FP64 table and of the binary16 table of
// the FP32 form (round to nearest even, saturated at +-65504).
__global__ void repack_control_kernel(const Params P, const double *src, double *c64, __half *c16)
{
    const long long rows = (long long)P.N * P.K;
    const int qp = P.q * P.p;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows;
         r += (long long)gridDim.x * blockDim.x) {
        for (int a = 0; a < qp; ++a) {
            const double v = src[r * qp + a];
            c64[r * P.rz64 + a] = v;
            c16[r * P.rc16 + srmc::c16_index(P, a / P.p, a % P.p)] = __double2half(fmin(fmax(v, -65504.0), 65504.0));
        }
    }
}
}  // namespace

srmc_status srmc_set_control(srmc_solver *s, const double *rows)
{
    if (!s || !rows) return fail(SRMC_ERR_INVALID_ARG, "srmc_set_control: NULL argument");
    if (!s->lp1) return fail(SRMC_ERR_UNSUPPORTED, "srmc_set_control: LP1 solvers only");
    if (s->mv == srmc::MV_AFFINE) return fail(SRMC_ERR_UNSUPPORTED, "srmc_set_control: not for the affine model");
    if (s->P.d >= srmc::SRMC_WIDE_DMIN_V) return fail(SRMC_ERR_UNSUPPORTED, "srmc_set_control: d <= 8 only");
    if (const int st = srmc_prepare_user_control(s)) return (srmc_status)st;
    const size_t nrow = (size_t)s->P.N * (size_t)s->P.K;
    const size_t n = nrow * (size_t)(s->P.q * s->P.p);
    if (!s->C64) {
        SRMC_CUDA(cudaMalloc(&s->C64, sizeof(double) * nrow * s->P.rz64), "cudaMalloc control");
        SRMC_CUDA(cudaMalloc(&s->C16, sizeof(__half) * nrow * s->P.rc16), "cudaMalloc control");
        SRMC_CUDA(cudaMemset(s->C64, 0, sizeof(double) * nrow * s->P.rz64), "cudaMemset control");
        SRMC_CUDA(cudaMemset(s->C16, 0, sizeof(__half) * nrow * s->P.rc16), "cudaMemset control");
    }
    double *staging = nullptr;
    SRMC_CUDA(cudaMalloc(&staging, sizeof(double) * n), "cudaMalloc control staging");
    cudaError_t e = cudaMemcpy(staging, rows, sizeof(double) * n, cudaMemcpyDefault);
    if (e == cudaSuccess) {
        repack_control_kernel<<<grid_for((long long)nrow, 256), 256>>>(s->P, staging, s->C64, s->C16);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(staging);
    if (e != cudaSuccess) return cuda_fail(e, "srmc_set_control");
    s->cv = true;
    s->cv_own = false;
    if (s->graph) { cudaGraphExecDestroy(s->graph); s->graph = nullptr; }
    return SRMC_OK;
}

srmc_status srmc_read_control(const srmc_solver *s, double *rows)
{
    if (!s || !rows) return fail(SRMC_ERR_INVALID_ARG, "srmc_read_control: NULL argument");
    if (!s->cv || s->cv_own || !s->C64)
        return fail(SRMC_ERR_STATE, "srmc_read_control: no control rows installed");
    const size_t nrow = (size_t)s->P.N * (size_t)s->P.K, qp = (size_t)(s->P.q * s->P.p);
    SRMC_CUDA(cudaMemcpy2D(rows, qp * sizeof(double), s->C64, (size_t)s->P.rz64 * sizeof(double),
                           qp * sizeof(double), nrow, cudaMemcpyDefault), "srmc_read_control");
    return SRMC_OK;
}

srmc_status srmc_set_own_control(srmc_solver *s)
{
    if (!s) return fail(SRMC_ERR_INVALID_ARG, "srmc_set_own_control: NULL solver");
    if (!s->lp1) return fail(SRMC_ERR_UNSUPPORTED, "srmc_set_own_control: LP1 solvers only");
    if (s->mv == srmc::MV_AFFINE)
        return fail(SRMC_ERR_UNSUPPORTED, "srmc_set_own_control: not for the affine model");
    if (s->P.d >= srmc::SRMC_WIDE_DMIN_V)
        return fail(SRMC_ERR_UNSUPPORTED, "srmc_set_own_control: d <= 8 only");
    if (const int st = srmc_prepare_user_control(s)) return (srmc_status)st;
    s->cv = true;
    s->cv_own = true;
    if (s->graph) { cudaGraphExecDestroy(s->graph); s->graph = nullptr; }
    return SRMC_OK;
}

srmc_status srmc_clear_control(srmc_solver *s)
{
    if (!s) return fail(SRMC_ERR_INVALID_ARG, "srmc_clear_control: NULL solver");
    s->cv = false;
    s->cv_own = false;
    if (s->graph) { cudaGraphExecDestroy(s->graph); s->graph = nullptr; }
    return SRMC_OK;
}

srmc_status srmc_stats(const srmc_solver *s, unsigned long long out[3])
{
    if (!s || !out) return fail(SRMC_ERR_INVALID_ARG, "srmc_stats: NULL argument");
    unsigned long long h[4];
    SRMC_CUDA(cudaDeviceSynchronize(), "srmc_stats: synchronize");
    SRMC_CUDA(cudaMemcpy(h, s->stats, sizeof(h), cudaMemcpyDeviceToHost), "srmc_stats: copy");
    out[0] = h[0];
    out[1] = h[1];
    long long steps = 0;
    for (int i = s->done_from; i < s->P.N; ++i) steps += (long long)(s->P.N - i);
    out[2] = (unsigned long long)(steps * s->M_sum);
    return SRMC_OK;
}

srmc_status srmc_philox(const uint32_t *ctr, const uint32_t key[2], long long n, uint32_t *out,
                        void *stream)
{
    if (n < 0 || !key) return fail(SRMC_ERR_INVALID_ARG, "srmc_philox: bad argument");
    if (n == 0) return SRMC_OK;
    if (!ctr || !out) return fail(SRMC_ERR_INVALID_ARG, "srmc_philox: NULL buffer");
    philox_kernel<<<grid_for(n, 128), 128, 0, (cudaStream_t)stream>>>(ctr, key[0], key[1], n, out);
    SRMC_CUDA(cudaGetLastError(), "philox kernel launch");
    return SRMC_OK;
}

srmc_status srmc_normals(const uint32_t *w, long long n, double *o64, float *o32, void *stream)
{
    if (n < 0) return fail(SRMC_ERR_INVALID_ARG, "srmc_normals: n < 0");
    if (n == 0) return SRMC_OK;
    if (!w || (!o64 && !o32)) return fail(SRMC_ERR_INVALID_ARG, "srmc_normals: NULL buffer");
    normals_kernel<<<grid_for(n, 128), 128, 0, (cudaStream_t)stream>>>(w, n, o64, o32);
    SRMC_CUDA(cudaGetLastError(), "normals kernel launch");
    return SRMC_OK;
}

srmc_status srmc_locate(const srmc_solver *s, const double *x64, const float *x32, long long n,
                        long long *k, void *stream)
{
    if (!s || n < 0) return fail(SRMC_ERR_INVALID_ARG, "srmc_locate: bad argument");
    if (n == 0) return SRMC_OK;
    if (!k || (!x64 == !x32)) return fail(SRMC_ERR_INVALID_ARG, "srmc_locate: need exactly one of x64, x32");
    locate_kernel<<<grid_for(n, 128), 128, 0, (cudaStream_t)stream>>>(s->P, x64, x32, n, k);
    SRMC_CUDA(cudaGetLastError(), "locate kernel launch");
    return SRMC_OK;
}

srmc_status srmc_start_points(const srmc_solver *s, int i, long long k, long long m0, long long n,
                              double *x, void *stream)
{
    if (!s || n < 0 || i < 0 || i >= s->P.N || k < 0 || k >= s->P.K || m0 < 0 ||
        m0 + n > 4294967296LL)
        return fail(SRMC_ERR_INVALID_ARG, "srmc_start_points: bad argument");
    if (n == 0) return SRMC_OK;
    if (!x) return fail(SRMC_ERR_INVALID_ARG, "srmc_start_points: NULL buffer");
    start_points_kernel<<<grid_for(n, 128), 128, 0, (cudaStream_t)stream>>>(s->P, s->fp64, i, k, m0, n, x);
    SRMC_CUDA(cudaGetLastError(), "start points kernel launch");
    return SRMC_OK;
}

}  // extern "C"
