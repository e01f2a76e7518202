// srmc_internal.h -- declarations shared by the translation units of libsrmc.
#pragma once

#include "srmc_device.cuh"

#include <string>

// A step launch solves the strata in Morton order of their cells (host-built
// table, 4 bytes per stratum) for d >= SRMC_ORDER_MIN_D and K up to
// SRMC_ORDER_MAX_K; below, index order already keeps neighbours together.
#ifndef SRMC_ORDER_MIN_D
#define SRMC_ORDER_MIN_D 3
#endif
#ifndef SRMC_ORDER_MAX_K
#define SRMC_ORDER_MAX_K (1LL << 25)
#endif

namespace srmc {

// Message returned by srmc_last_error() for the calling thread; every entry
// point of the library reports through it.
void set_last_error(const std::string &msg);

// Model variants of the step kernel: the driver needs z only for the cos
// model with kapz != 0 and for the logistic model.
enum ModelVariant { MV_COS = 0, MV_COS_Z = 1, MV_LOGISTIC = 2, MV_AFFINE = 3 };

// One round of the batched form: the strata of every active instance, laid
// end to end (instance a owns work items kofs[a] .. kofs[a+1]-1 and solves
// its step step[a]).
struct BatchRound {
    const Params *params;           // [instances] on the device
    const int *inst;                // [n_active] instance of active entry a
    const int *step;                // [n_active] step index i of that instance
    const long long *kofs;          // [n_active + 1] prefix sums of K
    int n_active;
    long long total;                // kofs[n_active]
};

// The persistent form of the batched solve: one launch per kernel variant
// over all of its rounds.  Segment a = (instance inst[a], step step[a]) owns
// the work items kofs[a] .. kofs[a+1]-1 (its strata); segments are listed in
// round order.  A block takes the next item from *next, waits until segment
// dep[a] (the same instance's step step[a] + 1; -1: none) has all its strata
// done, solves the item and counts it in done[a].  A wait that runs past its
// iteration limit sets *error and goes on (no hang; the tables are then not
// valid and srmc_batch_stats reports it).
struct FlowPlan {
    const Params *params;           // [instances] on the device
    const int *inst;                // [n_seg]
    const int *step;                // [n_seg]
    const long long *kofs;          // [n_seg + 1]
    const int *dep;                 // [n_seg]
    unsigned long long *done;       // [n_seg], zeroed before every launch
    unsigned long long *next;       // [1], zeroed before every launch
    unsigned *error;                // [1]
    int n_seg;
    long long total;                // kofs[n_seg]
};

#define SRMC_LAUNCH_STEP_NAME(D) SRMC_LAUNCH_STEP_NAME_(D)
#define SRMC_LAUNCH_BATCH_NAME(D) SRMC_LAUNCH_BATCH_NAME_(D)
#define SRMC_LAUNCH_BATCH_NAME_(D) launch_batch_d##D
#define SRMC_OCC_BATCH_NAME(D) SRMC_OCC_BATCH_NAME_(D)
#define SRMC_OCC_BATCH_NAME_(D) occupancy_batch_d##D
#define SRMC_LAUNCH_FLOW_NAME(D) SRMC_LAUNCH_FLOW_NAME_(D)
#define SRMC_LAUNCH_FLOW_NAME_(D) launch_flow_d##D
#define SRMC_OCC_FLOW_NAME(D) SRMC_OCC_FLOW_NAME_(D)
#define SRMC_OCC_FLOW_NAME_(D) occupancy_flow_d##D
#define SRMC_LAUNCH_STEP_NAME_(D) launch_step_d##D
#define SRMC_LAUNCH_STEP_PROB_NAME(D) SRMC_LAUNCH_STEP_PROB_NAME_(D)
#define SRMC_LAUNCH_STEP_PROB_NAME_(D) launch_step_prob_d##D
#define SRMC_LAUNCH_STEP_EXACT_NAME(D) SRMC_LAUNCH_STEP_EXACT_NAME_(D)
#define SRMC_LAUNCH_STEP_EXACT_NAME_(D) launch_step_exact_d##D
#define SRMC_LAUNCH_STEP_DENSE_NAME(D) SRMC_LAUNCH_STEP_DENSE_NAME_(D)
#define SRMC_LAUNCH_STEP_DENSE_NAME_(D) launch_step_dense_d##D
#define SRMC_LAUNCH_STEP_DENSEQ_NAME(D, Q) SRMC_LAUNCH_STEP_DENSEQ_NAME_(D, Q)
#define SRMC_LAUNCH_STEP_DENSEQ_NAME_(D, Q) launch_step_dense_d##D##_q##Q
#define SRMC_LAUNCH_STEP_QUAD_NAME(D) SRMC_LAUNCH_STEP_QUAD_NAME_(D)
#define SRMC_LAUNCH_STEP_QUAD_NAME_(D) launch_step_quad_d##D
// LP2 step kernels are built for d <= SRMC_LP2_DMAX.
#define SRMC_LP2_DMAX 3

#define SRMC_DECLARE_STEP(D)                                                              \
    cudaError_t launch_step_d##D(const Params &P, int i, bool fp64, bool lp1, int mv, int grid, \
                                 int threads, cudaStream_t st);                               \
    cudaError_t launch_step_prob_d##D(const Params &P, int i, bool fp64, bool lp1, int mv,    \
                                      int grid, int threads, cudaStream_t st);                \
    cudaError_t launch_step_exact_d##D(const Params &P, int i, bool fp64, bool lp1, int mv,   \
                                       int grid, int threads, cudaStream_t st);                \
    cudaError_t launch_step_dense_d##D(const Params &P, int i, bool fp64, bool lp1, int mv,   \
                                       int grid, int threads, cudaStream_t st);
SRMC_DECLARE_STEP(1)
SRMC_DECLARE_STEP(2)
SRMC_DECLARE_STEP(3)
SRMC_DECLARE_STEP(4)
SRMC_DECLARE_STEP(5)
SRMC_DECLARE_STEP(6)
SRMC_DECLARE_STEP(7)
SRMC_DECLARE_STEP(8)
#undef SRMC_DECLARE_STEP
// A d x q sigma with q != d (non-diagonal-sigma dynamics): d, q <= SRMC_DENSEQ_MAX.
#define SRMC_DENSEQ_MAX 4
#define SRMC_DECLARE_STEP_Q(D, Q)                                                                \
    cudaError_t launch_step_dense_d##D##_q##Q(const Params &P, int i, bool fp64, bool lp1, int mv, \
                                              int grid, int threads, cudaStream_t st);
SRMC_DECLARE_STEP_Q(1, 2) SRMC_DECLARE_STEP_Q(1, 3) SRMC_DECLARE_STEP_Q(1, 4)
SRMC_DECLARE_STEP_Q(2, 1) SRMC_DECLARE_STEP_Q(2, 3) SRMC_DECLARE_STEP_Q(2, 4)
SRMC_DECLARE_STEP_Q(3, 1) SRMC_DECLARE_STEP_Q(3, 2) SRMC_DECLARE_STEP_Q(3, 4)
SRMC_DECLARE_STEP_Q(4, 1) SRMC_DECLARE_STEP_Q(4, 2) SRMC_DECLARE_STEP_Q(4, 3)
#undef SRMC_DECLARE_STEP_Q
// d = 9..11: equal-size strata, Euler dynamics, the FP32 form, no controls.
constexpr int SRMC_WIDE_DMIN_V = 9;
cudaError_t launch_step_d9(const Params &P, int i, bool fp64, bool lp1, int mv, int grid, int threads,
                           cudaStream_t st);
cudaError_t launch_step_d10(const Params &P, int i, bool fp64, bool lp1, int mv, int grid, int threads,
                            cudaStream_t st);
cudaError_t launch_step_d11(const Params &P, int i, bool fp64, bool lp1, int mv, int grid, int threads,
                            cudaStream_t st);
// d = 12..19: the same, with the block's shared memory dynamic (prepare_step_dD
// sets the kernels' attribute once, at solver creation).
#define SRMC_PREPARE_STEP_NAME(D) SRMC_PREPARE_STEP_NAME_(D)
#define SRMC_PREPARE_STEP_NAME_(D) prepare_step_d##D
#define SRMC_DECLARE_XL(D)                                                                     \
    cudaError_t launch_step_d##D(const Params &P, int i, bool fp64, bool lp1, int mv, int grid, \
                                 int threads, cudaStream_t st);                                \
    cudaError_t prepare_step_d##D();
SRMC_DECLARE_XL(12)
SRMC_DECLARE_XL(13)
SRMC_DECLARE_XL(14)
SRMC_DECLARE_XL(15)
SRMC_DECLARE_XL(16)
SRMC_DECLARE_XL(17)
SRMC_DECLARE_XL(18)
SRMC_DECLARE_XL(19)
#undef SRMC_DECLARE_XL
cudaError_t launch_step_quad_d1(const Params &P, int i, bool fp64, bool lp1, int mv, int grid, int threads,
                                cudaStream_t st);
cudaError_t launch_step_quad_d2(const Params &P, int i, bool fp64, bool lp1, int mv, int grid, int threads,
                                cudaStream_t st);
cudaError_t launch_step_quad_d3(const Params &P, int i, bool fp64, bool lp1, int mv, int grid, int threads,
                                cudaStream_t st);

#define SRMC_DECLARE_BATCH(D)                                                                 \
    cudaError_t launch_batch_d##D(const BatchRound &B, bool fp64, bool lp1, int mv, bool cv,  \
                                  int grid, int threads, cudaStream_t st);                    \
    int occupancy_batch_d##D(bool fp64, bool lp1, int mv, bool cv, int threads);              \
    cudaError_t launch_flow_d##D(const FlowPlan &F, bool lp1, int mv, bool cv, int grid,      \
                                 int threads, cudaStream_t st);                              \
    int occupancy_flow_d##D(bool lp1, int mv, bool cv, int threads);
SRMC_DECLARE_BATCH(1)
SRMC_DECLARE_BATCH(2)
SRMC_DECLARE_BATCH(3)
SRMC_DECLARE_BATCH(4)
SRMC_DECLARE_BATCH(5)
SRMC_DECLARE_BATCH(6)
SRMC_DECLARE_BATCH(7)
SRMC_DECLARE_BATCH(8)
#undef SRMC_DECLARE_BATCH

// Cell of x along axis l for either kind of strata, and the centred basis
// coordinate (x - centre)/unit of that cell, in FP64 and in FP32.
__device__ __forceinline__ int cell_of(const Params &P, int l, double x, double &phi)
{
    if (P.kind != 0) return locate_prob(x, P.cellB + 4 * P.cell_off[l], P.cells[l], P.mu, phi);
    double t;
    const int c = locate_dim(x, P.lo[l], P.h[l], P.cells[l], t);
    phi = 2.0 * (t - (double)c) - 1.0;
    return c;
}
__device__ __forceinline__ int cell_of(const Params &P, int l, float x, float &phi)
{
    if (P.kind != 0) return locate_prob(x, P.cellB_f + 4 * P.cell_off[l], P.cells[l], P.mu_f, phi);
    float t;
    const int c = locate_dim(x, P.lo_f[l], P.r_f[l], P.cells[l], t);
    phi = 2.0f * (t - (float)c) - 1.0f;
    return c;
}

// Basis centre and unit of cell c along axis l (FP64 table).
__device__ __forceinline__ double cell_centre(const Params &P, int l, int c)
{
    return P.cellB[4 * (P.cell_off[l] + c) + 2];
}
__device__ __forceinline__ double cell_unit(const Params &P, int l, int c)
{
    return 1.0 / P.cellB[4 * (P.cell_off[l] + c) + 3];
}

// Table-row evaluation of y_i(x) in FP64 (truncated), x in double; the
// kernel-side twin of srmc_eval used by the MLP data generator.
__device__ __forceinline__ double eval_y64(const Params &P, int i, const double *x)
{
    double phi[PBMAX];
    phi[0] = 1.0;
    long long k = 0;
    for (int l = 0; l < P.d; ++l) {
        const int c = cell_of(P, l, x[l], phi[1 + l]);
        k += (long long)c * P.stride[l];
    }
    add_quadratic_rt(phi, P.d, P.p);
    const double *al = P.Y64 + ((long long)i * P.K + k) * P.ry64;
    double v = al[0];
    for (int c = 1; c < P.p; ++c) v += al[c] * phi[c];
    return fmin(fmax(v, -P.Cy), P.Cy);
}

}  // namespace srmc

using srmc::Params;

// One step launch of a single-instance solver on a stream (srmc_capi.cu).
cudaError_t srmc_launch_solver_step(const struct srmc_solver *s, int i, cudaStream_t st);

namespace srmc {
// A run-time compiled step kernel (user models, srmc_rtc.cu).
struct RtcKernel {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kernel = nullptr;
};
bool rtc_compile(const std::string &user_source, int d, bool fp64, bool lp1, bool cv, bool user_dynamics,
                 RtcKernel &out, std::string &log);
cudaError_t rtc_launch(const RtcKernel &k, const Params &P, int i, int grid, int threads, cudaStream_t st);
void rtc_release(RtcKernel &k);
}  // namespace srmc

// For a user-model solver, compile its control-variate step kernel if it is
// not compiled yet (called when a control is installed, outside any stream
// capture).  Returns 0, or a status with srmc_last_error set.
int srmc_prepare_user_control(struct srmc_solver *s);

// The solver object behind the opaque srmc_solver handle.
struct srmc_solver {
    Params P;                   // device pointers inside point to the buffers below
    int device;
    bool fp64, lp1;
    int mv;                     // model variant of the step kernel
    int threads;
    int done_from;              // every step >= done_from has been enqueued
    double *cellF = nullptr;
    float *cellF_f = nullptr;
    double *cellB = nullptr;             // per cell: edges, basis centre, 1/unit
    float *cellB_f = nullptr;
    double *stepc = nullptr;
    float *stepc_f = nullptr;
    float *Y32 = nullptr, *Z32 = nullptr;
    double *Y64 = nullptr, *Z64 = nullptr;
    unsigned long long *stats = nullptr;
    __half *C16 = nullptr;               // control rows of the FP32 form (binary16, [q][ph] per row)
    double *C64 = nullptr;               // control rows (FP64, padded like Z64)
    unsigned *order = nullptr;           // locality order of the strata (NULL: index order)
    unsigned *Mk = nullptr;              // paths of each stratum (NULL: M for all)
    long long M_sum = 0;                 // sum of the paths over the strata
    bool cv = false;                     // control installed
    bool cv_own = false;                 // ... and it is the run's own fitted z
    bool exact = false;                  // exact dynamics (Alg. 1)
    bool dense = false;                  // Euler dynamics with a non-diagonal constant sigma
    bool lp2 = false;                    // quadratic local polynomials
    std::string user_source;             // user model (SRMC_MODEL_USER): g and f as source
    bool user_dynamics = false;          // ... with its own drift and diffusion
    srmc::RtcKernel rtc[2];              // its step kernels: plain, control variate
    cudaStream_t cap_stream = nullptr;   // private stream for graph capture
    cudaGraphExec_t graph = nullptr;     // the N step launches of one solve
};

namespace srmc {
// Step-kernel model variant of a solver: the run's own control needs z_j at
// every path point, so the cos model without z in its driver runs the
// variant that evaluates z (whose z term then has coefficient kapz = 0).
inline int kernel_mv(const srmc_solver *s)
{
    return (s->cv && s->cv_own && s->mv == MV_COS) ? (int)MV_COS_Z : s->mv;
}
}  // namespace srmc


