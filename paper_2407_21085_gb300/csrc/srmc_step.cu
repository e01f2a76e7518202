// srmc_step.cu -- one backward step i of Alg. SRMDP for every stratum.
//
// Compiled once per dimension D (-DSRMC_STEP_D=D) so that every per-path
// array lives in registers.  One thread block owns one stratum H_k at a time
// (grid-stride over k); its threads share the M paths of the cloud C_{i,k}.
//
//   phase A  per path m: start point x_i ~ nu_k (Alg. 3), Euler to t_N
//            (Alg. 2), at every later step locate the stratum of X_{j+1},
//            read its fitted row and evaluate y_{j+1}(X_{j+1}), z_{j+1}(X_{j+1})
//            (truncated), accumulate S_{Y,i+1} = g(X_N) + sum_{j>i} f_j dt
//            (eq. PsiM); add phi phi^T, phi S dW_i/dt, phi S to the moments.
//   Z fit    Cholesky of the Gram matrix in FP64, beta = G^{-1} r_Z.
//   phase B  per path: regenerate x_i, dW_i, X_{i+1} from the same counters,
//            f_i(x_i, y_{i+1}(X_{i+1}), z_i(x_i)) with the new beta (Z before Y),
//            add phi f_i to the moments.  Only drivers that read z need it:
//            otherwise f_i is added to the Y response in phase A.
//   Y fit    alpha = G^{-1} (r_S + dt r_F); write row (i, k).
//
// Moments: FP64 form accumulates in double per thread.  FP32 form
// accumulates in float per thread over blocks of FLUSH paths, then reduces
// each entry across the warp and carries the warp sums in double, so the
// rounding error of a moment does not grow with M.
//
// The same source is compiled at run time by NVRTC for user models
// (__CUDACC_RTC__, -DSRMC_USER_MODEL): device code only, with the entry
// kernel srmc_user_step at the end; the host launchers are left out.
#ifdef __CUDACC_RTC__
#include "srmc_device.cuh"
#else
#include "srmc_internal.h"
#endif

#ifndef SRMC_STEP_D
#error "compile with -DSRMC_STEP_D=<dimension>"
#endif
// Kind of strata the unit is compiled for: 0 equal size (the launchers
// launch_step_dD, launch_batch_dD), 1 equal nu-probability (launch_step_prob_dD;
// the batched form is built for equal-size strata only).
#ifndef SRMC_STEP_KIND
#define SRMC_STEP_KIND 0
#endif
// Dynamics of the unit: 0 the Euler scheme (Alg. 2), 1 the exact affine-drift
// SDE (Alg. 1; launch_step_exact_dD), which draws a second block of q normals
// per step, 2 the Euler scheme with a non-diagonal constant sigma
// (launch_step_dense_dD: X'_l = A_l X_l + c_l + sum_r sigma_lr dW_r).  Exact
// and dense dynamics are built for equal-size strata only.
#ifndef SRMC_STEP_DYN
#define SRMC_STEP_DYN 0
#endif
// Local polynomials of the unit's LP1 kernels: 1 affine (Sec. 4.1), 2
// quadratic (LP2: [1, u, u_a u_b (a <= b)]; launch_step_quad_dD, d <= 3,
// equal-size strata and Euler dynamics).
#ifndef SRMC_STEP_BASIS
#define SRMC_STEP_BASIS 1
#endif
// Brownian components q of the unit: q = d, except in the units of the
// non-diagonal-sigma dynamics compiled with -DSRMC_STEP_Q=q (a d x q sigma).
#ifndef SRMC_STEP_Q
#define SRMC_STEP_Q SRMC_STEP_D
#endif
static_assert(SRMC_STEP_Q == SRMC_STEP_D || SRMC_STEP_DYN == 2, "q != d is built for the dense-sigma units only");

namespace srmc {
namespace {

constexpr int FLUSH = 16;

// q of a d-dimensional kernel in this unit (dW_j, z, the Z fits and the
// control rows have q components; x, the strata and the basis have d).
template <int D>
struct QOf {
    static constexpr int value = D == SRMC_STEP_D ? SRMC_STEP_Q : D;
};
constexpr int NW = SRMC_STEP_DYN == 1 ? 2 : 1;     // blocks of q normals per step

// Basis dimension: 1 (LP0), d + 1 (LP1) or 1 + d + d(d+1)/2 (LP2 units).
template <int D, bool LP1>
struct BasisDim {
    static constexpr int value = !LP1 ? 1 : SRMC_STEP_BASIS == 2 ? 1 + D + D * (D + 1) / 2 : D + 1;
};

// The quadratic monomials u_a u_b (a <= b, row order) after the linear ones.
template <typename R, int D, int p>
__device__ __forceinline__ void add_quadratic(R (&phi)[p])
{
    if constexpr (p > D + 1) {
        int e = 1 + D;
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = a; b < D; ++b) phi[e++] = phi[1 + a] * phi[1 + b];
    }
}

// One step of the chain for coordinate l: X' = A X + c + s1 dW (+ s2 xi2 for
// the exact dynamics).
template <typename R>
__device__ __forceinline__ R chain_step(const Params &P, int l, R x, R dw, R xi2)
{
    R v = fma(Form<R>::A(P, l), x, Form<R>::c(P, l)) + Form<R>::s1(P, l) * dw;
    if constexpr (NW == 2) v += Form<R>::s2(P, l) * xi2;
    return v;
}

// Coordinate l of the step from X_j = x (the whole vector): the affine-drift
// step above, or, for user models with their own dynamics (run-time units,
// -DSRMC_USER_DYNAMICS), the Euler step (Alg. 2) with the user's drift and
// diagonal diffusion at (t_j, X_j).
template <typename R, int D>
__device__ __forceinline__ R next_coord(const Params &P, int j, int l, const R (&x)[D], R dw, R xi2)
{
#ifdef SRMC_USER_DYNAMICS
    const R t = (R)j * Form<R>::dt(P);
    return x[l] + srmc_user_b(t, x, l, D, P.prm) * Form<R>::dt(P) + srmc_user_sigma(t, x, l, D, P.prm) * dw;
#else
    return chain_step<R>(P, l, x[l], dw, xi2);
#endif
}

// Whether the FP32 Euler step and cell location of equal-size strata take
// coordinates two at a time with the packed FP32 instructions (same
// operations and roundings as the scalar forms).
#ifndef SRMC_COORD_PAIRS
#define SRMC_COORD_PAIRS 1
#endif
#if SRMC_COORD_PAIRS && SRMC_NORMAL_PAIRS && !defined(__CUDACC_RTC__) && SRMC_STEP_DYN == 0
#define SRMC_PAIRS_ON 1
#else
#define SRMC_PAIRS_ON 0
#endif

// X_{j+1} from X_j = x and the increments dw (the whole vector).
template <typename R, int D>
__device__ __forceinline__ void advance(const Params &P, int j, const R (&x)[D],
                                        const R (&dw)[QOf<D>::value], R (&xn)[D])
{
#if SRMC_STEP_DYN == 2
    constexpr int Q = QOf<D>::value;
    static_assert(D <= SD_DMAX && Q <= SD_DMAX, "non-diagonal sigma units are built for d, q <= SD_DMAX");
    // the full d x q matrix: coordinate l takes every increment
#pragma unroll
    for (int l = 0; l < D; ++l) {
        R v = fma(Form<R>::A(P, l), x[l], Form<R>::c(P, l));
#pragma unroll
        for (int r = 0; r < Q; ++r) v = fma(Form<R>::sd(P, l * Q + r), dw[r], v);
        xn[l] = v;
    }
#else
#if SRMC_PAIRS_ON && !defined(SRMC_USER_DYNAMICS)
    if constexpr (sizeof(R) == 4) {
        if (P.unit_drift) {
            // A = 1, c = 0 in every coordinate (no drift): A x + c = x exactly
#pragma unroll
            for (int l = 0; l + 1 < D; l += 2) {
                const float2 v = __ffma2_rn(make_float2(P.s1_f[l], P.s1_f[l + 1]), make_float2(dw[l], dw[l + 1]),
                                            make_float2(x[l], x[l + 1]));
                xn[l] = v.x;
                xn[l + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int l = 0; l + 1 < D; l += 2) {
                const float2 v = __ffma2_rn(make_float2(P.s1_f[l], P.s1_f[l + 1]), make_float2(dw[l], dw[l + 1]),
                                            __ffma2_rn(make_float2(P.A_f[l], P.A_f[l + 1]),
                                                       make_float2(x[l], x[l + 1]),
                                                       make_float2(P.c_f[l], P.c_f[l + 1])));
                xn[l] = v.x;
                xn[l + 1] = v.y;
            }
        }
        if constexpr ((D & 1) != 0) xn[D - 1] = next_coord<R, D>(P, j, D - 1, x, dw[D - 1], (R)0);
        return;
    }
#endif
#pragma unroll
    for (int l = 0; l < D; ++l) xn[l] = next_coord<R, D>(P, j, l, x, dw[l], (R)0);
#endif
}

// Cells of x on equal-size strata: kk = sum_l c_l stride_l, and (LP1) the
// centred coordinates phi[1 + l] = 2 (t_l - c_l) - 1, t_l = (x_l - lo_l) / h_l.
//
// With SRMC_LOCATE_RD the FP32 cell c = clamp(floor(t), 0, C - 1) is taken by
// one addition rounded toward -inf: for 0 <= tc < 2^23, tc + 2^23 rounded down
// is exactly 2^23 + floor(tc), whose bits are 0x4B000000 + floor(tc), so with
// tc = clamp(t, 0, C - 1) (NaN -> 0) the bits are 0x4B000000 + c and the float
// minus 2^23 is c itself: the same decision and basis value as floorf, with no
// conversion.  The stride-weighted 0x4B000000 terms are removed at the end
// (P.kbias, all modulo 2^32).
#ifndef SRMC_LOCATE_RD
#define SRMC_LOCATE_RD 1
#endif
template <typename R, int D, bool LP1, int p>
__device__ __forceinline__ unsigned locate_point(const Params &P, const R (&x)[D], R (&phi)[p])
{
    unsigned kk = 0;
#if SRMC_PAIRS_ON && SRMC_LOCATE_RD
    if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int l = 0; l + 1 < D; l += 2) {
            const float2 t = __fmul2_rn(__fadd2_rn(make_float2(x[l], x[l + 1]),
                                                   make_float2(-P.lo_f[l], -P.lo_f[l + 1])),
                                        make_float2(P.r_f[l], P.r_f[l + 1]));
            const float2 tc = make_float2(fminf(fmaxf(t.x, 0.0f), (float)(P.cells[l] - 1)),
                                          fminf(fmaxf(t.y, 0.0f), (float)(P.cells[l + 1] - 1)));
            const float2 f = __fadd2_rd(tc, f2(0x1p23f));
            kk += __float_as_uint(f.x) * (unsigned)P.stride[l] + __float_as_uint(f.y) * (unsigned)P.stride[l + 1];
            if (LP1) {
                const float2 c = __fadd2_rn(f, f2(-0x1p23f));
                const float2 u = __ffma2_rn(f2(2.0f), __fadd2_rn(t, make_float2(-c.x, -c.y)), f2(-1.0f));
                phi[1 + l] = u.x;
                phi[2 + l] = u.y;
            }
        }
        if constexpr ((D & 1) != 0) {
            const float t = __fmul_rn(__fsub_rn(x[D - 1], P.lo_f[D - 1]), P.r_f[D - 1]);
            const float f = __fadd_rd(fminf(fmaxf(t, 0.0f), (float)(P.cells[D - 1] - 1)), 0x1p23f);
            kk += __float_as_uint(f) * (unsigned)P.stride[D - 1];
            if (LP1) phi[D] = 2.0f * (t - (f - 0x1p23f)) - 1.0f;
        }
        return kk - P.kbias;
    }
#elif SRMC_PAIRS_ON
    if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int l = 0; l + 1 < D; l += 2) {
            const float2 t = __fmul2_rn(__fadd2_rn(make_float2(x[l], x[l + 1]),
                                                   make_float2(-P.lo_f[l], -P.lo_f[l + 1])),
                                        make_float2(P.r_f[l], P.r_f[l + 1]));
            const float c0 = fminf(fmaxf(floorf(t.x), 0.0f), (float)(P.cells[l] - 1));
            const float c1 = fminf(fmaxf(floorf(t.y), 0.0f), (float)(P.cells[l + 1] - 1));
            kk += (unsigned)(int)c0 * (unsigned)P.stride[l] + (unsigned)(int)c1 * (unsigned)P.stride[l + 1];
            if (LP1) {
                const float2 u = __ffma2_rn(make_float2(2.0f, 2.0f), __fadd2_rn(t, make_float2(-c0, -c1)),
                                            make_float2(-1.0f, -1.0f));
                phi[1 + l] = u.x;
                phi[2 + l] = u.y;
            }
        }
        if constexpr ((D & 1) != 0) {
            R t;
            const int c = locate_dim(x[D - 1], P.lo_f[D - 1], P.r_f[D - 1], P.cells[D - 1], t);
            kk += (unsigned)c * (unsigned)P.stride[D - 1];
            if (LP1) phi[D] = 2.0f * (t - (float)c) - 1.0f;
        }
        return kk;
    }
#endif
#pragma unroll
    for (int l = 0; l < D; ++l) {
        R t;
        const int c = locate_dim(x[l], Form<R>::lo(P, l), Form<R>::scale(P, l), P.cells[l], t);
        kk += (unsigned)c * (unsigned)P.stride[l];
        if (LP1) phi[1 + l] = (R)2 * (t - (R)c) - (R)1;
    }
    return kk;
}

template <int E>
struct Moments64 {
    double a[E];
    __device__ void zero() {
#pragma unroll
        for (int e = 0; e < E; ++e) a[e] = 0.0;
    }
    __device__ void add(int e, double v) { a[e] += v; }
    __device__ void flush(int) {}
    // Leaves the warp total of entry e in lane (e & 31), slot e >> 5.
    __device__ void finish(double (&out)[(E + 31) / 32], int lane) {
#pragma unroll
        for (int s = 0; s < (E + 31) / 32; ++s) out[s] = 0.0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            double v = a[e];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == (e & 31)) out[e >> 5] = v;
        }
    }
};

template <int E>
struct Moments32 {
    float a[E];
    double c[(E + 31) / 32];
    __device__ void zero() {
#pragma unroll
        for (int e = 0; e < E; ++e) a[e] = 0.0f;
#pragma unroll
        for (int s = 0; s < (E + 31) / 32; ++s) c[s] = 0.0;
    }
    __device__ void add(int e, float v) { a[e] += v; }
    __device__ void flush(int lane) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            float v = a[e];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == (e & 31)) c[e >> 5] += (double)v;
            a[e] = 0.0f;
        }
    }
    __device__ void finish(double (&out)[(E + 31) / 32], int lane) {
        flush(lane);
#pragma unroll
        for (int s = 0; s < (E + 31) / 32; ++s) out[s] = c[s];
    }
};

// FP32 moments for long moment vectors: the path's E products are formed
// after its time loop and summed over the warp by recursive halving
// (reduce-scatter): in round r every lane keeps one half of its vector and
// adds the partner's copy of that half, so after five rounds each lane holds
// LF = E / 32 (rounded up level by level) warp sums, which it adds to running
// sums in double.  Nothing of size E stays live across the time loop, so the
// registers of the path simulation do not grow with E, and no shared memory
// is taken from L1.
__host__ __device__ constexpr int halve(int L) { return (L + 1) / 2; }
__host__ __device__ constexpr int rs_len(int E, int r) { return r == 0 ? E : halve(rs_len(E, r - 1)); }

template <int E>
struct MomentsRS {
    static constexpr int LF = rs_len(E, 5);
    double c[LF];
    int base;                          // entry index of c[0] held by this lane
    int rend;                          // end of the real entries of this lane's slice
    __device__ void zero(int lane) {
#pragma unroll
        for (int s = 0; s < LF; ++s) c[s] = 0.0;
        // In round r the slice [base, base + L_{r-1}) splits at L_r = rs_len(E, r):
        // the upper half [base + L_r, ...) ends where the parent's real entries
        // end; the lower half ends at base + L_r.  Slots past rend are padding.
        base = 0;
        rend = E;
#pragma unroll
        for (int r = 1; r <= 5; ++r) {
            const int L = rs_len(E, r);
            if (lane & (32 >> r)) base += L;
            else rend = min(rend, base + L);
        }
    }
    template <int L, int O>
    __device__ __forceinline__ static void round(const float (&v)[L], float (&o)[halve(L)], int lane) {
        constexpr int H = halve(L);
        const bool up = (lane & O) != 0;
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const float lo = v[k];
            const float hi = (k + H < L) ? v[k + H] : 0.0f;
            const float mine = up ? hi : lo;
            const float other = up ? lo : hi;
            o[k] = mine + __shfl_xor_sync(0xffffffffu, other, O);
        }
    }
    __device__ __forceinline__ void add_path(const float (&v)[E], int lane) {
        float a1[rs_len(E, 1)], a2[rs_len(E, 2)], a3[rs_len(E, 3)], a4[rs_len(E, 4)], a5[LF];
        round<E, 16>(v, a1, lane);
        round<rs_len(E, 1), 8>(a1, a2, lane);
        round<rs_len(E, 2), 4>(a2, a3, lane);
        round<rs_len(E, 3), 2>(a3, a4, lane);
        round<rs_len(E, 4), 1>(a4, a5, lane);
#pragma unroll
        for (int s = 0; s < LF; ++s) c[s] += (double)a5[s];
    }
};

// Block totals of reduce-scattered moments: lane values go to their entries.
template <int E, int LF>
__device__ void block_totals_rs(const double (&c)[LF], int base, int rend, double (*red)[E],
                                double *tot, int warp, int nwarps)
{
#pragma unroll
    for (int s = 0; s < LF; ++s)
        if (base + s < rend) red[warp][base + s] = c[s];
    __syncthreads();
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        double v = 0.0;
        for (int w = 0; w < nwarps; ++w) v += red[w][e];
        tot[e] = v;
    }
    __syncthreads();
}

// Position (a, b), a <= b, of entry e of the packed upper triangle of a
// p x p matrix stored row by row.
__host__ __device__ constexpr int tri_a(int e, int p) { return e < p ? 0 : 1 + tri_a(e - p, p - 1); }
__host__ __device__ constexpr int tri_b(int e, int p) { return e < p ? e : 1 + tri_b(e - p, p - 1); }

template <typename R, int E> struct MomentsOf;
template <int E> struct MomentsOf<double, E> { using type = Moments64<E>; };
template <int E> struct MomentsOf<float, E> { using type = Moments32<E>; };

// Block-wide totals of E entries: every warp parks its totals in smem, then
// threads sum the warps in a fixed order (deterministic).
template <int E>
__device__ void block_totals(const double (&lanev)[(E + 31) / 32], double (*red)[E], double *tot,
                             int lane, int warp, int nwarps)
{
#pragma unroll
    for (int s = 0; s < (E + 31) / 32; ++s) {
        const int e = s * 32 + lane;
        if (e < E) red[warp][e] = lanev[s];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        double v = 0.0;
        for (int w = 0; w < nwarps; ++w) v += red[w][e];
        tot[e] = v;
    }
    __syncthreads();
}

// Cholesky factor L (row-major p x p, shared memory) of the Gram matrix
// given as its packed upper triangle (pairs a <= b, row by row), computed by
// one warp (right-looking: pivot by lane 0, column and trailing update spread
// over the lanes); Linv holds 1 / L[a][a].  Returns false (in every lane) if
// a pivot is below 1e-12 of the trace: numerically singular.  G is a
// p x p shared-memory work array.
template <int p>
__device__ bool cholesky_warp(const double *Gp, double *G, double *L, double *Linv, int lane)
{
    for (int e = lane; e < p * p; e += 32) {
        const int a = e / p, b = e % p;
        const int r = a < b ? a : b, c = a < b ? b : a;
        G[e] = Gp[r * p - r * (r - 1) / 2 + (c - r)];
        L[e] = 0.0;
    }
    __syncwarp();
    double tr = 0.0;
    for (int a = 0; a < p; ++a) tr += G[a * p + a];
    for (int b = 0; b < p; ++b) {
        const double piv = G[b * p + b];
        if (!(piv > 1e-12 * tr)) return false;          // uniform: every lane reads the same value
        const double ld = sqrt(piv), inv = 1.0 / ld;
        for (int a = b + 1 + lane; a < p; a += 32) L[a * p + b] = G[a * p + b] * inv;
        if (lane == 0) { L[b * p + b] = ld; Linv[b] = inv; }
        __syncwarp();
        const int m = p - 1 - b;                          // trailing (m x m) lower part
        for (int t = lane; t < m * m; t += 32) {
            const int a = b + 1 + t / m, c = b + 1 + t % m;
            if (c <= a) G[a * p + c] -= L[a * p + b] * L[c * p + b];
        }
        __syncwarp();
    }
    return true;
}

// Solve L L^T x = r (L, Linv from cholesky_warp) into x (may alias r).
template <int p>
__device__ void chol_solve(const double *L, const double *Linv, const double *r, double *x)
{
    for (int a = 0; a < p; ++a) {
        double s = r[a];
        for (int c = 0; c < a; ++c) s -= L[a * p + c] * x[c];
        x[a] = s * Linv[a];
    }
    for (int a = p - 1; a >= 0; --a) {
        double s = x[a];
        for (int c = a + 1; c < p; ++c) s -= L[c * p + a] * x[c];
        x[a] = s * Linv[a];
    }
}

// Padded length of a table row of n entries: 16 bytes (4 floats or 2
// doubles) per vector load.
template <typename R>
__host__ __device__ constexpr int row_pad(int n) { return sizeof(R) == 4 ? (n + 3) / 4 * 4 : (n + 1) / 2 * 2; }

// y_{j}(x), z_{j}(x) from the row of the stratum holding x (truncated), or
// g(x) when j == N.
// With CV, also hands back phi(x) and the row index of (j, stratum of x), from
// which the control of the next increment is evaluated.
template <typename R, int D, bool LP1, int MODEL, bool ZIN, bool CV, bool FLOW = false>
__device__ __forceinline__ void eval_at(const Params &P, int j, const R (&x)[D], R &y,
                                        R (&z)[QOf<D>::value], R (&phio)[BasisDim<D, LP1>::value],
                                        unsigned &rowo)
{
    constexpr int p = BasisDim<D, LP1>::value;
    constexpr int Q = QOf<D>::value;
    if (j == P.N) {
        y = model_g<R, D, MODEL>(P, x);
        return;
    }
    unsigned kk = 0;
    R phi[p];
    phi[0] = (R)1;
    if constexpr (SRMC_STEP_KIND == 0) {
        kk = locate_point<R, D, LP1, p>(P, x, phi);
    } else {
#pragma unroll
        for (int l = 0; l < D; ++l) {
            R u;
            const int c = locate_prob(x[l], Form<R>::cellB(P) + 4 * P.cell_off[l], P.cells[l],
                                      Form<R>::mu(P), u);
            kk += (unsigned)c * (unsigned)P.stride[l];
            if (LP1) phi[1 + l] = u;
        }
    }
    add_quadratic<R, D, p>(phi);
    const unsigned row = (unsigned)j * (unsigned)P.K + kk;     // N K < 2^32 (checked at create)
    // The row strides are those srmc_create sets (rows padded to 16 bytes),
    // as constants of the kernel's basis dimension.
    constexpr unsigned RY = (unsigned)row_pad<R>(p), RZ = (unsigned)row_pad<R>(Q * p);
    R a[p];
    load_row<p, FLOW>(Form<R>::Ytab(P) + row * RY, a);
    R v = a[0];
#pragma unroll
    for (int c = 1; c < p; ++c) v += a[c] * phi[c];
    y = clamp_r(v, Form<R>::Cy(P));
    if (ZIN) {
        if constexpr (sizeof(R) == 4 && Q * p > 64) {
            // long rows (d >= 8): each 16-byte vector is folded into z as it
            // arrives, so that the row never sits in registers whole
            const float4 *z4 = reinterpret_cast<const float4 *>(Form<R>::Ztab(P) + row * RZ);
            R w[Q];
#pragma unroll
            for (int l = 0; l < Q; ++l) w[l] = (R)0;
#pragma unroll
            for (int v = 0; v < (Q * p + 3) / 4; ++v) {
                const float4 t = ld_row4<FLOW>(z4 + v);
                const float tv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int e = 4 * v + u;
                    if (e < Q * p) w[e / p] = (e % p == 0) ? w[e / p] + tv[u] : fmaf(tv[u], phi[e % p], w[e / p]);
                }
            }
#pragma unroll
            for (int l = 0; l < Q; ++l) z[l] = clamp_r(w[l], Form<R>::Cz(P));
        } else {
            R bz[Q * p];
            load_row<Q * p, FLOW>(Form<R>::Ztab(P) + row * RZ, bz);
#pragma unroll
            for (int l = 0; l < Q; ++l) {
                R w = bz[l * p];
#pragma unroll
                for (int c = 1; c < p; ++c) w += bz[l * p + c] * phi[c];
                z[l] = clamp_r(w, Form<R>::Cz(P));
            }
        }
    }
    if constexpr (CV) {
#pragma unroll
        for (int c = 0; c < p; ++c) phio[c] = phi[c];
        rowo = row;
    }
}

// zc(x) = T_Cz(beta_l . phi) for the control row `row` and the basis values
// phi of x: the values of the martingale control's integrand (clamped).
template <typename R, int D, int p>
__device__ __forceinline__ void control_vals(const Params &P, unsigned row, const R (&phi)[p],
                                             R (&zc)[QOf<D>::value])
{
    constexpr int Q = QOf<D>::value;
    if constexpr (sizeof(R) == 4) {
        // FP32 form: binary16 rows, coefficient-major (the halves of a 32-bit
        // word are coefficient a of components 2m and 2m + 1, c16_index), read
        // in 16-byte vectors and folded in as they arrive: each word widens to
        // an FP32 pair that enters both components' dot products with one
        // packed FMA; the order of the terms of each component is that of the
        // scalar form (constant first, then a = 1 .. p - 1).
        constexpr int QH = (Q + 1) / 2;                  // component pairs
        constexpr int NWD = p * QH;                      // 32-bit words of a row in use
        constexpr int RCW = (2 * NWD + 7) / 8 * 4;       // 32-bit words per row (16-byte rows)
        const uint4 *b4 = reinterpret_cast<const uint4 *>(reinterpret_cast<const unsigned *>(P.C16) +
                                                          row * (unsigned)RCW);
        float2 w2[QH];
#pragma unroll
        for (int v = 0; v < (NWD + 3) / 4; ++v) {
            const uint4 t = __ldg(b4 + v);
            const unsigned tw[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = 4 * v + u;
                if (e < NWD) {
                    const int a = e / QH, m = e % QH;
                    const float2 c = __half22float2(*reinterpret_cast<const __half2 *>(&tw[u]));
                    w2[m] = a == 0 ? c : __ffma2_rn(c, make_float2(phi[a], phi[a]), w2[m]);
                }
            }
        }
        const float L = Form<R>::Cz(P);
#pragma unroll
        for (int m = 0; m < QH; ++m) {
            zc[2 * m] = clamp_r(w2[m].x, L);
            if (2 * m + 1 < Q) zc[2 * m + 1] = clamp_r(w2[m].y, L);
        }
    } else {
        const double *b = P.C64 + row * (unsigned)P.rz64;
#pragma unroll
        for (int l = 0; l < Q; ++l) {
            double w = __ldg(b + l * p);
#pragma unroll
            for (int a = 1; a < p; ++a) w += __ldg(b + l * p + a) * phi[a];
            zc[l] = clamp_r(w, Form<R>::Cz(P));
        }
    }
}

// zc . dw: the martingale control of one increment (FP32: two components
// per packed FMA, the pair sums added at the end).
template <typename R, int D>
__device__ __forceinline__ R control_apply(const R (&zc)[D], const R (&dw)[D])
{
    if constexpr (sizeof(R) == 4) {
        float2 s2 = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int m = 0; m < (D + 1) / 2; ++m)
            s2 = __ffma2_rn(make_float2(zc[2 * m], 2 * m + 1 < D ? zc[2 * m + 1] : 0.0f),
                            make_float2(dw[2 * m], 2 * m + 1 < D ? dw[2 * m + 1] : 0.0f), s2);
        return s2.x + s2.y;
    } else {
        R acc = (R)0;
#pragma unroll
        for (int l = 0; l < D; ++l) acc += zc[l] * dw[l];
        return acc;
    }
}

template <typename R, int D, int p>
__device__ __forceinline__ R control_dot(const Params &P, unsigned row, const R (&phi)[p],
                                         const R (&dw)[QOf<D>::value])
{
    R zc[QOf<D>::value];
    control_vals<R, D, p>(P, row, phi, zc);
    return control_apply<R, QOf<D>::value>(zc, dw);
}

// Blocks per SM the compiler must fit (register budget): FP32 forms of
// higher dimension would otherwise take > 100 registers and run 2 blocks/SM.
// (Measured on GB300: 5 blocks for d <= 2 and 4 for d >= 3 are best; the
// control-variate kernel at d = 6 runs 6 % faster with 4 blocks and a
// 96-byte spill than with 3 blocks and none.)
#ifndef SRMC_MINB_LO
#define SRMC_MINB_LO 5
#endif
#ifndef SRMC_MINB_HI
#define SRMC_MINB_HI 4
#endif
#ifndef SRMC_CVMINB_HI
#define SRMC_CVMINB_HI 4
#endif
#ifndef SRMC_CVZMINB_HI
#define SRMC_CVZMINB_HI 3
#endif
#ifndef SRMC_MINB_XL
#define SRMC_MINB_XL 3
#endif
template <typename R, int D, bool CV, bool ZIN>
struct MinBlocks {
    static constexpr int value = sizeof(R) == 8 ? 1
                               : CV ? (D <= 2 ? 4 : ZIN ? SRMC_CVZMINB_HI : SRMC_CVMINB_HI)
                                    : (D <= 2 ? SRMC_MINB_LO : D >= 12 ? 2 : D >= 9 ? SRMC_MINB_XL
                                                                                     : SRMC_MINB_HI);
};

// Units of d >= 12 hold their block's shared memory dynamically (above the
// 48 KB of static shared memory a block may declare; about 94 KB at d = 19).
constexpr bool DYN_SMEM = SRMC_STEP_D >= 12;

// Whether phase A parks a path's basis values phi(x_i) and increments dW_i
// in shared memory across its time loop (FP32 form, d >= SRMC_STAGE_MIN_D):
// they are needed only for the moments after the loop, and in registers they
// would stay live through every step (at d = 6, 12 registers, which made the
// kernel spill at its 64-register budget).  One column per thread, read back
// with volatile loads so that the compiler cannot keep the values instead.
#ifndef SRMC_STAGE_MIN_D
#define SRMC_STAGE_MIN_D 5
#endif
template <typename R, int D>
struct Stage {
    static constexpr bool value = sizeof(R) == 4 && D >= SRMC_STAGE_MIN_D;
};

// FP32 moments of long vectors (E > 24 entries: LP1 at d >= 4, LP2 at d >= 2)
// by warp tiles: after its time loop every thread writes its path's columns
// (1 or 0 for a path past M_k, phi_1..phi_{p-1}, w_l = S_Z dW_l / dt, S_Y;
// zeros past M_k) into shared memory, and lane s of the warp forms entries
// e = s, s + 32, ... of the moment vector as dot products over the warp's 32
// paths -- the Gram entries sum phi_a phi_b, the Z right-hand sides
// sum phi_a w_l, the Y right-hand side sum phi_a S_Y -- in FP32, then adds
// them to running sums in FP64.  Each FP32 partial sums 32 terms, so the
// rounding error of a moment is bounded by ~31 u sum |terms| whatever M is.
// (The alternative, SRMC_TILE_MOMENTS=0, reduces each path's products across
// the warp by shuffles, which costs ~3 E instructions per path.)
#ifndef SRMC_TILE_MOMENTS
#define SRMC_TILE_MOMENTS 1
#endif
// (Also for every FP32 kernel of d >= SRMC_TILE_MIN_D, whose path state
// leaves no room for per-thread accumulators.)
#ifndef SRMC_TILE_MIN_D
#define SRMC_TILE_MIN_D 5
#endif
template <typename R, int D, int EA>
struct TileMoments {
    static constexpr bool value =
        SRMC_TILE_MOMENTS && sizeof(R) == 4 && (EA > 24 || D >= SRMC_TILE_MIN_D);
};

// Shared memory of one stratum block.
template <typename R, int D, bool LP1>
struct StepSmem {
    static constexpr int p = BasisDim<D, LP1>::value;
    static constexpr int q = QOf<D>::value;
    static constexpr int EG = LP1 ? p * (p + 1) / 2 : 0;
    static constexpr int EA = EG + q * p + p;
    // Path columns (one per thread; rows padded by four words, so that rows
    // stay 16-byte aligned for vector loads along a row and lanes reading
    // different rows at one column fall in different banks): [0] 1 or 0,
    // [1, p) phi_a, [p, p + q) dW_l and later w_l, [p + q] S_Y.
    static constexpr bool COLS = Stage<R, D>::value || TileMoments<R, D, EA>::value;
    static constexpr int NT = COLS ? p + q + 1 : 1;
    static constexpr int TS = COLS ? MAX_THREADS + 4 : 4;
    __align__(16) float tile[NT][TS];
    // Warp tiles with more than 8 entries per lane (d >= 12) keep their running
    // sums in redA (each warp its own row) and their column pairs here.
    static constexpr bool TSM = TileMoments<R, D, EA>::value && (EA + 31) / 32 > 8;
    short2 tcol[TSM ? EA : 1];
    static constexpr int EB = p;
    double redA[MAX_WARPS][EA];
    double totA[EA];
    double redB[MAX_WARPS][EB];
    double totB[EB];
    double Ls[p * p];
    double Gw[p * p];
    double Linv[p];
    double beta_s[q * p];
    R beta_r[q * p];
    int ok_s;
};

// Fits of stratum k at step i (the whole of Alg. SRMDP for one (i, k)) by the
// calling block: phase A, Z fit, phase B, Y fit, row store.
template <typename R, int D, bool LP1, int MODEL, bool ZIN, bool CV, bool FLOW = false>
__device__ __forceinline__ void solve_stratum(const Params &P, const int i, const long long k,
                                              StepSmem<R, D, LP1> &sm)
{
    constexpr int p = BasisDim<D, LP1>::value;
    constexpr int q = QOf<D>::value;                 // Brownian components
    constexpr int EG = LP1 ? p * (p + 1) / 2 : 0;
    constexpr int EZ = q * p;
    constexpr int EA = EG + EZ + p;
    constexpr int EB = p;
    constexpr bool TILE = TileMoments<R, D, EA>::value;
    // The paper's logistic driver reads z only through sum_l z_l (of the
    // truncated components): then only that sum is carried from step to step.
    constexpr bool ZSUM = ZIN && MODEL == MODEL_LOGISTIC && !CV;
    constexpr bool RS = sizeof(R) == 4 && EA > 24 && !TILE;
    using MA = typename Select<RS, MomentsRS<EA>, typename MomentsOf<R, EA>::type>::type;
    constexpr int TS = StepSmem<R, D, LP1>::TS;
    constexpr bool TSM = StepSmem<R, D, LP1>::TSM;  // tile sums in shared memory
    constexpr int LF = TSM ? 1 : (EA + 31) / 32;   // moment entries per lane held in registers (TILE)
    using MB = typename MomentsOf<R, EB>::type;
    auto &redA = sm.redA;
    auto &totA = sm.totA;
    auto &redB = sm.redB;
    auto &totB = sm.totB;
    auto &Ls = sm.Ls;
    auto &Gw = sm.Gw;
    auto &Linv = sm.Linv;
    auto &beta_s = sm.beta_s;
    auto &beta_r = sm.beta_r;
    auto &ok_s = sm.ok_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const R dt = Form<R>::dt(P), sdt = Form<R>::sdt(P), inv_dt = (R)1 / dt;
    const long long Mk = P.Mk ? (long long)__ldg(P.Mk + k) : P.M;     // paths of this cloud
    // Cells of H_k; the sampler constants of its sides are re-read (L1
    // hits) at every path start rather than held in registers.
    int cell[D];
    {
        long long rem = k;
#pragma unroll
        for (int l = 0; l < D; ++l) {
            cell[l] = (int)(rem % P.cells[l]);
            rem /= P.cells[l];
        }
    }
    // Centred basis coordinate of a start point x of cell cell[l] (the cell is
    // known: a start point is never located).
    auto start_phi = [&](R x, int l) -> R {
        if constexpr (SRMC_STEP_KIND != 0) {
            const R *b = Form<R>::cellB(P) + 4 * (P.cell_off[l] + cell[l]);
            return (x - __ldg(b + 2)) * __ldg(b + 3);
        } else {
            R t;
            if (sizeof(R) == 8) t = (x - (R)P.lo[l]) / (R)P.h[l];
            else t = (x - (R)P.lo_f[l]) * (R)P.r_f[l];
            return (R)2 * (t - (R)cell[l]) - (R)1;
        }
    };
    auto sample_start = [&](unsigned w, int l) -> R {
        const R *cf = Form<R>::cellF(P) + 3 * (P.cell_off[l] + cell[l]);
        return sample_cell(w, __ldg(cf), __ldg(cf + 1), __ldg(cf + 2), Form<R>::mu_arg(P));
    };

    // ---------------- phase A: responses of the Z and Y fits ---------------
    MA mA;
    if constexpr (RS) mA.zero(lane); else mA.zero();
    int since_flush = 0;
    // TILE: the two columns whose dot product is this lane's entry e = lane + 32 s,
    // and the entry's running sum
    [[maybe_unused]] int colA[LF], colB[LF];
    [[maybe_unused]] double csum[LF];
    // The column pair (a, b) of moment entry e: Gram (a, b) row by row for
    // a <= b, then the Z right-hand sides (phi_a, w_l), then the Y one (phi_a, S_Y).
    auto tile_pair = [&](int e, int &a, int &b) {
        a = 0; b = 0;
        if (e < EG) {
            int rem = e;
            while (rem >= p - a) { rem -= p - a; ++a; }
            b = a + rem;
        } else if (e < EG + EZ) {
            a = (e - EG) % p;
            b = p + (e - EG) / p;
        } else if (e < EA) {
            a = e - EG - EZ;
            b = p + q;
        }
    };
    if constexpr (TSM) {
        for (int e = threadIdx.x; e < EA; e += blockDim.x) {
            int a, b;
            tile_pair(e, a, b);
            sm.tcol[e] = make_short2((short)a, (short)b);
        }
        for (int e = lane; e < EA; e += 32) redA[warp][e] = 0.0;
        __syncthreads();
    } else if constexpr (TILE) {
#pragma unroll
        for (int t = 0; t < LF; ++t) {
            const int e = lane + 32 * t;
            int a, b;
            tile_pair(e, a, b);
            colA[t] = a * TS + 32 * warp;
            colB[t] = b * TS + 32 * warp;
            csum[t] = 0.0;
        }
    }
    for (long long m0 = 0; m0 < Mk; m0 += blockDim.x) {
        const long long m = m0 + threadIdx.x;
        const bool valid = m < Mk;
        Words W;
        W.init(P, (unsigned)m, (unsigned)k, (unsigned)i);
        R x[D], phi[p], dwi[q], xj[D], zj[q], yn;
        phi[0] = (R)1;
        {
            unsigned ws[D];
            W.template take<0, D, true>(P, ws);
#pragma unroll
            for (int l = 0; l < D; ++l) {
                x[l] = sample_start(ws[l], l);
                if (LP1) phi[1 + l] = start_phi(x[l], l);
            }
            add_quadratic<R, D, p>(phi);
        }
        {
            unsigned wd[q], we[q];
            W.template take<D % 4, q, false>(P, wd);
            if constexpr (NW == 2) W.template take<(D + q) % 4, q, false>(P, we);
            scaled_normals<q>(wd, sdt, dwi);
            if constexpr (SRMC_STEP_DYN == 2) {
                advance<R, D>(P, i, x, dwi, xj);
            } else {
#pragma unroll
                for (int l = 0; l < D; ++l) {
                    xj[l] = next_coord<R, D>(P, i, l, x, dwi[l], NW == 2 ? normal_of(we[l], (R)0) : (R)0);
                }
            }
        }
        // (CI below reads phi and dwi before they are parked)
        [[maybe_unused]] R CI = (R)0, CZ = (R)0;
        if constexpr (CV) {
            if (!P.cv_own) CI = control_dot<R, D, p>(P, (unsigned)i * (unsigned)P.K + (unsigned)k, phi, dwi);
        }
        if constexpr (Stage<R, D>::value) {
#pragma unroll
            for (int a = 1; a < p; ++a) sm.tile[a][threadIdx.x] = (float)phi[a];
#pragma unroll
            for (int l = 0; l < q; ++l) sm.tile[p + l][threadIdx.x] = (float)dwi[l];
        }
        // Martingale control: CI = zc_i(x_i).dW_i (stratum k), CZ = sum_{j>i} zc_j(X_j).dW_j,
        // zc_j evaluated at X_j from the control row of (j, stratum of X_j); with the
        // run's own control zc_j = z_j, the fitted z of step j, and CI = 0.
        // the control's integrand zc_j(X_j) (from the control row of (j, stratum
        // of X_j)), evaluated when X_j is located and carried to step j
        [[maybe_unused]] R phij[p];
        [[maybe_unused]] unsigned rowj = 0;
        [[maybe_unused]] R zcj[q];
        // A driver that does not read z: f_i(x_i, y_{i+1}(X_{i+1})) is known
        // after this first step, so the Y response is complete in phase A (no
        // phase B).  Its part in x_i is taken before X_{i+1} is located.
        [[maybe_unused]] R fdt = (R)0;
        if constexpr (!ZIN) fdt = model_f_x<R, D, MODEL>(P, i, x);
        eval_at<R, D, LP1, MODEL, ZIN, CV, FLOW>(P, i + 1, xj, yn, zj, phij, rowj);
        if constexpr (CV) {
            if (!P.cv_own && i + 1 < P.N) control_vals<R, D, p>(P, rowj, phij, zcj);
        }
        if constexpr (!ZIN) fdt = dt * model_f_y<R, D, MODEL>(P, yn, fdt);
        [[maybe_unused]] R zsum = (R)0;
        if constexpr (ZSUM) {
#pragma unroll
            for (int l = 0; l < q; ++l) zsum += zj[l];
        }
        R S = (R)0;
        // Steps j = i+1 .. N-1 in groups of G, so that the word phase of
        // every step in a group is a compile-time constant.
        constexpr int G = 4 / gcd_c(NW * q, 4);
        for (int j0 = i + 1; j0 < P.N; j0 += G) {
            static_for<0, G>([&](auto gc) {
                constexpr int g = decltype(gc)::value;
                const int j = j0 + g;
                if (j >= P.N) return;
                unsigned wn[q];
                [[maybe_unused]] unsigned we[q];
                W.template take<(D + NW * q * (1 + g)) % 4, q, false>(P, wn);
                if constexpr (NW == 2) W.template take<(D + q + NW * q * (1 + g)) % 4, q, false>(P, we);
                R xn[D], zn[q], dw[q];
                scaled_normals<q>(wn, sdt, dw);
                if constexpr (NW == 1) {
                    advance<R, D>(P, j, xj, dw, xn);
                } else {
#pragma unroll
                    for (int l = 0; l < D; ++l)
                        xn[l] = next_coord<R, D>(P, j, l, xj, dw[l], normal_of(we[l], (R)0));
                }
                if constexpr (CV) {
                    // own control: z_j(X_j), already evaluated for the driver
                    bool own = false;
                    if constexpr (ZIN) {
                        if (P.cv_own) {
                            own = true;
#pragma unroll
                            for (int l = 0; l < q; ++l) CZ += zj[l] * dw[l];
                        }
                    }
                    if (!own) CZ += control_apply<R, q>(zcj, dw);
                }
                [[maybe_unused]] R fx = (R)0;
                if constexpr (!ZIN) fx = model_f_x<R, D, MODEL>(P, j, xj);
                eval_at<R, D, LP1, MODEL, ZIN, CV, FLOW>(P, j + 1, xn, yn, zn, phij, rowj);
                if constexpr (CV) {
                    if (!P.cv_own && j + 1 < P.N) control_vals<R, D, p>(P, rowj, phij, zcj);
                }
                if constexpr (ZSUM) {
                    S += dt * logistic_f<R, q>(yn, zsum);
                    zsum = (R)0;
#pragma unroll
                    for (int l = 0; l < q; ++l) zsum += zn[l];
                } else if constexpr (ZIN) {
                    S += dt * model_f<R, D, MODEL, ZIN, q>(P, j, xj, yn, zj);
                } else {
                    S += dt * model_f_y<R, D, MODEL>(P, yn, fx);
                }
#pragma unroll
                for (int l = 0; l < D; ++l) xj[l] = xn[l];
#pragma unroll
                for (int l = 0; l < q; ++l) zj[l] = zn[l];
            });
        }
        S += model_g<R, D, MODEL>(P, xj);
        if constexpr (Stage<R, D>::value) {
            const volatile float *st = &sm.tile[0][threadIdx.x];
            if constexpr (!TILE) {
#pragma unroll
                for (int a = 1; a < p; ++a) phi[a] = (R)st[a * TS];
            }
#pragma unroll
            for (int l = 0; l < q; ++l) dwi[l] = (R)st[(p + l) * TS];
        }
        // Z response uses S - CZ; the phase-A part of the Y response S - CZ - CI.
        R SZ = S, SY = S;
        if constexpr (CV) { SZ = S - CZ; SY = SZ - CI; }
        if constexpr (!ZIN) SY += fdt;
        if constexpr (TILE) {
            // this path's columns (zeros past M_k), then the warp's dot products
            float *col = &sm.tile[0][threadIdx.x];
            col[0] = valid ? 1.0f : 0.0f;
            if (!Stage<R, D>::value || !valid) {
#pragma unroll
                for (int a = 1; a < p; ++a) col[a * TS] = valid ? (float)phi[a] : 0.0f;
            }
#pragma unroll
            for (int l = 0; l < q; ++l) col[(p + l) * TS] = valid ? (float)(SZ * dwi[l] * inv_dt) : 0.0f;
            col[(p + q) * TS] = valid ? (float)SY : 0.0f;
            __syncwarp();
            const float *tb = &sm.tile[0][0];
            if constexpr (TSM) {
                for (int e = lane; e < EA; e += 32) {
                    const short2 c = sm.tcol[e];
                    const float *ca = tb + c.x * TS + 32 * warp, *cb = tb + c.y * TS + 32 * warp;
                    float acc1 = 0.0f;
#pragma unroll 2
                    for (int r = 0; r < 32; r += 4) {
                        const float4 a4 = *reinterpret_cast<const float4 *>(ca + r);
                        const float4 b4 = *reinterpret_cast<const float4 *>(cb + r);
                        acc1 = fmaf(a4.x, b4.x, acc1);
                        acc1 = fmaf(a4.y, b4.y, acc1);
                        acc1 = fmaf(a4.z, b4.z, acc1);
                        acc1 = fmaf(a4.w, b4.w, acc1);
                    }
                    redA[warp][e] += (double)acc1;
                }
                __syncwarp();
            } else {
            float acc[LF];
#pragma unroll
            for (int t = 0; t < LF; ++t) acc[t] = 0.0f;
#pragma unroll 1
            for (int r = 0; r < 32; r += 4)
#pragma unroll
                for (int t = 0; t < LF; ++t) {
                    const float4 a4 = *reinterpret_cast<const float4 *>(tb + colA[t] + r);
                    const float4 b4 = *reinterpret_cast<const float4 *>(tb + colB[t] + r);
                    acc[t] = fmaf(a4.x, b4.x, acc[t]);
                    acc[t] = fmaf(a4.y, b4.y, acc[t]);
                    acc[t] = fmaf(a4.z, b4.z, acc[t]);
                    acc[t] = fmaf(a4.w, b4.w, acc[t]);
                }
#pragma unroll
            for (int t = 0; t < LF; ++t) csum[t] += (double)acc[t];
            __syncwarp();
            }
        } else if constexpr (RS) {
            // this path's products (zero for lanes past M)
            const float Sv = valid ? (float)SZ : 0.0f;
            const float Sy = valid ? (float)SY : 0.0f;
            const float g1 = valid ? 1.0f : 0.0f;
            float v[EA];
#pragma unroll
            for (int e = 0; e < EG; ++e) v[e] = g1 * phi[tri_a(e, p)] * phi[tri_b(e, p)];
#pragma unroll
            for (int l = 0; l < q; ++l) {
                const float wz = Sv * (float)dwi[l] * (float)inv_dt;
#pragma unroll
                for (int a = 0; a < p; ++a) v[EG + l * p + a] = (float)phi[a] * wz;
            }
#pragma unroll
            for (int a = 0; a < p; ++a) v[EG + EZ + a] = (float)phi[a] * Sy;
            mA.add_path(v, lane);
        } else {
            if (valid) {
                int e = 0;
                if (LP1) {
#pragma unroll
                    for (int a = 0; a < p; ++a)
#pragma unroll
                        for (int b = a; b < p; ++b) mA.add(e++, phi[a] * phi[b]);
                }
#pragma unroll
                for (int l = 0; l < q; ++l) {
                    const R wz = SZ * dwi[l] * inv_dt;
#pragma unroll
                    for (int a = 0; a < p; ++a) mA.add(EG + l * p + a, phi[a] * wz);
                }
#pragma unroll
                for (int a = 0; a < p; ++a) mA.add(EG + EZ + a, phi[a] * SY);
            }
            if (++since_flush == FLUSH) { mA.flush(lane); since_flush = 0; }
        }
    }
    if constexpr (TSM) {
        __syncthreads();
        for (int e = threadIdx.x; e < EA; e += blockDim.x) {
            double v = 0.0;
            for (int w = 0; w < nwarps; ++w) v += redA[w][e];
            totA[e] = v;
        }
        __syncthreads();
    } else if constexpr (TILE) {
        block_totals<EA>(csum, redA, totA, lane, warp, nwarps);
    } else if constexpr (RS) {
        block_totals_rs<EA>(mA.c, mA.base, mA.rend, redA, totA, warp, nwarps);
    } else {
        double lv[(EA + 31) / 32];
        mA.finish(lv, lane);
        block_totals<EA>(lv, redA, totA, lane, warp, nwarps);
    }

    // ---------------- Z fit (FP64, one warp) -----------------------------
    if (warp == 0) {
        const double Md = (double)Mk;
        bool ok = true;
        if (LP1) ok = cholesky_warp<p>(totA, Gw, Ls, Linv, lane);
        __syncwarp();
        for (int l = lane; l < q; l += 32) {
            if (LP1 && ok) {
                chol_solve<p>(Ls, Linv, totA + EG + l * p, beta_s + l * p);
            } else {
                const double m0 = totA[EG + l * p] / Md;
                for (int a = 0; a < p; ++a) beta_s[l * p + a] = (a == 0) ? m0 : 0.0;
            }
        }
        __syncwarp();
        for (int a = lane; a < q * p; a += 32) beta_r[a] = (R)beta_s[a];
        if (lane == 0) ok_s = ok ? 1 : 0;
    }
    __syncthreads();

    // ---------------- phase B: the f_i term of the Y response ----------------
    // Only for drivers that read z: f_i then needs z_i(x_i) from the Z fit
    // above (Z before Y), so the paths of the cloud are regenerated.
    if constexpr (ZIN) {
        MB mB;
        mB.zero();
        since_flush = 0;
        for (long long m0 = 0; m0 < Mk; m0 += blockDim.x) {
            const long long m = m0 + threadIdx.x;
            const bool valid = m < Mk;
            Words W;
            W.init(P, (unsigned)m, (unsigned)k, (unsigned)i);
            R x[D], phi[p], x1[D], y1, z1[q], zi[q];
            phi[0] = (R)1;
            {
                unsigned ws[D];
                W.template take<0, D, true>(P, ws);
#pragma unroll
                for (int l = 0; l < D; ++l) {
                    x[l] = sample_start(ws[l], l);
                    if (LP1) phi[1 + l] = start_phi(x[l], l);
                }
                add_quadratic<R, D, p>(phi);
            }
            {
                unsigned wd[q], we[q];
                W.template take<D % 4, q, false>(P, wd);
                if constexpr (NW == 2) W.template take<(D + q) % 4, q, false>(P, we);
                R dwb[q];
                scaled_normals<q>(wd, sdt, dwb);
                if constexpr (SRMC_STEP_DYN == 2) {
                    advance<R, D>(P, i, x, dwb, x1);
                } else {
#pragma unroll
                    for (int l = 0; l < D; ++l) {
                        x1[l] = next_coord<R, D>(P, i, l, x, dwb[l], NW == 2 ? normal_of(we[l], (R)0) : (R)0);
                    }
                }
            }
            {
                [[maybe_unused]] R phi1[p];
                [[maybe_unused]] unsigned row1;
                eval_at<R, D, LP1, MODEL, ZIN, false, FLOW>(P, i + 1, x1, y1, z1, phi1, row1);
            }
            {
                // z_i(x_i) from the fresh Z fit; long coefficient vectors are read
                // from shared memory at every path (volatile) rather than hoisted
                // into registers for the whole loop
                using BR = typename Select<(q * p > 24), const volatile R, const R>::type;
                BR *br = beta_r;
#pragma unroll
                for (int l = 0; l < q; ++l) {
                    R w = br[l * p];
#pragma unroll
                    for (int a = 1; a < p; ++a) w += br[l * p + a] * phi[a];
                    zi[l] = clamp_r(w, Form<R>::Cz(P));
                }
            }
            const R fi = model_f<R, D, MODEL, ZIN, q>(P, i, x, y1, zi);
            if (valid) {
#pragma unroll
                for (int a = 0; a < p; ++a) mB.add(a, phi[a] * fi);
            }
            if (++since_flush == FLUSH) { mB.flush(lane); since_flush = 0; }
        }
        {
            double lv[(EB + 31) / 32];
            mB.finish(lv, lane);
            block_totals<EB>(lv, redB, totB, lane, warp, nwarps);
        }
    }

    // ---------------- Y fit (FP64) and the row (i, k) -----------------------
    if (threadIdx.x == 0) {
        const double Md = (double)Mk;
        const double dtd = P.dt;
        double *alpha = totB;                      // solved in place
        for (int a = 0; a < p; ++a) alpha[a] = totA[EG + EZ + a] + (ZIN ? dtd * totB[a] : 0.0);
        if (LP1 && ok_s) {
            chol_solve<p>(Ls, Linv, alpha, alpha);
        } else {
            const double m0 = alpha[0] / Md;
            for (int a = 0; a < p; ++a) alpha[a] = (a == 0) ? m0 : 0.0;
        }
        const long long row = (long long)i * P.K + k;
        bool finite = true;
        for (int a = 0; a < p; ++a) {
            finite = finite && isfinite(alpha[a]);
            P.Y64[row * P.ry64 + a] = alpha[a];
            if (P.Y32) P.Y32[row * P.ry32 + a] = (float)alpha[a];
        }
        for (int a = 0; a < q * p; ++a) {
            finite = finite && isfinite(beta_s[a]);
            P.Z64[row * P.rz64 + a] = beta_s[a];
            if (P.Z32) P.Z32[row * P.rz32 + a] = (float)beta_s[a];
        }
        if (LP1 && !ok_s) atomicAdd(P.stats + 0, 1ull);
        if (!finite) atomicAdd(P.stats + 1, 1ull);
    }
    __syncthreads();
}

template <typename R, int D, bool LP1, int MODEL, bool ZIN, bool CV>
__global__ void __launch_bounds__(MAX_THREADS, MinBlocks<R, D, CV, ZIN>::value)
step_kernel(const Params P, const int i)
{
    auto strata = [&](StepSmem<R, D, LP1> &sm) {
        for (long long t = blockIdx.x; t < P.K; t += gridDim.x) {
            const long long k = P.order ? (long long)__ldg(P.order + t) : t;
            solve_stratum<R, D, LP1, MODEL, ZIN, CV>(P, i, k, sm);
        }
    };
    if constexpr (DYN_SMEM) {
        extern __shared__ __align__(16) unsigned char srmc_dyn_smem[];
        strata(*reinterpret_cast<StepSmem<R, D, LP1> *>(srmc_dyn_smem));
    } else {
        __shared__ StepSmem<R, D, LP1> sm;
        strata(sm);
    }
}

#ifndef __CUDACC_RTC__
// Batched form: one launch per round and group of instances with the same
// kernel variant.  Work item t is stratum t - kofs[a] of active instance a;
// the block copies that instance's parameters into shared memory whenever
// its work items move to another instance (the items of one instance are
// contiguous, and the grid strides through them).
template <typename R, int D, bool LP1, int MODEL, bool ZIN, bool CV>
__global__ void __launch_bounds__(MAX_THREADS, MinBlocks<R, D, CV, ZIN>::value)
step_kernel_batch(const BatchRound B)
{
    __shared__ StepSmem<R, D, LP1> sm;
    __shared__ __align__(16) Params Ps;
    int cur = -1;
    for (long long t = blockIdx.x; t < B.total; t += gridDim.x) {
        int lo = 0, hi = B.n_active - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(B.kofs + mid) <= t) lo = mid; else hi = mid - 1;
        }
        if (lo != cur) {                          // the same decision in every thread
            __syncthreads();
            const int *src = reinterpret_cast<const int *>(B.params + __ldg(B.inst + lo));
            int *dst = reinterpret_cast<int *>(&Ps);
            for (int e = threadIdx.x; e < (int)(sizeof(Params) / sizeof(int)); e += blockDim.x)
                dst[e] = __ldg(src + e);
            __syncthreads();
            cur = lo;
        }
        solve_stratum<R, D, LP1, MODEL, ZIN, CV>(Ps, __ldg(B.step + lo), t - __ldg(B.kofs + lo), sm);
    }
}

// The persistent batched form (FlowPlan): one launch per kernel variant over
// all rounds of all its instances.  Blocks take work items in round order
// from a global counter; an item of step i waits for the whole step i + 1 of
// its instance (written by other blocks of the same launch), then reads
// those rows with cached coherent loads (FLOW) after a device-scope fence.
// Every item waited for was handed out earlier to a running block whose own
// waits are for still earlier items, so the waits always end; each also has
// an iteration limit, after which it flags *error and goes on.
constexpr unsigned FLOW_SPIN_LIMIT = 1u << 23;      // x ~128 ns sleep: about a second

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

template <typename R, int D, bool LP1, int MODEL, bool ZIN, bool CV>
__global__ void __launch_bounds__(MAX_THREADS, MinBlocks<R, D, CV, ZIN>::value)
step_kernel_flow(const FlowPlan F)
{
    __shared__ StepSmem<R, D, LP1> sm;
    __shared__ __align__(16) Params Ps;
    __shared__ long long item_s;
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) item_s = (long long)atomicAdd(F.next, 1ull);
        __syncthreads();
        const long long t = item_s;
        if (t >= F.total) break;
        int lo = 0, hi = F.n_seg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(F.kofs + mid) <= t) lo = mid; else hi = mid - 1;
        }
        if (threadIdx.x == 0) {
            const int dseg = __ldg(F.dep + lo);
            if (dseg >= 0) {
                const unsigned long long need =
                    (unsigned long long)(__ldg(F.kofs + dseg + 1) - __ldg(F.kofs + dseg));
                unsigned spins = 0;
                while (ld_acquire_u64(F.done + dseg) < need) {
                    if (++spins > FLOW_SPIN_LIMIT) { atomicExch(F.error, 1u); break; }
                    __nanosleep(128);
                }
            }
            __threadfence();
        }
        const int r = __ldg(F.inst + lo);
        if (r != cur) {                           // the same decision in every thread
            __syncthreads();
            const int *src = reinterpret_cast<const int *>(F.params + r);
            int *dst = reinterpret_cast<int *>(&Ps);
            for (int e = threadIdx.x; e < (int)(sizeof(Params) / sizeof(int)); e += blockDim.x)
                dst[e] = __ldg(src + e);
            cur = r;
        }
        __syncthreads();
        solve_stratum<R, D, LP1, MODEL, ZIN, CV, true>(Ps, __ldg(F.step + lo), t - __ldg(F.kofs + lo), sm);
        if (threadIdx.x == 0) {
            __threadfence();                       // the rows of (step, stratum) before the count
            atomicAdd(F.done + lo, 1ull);
        }
    }
}

template <typename R, bool LP1, int MODEL, bool ZIN, bool CV>
cudaError_t launch_flow_one(const FlowPlan &F, int grid, int threads, cudaStream_t st)
{
    step_kernel_flow<R, SRMC_STEP_D, LP1, MODEL, ZIN, CV><<<grid, threads, 0, st>>>(F);
    return cudaGetLastError();
}

template <typename R, bool LP1, int MODEL, bool ZIN, bool CV>
int occ_flow_one(int threads)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, step_kernel_flow<R, SRMC_STEP_D, LP1, MODEL, ZIN, CV>, threads, 0) != cudaSuccess)
        return 0;
    return n;
}

template <typename R, bool LP1, int MODEL, bool ZIN, bool CV>
cudaError_t launch_batch_one(const BatchRound &B, int grid, int threads, cudaStream_t st)
{
    step_kernel_batch<R, SRMC_STEP_D, LP1, MODEL, ZIN, CV><<<grid, threads, 0, st>>>(B);
    return cudaGetLastError();
}

template <typename R, bool LP1, int MODEL, bool ZIN, bool CV>
int occ_batch_one(int threads)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, step_kernel_batch<R, SRMC_STEP_D, LP1, MODEL, ZIN, CV>, threads, 0) != cudaSuccess)
        return 0;
    return n;
}

// Dispatch of the batched kernels over (precision, basis, model variant,
// control): F is called with the template arguments as a functor.
template <typename R, typename F>
auto dispatch_variant(bool lp1, int mv, bool cv, F &&f) -> decltype(f.template operator()<R, true, MODEL_COS, false, false>())
{
    using Ret = decltype(f.template operator()<R, true, MODEL_COS, false, false>());
    if (cv) {
        if (!lp1) return Ret{};
        switch (mv) {
        case MV_COS:      return f.template operator()<R, true, MODEL_COS, false, true>();
        case MV_COS_Z:    return f.template operator()<R, true, MODEL_COS, true, true>();
        case MV_LOGISTIC: return f.template operator()<R, true, MODEL_LOGISTIC, true, true>();
        }
        return Ret{};
    }
    switch (mv) {
    case MV_COS:      return lp1 ? f.template operator()<R, true, MODEL_COS, false, false>()
                                 : f.template operator()<R, false, MODEL_COS, false, false>();
    case MV_COS_Z:    return lp1 ? f.template operator()<R, true, MODEL_COS, true, false>()
                                 : f.template operator()<R, false, MODEL_COS, true, false>();
    case MV_LOGISTIC: return lp1 ? f.template operator()<R, true, MODEL_LOGISTIC, true, false>()
                                 : f.template operator()<R, false, MODEL_LOGISTIC, true, false>();
    case MV_AFFINE:   return lp1 ? f.template operator()<R, true, MODEL_AFFINE, false, false>()
                                 : f.template operator()<R, false, MODEL_AFFINE, false, false>();
    }
    return Ret{};
}

template <typename R, bool LP1, int MODEL, bool ZIN, bool CV = false>
cudaError_t launch_one(const Params &P, int i, int grid, int threads, cudaStream_t st)
{
    const size_t smem = DYN_SMEM ? sizeof(StepSmem<R, SRMC_STEP_D, LP1>) : 0;
    step_kernel<R, SRMC_STEP_D, LP1, MODEL, ZIN, CV><<<grid, threads, smem, st>>>(P, i);
    return cudaGetLastError();
}

// Units of d >= 12: allow each FP32 LP0/LP1 kernel its dynamic shared memory
// (a function attribute, set once before the first launch, outside any
// stream capture).
template <typename R, bool LP1, int MODEL, bool ZIN>
cudaError_t allow_smem_one()
{
    if constexpr (!DYN_SMEM) {
        return cudaSuccess;
    } else {
        return cudaFuncSetAttribute(step_kernel<R, SRMC_STEP_D, LP1, MODEL, ZIN, false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sizeof(StepSmem<R, SRMC_STEP_D, LP1>));
    }
}

// Units of d >= 9 carry the FP32 form without controls only (create rejects
// the rest), which keeps their compile time and code size down.
constexpr bool WIDE_UNIT = SRMC_STEP_D >= 9;

template <typename R>
cudaError_t launch_prec(const Params &P, int i, bool lp1, int mv, int grid, int threads,
                        cudaStream_t st)
{
    if constexpr (WIDE_UNIT && sizeof(R) == 8) {
        return cudaErrorInvalidValue;
    } else {
    if (P.C64 != nullptr || P.cv_own) { // control variate form (LP1 only)
        if constexpr (WIDE_UNIT) return cudaErrorInvalidValue;
        else {
        if (!lp1) return cudaErrorInvalidValue;
        switch (mv) {
        case MV_COS:      return launch_one<R, true, MODEL_COS, false, true>(P, i, grid, threads, st);
        case MV_COS_Z:    return launch_one<R, true, MODEL_COS, true, true>(P, i, grid, threads, st);
        case MV_LOGISTIC: return launch_one<R, true, MODEL_LOGISTIC, true, true>(P, i, grid, threads, st);
        }
        return cudaErrorInvalidValue;
        }
    }
    switch (mv) {
    case MV_COS:      return lp1 ? launch_one<R, true, MODEL_COS, false>(P, i, grid, threads, st)
                                 : launch_one<R, false, MODEL_COS, false>(P, i, grid, threads, st);
    case MV_COS_Z:    return lp1 ? launch_one<R, true, MODEL_COS, true>(P, i, grid, threads, st)
                                 : launch_one<R, false, MODEL_COS, true>(P, i, grid, threads, st);
    case MV_LOGISTIC: return lp1 ? launch_one<R, true, MODEL_LOGISTIC, true>(P, i, grid, threads, st)
                                 : launch_one<R, false, MODEL_LOGISTIC, true>(P, i, grid, threads, st);
    case MV_AFFINE:   return lp1 ? launch_one<R, true, MODEL_AFFINE, false>(P, i, grid, threads, st)
                                 : launch_one<R, false, MODEL_AFFINE, false>(P, i, grid, threads, st);
    }
    return cudaErrorInvalidValue;
    }
}

}  // namespace

#if SRMC_STEP_KIND == 0 && SRMC_STEP_DYN == 0 && SRMC_STEP_BASIS == 1 && SRMC_STEP_D <= 8
namespace {
struct BatchLauncher {
    const BatchRound &B; int grid, threads; cudaStream_t st;
    template <typename R, bool LP1, int MODEL, bool ZIN, bool CV>
    cudaError_t operator()() { return launch_batch_one<R, LP1, MODEL, ZIN, CV>(B, grid, threads, st); }
};
struct BatchOccupancy {
    int threads;
    template <typename R, bool LP1, int MODEL, bool ZIN, bool CV>
    int operator()() { return occ_batch_one<R, LP1, MODEL, ZIN, CV>(threads); }
};
struct FlowLauncher {
    const FlowPlan &F; int grid, threads; cudaStream_t st;
    template <typename R, bool LP1, int MODEL, bool ZIN, bool CV>
    cudaError_t operator()() { return launch_flow_one<R, LP1, MODEL, ZIN, CV>(F, grid, threads, st); }
};
struct FlowOccupancy {
    int threads;
    template <typename R, bool LP1, int MODEL, bool ZIN, bool CV>
    int operator()() { return occ_flow_one<R, LP1, MODEL, ZIN, CV>(threads); }
};
}  // namespace

cudaError_t SRMC_LAUNCH_FLOW_NAME(SRMC_STEP_D)(const FlowPlan &F, bool lp1, int mv, bool cv, int grid, int threads,
                                                cudaStream_t st)
{
    const bool ok = !(cv && !lp1) && mv >= MV_COS && mv <= MV_AFFINE && !(cv && mv == MV_AFFINE);
    if (!ok) return cudaErrorInvalidValue;
    FlowLauncher f{F, grid, threads, st};
    return dispatch_variant<float>(lp1, mv, cv, f);
}

int SRMC_OCC_FLOW_NAME(SRMC_STEP_D)(bool lp1, int mv, bool cv, int threads)
{
    FlowOccupancy f{threads};
    return dispatch_variant<float>(lp1, mv, cv, f);
}

cudaError_t SRMC_LAUNCH_BATCH_NAME(SRMC_STEP_D)(const BatchRound &B, bool fp64, bool lp1, int mv, bool cv,
                                                 int grid, int threads, cudaStream_t st)
{
    // combinations without a kernel (dispatch_variant would return Ret{} = 0)
    const bool ok = !(cv && !lp1) && mv >= MV_COS && mv <= MV_AFFINE && !(cv && mv == MV_AFFINE);
    if (!ok) return cudaErrorInvalidValue;
    if (fp64) return cudaErrorInvalidValue;     // the batched form is built for FP32 paths
    BatchLauncher f{B, grid, threads, st};
    return dispatch_variant<float>(lp1, mv, cv, f);
}

int SRMC_OCC_BATCH_NAME(SRMC_STEP_D)(bool fp64, bool lp1, int mv, bool cv, int threads)
{
    if (fp64) return 0;
    BatchOccupancy f{threads};
    return dispatch_variant<float>(lp1, mv, cv, f);
}

#endif  // batched form

#if SRMC_STEP_KIND == 0 && SRMC_STEP_DYN == 0 && SRMC_STEP_BASIS == 1 && SRMC_STEP_D >= 12
cudaError_t SRMC_PREPARE_STEP_NAME(SRMC_STEP_D)()
{
    cudaError_t e = cudaSuccess;
    const cudaError_t r[8] = {
        allow_smem_one<float, true, MODEL_COS, false>(), allow_smem_one<float, false, MODEL_COS, false>(),
        allow_smem_one<float, true, MODEL_COS, true>(), allow_smem_one<float, false, MODEL_COS, true>(),
        allow_smem_one<float, true, MODEL_LOGISTIC, true>(), allow_smem_one<float, false, MODEL_LOGISTIC, true>(),
        allow_smem_one<float, true, MODEL_AFFINE, false>(), allow_smem_one<float, false, MODEL_AFFINE, false>()};
    for (cudaError_t v : r)
        if (v != cudaSuccess) e = v;
    return e;
}
#endif

#if SRMC_STEP_BASIS == 2
cudaError_t SRMC_LAUNCH_STEP_QUAD_NAME(SRMC_STEP_D)(const Params &P, int i, bool fp64, bool lp1, int mv,
                                                     int grid, int threads, cudaStream_t st)
#elif SRMC_STEP_DYN == 1
cudaError_t SRMC_LAUNCH_STEP_EXACT_NAME(SRMC_STEP_D)(const Params &P, int i, bool fp64, bool lp1, int mv,
                                                      int grid, int threads, cudaStream_t st)
#elif SRMC_STEP_DYN == 2 && SRMC_STEP_Q != SRMC_STEP_D
cudaError_t SRMC_LAUNCH_STEP_DENSEQ_NAME(SRMC_STEP_D, SRMC_STEP_Q)(const Params &P, int i, bool fp64, bool lp1,
                                                                    int mv, int grid, int threads, cudaStream_t st)
#elif SRMC_STEP_DYN == 2
cudaError_t SRMC_LAUNCH_STEP_DENSE_NAME(SRMC_STEP_D)(const Params &P, int i, bool fp64, bool lp1, int mv,
                                                      int grid, int threads, cudaStream_t st)
#elif SRMC_STEP_KIND == 0
cudaError_t SRMC_LAUNCH_STEP_NAME(SRMC_STEP_D)(const Params &P, int i, bool fp64, bool lp1, int mv,
                                                int grid, int threads, cudaStream_t st)
#else
cudaError_t SRMC_LAUNCH_STEP_PROB_NAME(SRMC_STEP_D)(const Params &P, int i, bool fp64, bool lp1, int mv,
                                                     int grid, int threads, cudaStream_t st)
#endif
{
    return fp64 ? launch_prec<double>(P, i, lp1, mv, grid, threads, st)
                : launch_prec<float>(P, i, lp1, mv, grid, threads, st);
}
#else
}  // namespace (the unit-local one; in library builds it closes above)
#endif  // !__CUDACC_RTC__

}  // namespace srmc

#ifdef __CUDACC_RTC__
// Entry point of a run-time compiled unit: a user model (MODEL_USER, z read at
// every path point) in the precision SRMC_RTC_REAL, with the affine part of the
// basis when SRMC_RTC_LP1 and the control variate when SRMC_RTC_CV.
extern "C" __global__ void
__launch_bounds__(srmc::MAX_THREADS,
                  srmc::MinBlocks<SRMC_RTC_REAL, SRMC_STEP_D, SRMC_RTC_CV != 0, true>::value)
srmc_user_step(const srmc::Params P, const int i)
{
    __shared__ srmc::StepSmem<SRMC_RTC_REAL, SRMC_STEP_D, SRMC_RTC_LP1 != 0> sm;
    for (long long t = blockIdx.x; t < P.K; t += gridDim.x) {
        const long long k = P.order ? (long long)__ldg(P.order + t) : t;
        srmc::solve_stratum<SRMC_RTC_REAL, SRMC_STEP_D, SRMC_RTC_LP1 != 0, srmc::MODEL_USER, true,
                            SRMC_RTC_CV != 0>(P, i, k, sm);
    }
}
#endif
