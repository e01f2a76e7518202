// srmc_device.cuh -- device building blocks of the SRMDP hot path (sm_103a).
//
// Every function here is one step of Alg. SRMDP or of the simulation it
// relies on; the passage is named beside each.  FP32 and FP64 forms are
// overloads of the same definition.
#pragma once

// Compiled by nvcc into the library and, for user models, by NVRTC at run
// time (__CUDACC_RTC__: device code only, no host headers).
#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#endif
#include <cuda_fp16.h>

namespace srmc {

constexpr int DMAX = 19;
// A non-diagonal constant diffusion matrix (q = d) is built for d <= SD_DMAX.
constexpr int SD_DMAX = 8;
constexpr int PBMAX = 20;            // largest basis dimension: LP1 at d = 19 (20), LP2 at d = 3 (10)

// The quadratic monomials u_a u_b (a <= b, row order) after the linear ones
// of a basis vector of dimension p, for d only known at run time.
__host__ __device__ __forceinline__ void add_quadratic_rt(double *phi, int d, int p)
{
    if (p <= d + 1) return;
    int e = 1 + d;
    for (int a = 0; a < d; ++a)
        for (int b = a; b < d; ++b) phi[e++] = phi[1 + a] * phi[1 + b];
}
constexpr int PMAX = 24;
constexpr int MAX_THREADS = 256;
constexpr int MAX_WARPS = MAX_THREADS / 32;

enum Model { MODEL_COS = 0, MODEL_LOGISTIC = 1, MODEL_AFFINE = 2, MODEL_USER = 3 };

// Everything a step launch needs, passed by value as the kernel parameter.
struct Params {
    int d, q, N, p;                 // dims, steps, basis dimension
    int ry32, rz32, ry64, rz64;     // row strides of the coefficient tables
    long long K, M;
    int model;
    int cells[DMAX];
    int stride[DMAX];               // stratum index stride of each dimension
    unsigned kbias;                 // sum_l 0x4B000000 stride_l mod 2^32 (cell location by rounding)
    int cell_off[DMAX];             // offset of dimension l in cellF
    double lo[DMAX], h[DMAX], b[DMAX], sig[DMAX];
    float lo_f[DMAX], r_f[DMAX], b_f[DMAX], sig_f[DMAX];
    // One step of the chain, per coordinate: X' = A X + c + s1 dW + s2 xi2
    // (Euler: A = 1 - theta dt, c = b dt, s1 = sigma, s2 = 0; exact OU: see
    // srmc_create), and the drift's mean reversion for the driver.
    double A[DMAX], c[DMAX], s1[DMAX], s2[DMAX], theta[DMAX];
    float A_f[DMAX], c_f[DMAX], s1_f[DMAX], s2_f[DMAX], theta_f[DMAX];
    // A non-diagonal constant sigma (dense != 0, Euler dynamics): the step adds
    // sum_r sigma[l][r] dW_r to coordinate l; sd holds sigma row-major with
    // stride d (the dense units read entry l d + r with d their compiled D).
    int dense;
    double sd[SD_DMAX * SD_DMAX];
    float sd_f[SD_DMAX * SD_DMAX];
    int drift;                      // cos model: driver carries -(1/s0) b(x).z
    int unit_drift;                 // A = 1 and c = 0 in every coordinate (FP32 copies)
    double inv_s0;
    float inv_s0_f;
    double T, dt, sdt, mu, sqrt_d;
    float dt_f, sdt_f, inv_mu_f, inv_sqrt_d_f, mu_f;
    int kind;                       // 0: equal-size cells on the box, 1: equal nu-probability
    double Cy, Cz;                  // +inf when disabled
    float Cy_f, Cz_f;
    unsigned key0, key1;
    unsigned rk0[10], rk1[10];      // Philox round keys: key + r (0x9E3779B9, 0xBB67AE85)
    double prm[PMAX];
    float prm_f[PMAX];
    double lin;                     // cos model: lam + s0^2/2
    float lin_f;
    const double *cellF;            // [sum cells][3]: F(x-), 1 - F(x+), F(x+) - F(x-)
    const float *cellF_f;
    const double *cellB;            // [sum cells][4]: x-, x+, basis centre, 1 / basis unit
    const float *cellB_f;
    const double *stepc;            // [N+1][2] per-step driver constants
    const float *stepc_f;
    float *Y32, *Z32;               // [N][K][ry32], [N][K][rz32]; N K r < 2^32
    double *Y64, *Z64;              // [N][K][ry64], [N][K][rz64]
    const __half *C16;              // control rows of the FP32 form in binary16, coefficient-major:
    int ph, rc16;                   // half (r, a, l) at r rc16 + a ph + l; ph = q rounded up to even,
                                    // rc16 = p ph rounded up to 8 (16-byte rows)
    const double *C64;              // control rows [N][K][rz64]
    unsigned long long *stats;      // [0] LP1->LP0 fallbacks, [1] non-finite rows
    const unsigned *order;          // [K] stratum solved by work item t (NULL: t itself)
    const unsigned *Mk;             // [K] paths of each stratum (NULL: M for all)
    int cv_own;                     // control from the fitted z of later steps (ZIN kernels)
};

// ---- Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) --------------------
// The 32 x 32 -> 64-bit product of a round's multiplier and counter word, as
// (hi, lo).  With SRMC_PHILOX_WIDE the product is one mul.wide.u32 whose two
// halves are the high and low words; otherwise the high and low words are
// formed separately (__umulhi and the wrapping product).  Measured on GB300:
// the wide form is 1 % faster for d <= 3 and 0.5 % slower for d = 6 (register
// allocation), so it is the default for the small dimensions only.
#ifndef SRMC_PHILOX_WIDE
#if defined(SRMC_STEP_D) && SRMC_STEP_D > 3
#define SRMC_PHILOX_WIDE 0
#else
#define SRMC_PHILOX_WIDE 1
#endif
#endif
__device__ __forceinline__ void mul_hilo(unsigned a, unsigned b, unsigned &hi, unsigned &lo)
{
#if SRMC_PHILOX_WIDE && !defined(__CUDACC_RTC__)
    unsigned long long r;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(r) : "r"(a), "r"(b));
    lo = (unsigned)r;
    hi = (unsigned)(r >> 32);
#else
    hi = __umulhi(a, b);
    lo = a * b;
#endif
}

__device__ __forceinline__ void philox10(unsigned &c0, unsigned &c1, unsigned &c2, unsigned &c3,
                                         const unsigned (&rk0)[10], const unsigned (&rk1)[10])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        unsigned hi0, lo0, hi1, lo1;
        mul_hilo(0xD2511F53u, c0, hi0, lo0);
        mul_hilo(0xCD9E8D57u, c2, hi1, lo1);
        const unsigned n0 = hi1 ^ c1 ^ rk0[r];
        const unsigned n2 = hi0 ^ c3 ^ rk1[r];
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
}

// The same with the round keys derived on the fly from the key (k0, k1).
__device__ __forceinline__ void philox10(unsigned &c0, unsigned &c1, unsigned &c2, unsigned &c3,
                                         unsigned k0, unsigned k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        unsigned hi0, lo0, hi1, lo1;
        mul_hilo(0xD2511F53u, c0, hi0, lo0);
        mul_hilo(0xCD9E8D57u, c2, hi1, lo1);
        const unsigned n0 = hi1 ^ c1 ^ k0;
        const unsigned n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
}

// The word stream of one path of cloud C_{i,k}: counter (n/4, m, k, i),
// word n = position n mod 4 of block n/4.  Callers take words in order with
// a compile-time phase PH = (index of the first word) mod 4, so that every
// word is read from a fixed register; a new block is generated whenever
// the stream crosses a block boundary (FRESH: block 0 is already there).
struct Words {
    unsigned m, k, i, blk;
    unsigned w[4];
    template <typename PP>
    __device__ __forceinline__ void gen(const PP &P)
    {
        w[0] = blk; w[1] = m; w[2] = k; w[3] = i;
        philox10(w[0], w[1], w[2], w[3], P.rk0, P.rk1);
    }
    template <typename PP>
    __device__ __forceinline__ void init(const PP &P, unsigned m_, unsigned k_, unsigned i_)
    {
        m = m_; k = k_; i = i_; blk = 0;
        gen(P);
    }
    template <int PH, int CNT, bool FRESH, typename PP>
    __device__ __forceinline__ void take(const PP &P, unsigned (&out)[CNT])
    {
#pragma unroll
        for (int c = 0; c < CNT; ++c) {
            const int p = (PH + c) & 3;
            if (p == 0 && !(FRESH && c == 0)) { ++blk; gen(P); }
            out[c] = w[p];
        }
    }
    // Word at a run-time position (used off the hot loop only).
    template <typename PP>
    __device__ __forceinline__ unsigned next_dynamic(const PP &P, int &pos)
    {
        if (pos == 4) { ++blk; gen(P); pos = 0; }
        const unsigned r = pos == 0 ? w[0] : pos == 1 ? w[1] : pos == 2 ? w[2] : w[3];
        ++pos;
        return r;
    }
};

// A compile-time integer, and a compile-time choice of type.
template <int V> struct IntC { static constexpr int value = V; };
template <bool B, typename T, typename F> struct Select { using type = T; };
template <typename T, typename F> struct Select<false, T, F> { using type = F; };

// Compile-time loop: f(IntC<g>) for g = G0 .. G-1.
template <int G0, int G, typename F>
__device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (G0 < G) {
        f(IntC<G0>{});
        static_for<G0 + 1, G>(f);
    }
}

__host__ __device__ constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }

// ---- standard normal by inversion: xi = Phi^{-1}((w + 1/2) 2^-32) ----------
// The upper half is taken from the exact complement (~w + 1/2) 2^-32.
__device__ __forceinline__ double normal_of(unsigned w, double)
{
    const bool up = w >= 0x80000000u;
    const unsigned v = up ? ~w : w;
    const double x = normcdfinv(((double)v + 0.5) * 0x1p-32);
    return up ? -x : x;
}
// Single-precision Phi^{-1}: erfinv-style reduction (Giles, "Approximating
// the erfinv function", GPU Computing Gems, 2010): with y = 2p - 1 and
// w = -log(4 p (1-p)), Phi^{-1}(p) = y h(w) where h is smooth in w.  h is
// approximated by degree-9 polynomials in (w - 3) for w < 6 and in
// (sqrt(w) - c) for w >= 6, with coefficients fitted by this project
// (weighted least squares towards minimax relative error against an FP64
// Phi^{-1}; max relative error 5e-8 and 9e-8 on the two pieces; the tail
// piece was fitted for w >= 5).  The central piece covers p >= 6.2e-4, so a
// warp meets a tail word in about 8 % of its pairs of normals (20 % with the
// switch at w = 5).  p is formed from the smaller of w and ~w (p <= 1/2), so
// 1 - p and 4 p (1 - p) keep full precision in the tails; the sign is that of
// w's upper half.  Coefficients of h, highest degree first: central piece (in
// w - 3) and tail piece (in sqrt(w) - 3.435767889).
__device__ constexpr float NRM_C[10] = {
    -8.240728988e-09f, -6.130190577e-09f, 6.442992913e-07f, -2.666269438e-06f, -1.804150088e-05f,
    2.764452947e-04f, -1.182383508e-03f, -8.115578443e-03f, 3.417168856e-01f, 2.296035290e+00f};
__device__ constexpr float NRM_T[10] = {
    6.402532017e-05f, -3.551483360e-06f, -4.645976005e-04f, 9.079263546e-04f, -1.158809988e-03f,
    1.824696665e-03f, -3.379537957e-03f, 5.249740090e-03f, 1.424003482e+00f, 4.625601292e+00f};

// The two SFU approximations the transform uses: base-2 logarithm and square
// root (the tail piece only; its argument w >= 6 is far from any special case).
__device__ __forceinline__ float lg2_approx(float x)
{
    float r;
    asm("lg2.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
#ifndef SRMC_NRM_SQRT_APPROX
#define SRMC_NRM_SQRT_APPROX 1
#endif
__device__ __forceinline__ float sqrt_approx(float x)
{
#if SRMC_NRM_SQRT_APPROX
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
#else
    return sqrtf(x);
#endif
}
constexpr float NRM_LN2 = 0.693147180559945f;

// h on the two pieces, from l = log2(4 p (1 - p)) (so w = -ln2 l): the central
// piece takes s = w - 3 in one fused multiply-add of l; the tail piece
// (w >= 6, i.e. s >= 3) takes sqrt(w) - c with w = s + 3 (so that only s
// stays live).
__device__ __forceinline__ float normal_h(float l)
{
    float h;
    const float s = __fmaf_rn(l, -NRM_LN2, -3.0f);
    if (s < 3.0f) {
        h = NRM_C[0];
#pragma unroll
        for (int c = 1; c < 10; ++c) h = __fmaf_rn(h, s, NRM_C[c]);
    } else {
        const float st = __fadd_rn(sqrt_approx(__fadd_rn(s, 3.0f)), -3.435767889f);
        h = NRM_T[0];
#pragma unroll
        for (int c = 1; c < 10; ++c) h = __fmaf_rn(h, st, NRM_T[c]);
    }
    return h;
}

// With SRMC_NORMAL_EXACT_Y, y = 2p - 1 comes from the integer complement
// 2^31 - 1 - v (full relative precision next to p = 1/2, at the price of a
// second conversion); otherwise from the float p itself, exact to 2^-24
// absolute -- the effect of rounding U to float, <= 8e-8 in xi next to 0.
#ifndef SRMC_NORMAL_EXACT_Y
#define SRMC_NORMAL_EXACT_Y 0
#endif
// (The scalar form is written with the _rn intrinsics, which the compiler
// neither contracts nor rearranges, so that every kernel that inlines it --
// and the packed form, which does the same operations -- gives the same bits.)
// 4 p (1 - p) is formed as p (4 - 4 p): 4 - 4 p = 4 (1 - p) rounded once, the
// same bits as (1 - p) 4, in one instruction less.
__device__ __forceinline__ float normal_of(unsigned w, float)
{
    const bool up = w >= 0x80000000u;
    const unsigned v = up ? ~w : w;                                     // p <= 1/2
    const float p = __fmaf_rn(__uint2float_rn(v), 0x1p-32f, 0x1p-33f);
#if SRMC_NORMAL_EXACT_Y
    const float y = __fmaf_rn(__uint2float_rn(0x7FFFFFFFu - v), -0x1p-31f, -0x1p-32f);   // 2p - 1
#else
    const float y = __fmaf_rn(p, 2.0f, -1.0f);                                          // 2p - 1
#endif
    const float l = lg2_approx(__fmul_rn(p, __fmaf_rn(p, -4.0f, 4.0f)));
    const float x = __fmul_rn(y, normal_h(l));
    return up ? -x : x;
}

// Two normals at once with the packed two-wide FP32 instructions of the
// sm_100 family (one instruction issue computes both values).  The operations
// and roundings are those of normal_of(w, float) for each word, so the values
// are identical.  The central piece is evaluated for both words, the tail
// piece (rare) only when a word of the pair needs it.
#ifndef SRMC_NORMAL_PAIRS
#define SRMC_NORMAL_PAIRS 1
#endif
#if SRMC_NORMAL_PAIRS && !defined(__CUDACC_RTC__)
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 normal_pair(unsigned w0, unsigned w1)
{
    const bool up0 = w0 >= 0x80000000u, up1 = w1 >= 0x80000000u;
    const unsigned v0 = up0 ? ~w0 : w0, v1 = up1 ? ~w1 : w1;
    const float2 p = __ffma2_rn(make_float2(__uint2float_rn(v0), __uint2float_rn(v1)),
                                f2(0x1p-32f), f2(0x1p-33f));
#if SRMC_NORMAL_EXACT_Y
    const float2 y = __ffma2_rn(make_float2(__uint2float_rn(0x7FFFFFFFu - v0),
                                            __uint2float_rn(0x7FFFFFFFu - v1)),
                                f2(-0x1p-31f), f2(-0x1p-32f));
#else
    const float2 y = __ffma2_rn(p, f2(2.0f), f2(-1.0f));
#endif
    const float2 r = __fmul2_rn(p, __ffma2_rn(p, f2(-4.0f), f2(4.0f)));
    const float2 l = make_float2(lg2_approx(r.x), lg2_approx(r.y));
    const float2 s = __ffma2_rn(l, f2(-NRM_LN2), f2(-3.0f));            // w - 3
    float2 h;
    // central piece for both words; the tail piece (w >= 6, rare) only when a
    // word needs it, and only for that word
    h = f2(NRM_C[0]);
#pragma unroll
    for (int c = 1; c < 10; ++c) h = __ffma2_rn(h, s, f2(NRM_C[c]));
    const bool tx = !(s.x < 3.0f), ty = !(s.y < 3.0f);
    if (tx || ty) {
        const float2 wv = __fadd2_rn(s, f2(3.0f));
        const float2 st = __fadd2_rn(make_float2(sqrt_approx(wv.x), sqrt_approx(wv.y)), f2(-3.435767889f));
        float2 ht = f2(NRM_T[0]);
#pragma unroll
        for (int c = 1; c < 10; ++c) ht = __ffma2_rn(ht, st, f2(NRM_T[c]));
        if (tx) h.x = ht.x;
        if (ty) h.y = ht.y;
    }
    const float2 x = __fmul2_rn(y, h);
    return make_float2(up0 ? -x.x : x.x, up1 ? -x.y : x.y);
}
#endif

// out[l] = sdt Phi^{-1}(U(w[l])): the Brownian increments of one step.
template <int D>
__device__ __forceinline__ void scaled_normals(const unsigned (&w)[D], double sdt, double (&out)[D])
{
#pragma unroll
    for (int l = 0; l < D; ++l) out[l] = sdt * normal_of(w[l], 0.0);
}
template <int D>
__device__ __forceinline__ void scaled_normals(const unsigned (&w)[D], float sdt, float (&out)[D])
{
#if SRMC_NORMAL_PAIRS && !defined(__CUDACC_RTC__)
#pragma unroll
    for (int l = 0; l + 1 < D; l += 2) {
        const float2 v = __fmul2_rn(f2(sdt), normal_pair(w[l], w[l + 1]));
        out[l] = v.x;
        out[l + 1] = v.y;
    }
    if constexpr ((D & 1) != 0) out[D - 1] = sdt * normal_of(w[D - 1], 0.0f);
#else
#pragma unroll
    for (int l = 0; l < D; ++l) out[l] = sdt * normal_of(w[l], 0.0f);
#endif
}

// ---- restricted logistic sampler (assumption A_nu, Alg. 3) ------------------
// x = log(p / qc) / mu, p = F(x-) + U w, qc = 1 - F(x+) + (1 - U) w,
// w = F(x+) - F(x-): the inverse of the cell's restricted CDF.
__device__ __forceinline__ double sample_cell(unsigned w, double Flo, double Fchi, double wid,
                                              double mu)
{
    const double U = ((double)w + 0.5) * 0x1p-32;
    const double Uc = ((double)(~w) + 0.5) * 0x1p-32;
    const double p = Flo + U * wid;
    const double qc = Fchi + Uc * wid;
    return log(p / qc) / mu;
}
__device__ __forceinline__ float sample_cell(unsigned w, float Flo, float Fchi, float wid,
                                             float inv_mu)
{
    const float U = fmaf(__uint2float_rn(w), 0x1p-32f, 0x1p-33f);
    const float Uc = fmaf(__uint2float_rn(~w), 0x1p-32f, 0x1p-33f);
    const float p = fmaf(U, wid, Flo);
    const float qc = fmaf(Uc, wid, Fchi);
    return __logf(__fdividef(p, qc)) * inv_mu;
}

// ---- stratum location (assumption A_Strat, half-open cells) ----------------
// Returns the cell and the cell coordinate t = (x - lo)/h, from which the
// centred LP1 basis value 2 (t - c) - 1 follows.
__device__ __forceinline__ int locate_dim(double x, double lo, double h, int C, double &t)
{
    t = __ddiv_rn(__dsub_rn(x, lo), h);
    if (!(t >= 0.0)) return 0;
    if (t >= (double)C) return C - 1;
    const int c = (int)floor(t);
    return c > C - 1 ? C - 1 : c;
}
__device__ __forceinline__ int locate_dim(float x, float lo, float r, int C, float &t)
{
    t = __fmul_rn(__fsub_rn(x, lo), r);
    // fmaxf maps NaN to 0, like the "!(t >= 0)" test of the FP64 form.
    return (int)fminf(fmaxf(floorf(t), 0.0f), (float)(C - 1));
}

// Equal-probability cells (assumption HS, example ii): the cell of x along
// an axis of C cells whose rows B[4c..4c+3] = (x-, x+, centre, 1/unit) are
// given, and the centred basis coordinate (x - centre)/unit.  The guess
// floor(C F(x)) from the logistic CDF is off by at most one cell (F is
// accurate to a few ulps, far below 1/C), and one comparison with the
// stored edges settles it; NaN lands in cell 0 like the equal-size form.
__device__ __forceinline__ int locate_prob(double x, const double *B, int C, double mu, double &phi)
{
    const double F = 1.0 / (1.0 + exp(-mu * x));
    int c = (int)fmin(fmax(floor(F * (double)C), 0.0), (double)(C - 1));
    if (c > 0 && x < __ldg(B + 4 * c)) --c;
    else if (c < C - 1 && x >= __ldg(B + 4 * c + 1)) ++c;
    phi = (x - __ldg(B + 4 * c + 2)) * __ldg(B + 4 * c + 3);
    return c;
}
__device__ __forceinline__ int locate_prob(float x, const float *B, int C, float mu, float &phi)
{
    const float F = __fdividef(1.0f, 1.0f + __expf(-mu * x));
    int c = (int)fminf(fmaxf(floorf(F * (float)C), 0.0f), (float)(C - 1));
    const float4 b = __ldg(reinterpret_cast<const float4 *>(B) + c);
    float ctr = b.z, inv = b.w;
    if (c > 0 && x < b.x) {
        --c;
        const float2 v = __ldg(reinterpret_cast<const float2 *>(B + 4 * c + 2));
        ctr = v.x; inv = v.y;
    } else if (c < C - 1 && x >= b.y) {
        ++c;
        const float2 v = __ldg(reinterpret_cast<const float2 *>(B + 4 * c + 2));
        ctr = v.x; inv = v.y;
    }
    phi = (x - ctr) * inv;
    return c;
}

// Precision traits: which parameter copies a form reads.
template <typename R> struct Form;
template <> struct Form<double> {
    __device__ static double lo(const Params &P, int l) { return P.lo[l]; }
    __device__ static double scale(const Params &P, int l) { return P.h[l]; }   // divide by h
    __device__ static double b(const Params &P, int l) { return P.b[l]; }
    __device__ static double A(const Params &P, int l) { return P.A[l]; }
    __device__ static double c(const Params &P, int l) { return P.c[l]; }
    __device__ static double s1(const Params &P, int l) { return P.s1[l]; }
    __device__ static double sd(const Params &P, int e) { return P.sd[e]; }
    __device__ static double s2(const Params &P, int l) { return P.s2[l]; }
    __device__ static double theta(const Params &P, int l) { return P.theta[l]; }
    __device__ static double inv_s0(const Params &P) { return P.inv_s0; }
    __device__ static double sig(const Params &P, int l) { return P.sig[l]; }
    __device__ static double dt(const Params &P) { return P.dt; }
    __device__ static double sdt(const Params &P) { return P.sdt; }
    __device__ static double Cy(const Params &P) { return P.Cy; }
    __device__ static double Cz(const Params &P) { return P.Cz; }
    __device__ static double prm(const Params &P, int a) { return P.prm[a]; }
    __device__ static double lin(const Params &P) { return P.lin; }
    __device__ static double mu_arg(const Params &P) { return P.mu; }
    __device__ static const double *cellF(const Params &P) { return P.cellF; }
    __device__ static const double *cellB(const Params &P) { return P.cellB; }
    __device__ static double mu(const Params &P) { return P.mu; }
    __device__ static const double *stepc(const Params &P) { return P.stepc; }
    __device__ static const double *Ytab(const Params &P) { return P.Y64; }
    __device__ static const double *Ztab(const Params &P) { return P.Z64; }
    __device__ static int ry(const Params &P) { return P.ry64; }
    __device__ static int rz(const Params &P) { return P.rz64; }
};
template <> struct Form<float> {
    __device__ static float lo(const Params &P, int l) { return P.lo_f[l]; }
    __device__ static float scale(const Params &P, int l) { return P.r_f[l]; }  // multiply by r
    __device__ static float b(const Params &P, int l) { return P.b_f[l]; }
    __device__ static float A(const Params &P, int l) { return P.A_f[l]; }
    __device__ static float c(const Params &P, int l) { return P.c_f[l]; }
    __device__ static float s1(const Params &P, int l) { return P.s1_f[l]; }
    __device__ static float sd(const Params &P, int e) { return P.sd_f[e]; }
    __device__ static float s2(const Params &P, int l) { return P.s2_f[l]; }
    __device__ static float theta(const Params &P, int l) { return P.theta_f[l]; }
    __device__ static float inv_s0(const Params &P) { return P.inv_s0_f; }
    __device__ static float sig(const Params &P, int l) { return P.sig_f[l]; }
    __device__ static float dt(const Params &P) { return P.dt_f; }
    __device__ static float sdt(const Params &P) { return P.sdt_f; }
    __device__ static float Cy(const Params &P) { return P.Cy_f; }
    __device__ static float Cz(const Params &P) { return P.Cz_f; }
    __device__ static float prm(const Params &P, int a) { return P.prm_f[a]; }
    __device__ static float lin(const Params &P) { return P.lin_f; }
    __device__ static float mu_arg(const Params &P) { return P.inv_mu_f; }
    __device__ static const float *cellF(const Params &P) { return P.cellF_f; }
    __device__ static const float *cellB(const Params &P) { return P.cellB_f; }
    __device__ static float mu(const Params &P) { return P.mu_f; }
    __device__ static const float *stepc(const Params &P) { return P.stepc_f; }
    __device__ static const float *Ytab(const Params &P) { return P.Y32; }
    __device__ static const float *Ztab(const Params &P) { return P.Z32; }
    __device__ static int ry(const Params &P) { return P.ry32; }
    __device__ static int rz(const Params &P) { return P.rz32; }
};

__device__ __forceinline__ void sincos_r(double s, double *sn, double *cs) { sincos(s, sn, cs); }
// The FP32 form takes the SFU versions (error ~1e-6 absolute for the
// arguments met here, far below the FP32 tolerance of the fits).
__device__ __forceinline__ void sincos_r(float s, float *sn, float *cs) { __sincosf(s, sn, cs); }
__device__ __forceinline__ double cos_r(double s) { return cos(s); }
__device__ __forceinline__ float cos_r(float s) { return __cosf(s); }
__device__ __forceinline__ double exp_r(double s) { return exp(s); }
__device__ __forceinline__ float exp_r(float s) { return __expf(s); }
__device__ __forceinline__ double clamp_r(double v, double L) { return fmin(fmax(v, -L), L); }
__device__ __forceinline__ float clamp_r(float v, float L) { return fminf(fmaxf(v, -L), L); }
__device__ __forceinline__ double sqrtd_of(const Params &P, double) { return P.sqrt_d; }

// ---- terminal condition g and driver f_j (Sec. 1, eq. fbsde; models) --------
template <typename R, int D, int MODEL>
__device__ __forceinline__ R model_g(const Params &P, const R (&x)[D])
{
#ifdef SRMC_USER_MODEL
    // user model (run-time compiled units): srmc_real is R there
    if constexpr (MODEL == MODEL_USER) return srmc_user_g(x, D, P.prm);
#endif
    R s = x[0];
#pragma unroll
    for (int l = 1; l < D; ++l) s += x[l];
    if (MODEL == MODEL_COS) {
        if (sizeof(R) == 8) return cos_r(s / (R)P.sqrt_d);
        return cos_r(s * (R)P.inv_sqrt_d_f);
    } else if (MODEL == MODEL_LOGISTIC) {
        const R w = exp_r((R)P.T + s);
        return w / ((R)1 + w);
    } else {
        R v = Form<R>::prm(P, 0);
#pragma unroll
        for (int l = 0; l < D; ++l) v += Form<R>::prm(P, 1 + l) * x[l];
        return v;
    }
}

// Drivers that do not read z (the cos family without kapz, the affine
// model) are a part in x plus a part in y: f_j(x, y) = fy(y) + fx_j(x).  The
// step kernel takes fx_j(X_j) before the next point is located, so that X_j
// need not stay live across the gather.
template <typename R, int D, int MODEL>
__device__ __forceinline__ R model_f_x(const Params &P, int j, const R (&x)[D])
{
    if constexpr (MODEL == MODEL_COS) {
        R s = x[0];
#pragma unroll
        for (int l = 1; l < D; ++l) s += x[l];
        s = (sizeof(R) == 8) ? s / (R)P.sqrt_d : s * (R)P.inv_sqrt_d_f;
        const R c1 = __ldg(Form<R>::stepc(P) + 2 * j);     // kap e_j^2
        const R cs = cos_r(s);
        return -(c1 * cs * cs);
    } else if constexpr (MODEL == MODEL_AFFINE) {
        R v = Form<R>::prm(P, 1 + D);
#pragma unroll
        for (int l = 0; l < D; ++l) v += Form<R>::prm(P, 2 + D + l) * x[l];
        return v;
    } else {
        return (R)0;
    }
}
template <typename R, int D, int MODEL>
__device__ __forceinline__ R model_f_y(const Params &P, R y, R fx)
{
    if constexpr (MODEL == MODEL_COS) {
        return Form<R>::lin(P) * y + Form<R>::prm(P, 1) * y * y + fx;   // (lam + s0^2/2) y + kap y^2
    } else if constexpr (MODEL == MODEL_AFFINE) {
        return fx + Form<R>::prm(P, 2 + 2 * D) * y;
    } else {
        return fx;
    }
}

// The driver of the paper's test BSDE (Sec. 5.1), f = (sum_l z_l)(y - (2 + d)/(2d)),
// from the sum of the components of z.
template <typename R, int D>
__device__ __forceinline__ R logistic_f(R y, R zsum)
{
    return zsum * (y - (R)(2 + D) / (R)(2 * D));
}

// f_j(x, y, z); z (Q components) is used only when ZIN.
template <typename R, int D, int MODEL, bool ZIN, int Q = D>
__device__ __forceinline__ R model_f(const Params &P, int j, const R (&x)[D], R y, const R *z)
{
#ifdef SRMC_USER_MODEL
    if constexpr (MODEL == MODEL_USER) return srmc_user_f((R)j * Form<R>::dt(P), x, y, z, D, P.prm);
#endif
    if (MODEL == MODEL_COS) {
        if (!ZIN) return model_f_y<R, D, MODEL>(P, y, model_f_x<R, D, MODEL>(P, j, x));
        R s = x[0];
#pragma unroll
        for (int l = 1; l < D; ++l) s += x[l];
        s = (sizeof(R) == 8) ? s / (R)P.sqrt_d : s * (R)P.inv_sqrt_d_f;
        const R kap = Form<R>::prm(P, 1);
        const R *sc = Form<R>::stepc(P) + 2 * j;
        const R c1 = __ldg(sc), c2 = __ldg(sc + 1);     // kap e_j^2, kapz s0^2 e_j^2
        R v = Form<R>::lin(P) * y + kap * y * y;        // (lam + s0^2/2) y + kap y^2
        if (ZIN) {
            R sn, cs;
            sincos_r(s, &sn, &cs);
            R zz = (R)0;
#pragma unroll
            for (int l = 0; l < Q; ++l) zz += z[l] * z[l];
            v += Form<R>::prm(P, 2) * zz - c1 * cs * cs - c2 * sn * sn;
            if constexpr (Q == D) {
                if (P.drift) {      // uniform: cancels the drift b(x).grad u = b(x).z / s0
                    R bz = (R)0;
#pragma unroll
                    for (int l = 0; l < D; ++l) bz += (Form<R>::b(P, l) - Form<R>::theta(P, l) * x[l]) * z[l];
                    v -= bz * Form<R>::inv_s0(P);
                }
            }
        } else {
            const R cs = cos_r(s);
            v -= c1 * cs * cs;
        }
        return v;
    } else if (MODEL == MODEL_LOGISTIC) {
        R sz = (R)0;
#pragma unroll
        for (int l = 0; l < Q; ++l) sz += z[l];
        return logistic_f<R, Q>(y, sz);
    } else {
        return model_f_y<R, D, MODEL>(P, y, model_f_x<R, D, MODEL>(P, j, x));
    }
}

// Index of coefficient c of component l in a binary16 control row.
__host__ __device__ __forceinline__ int c16_index(const Params &P, int l, int c) { return c * P.ph + l; }

// ---- table rows ----------------------------------------------------------
// COH: the rows may have been written by other blocks of the same launch (the
// persistent batched form), so they are read with ordinary cached loads, not
// through the read-only path.
template <bool COH>
__device__ __forceinline__ float4 ld_row4(const float4 *p) { return COH ? __ldca(p) : __ldg(p); }
template <bool COH>
__device__ __forceinline__ double2 ld_row2(const double2 *p) { return COH ? __ldca(p) : __ldg(p); }

template <int PP, bool COH = false>
__device__ __forceinline__ void load_row(const float *ptr, float (&out)[PP])
{
    constexpr int V = (PP + 3) / 4;
    const float4 *p4 = reinterpret_cast<const float4 *>(ptr);
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const float4 t = ld_row4<COH>(p4 + v);
        if (4 * v + 0 < PP) out[4 * v + 0] = t.x;
        if (4 * v + 1 < PP) out[4 * v + 1] = t.y;
        if (4 * v + 2 < PP) out[4 * v + 2] = t.z;
        if (4 * v + 3 < PP) out[4 * v + 3] = t.w;
    }
}
template <int PP, bool COH = false>
__device__ __forceinline__ void load_row(const double *ptr, double (&out)[PP])
{
    constexpr int V = (PP + 1) / 2;
    const double2 *p2 = reinterpret_cast<const double2 *>(ptr);
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const double2 t = ld_row2<COH>(p2 + v);
        if (2 * v + 0 < PP) out[2 * v + 0] = t.x;
        if (2 * v + 1 < PP) out[2 * v + 1] = t.y;
    }
}

}  // namespace srmc
