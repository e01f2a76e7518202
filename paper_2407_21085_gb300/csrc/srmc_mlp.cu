// srmc_mlp.cu -- the learned control variate: a small MLP u_theta(t, x)
// (n_in -> 64 -> 64 -> 1, SiLU) on BF16 tensor-core tiles, its training
// (loss gradient + Adam) and the tabulation of sigma^T grad_x u_theta as the
// martingale-control rows of a solver.
//
// One warp processes a tile of 16 samples with mma.sync m16n8k16 (bf16 in,
// fp32 accumulate).  The accumulator fragments of one layer are repacked in
// registers as the A fragments of the next (rows = samples, columns =
// features), so the forward pass and the input gradient never leave the
// register file; the weight gradients of the backward pass (samples are the
// contraction index there) go through per-warp shared-memory transposes.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/srmc.h"
#include "srmc_internal.h"

namespace {

constexpr int H = 64;       // hidden width
constexpr int KIN = 16;     // padded input width (one k-tile)
constexpr int WARPS = 4;    // warps per block

srmc_status mfail(srmc_status st, const std::string &m)
{
    srmc::set_last_error(m);
    return st;
}

#define MLP_CUDA(call, what)                                                                   \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return mfail(e_ == cudaErrorMemoryAllocation ? SRMC_ERR_OOM : SRMC_ERR_CUDA,       \
                         std::string(what) + ": " + cudaGetErrorString(e_));                   \
    } while (0)

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);           // .x (low half) = lo
    return *reinterpret_cast<uint32_t *>(&v);
}
__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ uint32_t bits16(__nv_bfloat16 v) { return (uint32_t)(*reinterpret_cast<unsigned short *>(&v)); }

// D += A B for one m16n8k16 tile (A row-major 16x16, B 16x8, bf16; D fp32).
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float sigm(float z) { return 1.0f / (1.0f + __expf(-z)); }

// Weights staged in shared memory (bf16 operand copies and fp32 vectors).
struct SmemW {
    __nv_bfloat16 W1[H * KIN];    // [out][in]
    __nv_bfloat16 W1T[KIN * H];   // [in][out]
    __nv_bfloat16 W2[H * H];      // [out][in]
    __nv_bfloat16 W2T[H * H];     // [in][out]
    float b1[H], b2[H], w3[H], b3;
};

// Per-warp staging for the weight gradients (training only).
struct SmemStage {
    __nv_bfloat16 G2[16 * H];     // [sample][out2]
    __nv_bfloat16 H1[16 * H];     // [sample][in2]
    __nv_bfloat16 G1[16 * H];     // [sample][out1]
    __nv_bfloat16 A1[16 * KIN];   // [sample][in]
};

struct SmemGrad {
    float dW1[H * KIN], dW2[H * H], db1[H], db2[H], dw3[H], db3;
};

struct Net {                      // device views of one network
    const __nv_bfloat16 *W1, *W1T, *W2, *W2T;
    const float *prm;             // fp32 master parameters
    int nin;
};

__device__ void load_weights(const Net &n, SmemW &w)
{
    for (int e = threadIdx.x; e < H * KIN; e += blockDim.x) { w.W1[e] = n.W1[e]; w.W1T[e] = n.W1T[e]; }
    for (int e = threadIdx.x; e < H * H; e += blockDim.x) { w.W2[e] = n.W2[e]; w.W2T[e] = n.W2T[e]; }
    const float *b1 = n.prm + H * n.nin, *b2 = b1 + H + H * H, *w3 = b2 + H;
    for (int e = threadIdx.x; e < H; e += blockDim.x) { w.b1[e] = b1[e]; w.b2[e] = b2[e]; w.w3[e] = w3[e]; }
    if (threadIdx.x == 0) w.b3 = w3[H];
}

// Forward pass of a 16-sample tile: in(r, c) gives input column c of tile
// row r.  Leaves the SiLU derivatives and h2 for the backward passes.
struct Tile {
    uint32_t A1[4];               // input fragment
    uint32_t A2[4][4];            // h1 as A fragments (bf16)
    float S1[8][4], S2[8][4], H2[8][4];
    float u0, u1;                 // outputs of rows g and g+8
    int g, tg;

    template <typename In>
    __device__ __forceinline__ void forward(const SmemW &w, In in)
    {
        const int lane = threadIdx.x & 31;
        g = lane >> 2; tg = lane & 3;
        A1[0] = pack_bf16(in(g, 2 * tg), in(g, 2 * tg + 1));
        A1[1] = pack_bf16(in(g + 8, 2 * tg), in(g + 8, 2 * tg + 1));
        A1[2] = pack_bf16(in(g, 2 * tg + 8), in(g, 2 * tg + 9));
        A1[3] = pack_bf16(in(g + 8, 2 * tg + 8), in(g + 8, 2 * tg + 9));
        float Z[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            Z[nt][0] = Z[nt][1] = Z[nt][2] = Z[nt][3] = 0.0f;
            const uint32_t b0 = *reinterpret_cast<const uint32_t *>(&w.W1[(nt * 8 + g) * KIN + 2 * tg]);
            const uint32_t b1 = *reinterpret_cast<const uint32_t *>(&w.W1[(nt * 8 + g) * KIN + 2 * tg + 8]);
            mma16816(Z[nt], A1, b0, b1);
        }
        float Hf[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int col = nt * 8 + 2 * tg + (e & 1);
                const float z = Z[nt][e] + w.b1[col];
                const float sg = sigm(z);
                Hf[nt][e] = z * sg;
                S1[nt][e] = sg * (1.0f + z * (1.0f - sg));
            }
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            A2[kt][0] = pack_bf16(Hf[2 * kt][0], Hf[2 * kt][1]);
            A2[kt][1] = pack_bf16(Hf[2 * kt][2], Hf[2 * kt][3]);
            A2[kt][2] = pack_bf16(Hf[2 * kt + 1][0], Hf[2 * kt + 1][1]);
            A2[kt][3] = pack_bf16(Hf[2 * kt + 1][2], Hf[2 * kt + 1][3]);
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            Z[nt][0] = Z[nt][1] = Z[nt][2] = Z[nt][3] = 0.0f;
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) {
                const uint32_t b0 = *reinterpret_cast<const uint32_t *>(&w.W2[(nt * 8 + g) * H + kt * 16 + 2 * tg]);
                const uint32_t b1 = *reinterpret_cast<const uint32_t *>(&w.W2[(nt * 8 + g) * H + kt * 16 + 2 * tg + 8]);
                mma16816(Z[nt], A2[kt], b0, b1);
            }
        }
        float p0 = 0.0f, p1 = 0.0f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int col = nt * 8 + 2 * tg + (e & 1);
                const float z = Z[nt][e] + w.b2[col];
                const float sg = sigm(z);
                H2[nt][e] = z * sg;
                S2[nt][e] = sg * (1.0f + z * (1.0f - sg));
                if (e < 2) p0 += w.w3[col] * H2[nt][e];
                else p1 += w.w3[col] * H2[nt][e];
            }
        p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
        p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
        p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
        p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
        u0 = p0 + w.b3;
        u1 = p1 + w.b3;
    }

    // From per-element dL/dz2 (rows g, g+8 scaled by s0, s1): the A fragments
    // of g_z2 (bf16, also returned rounded in G2r) and the product g_z2 W2
    // times the SiLU derivatives of layer 1 (g_z1, rounded to bf16 in G1r).
    __device__ __forceinline__ void back_to_layer1(const SmemW &w, float s0, float s1, float (&G2r)[8][4],
                                                   float (&G1r)[8][4], uint32_t (&AG1)[4][4])
    {
        uint32_t AG2[4][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int col = nt * 8 + 2 * tg + (e & 1);
                G2r[nt][e] = bf16r((e < 2 ? s0 : s1) * w.w3[col] * S2[nt][e]);
            }
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            AG2[kt][0] = pack_bf16(G2r[2 * kt][0], G2r[2 * kt][1]);
            AG2[kt][1] = pack_bf16(G2r[2 * kt][2], G2r[2 * kt][3]);
            AG2[kt][2] = pack_bf16(G2r[2 * kt + 1][0], G2r[2 * kt + 1][1]);
            AG2[kt][3] = pack_bf16(G2r[2 * kt + 1][2], G2r[2 * kt + 1][3]);
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float D[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) {
                const uint32_t b0 = *reinterpret_cast<const uint32_t *>(&w.W2T[(nt * 8 + g) * H + kt * 16 + 2 * tg]);
                const uint32_t b1 = *reinterpret_cast<const uint32_t *>(&w.W2T[(nt * 8 + g) * H + kt * 16 + 2 * tg + 8]);
                mma16816(D, AG2[kt], b0, b1);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) G1r[nt][e] = bf16r(D[e] * S1[nt][e]);
        }
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            AG1[kt][0] = pack_bf16(G1r[2 * kt][0], G1r[2 * kt][1]);
            AG1[kt][1] = pack_bf16(G1r[2 * kt][2], G1r[2 * kt][3]);
            AG1[kt][2] = pack_bf16(G1r[2 * kt + 1][0], G1r[2 * kt + 1][1]);
            AG1[kt][3] = pack_bf16(G1r[2 * kt + 1][2], G1r[2 * kt + 1][3]);
        }
    }

    // du/da for the tile rows: GA[nt2][e], columns nt2*8 + 2tg + (e&1).
    __device__ __forceinline__ void input_grad(const SmemW &w, float (&GA)[2][4])
    {
        float G2r[8][4], G1r[8][4];
        uint32_t AG1[4][4];
        back_to_layer1(w, 1.0f, 1.0f, G2r, G1r, AG1);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            GA[nt][0] = GA[nt][1] = GA[nt][2] = GA[nt][3] = 0.0f;
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) {
                const uint32_t b0 = *reinterpret_cast<const uint32_t *>(&w.W1T[(nt * 8 + g) * H + kt * 16 + 2 * tg]);
                const uint32_t b1 = *reinterpret_cast<const uint32_t *>(&w.W1T[(nt * 8 + g) * H + kt * 16 + 2 * tg + 8]);
                mma16816(GA[nt], AG1[kt], b0, b1);
            }
        }
    }
};

// Sum of v over the 8 lanes sharing tg (rows of the tile), result in g == 0.
__device__ __forceinline__ float sum_rows(float v)
{
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    return v;
}

// ---- inference: u and du/da ---------------------------------------------------
__global__ void __launch_bounds__(WARPS * 32) mlp_eval_kernel(Net net, const float *a, long long n,
                                                              float *u, float *grad)
{
    extern __shared__ __align__(16) unsigned char smem[];
    SmemW &w = *reinterpret_cast<SmemW *>(smem);
    load_weights(net, w);
    __syncthreads();
    const int warp = threadIdx.x >> 5, nin = net.nin;
    const long long tiles = (n + 15) / 16;
    for (long long t = (long long)blockIdx.x * WARPS + warp; t < tiles; t += (long long)gridDim.x * WARPS) {
        const long long s0 = t * 16;
        Tile T;
        T.forward(w, [&](int r, int c) -> float {
            const long long s = s0 + r;
            return (s < n && c < nin) ? a[s * nin + c] : 0.0f;
        });
        const long long r0 = s0 + T.g, r1 = s0 + T.g + 8;
        if (T.tg == 0) {
            if (r0 < n) u[r0] = T.u0;
            if (r1 < n) u[r1] = T.u1;
        }
        if (grad) {
            float GA[2][4];
            T.input_grad(w, GA);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int col = nt * 8 + 2 * T.tg + (e & 1);
                    const long long r = e < 2 ? r0 : r1;
                    if (col < nin && r < n) grad[r * nin + col] = GA[nt][e];
                }
        }
    }
}

// ---- training: loss gradient accumulated over the batch -----------------------
__global__ void __launch_bounds__(WARPS * 32) mlp_grad_kernel(Net net, const float *a, const float *y,
                                                              long long n, float inv_n, float *grad,
                                                              float *loss)
{
    extern __shared__ __align__(16) unsigned char smem[];
    SmemW &w = *reinterpret_cast<SmemW *>(smem);
    SmemGrad &gs = *reinterpret_cast<SmemGrad *>(smem + sizeof(SmemW));
    SmemStage *stage = reinterpret_cast<SmemStage *>(smem + sizeof(SmemW) + sizeof(SmemGrad));
    load_weights(net, w);
    float *gflat = reinterpret_cast<float *>(&gs);
    for (int e = threadIdx.x; e < (int)(sizeof(SmemGrad) / 4); e += blockDim.x) gflat[e] = 0.0f;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nin = net.nin;
    SmemStage &st = stage[warp];
    float lsum = 0.0f;
    const long long tiles = (n + 15) / 16;
    for (long long t = (long long)blockIdx.x * WARPS + warp; t < tiles; t += (long long)gridDim.x * WARPS) {
        const long long s0 = t * 16;
        auto in = [&](int r, int c) -> float {
            const long long s = s0 + r;
            return (s < n && c < nin) ? a[s * nin + c] : 0.0f;
        };
        Tile T;
        T.forward(w, in);
        const int g = T.g, tg = T.tg;
        const long long r0 = s0 + g, r1 = s0 + g + 8;
        const float e0 = r0 < n ? T.u0 - y[r0] : 0.0f;
        const float e1 = r1 < n ? T.u1 - y[r1] : 0.0f;
        if (tg == 0) lsum += e0 * e0 + e1 * e1;
        const float du0 = 2.0f * e0 * inv_n, du1 = 2.0f * e1 * inv_n;
        float G2r[8][4], G1r[8][4];
        uint32_t AG1[4][4];
        T.back_to_layer1(w, du0, du1, G2r, G1r, AG1);
        // bias and output-layer gradients, summed over the tile rows
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int col = nt * 8 + 2 * tg + c;
                const float db2 = sum_rows(G2r[nt][c] + G2r[nt][c + 2]);
                const float dw3 = sum_rows(du0 * T.H2[nt][c] + du1 * T.H2[nt][c + 2]);
                const float db1 = sum_rows(G1r[nt][c] + G1r[nt][c + 2]);
                if (g == 0) {
                    atomicAdd(&gs.db2[col], db2);
                    atomicAdd(&gs.dw3[col], dw3);
                    atomicAdd(&gs.db1[col], db1);
                }
            }
        {
            float d3 = (tg == 0) ? du0 + du1 : 0.0f;
            d3 = sum_rows(d3);
            d3 += __shfl_xor_sync(0xffffffffu, d3, 1);
            d3 += __shfl_xor_sync(0xffffffffu, d3, 2);
            if (lane == 0) atomicAdd(&gs.db3, d3);
        }
        // stage g_z2, h1, g_z1 and the inputs (bf16) for the weight gradients
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int col = nt * 8 + 2 * tg + (e & 1), row = g + (e < 2 ? 0 : 8);
                st.G2[row * H + col] = __float2bfloat16_rn(G2r[nt][e]);
                st.G1[row * H + col] = __float2bfloat16_rn(G1r[nt][e]);
            }
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            const uint32_t v[4] = {T.A2[kt][0], T.A2[kt][1], T.A2[kt][2], T.A2[kt][3]};
            const int c0 = kt * 16 + 2 * tg;
            *reinterpret_cast<uint32_t *>(&st.H1[g * H + c0]) = v[0];
            *reinterpret_cast<uint32_t *>(&st.H1[(g + 8) * H + c0]) = v[1];
            *reinterpret_cast<uint32_t *>(&st.H1[g * H + c0 + 8]) = v[2];
            *reinterpret_cast<uint32_t *>(&st.H1[(g + 8) * H + c0 + 8]) = v[3];
        }
        *reinterpret_cast<uint32_t *>(&st.A1[g * KIN + 2 * tg]) = T.A1[0];
        *reinterpret_cast<uint32_t *>(&st.A1[(g + 8) * KIN + 2 * tg]) = T.A1[1];
        *reinterpret_cast<uint32_t *>(&st.A1[g * KIN + 2 * tg + 8]) = T.A1[2];
        *reinterpret_cast<uint32_t *>(&st.A1[(g + 8) * KIN + 2 * tg + 8]) = T.A1[3];
        __syncwarp();
        // dW2[out][in] = sum_s g_z2[s][out] h1[s][in]; dW1[out][in] = sum_s g_z1[s][out] a[s][in]
        auto tA = [&](const __nv_bfloat16 *M, int ld, int mrow, int k) -> uint32_t {
            return bits16(M[k * ld + mrow]) | (bits16(M[(k + 1) * ld + mrow]) << 16);
        };
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
            const int m0 = mt * 16 + g;
            const uint32_t A2t[4] = {tA(st.G2, H, m0, 2 * tg), tA(st.G2, H, m0 + 8, 2 * tg),
                                     tA(st.G2, H, m0, 2 * tg + 8), tA(st.G2, H, m0 + 8, 2 * tg + 8)};
            const uint32_t A1t[4] = {tA(st.G1, H, m0, 2 * tg), tA(st.G1, H, m0 + 8, 2 * tg),
                                     tA(st.G1, H, m0, 2 * tg + 8), tA(st.G1, H, m0 + 8, 2 * tg + 8)};
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const int n0 = nt * 8 + g;
                const uint32_t b0 = tA(st.H1, H, n0, 2 * tg), b1 = tA(st.H1, H, n0, 2 * tg + 8);
                float D[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                mma16816(D, A2t, b0, b1);
                const int cn = nt * 8 + 2 * tg;
                atomicAdd(&gs.dW2[m0 * H + cn], D[0]);
                atomicAdd(&gs.dW2[m0 * H + cn + 1], D[1]);
                atomicAdd(&gs.dW2[(m0 + 8) * H + cn], D[2]);
                atomicAdd(&gs.dW2[(m0 + 8) * H + cn + 1], D[3]);
            }
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const int n0 = nt * 8 + g;
                const uint32_t b0 = tA(st.A1, KIN, n0, 2 * tg), b1 = tA(st.A1, KIN, n0, 2 * tg + 8);
                float D[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                mma16816(D, A1t, b0, b1);
                const int cn = nt * 8 + 2 * tg;
                atomicAdd(&gs.dW1[m0 * KIN + cn], D[0]);
                atomicAdd(&gs.dW1[m0 * KIN + cn + 1], D[1]);
                atomicAdd(&gs.dW1[(m0 + 8) * KIN + cn], D[2]);
                atomicAdd(&gs.dW1[(m0 + 8) * KIN + cn + 1], D[3]);
            }
        }
        __syncwarp();
    }
    lsum += __shfl_xor_sync(0xffffffffu, lsum, 4);
    lsum += __shfl_xor_sync(0xffffffffu, lsum, 8);
    lsum += __shfl_xor_sync(0xffffffffu, lsum, 16);
    if (lane == 0 && loss) atomicAdd(loss, lsum * inv_n);
    __syncthreads();
    // block sums -> global gradient (parameter layout W1 [H][nin], b1, W2, b2, w3, b3)
    float *gW1 = grad, *gb1 = gW1 + H * nin, *gW2 = gb1 + H, *gb2 = gW2 + H * H, *gw3 = gb2 + H, *gb3 = gw3 + H;
    for (int e = threadIdx.x; e < H * nin; e += blockDim.x) atomicAdd(&gW1[e], gs.dW1[(e / nin) * KIN + e % nin]);
    for (int e = threadIdx.x; e < H * H; e += blockDim.x) atomicAdd(&gW2[e], gs.dW2[e]);
    for (int e = threadIdx.x; e < H; e += blockDim.x) {
        atomicAdd(&gb1[e], gs.db1[e]);
        atomicAdd(&gb2[e], gs.db2[e]);
        atomicAdd(&gw3[e], gs.dw3[e]);
    }
    if (threadIdx.x == 0) atomicAdd(gb3, gs.db3);
}

// fp32 master parameters -> bf16 operand copies (W1, W1^T, W2, W2^T; pads zero)
__global__ void mlp_pack_kernel(const float *prm, int nin, __nv_bfloat16 *W1, __nv_bfloat16 *W1T,
                                __nv_bfloat16 *W2, __nv_bfloat16 *W2T)
{
    const float *pW2 = prm + H * nin + H;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < H * H; e += gridDim.x * blockDim.x) {
        const int o = e / H, c = e % H;
        W2[e] = __float2bfloat16_rn(pW2[e]);
        W2T[c * H + o] = __float2bfloat16_rn(pW2[e]);
        if (e < H * KIN) {
            const int oo = e / KIN, cc = e % KIN;
            const float v = cc < nin ? prm[oo * nin + cc] : 0.0f;
            W1[e] = __float2bfloat16_rn(v);
            W1T[cc * H + oo] = __float2bfloat16_rn(v);
        }
    }
}

__global__ void mlp_adam_kernel(float *w, float *m, float *v, float *g, int P, float lr, float c1,
                                float c2)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= P) return;
    const float gq = g[q];
    const float mq = 0.9f * m[q] + 0.1f * gq;
    const float vq = 0.999f * v[q] + 0.001f * gq * gq;
    m[q] = mq;
    v[q] = vq;
    w[q] -= lr * (mq * c1) / (sqrtf(vq * c2) + 1e-8f);
    g[q] = 0.0f;
}

// Training points from a finished solve: (i, k) uniform, x ~ nu_k (Alg. 3),
// a = (t_i, x), target y_i(x) from the FP64 table.  Philox on (seed, s).
__global__ void mlp_data_kernel(const Params P, long long n, unsigned k0, unsigned k1, float *a,
                                float *y)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        unsigned w[4 * 3];
        for (int b = 0; b < 3; ++b) {
            unsigned c0 = (unsigned)b, c1 = (unsigned)s, c2 = (unsigned)(s >> 32), c3 = 0x5EEDu;
            srmc::philox10(c0, c1, c2, c3, k0, k1);
            w[4 * b] = c0; w[4 * b + 1] = c1; w[4 * b + 2] = c2; w[4 * b + 3] = c3;
        }
        const int i = (int)(((unsigned long long)w[0] * (unsigned long long)P.N) >> 32);
        long long k = (long long)(((unsigned long long)w[1] * (unsigned long long)P.K) >> 32);
        double x[srmc::DMAX];
        for (int l = 0; l < P.d; ++l) {
            const int c = (int)(k % P.cells[l]);
            k /= P.cells[l];
            const int o = 3 * (P.cell_off[l] + c);
            x[l] = srmc::sample_cell(w[2 + l], P.cellF[o], P.cellF[o + 1], P.cellF[o + 2], P.mu);
        }
        const int nin = P.d + 1;
        a[s * nin] = (float)((double)i * P.dt);
        for (int l = 0; l < P.d; ++l) a[s * nin + 1 + l] = (float)x[l];
        y[s] = (float)srmc::eval_y64(P, i, x);
    }
}

// Control rows from the network: one warp per (j, k) tile; tile rows are the
// stratum's basis centre (row 0) and c +- (unit_m/2) e_m (rows 1 + 2m, 2 + 2m),
// unit_m the basis unit of the stratum's cell along axis m (h_m/2 for
// equal-size cells).
__global__ void __launch_bounds__(WARPS * 32) mlp_tabulate_kernel(Net net, const Params P, double *c64,
                                                                  __half *c16)
{
    extern __shared__ __align__(16) unsigned char smem[];
    SmemW &w = *reinterpret_cast<SmemW *>(smem);
    float (*GAs)[16][KIN] = reinterpret_cast<float (*)[16][KIN]>(smem + sizeof(SmemW));
    load_weights(net, w);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, d = P.d, p = P.p;
    const long long tiles = (long long)P.N * P.K;
    for (long long t = (long long)blockIdx.x * WARPS + warp; t < tiles; t += (long long)gridDim.x * WARPS) {
        const int j = (int)(t / P.K);
        const long long k = t % P.K;
        double ctr[srmc::DMAX], half[srmc::DMAX];      // basis centre, half a basis unit
        {
            long long rem = k;
            for (int l = 0; l < d; ++l) {
                const int c = (int)(rem % P.cells[l]);
                rem /= P.cells[l];
                ctr[l] = srmc::cell_centre(P, l, c);
                half[l] = 0.5 * srmc::cell_unit(P, l, c);
            }
        }
        const float tj = (float)((double)j * P.dt);
        Tile T;
        T.forward(w, [&](int r, int c) -> float {
            if (c == 0) return tj;
            if (c > d) return 0.0f;
            const int l = c - 1;
            double x = ctr[l];
            if (r >= 1 && r <= 2 * d) {
                const int m = (r - 1) >> 1;
                if (m == l) x += (r & 1) ? half[l] : -half[l];
            }
            return (float)x;
        });
        float GA[2][4];
        T.input_grad(w, GA);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e)
                GAs[warp][T.g + (e < 2 ? 0 : 8)][nt * 8 + 2 * T.tg + (e & 1)] = GA[nt][e];
        __syncwarp();
        const long long row = (long long)j * P.K + k;
        for (int a = lane; a < d * p; a += 32) {
            const int l = a / p, c = a % p;
            // zc = sigma^T grad u: component l of the value (c = 0) or of the
            // central difference along axis c - 1 (c > 0)
            auto g = [&](int m) {
                return c == 0 ? (double)GAs[warp][0][1 + m]
                              : (double)GAs[warp][1 + 2 * (c - 1)][1 + m] - (double)GAs[warp][2 + 2 * (c - 1)][1 + m];
            };
            double v;
            if (P.dense) {
                v = 0.0;
                for (int m = 0; m < d; ++m) v += P.sd[m * P.q + l] * g(m);
            } else {
                v = P.sig[l] * g(l);
            }
            c64[row * P.rz64 + a] = v;
            c16[row * P.rc16 + srmc::c16_index(P, l, c)] = __double2half(fmin(fmax(v, -65504.0), 65504.0));
        }
        __syncwarp();
    }
}

size_t smem_eval() { return sizeof(SmemW); }
size_t smem_grad() { return sizeof(SmemW) + sizeof(SmemGrad) + WARPS * sizeof(SmemStage); }
size_t smem_tab() { return sizeof(SmemW) + WARPS * 16 * KIN * sizeof(float); }

int grid_tiles(long long tiles)
{
    long long g = (tiles + WARPS - 1) / WARPS;
    if (g > 152LL * 16) g = 152LL * 16;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

// Scratch of srmc_mlp_fit_noalloc: static device memory, one copy per GPU
// that loads the library.  Host code may not use the symbol as an address;
// its device address is looked up once per device (noalloc_scratch).
constexpr long long kNoallocFloats = 1LL << 21;          // 8 MiB
static __device__ __align__(256) float g_noalloc_scratch[kNoallocFloats];

namespace {
std::mutex g_noalloc_mu;
float *g_noalloc_ptr[256] = {};

// Device address of the scratch array on the current device (looked up on the
// first call for that device, with that device current).
srmc_status noalloc_scratch(float **out)
{
    int dev = 0;
    MLP_CUDA(cudaGetDevice(&dev), "srmc_mlp_fit_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 256) return mfail(SRMC_ERR_UNSUPPORTED, "srmc_mlp_fit_noalloc: device id >= 256");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        MLP_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch), "srmc_mlp_fit_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = static_cast<float *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return SRMC_OK;
}
}  // namespace

struct srmc_mlp {
    int nin = 0, P = 0, device = 0, step = 0;
    float *prm = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *loss = nullptr;
    __nv_bfloat16 *W1 = nullptr, *W1T = nullptr, *W2 = nullptr, *W2T = nullptr;
    Net net() const { return Net{W1, W1T, W2, W2T, prm, nin}; }
};

namespace {
void mlp_free(srmc_mlp *m)
{
    cudaFree(m->prm); cudaFree(m->m); cudaFree(m->v); cudaFree(m->grad); cudaFree(m->loss);
    cudaFree(m->W1); cudaFree(m->W1T); cudaFree(m->W2); cudaFree(m->W2T);
}

cudaError_t set_smem_limits()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_grad());
    if (e == cudaSuccess) done = true;
    return e;
}

srmc_status repack(srmc_mlp *m, cudaStream_t st)
{
    mlp_pack_kernel<<<16, 256, 0, st>>>(m->prm, m->nin, m->W1, m->W1T, m->W2, m->W2T);
    MLP_CUDA(cudaGetLastError(), "mlp pack");
    return SRMC_OK;
}
}  // namespace

extern "C" {

srmc_status srmc_mlp_create(int n_in, int hidden, unsigned long long seed, srmc_mlp **out)
{
    if (!out) return mfail(SRMC_ERR_INVALID_ARG, "srmc_mlp_create: out is NULL");
    *out = nullptr;
    if (hidden != H) return mfail(SRMC_ERR_UNSUPPORTED, "srmc_mlp_create: hidden must be 64");
    if (n_in < 1 || n_in > KIN - 1) return mfail(SRMC_ERR_INVALID_ARG, "srmc_mlp_create: n_in in [1, 15]");
    srmc_mlp *m = new srmc_mlp();
    m->nin = n_in;
    m->P = H * n_in + H + H * H + H + H + 1;
    cudaGetDevice(&m->device);
    // seeded initialisation: uniform +-sqrt(6/fan_in) (splitmix64 stream)
    std::vector<float> h(m->P, 0.0f);
    unsigned long long z = seed ^ 0x9E3779B97F4A7C15ull;
    auto next = [&]() {
        z += 0x9E3779B97F4A7C15ull;
        unsigned long long x = z;
        x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
        x ^= x >> 31;
        return ((double)(x >> 11) + 0.5) * 0x1p-53;
    };
    const double a1 = std::sqrt(6.0 / n_in), a2 = std::sqrt(6.0 / H);
    for (int e = 0; e < H * n_in; ++e) h[e] = (float)((2.0 * next() - 1.0) * a1);
    float *pW2 = h.data() + H * n_in + H;
    for (int e = 0; e < H * H; ++e) pW2[e] = (float)((2.0 * next() - 1.0) * a2);
    float *pw3 = pW2 + H * H + H;
    for (int e = 0; e < H; ++e) pw3[e] = (float)((2.0 * next() - 1.0) * a2);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t b) { if (e == cudaSuccess) e = cudaMalloc(p, b); };
    alloc((void **)&m->prm, sizeof(float) * m->P);
    alloc((void **)&m->m, sizeof(float) * m->P);
    alloc((void **)&m->v, sizeof(float) * m->P);
    alloc((void **)&m->grad, sizeof(float) * m->P);
    alloc((void **)&m->loss, sizeof(float) * 2);
    alloc((void **)&m->W1, sizeof(__nv_bfloat16) * H * KIN);
    alloc((void **)&m->W1T, sizeof(__nv_bfloat16) * H * KIN);
    alloc((void **)&m->W2, sizeof(__nv_bfloat16) * H * H);
    alloc((void **)&m->W2T, sizeof(__nv_bfloat16) * H * H);
    if (e == cudaSuccess) e = cudaMemcpy(m->prm, h.data(), sizeof(float) * m->P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->m, 0, sizeof(float) * m->P);
    if (e == cudaSuccess) e = cudaMemset(m->v, 0, sizeof(float) * m->P);
    if (e == cudaSuccess) e = cudaMemset(m->grad, 0, sizeof(float) * m->P);
    if (e == cudaSuccess) e = set_smem_limits();
    if (e != cudaSuccess) {
        mlp_free(m);
        delete m;
        return mfail(e == cudaErrorMemoryAllocation ? SRMC_ERR_OOM : SRMC_ERR_CUDA,
                     std::string("srmc_mlp_create: ") + cudaGetErrorString(e));
    }
    srmc_status st = repack(m, 0);
    if (st != SRMC_OK) { mlp_free(m); delete m; return st; }
    MLP_CUDA(cudaDeviceSynchronize(), "srmc_mlp_create");
    *out = m;
    return SRMC_OK;
}

void srmc_mlp_destroy(srmc_mlp *m)
{
    if (!m) return;
    mlp_free(m);
    delete m;
}

int srmc_mlp_nparams(const srmc_mlp *m) { return m ? m->P : 0; }

srmc_status srmc_mlp_set_params(srmc_mlp *m, const float *params)
{
    if (!m || !params) return mfail(SRMC_ERR_INVALID_ARG, "srmc_mlp_set_params: NULL argument");
    MLP_CUDA(cudaMemcpy(m->prm, params, sizeof(float) * m->P, cudaMemcpyDefault), "srmc_mlp_set_params");
    MLP_CUDA(cudaMemset(m->m, 0, sizeof(float) * m->P), "reset adam");
    MLP_CUDA(cudaMemset(m->v, 0, sizeof(float) * m->P), "reset adam");
    m->step = 0;
    srmc_status st = repack(m, 0);
    if (st != SRMC_OK) return st;
    MLP_CUDA(cudaDeviceSynchronize(), "srmc_mlp_set_params");
    return SRMC_OK;
}

srmc_status srmc_mlp_get_params(const srmc_mlp *m, float *params)
{
    if (!m || !params) return mfail(SRMC_ERR_INVALID_ARG, "srmc_mlp_get_params: NULL argument");
    MLP_CUDA(cudaMemcpy(params, m->prm, sizeof(float) * m->P, cudaMemcpyDefault), "srmc_mlp_get_params");
    return SRMC_OK;
}

srmc_status srmc_mlp_eval(const srmc_mlp *m, const float *a, long long n, float *u, float *grad,
                          void *stream)
{
    if (!m || n < 0) return mfail(SRMC_ERR_INVALID_ARG, "srmc_mlp_eval: bad argument");
    if (n == 0) return SRMC_OK;
    if (!a || !u) return mfail(SRMC_ERR_INVALID_ARG, "srmc_mlp_eval: NULL buffer");
    const long long tiles = (n + 15) / 16;
    mlp_eval_kernel<<<grid_tiles(tiles), WARPS * 32, smem_eval(), (cudaStream_t)stream>>>(m->net(), a, n, u, grad);
    MLP_CUDA(cudaGetLastError(), "mlp eval launch");
    return SRMC_OK;
}

srmc_status srmc_mlp_loss_grad(srmc_mlp *m, const float *a, const float *y, long long n, float *grad,
                               float *loss, void *stream)
{
    if (!m || n <= 0 || !a || !y || !grad) return mfail(SRMC_ERR_INVALID_ARG, "srmc_mlp_loss_grad: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    MLP_CUDA(cudaMemsetAsync(grad, 0, sizeof(float) * m->P, st), "zero grad");
    if (loss) MLP_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), st), "zero loss");
    const long long tiles = (n + 15) / 16;
    mlp_grad_kernel<<<grid_tiles(tiles), WARPS * 32, smem_grad(), st>>>(m->net(), a, y, n, 1.0f / (float)n,
                                                                       grad, loss);
    MLP_CUDA(cudaGetLastError(), "mlp grad launch");
    return SRMC_OK;
}

srmc_status srmc_mlp_fit(srmc_mlp *m, const srmc_solver *s, long long n_data, int iters, int batch,
                         float lr, unsigned long long seed, float *loss_curve, void *stream)
{
    if (!m || !s || n_data <= 0 || iters < 0 || batch <= 0 || n_data % batch)
        return mfail(SRMC_ERR_INVALID_ARG, "srmc_mlp_fit: bad argument");
    if (m->nin != s->P.d + 1) return mfail(SRMC_ERR_INVALID_ARG, "srmc_mlp_fit: n_in must be d + 1");
    if (s->done_from > 0) return mfail(SRMC_ERR_STATE, "srmc_mlp_fit: the coarse solve is not finished");
    // 2^40 points (16 TiB of inputs at d = 3) is beyond any device, and keeps
    // the byte counts below far from wrapping
    if (n_data > (1LL << 40)) return mfail(SRMC_ERR_INVALID_ARG, "srmc_mlp_fit: n_data > 2^40");
    cudaStream_t st = (cudaStream_t)stream;
    float *a = nullptr, *y = nullptr;
    MLP_CUDA(cudaMalloc(&a, sizeof(float) * n_data * m->nin), "cudaMalloc training inputs");
    if (cudaMalloc(&y, sizeof(float) * n_data) != cudaSuccess) {
        cudaFree(a);
        return mfail(SRMC_ERR_OOM, "srmc_mlp_fit: cudaMalloc training targets");
    }
    mlp_data_kernel<<<grid_tiles((n_data + 63) / 64) * 2, 256, 0, st>>>(
        s->P, n_data, (unsigned)(seed & 0xFFFFFFFFu), (unsigned)(seed >> 32), a, y);
    cudaError_t e = cudaGetLastError();
    const long long tiles = (batch + 15) / 16;
    const float decay = iters > 1 ? std::pow(0.1f, 1.0f / (float)(iters - 1)) : 1.0f;
    float lr_t = lr, b1t = 1.0f, b2t = 1.0f;
    for (int it = 0; it < iters && e == cudaSuccess; ++it) {
        const long long off = ((long long)it * batch) % n_data;
        float *lp = loss_curve ? loss_curve + it : m->loss;
        e = cudaMemsetAsync(lp, 0, sizeof(float), st);
        if (e != cudaSuccess) break;
        mlp_grad_kernel<<<grid_tiles(tiles), WARPS * 32, smem_grad(), st>>>(
            m->net(), a + off * m->nin, y + off, batch, 1.0f / (float)batch, m->grad, lp);
        ++m->step;
        b1t *= 0.9f; b2t *= 0.999f;
        mlp_adam_kernel<<<(m->P + 255) / 256, 256, 0, st>>>(m->prm, m->m, m->v, m->grad, m->P, lr_t,
                                                            1.0f / (1.0f - b1t), 1.0f / (1.0f - b2t));
        mlp_pack_kernel<<<16, 256, 0, st>>>(m->prm, m->nin, m->W1, m->W1T, m->W2, m->W2T);
        e = cudaGetLastError();
        lr_t *= decay;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(a);
    cudaFree(y);
    if (e != cudaSuccess) return mfail(SRMC_ERR_CUDA, std::string("srmc_mlp_fit: ") + cudaGetErrorString(e));
    return SRMC_OK;
}

srmc_status srmc_mlp_fit_noalloc(srmc_mlp *m, const srmc_solver *s, long long n_data, int iters,
                                 int batch, float lr, unsigned long long seed, float *loss_curve,
                                 void *stream)
{
    if (!m || !s || n_data <= 0 || iters < 0 || batch <= 0 || n_data % batch)
        return mfail(SRMC_ERR_INVALID_ARG, "srmc_mlp_fit_noalloc: bad argument");
    if (m->nin != s->P.d + 1) return mfail(SRMC_ERR_INVALID_ARG, "srmc_mlp_fit_noalloc: n_in must be d + 1");
    if (s->done_from > 0) return mfail(SRMC_ERR_STATE, "srmc_mlp_fit_noalloc: the coarse solve is not finished");
    {
        // the scratch is looked up on the current device, where the network must live
        int dev = -1;
        MLP_CUDA(cudaGetDevice(&dev), "srmc_mlp_fit_noalloc: cudaGetDevice");
        if (dev != m->device)
            return mfail(SRMC_ERR_INVALID_ARG, "srmc_mlp_fit_noalloc: the network's device is not the current one");
    }
    // bound n_data first, so that the size below cannot wrap
    if (n_data > kNoallocFloats)
        return mfail(SRMC_ERR_INVALID_ARG,
                     "srmc_mlp_fit_noalloc: n_data exceeds the 2^21-float scratch of the allocation-free path "
                     "(use srmc_mlp_fit)");
    // scratch layout (floats): [gradient, padded to 64][loss slot, 64][inputs n_data x n_in][targets n_data]
    const long long gpad = ((long long)m->P + 63) / 64 * 64;
    const long long need = gpad + 64 + n_data * (long long)(m->nin + 1);
    if (need > kNoallocFloats)
        return mfail(SRMC_ERR_INVALID_ARG,
                     "srmc_mlp_fit_noalloc: n_data * (n_in + 1) + nparams + 64 exceeds the 2^21-float "
                     "scratch of the allocation-free path (use srmc_mlp_fit)");
    float *base = nullptr;
    srmc_status st = noalloc_scratch(&base);
    if (st != SRMC_OK) return st;
    float *grad = base, *loss1 = base + gpad, *a = base + gpad + 64, *y = a + n_data * m->nin;
    cudaStream_t cs = (cudaStream_t)stream;
    // the array keeps the previous call's contents: clear the accumulators
    MLP_CUDA(cudaMemsetAsync(grad, 0, sizeof(float) * (size_t)(gpad + 64), cs), "srmc_mlp_fit_noalloc: clear");
    mlp_data_kernel<<<grid_tiles((n_data + 63) / 64) * 2, 256, 0, cs>>>(
        s->P, n_data, (unsigned)(seed & 0xFFFFFFFFu), (unsigned)(seed >> 32), a, y);
    cudaError_t e = cudaGetLastError();
    const long long tiles = (batch + 15) / 16;
    const float decay = iters > 1 ? std::pow(0.1f, 1.0f / (float)(iters - 1)) : 1.0f;
    float lr_t = lr, b1t = 1.0f, b2t = 1.0f;
    for (int it = 0; it < iters && e == cudaSuccess; ++it) {
        const long long off = ((long long)it * batch) % n_data;
        float *lp = loss_curve ? loss_curve + it : loss1;
        e = cudaMemsetAsync(lp, 0, sizeof(float), cs);
        if (e != cudaSuccess) break;
        mlp_grad_kernel<<<grid_tiles(tiles), WARPS * 32, smem_grad(), cs>>>(
            m->net(), a + off * m->nin, y + off, batch, 1.0f / (float)batch, grad, lp);
        ++m->step;
        b1t *= 0.9f; b2t *= 0.999f;
        mlp_adam_kernel<<<(m->P + 255) / 256, 256, 0, cs>>>(m->prm, m->m, m->v, grad, m->P, lr_t,
                                                            1.0f / (1.0f - b1t), 1.0f / (1.0f - b2t));
        mlp_pack_kernel<<<16, 256, 0, cs>>>(m->prm, m->nin, m->W1, m->W1T, m->W2, m->W2T);
        e = cudaGetLastError();
        lr_t *= decay;
    }
    if (e != cudaSuccess)
        return mfail(SRMC_ERR_CUDA, std::string("srmc_mlp_fit_noalloc: ") + cudaGetErrorString(e));
    return SRMC_OK;
}

srmc_status srmc_cv_tabulate(const srmc_mlp *m, srmc_solver *s, void *stream)
{
    if (!m || !s) return mfail(SRMC_ERR_INVALID_ARG, "srmc_cv_tabulate: NULL argument");
    if (!s->lp1 || s->lp2 || s->P.d > 7 || m->nin != s->P.d + 1 || s->mv == srmc::MV_AFFINE || s->P.q != s->P.d)
        return mfail(SRMC_ERR_UNSUPPORTED, "srmc_cv_tabulate: LP1, d <= 7, q = d, n_in = d + 1 only");
    if (const int st = srmc_prepare_user_control(s)) return (srmc_status)st;
    const size_t nrow = (size_t)s->P.N * (size_t)s->P.K;
    if (!s->C64) {
        MLP_CUDA(cudaMalloc(&s->C64, sizeof(double) * nrow * s->P.rz64), "cudaMalloc control");
        MLP_CUDA(cudaMalloc(&s->C16, sizeof(__half) * nrow * s->P.rc16), "cudaMalloc control");
        MLP_CUDA(cudaMemset(s->C64, 0, sizeof(double) * nrow * s->P.rz64), "cudaMemset control");
        MLP_CUDA(cudaMemset(s->C16, 0, sizeof(__half) * nrow * s->P.rc16), "cudaMemset control");
    }
    const long long tiles = (long long)nrow;
    mlp_tabulate_kernel<<<grid_tiles(tiles), WARPS * 32, smem_tab(), (cudaStream_t)stream>>>(
        m->net(), s->P, s->C64, s->C16);
    MLP_CUDA(cudaGetLastError(), "mlp tabulate launch");
    s->cv = true;
    s->cv_own = false;
    if (s->graph) { cudaGraphExecDestroy(s->graph); s->graph = nullptr; }
    return SRMC_OK;
}

}  // extern "C"
