// srmc_peak.cu -- FP32 FMA throughput probe (a measurement aid for the
// roofline of the path kernels; not part of the method).
//
// Every thread runs `iters` rounds of 16 independent fused multiply-adds:
// 8 two-wide packed FFMA2 (the packed FP32 instruction of the sm_100 family)
// or 16 scalar FFMA, then writes one sum so that the work is kept.  Either
// form performs 32 FLOP per round per thread.
#include "../../include/srmc.h"
#include "srmc_internal.h"

namespace {

template <bool PACKED>
__global__ void fma_probe_kernel(int iters, float a, float b, float *out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    float s = 0.0f;
    if constexpr (PACKED) {
        float2 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = make_float2(1e-7f * (float)t + (float)j, 0.5f * (float)j);
        const float2 A = make_float2(a, a), B = make_float2(b, b);
#pragma unroll 4
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = __ffma2_rn(v[j], A, B);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) s += v[j].x + v[j].y;
    } else {
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 1e-7f * (float)t + (float)j;
#pragma unroll 4
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = fmaf(v[j], a, b);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) s += v[j];
    }
    out[t] = s;
}

}  // namespace

extern "C" srmc_status srmc_fp32_fma_probe(int grid, int threads, int iters, int packed, float *dev_out,
                                           void *stream)
{
    if (grid < 1 || threads < 32 || threads > 1024 || threads % 32 || iters < 1 || !dev_out) {
        srmc::set_last_error("srmc_fp32_fma_probe: bad argument");
        return SRMC_ERR_INVALID_ARG;
    }
    const float a = 0.99999994f, b = 1e-6f;
    if (packed)
        fma_probe_kernel<true><<<grid, threads, 0, (cudaStream_t)stream>>>(iters, a, b, dev_out);
    else
        fma_probe_kernel<false><<<grid, threads, 0, (cudaStream_t)stream>>>(iters, a, b, dev_out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        srmc::set_last_error(std::string("srmc_fp32_fma_probe: ") + cudaGetErrorString(e));
        return SRMC_ERR_CUDA;
    }
    return SRMC_OK;
}
