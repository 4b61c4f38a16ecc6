// rr_fp32_peak: an FP32 fused multiply-add throughput kernel, the measured
// denominator of the cell walk's arithmetic roofline (the walk is bound by
// instruction issue and the FP32 pipe, not by DRAM; the paper has no
// counterpart). Every thread runs independent FMA chains long enough that
// latency is hidden by the other chains and warps; the caller times the
// launch with events and divides the FMA count by the time.
#include "rr_internal.h"

namespace {

constexpr int kChains = 8;   // independent chains per thread
constexpr int kUnroll = 16;  // chain steps per loop iteration

// scalar FFMA: kChains * kUnroll FMAs per thread and iteration
__global__ void fma_scalar_kernel(float* out, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = (float)(threadIdx.x & 31) * 1e-3f + (float)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < kUnroll; ++r) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == -1.f) out[blockIdx.x] = s;   // never true for the arguments below; keeps the chains live
}

// packed FFMA2: two FMAs per lane and instruction, 2 * kChains * kUnroll per
// thread and iteration
__global__ void fma_packed_kernel(float* out, int iters, float a, float b)
{
    float2 x[kChains];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        x[i].x = (float)(threadIdx.x & 31) * 1e-3f + (float)i;
        x[i].y = x[i].x + 0.5f;
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < kUnroll; ++r) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i].x + x[i].y;
    if (s == -1.f) out[blockIdx.x] = s;
}

}  // namespace

extern "C" rr_status rr_fp32_peak(int32_t packed, int32_t blocks, int32_t threads, int32_t iters, float* out,
                                  int64_t* fmas, void* stream)
{
    if (blocks < 1 || threads < 32 || threads > 1024 || (threads & 31) || iters < 1 || !out || !fmas)
        return RR_ERR_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    // a just below 1 and b > 0: the chains converge to b / (1 - a), finite and positive
    const float a = 0.99999994f, b = 1e-3f;
    if (packed)
        fma_packed_kernel<<<blocks, threads, 0, s>>>(out, iters, a, b);
    else
        fma_scalar_kernel<<<blocks, threads, 0, s>>>(out, iters, a, b);
    *fmas = (int64_t)blocks * threads * iters * kChains * kUnroll * (packed ? 2 : 1);
    return cudaGetLastError() == cudaSuccess ? RR_OK : RR_ERR_CUDA;
}
