// A conversion from FP64 to FP32 on the integer pipes.
#pragma once

#include <cuda_runtime.h>

namespace rr {

// double -> float on the integer pipes instead of the conversion unit (which
// on GB300 shares the slow FP64 pipe): rounds toward zero (within 1 ulp of
// FP32); magnitudes below the FP32 normal range become zeros of their sign,
// above it infinities; NaNs stay NaNs.
static __device__ __forceinline__ float d2f_bits(double d)
{
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const unsigned s = hi & 0x80000000u, e = (hi >> 20) & 0x7ffu;
    unsigned u = s | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    if (e < 897u) u = s;                                  // zero, or below the FP32 normal range
    if (e > 1150u) u = s | 0x7f800000u | (e == 0x7ffu && ((hi & 0xfffffu) | lo) ? 0x400000u : 0u);
    return __uint_as_float(u);
}

}  // namespace rr
