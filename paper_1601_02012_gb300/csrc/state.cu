// Ray directions (Eq. txty, Eq. raypos) and the finalize pass (maps in rayid order).
#include "rr_internal.h"

namespace rr {
namespace {

__global__ void init_directions_kernel(int nx, int ny, double fov_x, double fov_y, double* dir, float4* dirh,
                                       float4* dirl)
{
    const long long rid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (rid >= (long long)nx * ny) return;
    const int ix = (int)(rid % nx), iy = (int)(rid / nx);
    // Eq. (txty) with 0-based pixel indices, as (2i - (N-1)) U / (2(N-1)): the
    // central pixel of an odd row is at exactly 0; a single ray per side sits at 0
    const double tx = nx > 1 ? (double)(2 * ix - (nx - 1)) * (fov_x / (2.0 * (nx - 1))) : 0.0;
    const double ty = ny > 1 ? (double)(2 * iy - (ny - 1)) * (fov_y / (2.0 * (ny - 1))) : 0.0;
    const double th = sqrt(tx * tx + ty * ty);
    double n0 = 0.0, n1 = 0.0, n2 = 1.0;
    if (th > 0.0) {
        // (sin th cos ph, sin th sin ph, cos th) with cos ph = tx/th, sin ph = ty/th
        double s, c;
        sincos(th, &s, &c);
        n0 = s * (tx / th);
        n1 = s * (ty / th);
        n2 = c;
    }
    dir[3 * rid] = n0;
    dir[3 * rid + 1] = n1;
    dir[3 * rid + 2] = n2;
    const float h0 = (float)n0, h1 = (float)n1, h2 = (float)n2;
    dirh[rid] = make_float4(h0, h1, h2, 0.f);
    dirl[rid] = make_float4((float)(n0 - (double)h0), (float)(n1 - (double)h1), (float)(n2 - (double)h2), 0.f);
}

__global__ void finalize_kernel(int nrays, const float2* __restrict__ kacc, const float2* __restrict__ bacc,
                                const uint32_t* __restrict__ nseg, double* out_kappa, double* out_kborn,
                                unsigned long long* total)
{
    unsigned long long local = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nrays;
         i += (long long)gridDim.x * blockDim.x) {
        if (out_kappa) out_kappa[i] = (double)kacc[i].x + (double)kacc[i].y;
        if (out_kborn) out_kborn[i] = (double)bacc[i].x + (double)bacc[i].y;
        local += nseg[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(total, local);
}

}  // namespace

cudaError_t launch_init_directions(const rr_bundle_desc& b, double* dir, float4* dirh, float4* dirl, cudaStream_t s)
{
    const long long nr = (long long)b.nx * b.ny;
    const int nt = 256;
    init_directions_kernel<<<(unsigned)((nr + nt - 1) / nt), nt, 0, s>>>(b.nx, b.ny, b.fov_x, b.fov_y, dir, dirh,
                                                                                    dirl);
    return cudaGetLastError();
}

cudaError_t launch_finalize(int nrays, const float2* kacc, const float2* bacc, const uint32_t* nseg,
                            double* out_kappa, double* out_kborn, unsigned long long* total, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(total, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nt = 256;
    long long blocks = ((long long)nrays + nt - 1) / nt;
    const long long cap = (long long)(sms > 0 ? sms : 1) * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    finalize_kernel<<<(unsigned)blocks, nt, 0, s>>>(nrays, kacc, bacc, nseg, out_kappa, out_kborn, total);
    return cudaGetLastError();
}

}  // namespace rr
