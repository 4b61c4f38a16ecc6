// Ray directions (Eq. txty, Eq. raypos) and the finalize pass (maps in rayid order).
#include "rr_internal.h"

namespace rr {
namespace {

__global__ void init_directions_kernel(int nx, int ny, double fov_x, double fov_y, double* dir)
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
}

__global__ void finalize_kernel(int nrays, const double* __restrict__ kappa, const double* __restrict__ kborn,
                                const uint32_t* __restrict__ nseg, double* out_kappa, double* out_kborn,
                                unsigned long long* total)
{
    unsigned long long local = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nrays;
         i += (long long)gridDim.x * blockDim.x) {
        if (out_kappa) out_kappa[i] = kappa[i];
        if (out_kborn) out_kborn[i] = kborn[i];
        local += nseg[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(total, local);
}

}  // namespace

cudaError_t launch_init_directions(const rr_bundle_desc& b, double* dir, cudaStream_t s)
{
    const long long nr = (long long)b.nx * b.ny;
    const int nt = 256;
    init_directions_kernel<<<(unsigned)((nr + nt - 1) / nt), nt, 0, s>>>(b.nx, b.ny, b.fov_x, b.fov_y, dir);
    return cudaGetLastError();
}

cudaError_t launch_finalize(int nrays, const double* kappa, const double* kborn, const uint32_t* nseg,
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
    finalize_kernel<<<(unsigned)blocks, nt, 0, s>>>(nrays, kappa, kborn, nseg, out_kappa, out_kborn, total);
    return cudaGetLastError();
}

}  // namespace rr
