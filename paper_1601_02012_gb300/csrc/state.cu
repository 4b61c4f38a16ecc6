// Ray directions (Eq. txty, Eq. raypos), the finalize pass (maps in rayid order),
// the source-redshift moments (Eqs. Isources, Isources1) and the shear maps.
#include "rr_internal.h"

namespace rr {
namespace {

// Rows [row0, row0 + nrows) of an nx x ny bundle; rid counts from row row0.
__global__ void init_directions_kernel(int nx, int ny, int row0, int nrows, double fov_x, double fov_y,
                                       double* dir, float4* dirh, float4* dirl)
{
    const long long rid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (rid >= (long long)nx * nrows) return;
    const int ix = (int)(rid % nx), iy = row0 + (int)(rid / nx);
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

__device__ __forceinline__ double ff(float2 v) { return (double)v.x + (double)v.y; }

// Maps from the accumulators; for the moments form (kmom, bmom not null)
// kappa = A - B / chi_s per channel (Eq. Isources); for Method A (add_born)
// kappa = the gradient and surface terms plus the density term (Eq. kappa2).
__global__ void finalize_kernel(int nrays, const float2* __restrict__ kacc, const float2* __restrict__ bacc,
                                const uint32_t* __restrict__ nseg, double* out_kappa, double* out_kborn,
                                unsigned long long* total, const float2* __restrict__ kmom,
                                const float2* __restrict__ bmom, double inv_chi_s, int add_born)
{
    unsigned long long local = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nrays;
         i += (long long)gridDim.x * blockDim.x) {
        if (out_kappa)
            out_kappa[i] = kmom ? ff(kacc[i]) - ff(kmom[i]) * inv_chi_s
                                : (add_born ? ff(kacc[i]) + ff(bacc[i]) : ff(kacc[i]));
        if (out_kborn) out_kborn[i] = bmom ? ff(bacc[i]) - ff(bmom[i]) * inv_chi_s : ff(bacc[i]);
        local += nseg[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(total, local);
}

// The four moments (A_kappa, B_kappa, A_born, B_born) as FP64 rows.
__global__ void moments_kernel(int nrays, const float2* __restrict__ kacc, const float2* __restrict__ kmom,
                               const float2* __restrict__ bacc, const float2* __restrict__ bmom, double* out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrays) return;
    out[i] = ff(kacc[i]);
    out[nrays + i] = ff(kmom[i]);
    out[2LL * nrays + i] = ff(bacc[i]);
    out[3LL * nrays + i] = ff(bmom[i]);
}

// The shear maps from their float-float accumulators.
__global__ void shear_out_kernel(int nrays, const float2* __restrict__ g1acc, const float2* __restrict__ g2acc,
                                 double* gamma1, double* gamma2)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrays) return;
    gamma1[i] = ff(g1acc[i]);
    gamma2[i] = ff(g2acc[i]);
}

// kappa for sources at chi_k from the moments at the end and at chi_k
// (Eqs. Isources, Isources1): A(chi_k) = A_end - A_k, B(chi_k) = B_end - B_k.
__global__ void source_kappa_kernel(const double* __restrict__ m_end, const double* __restrict__ m_k,
                                    long long nrays, double inv_chi_k, double* kappa, double* kborn)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrays) return;
    double a = m_end[i], b = m_end[nrays + i], ab = m_end[2 * nrays + i], bb = m_end[3 * nrays + i];
    if (m_k) {
        a -= m_k[i];
        b -= m_k[nrays + i];
        ab -= m_k[2 * nrays + i];
        bb -= m_k[3 * nrays + i];
    }
    kappa[i] = a - b * inv_chi_k;
    if (kborn) kborn[i] = ab - bb * inv_chi_k;
}

}  // namespace

cudaError_t launch_moments(int nrays, const float2* kacc, const float2* kmom, const float2* bacc, const float2* bmom,
                           double* out, cudaStream_t s)
{
    const int nt = 256;
    moments_kernel<<<(unsigned)(((long long)nrays + nt - 1) / nt), nt, 0, s>>>(nrays, kacc, kmom, bacc, bmom, out);
    return cudaGetLastError();
}

cudaError_t launch_shear_out(int nrays, const float2* g1acc, const float2* g2acc, double* gamma1, double* gamma2,
                             cudaStream_t s)
{
    const int nt = 256;
    shear_out_kernel<<<(unsigned)(((long long)nrays + nt - 1) / nt), nt, 0, s>>>(nrays, g1acc, g2acc, gamma1, gamma2);
    return cudaGetLastError();
}

cudaError_t launch_source_kappa(const double* m_end, const double* m_k, long long nrays, double chi_k, double* kappa,
                                double* kborn, cudaStream_t s)
{
    const int nt = 256;
    source_kappa_kernel<<<(unsigned)((nrays + nt - 1) / nt), nt, 0, s>>>(m_end, m_k, nrays, 1.0 / chi_k, kappa, kborn);
    return cudaGetLastError();
}

cudaError_t launch_init_directions(const rr_bundle_desc& b, double* dir, float4* dirh, float4* dirl, cudaStream_t s,
                                   int row0, int nrows)
{
    if (nrows < 0) nrows = b.ny;
    const long long nr = (long long)b.nx * nrows;
    const int nt = 256;
    init_directions_kernel<<<(unsigned)((nr + nt - 1) / nt), nt, 0, s>>>(b.nx, b.ny, row0, nrows, b.fov_x, b.fov_y,
                                                                          dir, dirh, dirl);
    return cudaGetLastError();
}

cudaError_t launch_finalize(int nrays, const float2* kacc, const float2* bacc, const uint32_t* nseg,
                            double* out_kappa, double* out_kborn, unsigned long long* total, cudaStream_t s,
                            const float2* kmom, const float2* bmom, double chi_s, bool add_born)
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
    finalize_kernel<<<(unsigned)blocks, nt, 0, s>>>(nrays, kacc, bacc, nseg, out_kappa, out_kborn, total, kmom, bmom,
                                                    (kmom && chi_s > 0) ? 1.0 / chi_s : 0.0, add_born ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace rr
