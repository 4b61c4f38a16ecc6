// Tidal tensor and vertex records (Sec. 3.3, Eq. tidalexample; Sec. 2.7).
//
// One CTA produces a 4 x 4 x 32 tile of records (z fastest). It stages the
// potential of the tile plus a halo of two cells in shared memory, evaluates
// the six central-difference second derivatives at every cell centre the tile
// needs, and then either averages the 8 cells around each vertex or copies
// the centre values. Reads are 4 B per point from HBM (halo re-reads hit L2),
// writes 32 B per point as contiguous float4 runs: the kernel is bound by HBM
// bandwidth, 36 algorithmic bytes per point.
#include "rr_internal.h"

namespace rr {
namespace {

constexpr int TX = 4, TY = 4, TZ = 32;
constexpr int NT = 256;

struct TidalArgs {
    const float* phi;
    const float* delta;
    float4* rec;
    int n0, n1, n2;
    int x0, y0, z0;   // first point of the box (may be negative; wrapped)
    int ex, ey, ez;   // box extents
    float ih2;        // 1/h^2
    float iq;         // 1/(4 h^2)
    float dinv;       // 1 / (1.5 Omega_m (H0/c)^2)
};

__device__ __forceinline__ int wrapi(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

// MODE 0: records at vertices; MODE 1: records at centres.
template <int MODE>
__global__ void __launch_bounds__(NT) tidal_kernel(TidalArgs a)
{
    constexpr int V = (MODE == 0) ? 1 : 0;           // extra cell below each point
    constexpr int CX = TX + V, CY = TY + V, CZ = TZ + V;
    constexpr int PX = CX + 2, PY = CY + 2, PZ = CZ + 2;
    constexpr int NC = CX * CY * CZ;
    __shared__ float sphi[PX * PY * PZ];
    __shared__ float sH[7][NC];

    const int px0 = blockIdx.z * TX, py0 = blockIdx.y * TY, pz0 = blockIdx.x * TZ;  // box-relative
    const int cx0 = a.x0 + px0 - V, cy0 = a.y0 + py0 - V, cz0 = a.z0 + pz0 - V;     // first cell

    for (int i = threadIdx.x; i < PX * PY * PZ; i += NT) {
        const int z = i % PZ, y = (i / PZ) % PY, x = i / (PZ * PY);
        const int gx = wrapi(cx0 - 1 + x, a.n0), gy = wrapi(cy0 - 1 + y, a.n1), gz = wrapi(cz0 - 1 + z, a.n2);
        sphi[i] = __ldg(a.phi + ((size_t)gx * a.n1 + gy) * a.n2 + gz);
    }
    __syncthreads();

    for (int i = threadIdx.x; i < NC; i += NT) {
        const int z = i % CZ, y = (i / CZ) % CY, x = i / (CZ * CY);
        const float* c = sphi + ((x + 1) * PY + (y + 1)) * PZ + (z + 1);
        constexpr int SX = PY * PZ, SY = PZ;
        const float p0 = c[0];
        // Eq. (tidalexample): (Phi_- - 2 Phi_0 + Phi_+)/h^2 and (Phi_++ + Phi_-- - Phi_+- - Phi_-+)/(4h^2)
        const float hxx = (c[-SX] - 2.f * p0 + c[SX]) * a.ih2;
        const float hyy = (c[-SY] - 2.f * p0 + c[SY]) * a.ih2;
        const float hzz = (c[-1] - 2.f * p0 + c[1]) * a.ih2;
        const float hxy = ((c[SX + SY] + c[-SX - SY]) - (c[SX - SY] + c[-SX + SY])) * a.iq;
        const float hxz = ((c[SX + 1] + c[-SX - 1]) - (c[SX - 1] + c[-SX + 1])) * a.iq;
        const float hyz = ((c[SY + 1] + c[-SY - 1]) - (c[SY - 1] + c[-SY + 1])) * a.iq;
        float d;
        if (a.delta) {
            const int gx = wrapi(cx0 + x, a.n0), gy = wrapi(cy0 + y, a.n1), gz = wrapi(cz0 + z, a.n2);
            d = __ldg(a.delta + ((size_t)gx * a.n1 + gy) * a.n2 + gz);
        } else {
            d = (hxx + hyy + hzz) * a.dinv;
        }
        sH[0][i] = hxx; sH[1][i] = hyy; sH[2][i] = hzz;
        sH[3][i] = hxy; sH[4][i] = hxz; sH[5][i] = hyz;
        sH[6][i] = d;
    }
    __syncthreads();

    // Output: 2 float4 per point, flattened so that consecutive threads write
    // consecutive 16-byte words (z-fastest runs of 32 points = 1 KiB).
    for (int f = threadIdx.x; f < TX * TY * TZ * 2; f += NT) {
        const int half = f & 1, p = f >> 1;
        const int z = p % TZ, y = (p / TZ) % TY, x = p / (TZ * TY);
        if (px0 + x >= a.ex || py0 + y >= a.ey || pz0 + z >= a.ez) continue;
        const int ch0 = half ? 4 : 0;
        const int nch = half ? 3 : 4;
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        if (MODE == 0) {
            // vertex (x, y, z) of the tile is shared by tile cells x..x+1, y..y+1, z..z+1
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (k < nch) {
                    const float* s = sH[ch0 + k];
                    float acc = 0.f;
#pragma unroll
                    for (int dx = 0; dx < 2; ++dx)
#pragma unroll
                        for (int dy = 0; dy < 2; ++dy) {
                            const int base = ((x + dx) * CY + (y + dy)) * CZ + z;
                            acc += s[base] + s[base + 1];
                        }
                    v[k] = acc * 0.125f;
                }
            }
        } else {
            const int ci = (x * CY + y) * CZ + z;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (k < nch) v[k] = sH[ch0 + k][ci];
        }
        const int gx = wrapi(a.x0 + px0 + x, a.n0), gy = wrapi(a.y0 + py0 + y, a.n1),
                  gz = wrapi(a.z0 + pz0 + z, a.n2);
        a.rec[2 * (((size_t)gx * a.n1 + gy) * a.n2 + gz) + half] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

}  // namespace

cudaError_t launch_tidal(const rr_grid_desc& g, const float* phi, const float* delta, float* rec, int where,
                         const int32_t* bbox, cudaStream_t s)
{
    TidalArgs a;
    a.phi = phi;
    a.delta = delta;
    a.rec = reinterpret_cast<float4*>(rec);
    a.n0 = g.n[0]; a.n1 = g.n[1]; a.n2 = g.n[2];
    if (bbox) {
        a.x0 = bbox[0]; a.ex = bbox[1] - bbox[0];
        a.y0 = bbox[2]; a.ey = bbox[3] - bbox[2];
        a.z0 = bbox[4]; a.ez = bbox[5] - bbox[4];
    } else {
        a.x0 = a.y0 = a.z0 = 0;
        a.ex = g.n[0]; a.ey = g.n[1]; a.ez = g.n[2];
    }
    const double h = g.box / g.n[0];
    a.ih2 = (float)(1.0 / (h * h));
    a.iq = (float)(0.25 / (h * h));
    a.dinv = (float)(1.0 / (1.5 * g.omega_m * kH0OverC * kH0OverC));
    dim3 grid((a.ez + TZ - 1) / TZ, (a.ey + TY - 1) / TY, (a.ex + TX - 1) / TX);
    if (where == RR_AT_VERTICES)
        tidal_kernel<0><<<grid, NT, 0, s>>>(a);
    else
        tidal_kernel<1><<<grid, NT, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace rr
