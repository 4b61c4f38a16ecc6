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

// i mod n; the integer division only runs for indices outside [0, n) (halo
// points at the periodic seam, or tiles larger than a small grid).
__device__ __forceinline__ int wrapi(int i, int n)
{
    if (i >= 0 && i < n) return i;
    const int r = i % n;
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


// ---------------------------------------------------------------------------
// Transpose of the above: gradient records (16 floats per point: the hi and lo
// words of 8 channels, at vertices or centres) -> dL/dPhi
// (and dL/ddelta when delta was an independent input).
//   vertices: gH(c) = (1/8) sum of the gradient records of the 8 vertices of c
//             (the transpose of the 8-cell mean);
//   delta derived from tr(H): gH_aa += gdelta / (1.5 Omega_m (H0/c)^2);
//   dL/dPhi(m) += sum_ab (D_ab^T gH_ab)(m), and the central differences are
//             symmetric on the periodic grid, so D_ab^T = D_ab.
// One CTA handles 4 x 4 x 16 cells; each output cell is written by one thread.
// ---------------------------------------------------------------------------

constexpr int AX = 4, AY = 4, AZ = 16;

struct TidalAdjArgs {
    const float4* grad;
    float* dphi;
    float* ddelta;
    int n0, n1, n2;
    float ih2, iq, dinv;
};

template <int MODE>
__global__ void __launch_bounds__(NT) tidal_adjoint_kernel(TidalAdjArgs a)
{
    constexpr int V = (MODE == 0) ? 1 : 0;
    // gH is needed on the cells of the tile plus a halo of one
    constexpr int HX = AX + 2, HY = AY + 2, HZ = AZ + 2, NH = HX * HY * HZ;
    // gradient records: vertices c..c+1 of those cells (MODE 0) or the cells themselves
    constexpr int GX = HX + V, GY = HY + V, GZ = HZ + V, NG = GX * GY * GZ;
    __shared__ float sg[7][NG];
    __shared__ float sh[6][NH];

    const int cx0 = blockIdx.z * AX, cy0 = blockIdx.y * AY, cz0 = blockIdx.x * AZ;   // first output cell
    for (int i = threadIdx.x; i < NG; i += NT) {
        const int z = i % GZ, y = (i / GZ) % GY, x = i / (GZ * GY);
        const int gx = wrapi(cx0 - 1 + x, a.n0), gy = wrapi(cy0 - 1 + y, a.n1), gz = wrapi(cz0 - 1 + z, a.n2);
        const size_t p = ((size_t)gx * a.n1 + gy) * a.n2 + gz;
        // hi + lo of each channel (see the gradient record layout in rr.h)
        const float4 h0 = __ldg(a.grad + 4 * p), h1 = __ldg(a.grad + 4 * p + 1);
        const float4 l0 = __ldg(a.grad + 4 * p + 2), l1 = __ldg(a.grad + 4 * p + 3);
        sg[0][i] = h0.x + l0.x; sg[1][i] = h0.y + l0.y; sg[2][i] = h0.z + l0.z; sg[3][i] = h0.w + l0.w;
        sg[4][i] = h1.x + l1.x; sg[5][i] = h1.y + l1.y; sg[6][i] = h1.z + l1.z;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NH; i += NT) {
        const int z = i % HZ, y = (i / HZ) % HY, x = i / (HZ * HY);
        float g[7];
#pragma unroll
        for (int ch = 0; ch < 7; ++ch) {
            if (MODE == 0) {
                float acc = 0.f;
#pragma unroll
                for (int dx = 0; dx < 2; ++dx)
#pragma unroll
                    for (int dy = 0; dy < 2; ++dy) {
                        const int base = ((x + dx) * GY + (y + dy)) * GZ + z;
                        acc += sg[ch][base] + sg[ch][base + 1];
                    }
                g[ch] = acc * 0.125f;
            } else {
                g[ch] = sg[ch][(x * GY + y) * GZ + z];
            }
        }
        if (!a.ddelta) {
            const float fd = g[6] * a.dinv;
            g[0] += fd; g[1] += fd; g[2] += fd;
        }
#pragma unroll
        for (int ch = 0; ch < 6; ++ch) sh[ch][i] = g[ch];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < AX * AY * AZ; i += NT) {
        const int z = i % AZ, y = (i / AZ) % AY, x = i / (AZ * AY);
        constexpr int SX = HY * HZ, SY = HZ;
        const int ci = ((x + 1) * HY + (y + 1)) * HZ + (z + 1);
        const float* xx = sh[0] + ci;
        const float* yy = sh[1] + ci;
        const float* zz = sh[2] + ci;
        const float* xy = sh[3] + ci;
        const float* xz = sh[4] + ci;
        const float* yz = sh[5] + ci;
        float d = (xx[-SX] - 2.f * xx[0] + xx[SX]) * a.ih2;
        d += (yy[-SY] - 2.f * yy[0] + yy[SY]) * a.ih2;
        d += (zz[-1] - 2.f * zz[0] + zz[1]) * a.ih2;
        d += ((xy[SX + SY] + xy[-SX - SY]) - (xy[SX - SY] + xy[-SX + SY])) * a.iq;
        d += ((xz[SX + 1] + xz[-SX - 1]) - (xz[SX - 1] + xz[-SX + 1])) * a.iq;
        d += ((yz[SY + 1] + yz[-SY - 1]) - (yz[SY - 1] + yz[-SY + 1])) * a.iq;
        if (cx0 + x >= a.n0 || cy0 + y >= a.n1 || cz0 + z >= a.n2) continue;
        const size_t p = ((size_t)(cx0 + x) * a.n1 + (cy0 + y)) * a.n2 + (cz0 + z);
        a.dphi[p] += d;
        if (a.ddelta) {
            float gd;
            if (MODE == 0) {
                float acc = 0.f;
#pragma unroll
                for (int dx = 0; dx < 2; ++dx)
#pragma unroll
                    for (int dy = 0; dy < 2; ++dy) {
                        const int base = ((x + 1 + dx) * GY + (y + 1 + dy)) * GZ + (z + 1);
                        acc += sg[6][base] + sg[6][base + 1];
                    }
                gd = acc * 0.125f;
            } else {
                gd = sg[6][((x + 1) * GY + (y + 1)) * GZ + (z + 1)];
            }
            a.ddelta[p] += gd;
        }
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
        // the box start taken into [0, n), so that most indices need no wrap
        a.x0 = ((bbox[0] % g.n[0]) + g.n[0]) % g.n[0]; a.ex = bbox[1] - bbox[0];
        a.y0 = ((bbox[2] % g.n[1]) + g.n[1]) % g.n[1]; a.ey = bbox[3] - bbox[2];
        a.z0 = ((bbox[4] % g.n[2]) + g.n[2]) % g.n[2]; a.ez = bbox[5] - bbox[4];
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

cudaError_t launch_tidal_adjoint(const rr_grid_desc& g, const float* grad_rec, int where, float* dphi, float* ddelta,
                                 cudaStream_t s)
{
    TidalAdjArgs a;
    a.grad = reinterpret_cast<const float4*>(grad_rec);
    a.dphi = dphi;
    a.ddelta = ddelta;
    a.n0 = g.n[0]; a.n1 = g.n[1]; a.n2 = g.n[2];
    const double h = g.box / g.n[0];
    a.ih2 = (float)(1.0 / (h * h));
    a.iq = (float)(0.25 / (h * h));
    a.dinv = (float)(1.0 / (1.5 * g.omega_m * kH0OverC * kH0OverC));
    dim3 grid((a.n2 + AZ - 1) / AZ, (a.n1 + AY - 1) / AY, (a.n0 + AX - 1) / AX);
    if (where == RR_AT_VERTICES)
        tidal_adjoint_kernel<0><<<grid, NT, 0, s>>>(a);
    else
        tidal_adjoint_kernel<1><<<grid, NT, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace rr
