// Tidal tensor and vertex records (Sec. 3.3, Eq. tidalexample; Sec. 2.7), and
// the gradient records of Method A (Eq. kappa2).
//
// One CTA of 8 warps owns a 16 (y) x 32 (z) block of cell centres, each warp
// two y-rows, each thread the two centres of its lane in them, and marches
// along x through a chunk of planes. Per plane it keeps three planes of the
// potential (with a one-cell halo) in a shared ring, and every thread
// evaluates the six central-difference second derivatives at its two centres
// (whose stencils share their middle rows: 28 shared-memory reads instead of
// 2 x 19). For records at vertices, vertex (y, z) of the plane is the upper
// corner of centres (y-1..y, z-1..z): the z pair is summed with a warp
// shuffle, the y pair in registers (the vertex between a thread's two rows)
// or through shared memory (the vertex between two warps), and the record is
// the mean of that 2 x 2 sum and the previous plane's (kept in registers) --
// the 8 cells around the vertex. The first centre row and column of the block
// are the halo of its 15 x 31 vertices. The next potential plane is loaded
// into registers while the current one is processed. HBM traffic per point:
// the potential read about 1.2 times (halo re-reads hit L2) and the 32-byte
// record written once: 36 algorithmic bytes per point. The gradient records
// (KIND 1) take the same march with the three central first differences and
// delta instead: one 16-byte record, 20 bytes per point.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "fpbits.cuh"
#include "rr_internal.h"

namespace rr {
namespace {

constexpr int TY = 16, TZ = 32;      // centres per CTA and plane
constexpr int NT = 256;              // 8 warps, two y-rows of 32 centres each
constexpr int XCHUNK_MAX = 32;       // planes per CTA, at most

struct TidalArgs {
    const float* phi;
    const float* delta;
    float4* rec;
    int n0, n1, n2;
    int x0, y0, z0;   // first point of the box (wrapped into [0, n))
    int ex, ey, ez;   // box extents
    float ih2;        // 1/h^2
    float iq;         // 1/(4 h^2)
    float dinv;       // 1 / (1.5 Omega_m (H0/c)^2)
    float ih2h;       // 1/(2h), gradient records
    int xchunk;       // planes per CTA
    int compact;      // records stored box-local (point (i, j, k) of the box at (i ey + j) ez + k)
};

// i mod n; the integer division only runs for indices outside [0, n) (halo
// points at the periodic seam, or tiles larger than a small grid).
__device__ __forceinline__ int wrapi(int i, int n)
{
    if (i >= 0 && i < n) return i;
    const int r = i % n;
    return r < 0 ? r + n : r;
}

// The channels of one centre from the three potential planes (P0, P1, P2 =
// planes x-1, x, x+1) read at the offsets of its stencil: KIND 0: the six
// second differences of Eq. (tidalexample) and delta; KIND 1: the three
// central first differences and delta. Differences of neighbours first.
template <int KIND>
__device__ __forceinline__ void centre_channels(float p0, float x0m, float x0p, float ym, float yp, float zm,
                                                float zp, float xyA, float xyB, float xzA, float xzB, float yzA,
                                                float yzB, float dlt, bool has_delta, const TidalArgs& a,
                                                float* h)
{
    // x0m / x0p: P0 and P2 at the centre; ym / yp, zm / zp: P1 neighbours;
    // xyA = P2[y+1] - P2[y-1], xyB = P0[y-1] - P0[y+1] (and so on)
    if constexpr (KIND == 0) {
        h[0] = ((x0m - p0) + (x0p - p0)) * a.ih2;
        h[1] = ((ym - p0) + (yp - p0)) * a.ih2;
        h[2] = ((zm - p0) + (zp - p0)) * a.ih2;
        h[3] = (xyA + xyB) * a.iq;
        h[4] = (xzA + xzB) * a.iq;
        h[5] = (yzA + yzB) * a.iq;
        h[6] = has_delta ? dlt : (h[0] + h[1] + h[2]) * a.dinv;
    } else {
        h[0] = (x0p - x0m) * a.ih2h;
        h[1] = (yp - ym) * a.ih2h;
        h[2] = (zp - zm) * a.ih2h;
        if (has_delta) {
            h[3] = dlt;
        } else {
            const float lap = (((x0m - p0) + (x0p - p0)) + ((ym - p0) + (yp - p0)) + ((zm - p0) + (zp - p0))) * a.ih2;
            h[3] = lap * a.dinv;
        }
    }
}

// first record of output plane c (unwrapped centre/vertex plane index);
// CMP: the box-local layout
template <bool CMP>
__device__ __forceinline__ size_t out_plane(const TidalArgs& a, int c)
{
    return CMP ? (size_t)(c - a.x0) * a.ey * a.ez : (size_t)wrapi(c, a.n0) * a.n1 * a.n2;
}

// one 32-byte tidal record {c0..c3}, {c4, c5, c6, 0} in a single 256-bit store
// (the record buffers are 32-byte aligned: the entry points check it)
__device__ __forceinline__ void store_rec(float4* r, float c0, float c1, float c2, float c3, float c4, float c5,
                                          float c6)
{
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 :: "l"(r), "f"(c0), "f"(c1), "f"(c2), "f"(c3), "f"(c4), "f"(c5), "f"(c6), "f"(0.f) : "memory");
}

// ---- the potential planes by TMA --------------------------------------------
// A plane tile of the ring: PY rows of RP floats (the centres' 34 columns plus
// the rounding of the first one down to a multiple of 4, which a tensor copy
// needs to start on a 16-byte boundary), slots 128-byte aligned.
constexpr int RP = TZ + 8;                          // 40 floats per row
constexpr int PYR = TY + 2;                         // 18 rows
constexpr int SLOT = ((PYR * RP * 4 + 127) / 128) * 128 / 4;   // floats per ring slot
constexpr int NSLOT = 5;                            // planes c - 1 .. c + 1 in use, c + 2, c + 3 arriving
constexpr unsigned kWaitTries = 1u << 22;           // bound of every wait on a copy

__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count));
}

// one tile of plane x = gx, rows y0 .., columns z0 .. of the potential into dst,
// completing on bar (the issuing thread also arms bar with the byte count)
__device__ __forceinline__ void tma_plane(const CUtensorMap* map, float* dst, unsigned long long* bar, int gx,
                                          int y0, int z0)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_u32(bar)), "r"((unsigned)(PYR * RP * 4)) : "memory");
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];"
                 :: "r"(smem_u32(dst)), "l"(map), "r"(z0), "r"(y0), "r"(gx), "r"(smem_u32(bar)) : "memory");
}

// waits until phase `parity` of bar has completed; false after kWaitTries polls
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity)
{
    for (unsigned i = 0; i < kWaitTries; ++i) {
        unsigned done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// MODE 0: records at vertices (15 x 31 per CTA and plane); MODE 1: records at
// centres (16 x 32). KIND 0: tidal records, 7 channels {Hxx, Hyy, Hzz, Hxy,
// Hxz, Hyz, delta} in 2 float4; KIND 1: gradient records, 4 channels
// {d_x Phi, d_y Phi, d_z Phi, delta} in 1 float4. Each thread owns the two
// centres (2 w, z) and (2 w + 1, z) of its warp w, lane z: the two stencils
// share their middle rows, so 28 shared-memory reads serve two centres (19 for
// one alone), and the vertex between the two rows sums its y pair in
// registers.
// TMA: the potential planes arrive in the ring by tensor copies (one thread
// issues them two planes ahead, each completing on the slot's mbarrier), for
// blocks whose tile needs no periodic wrap in y and z; the other blocks (at
// the seam) and grids whose rows are not a multiple of 16 bytes load them
// through registers, a plane ahead. A copy that does not complete within
// kWaitTries polls makes the block write NaN records (the trace then reports
// a non-finite sum) after waiting, bounded again, for its copies in flight.
// (3 resident CTAs per SM: 80 registers, no spills. With the planes staged
// through registers, 4 CTAs at 64 registers had been 9 % faster; with the
// tensor copies, 3 CTAs measure 5 % faster than 4, whose cap spills)
template <int MODE, int KIND, bool TMA, bool CMP = false>
__global__ void __launch_bounds__(NT, 3) tidal_kernel(const TidalArgs a, const __grid_constant__ CUtensorMap map)
{
    constexpr int V = (MODE == 0) ? 1 : 0;
    constexpr int NC = KIND == 0 ? 7 : 4;            // channels
    constexpr int OY = TY - V, OZ = TZ - V;          // output points per CTA and plane
    constexpr int PZ = TZ + 2;                       // potential columns a block needs (halo 1)
    constexpr int NP = PYR * PZ;
    constexpr int LP = (NP + NT - 1) / NT;           // potential loads per thread and plane (register path)
    constexpr int NW = NT / 32;                      // warps
    __shared__ __align__(128) float ring[NSLOT * SLOT];
    __shared__ __align__(8) unsigned long long mbar[NSLOT];
    __shared__ float sP[2][MODE == 0 ? NC : 1][MODE == 0 ? NT : 1];   // z-pair sums of each warp's second row

    const int w = threadIdx.x / 32, tz = threadIdx.x % 32;
    const int r0 = 2 * w;                                                  // this thread's first centre row
    const int py0 = blockIdx.y * OY, pz0 = blockIdx.x * OZ;               // box-relative first output
    const int xb = blockIdx.z * a.xchunk, xe = min(xb + a.xchunk, a.ex);   // output planes [xb, xe)
    const int cy0 = a.y0 + py0 - V, cz0 = a.z0 + pz0 - V;                 // centre (0, 0) of the block
    const int c_first = a.x0 + xb - V, c_last = a.x0 + xe - 1;            // centre planes (unwrapped)
    const int p0 = c_first - 1;                                           // first plane in the ring

    // tensor copies for this block: rows cy0 - 1 .. cy0 + 16 and columns
    // zs .. zs + 39 (zs: cz0 - 1 rounded down to a multiple of 4) inside the grid
    const int zs = (cz0 - 1) & ~3;
    const bool tma = TMA && cy0 - 1 >= 0 && cy0 - 1 + PYR <= a.n1 && cz0 - 1 >= 0 && zs + RP <= a.n2;
    const int dz = tma ? (cz0 - 1) - zs : 0;                              // column of the tile's first centre - 1

    // register path: potential plane gx into registers / into a ring slot
    int poff[LP];
#pragma unroll
    for (int k = 0; k < LP; ++k) {
        const int i = threadIdx.x + k * NT;
        const int y = i / PZ, z = i % PZ;
        poff[k] = i < NP ? wrapi(cy0 - 1 + y, a.n1) * a.n2 + wrapi(cz0 - 1 + z, a.n2) : -1;
    }
    auto fetch = [&](int gx, float r[LP]) {
        const size_t base = (size_t)wrapi(gx, a.n0) * a.n1 * a.n2;
#pragma unroll
        for (int k = 0; k < LP; ++k) r[k] = poff[k] >= 0 ? __ldg(a.phi + base + poff[k]) : 0.f;
    };
    auto slot = [&](int p) { return (p - p0) % NSLOT; };
    auto put = [&](int sl, const float r[LP]) {
#pragma unroll
        for (int k = 0; k < LP; ++k) {
            const int i = threadIdx.x + k * NT;
            if (i < NP) ring[sl * SLOT + (i / PZ) * RP + (i % PZ)] = r[k];
        }
    };
    // TMA path: plane p into its slot (thread 0), and the wait for it (all)
    auto issue = [&](int p) {
        tma_plane(&map, ring + slot(p) * SLOT, &mbar[slot(p)], wrapi(p, a.n0), cy0 - 1, zs);
    };
    auto arrived = [&](int p) { return mbar_wait(&mbar[slot(p)], (unsigned)(((p - p0) / NSLOT) & 1)); };
    bool ok = true;   // every wait of this thread ended with its copy

    float nxt[LP];   // register path: the plane two ahead of the current one, on its way to the ring
    if (tma) {
        if (threadIdx.x == 0) {
            for (int k = 0; k < NSLOT; ++k) mbar_init(&mbar[k], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            for (int p = p0; p <= p0 + 3 && p <= c_last + 1; ++p) issue(p);
        }
        __syncthreads();
        ok = arrived(p0) && arrived(p0 + 1);
    } else {
        float r[LP];
        fetch(p0, r); put(slot(p0), r);
        fetch(p0 + 1, r); put(slot(p0 + 1), r);
        fetch(p0 + 2, r); put(slot(p0 + 2), r);
        fetch(p0 + 3, nxt);
        __syncthreads();
    }

    // outputs: centre rows r0 and r0 + 1 (MODE 1), or the vertices on rows r0
    // and r0 + 1 (MODE 0: vertex row r is the upper corner of centre rows
    // r - 1 and r; row 0 and column 0 are the halo)
    const int oz = pz0 + tz - V;
    const bool oz_ok = tz >= V && oz < a.ez;
    int oy[2];
    bool out_ok[2];
    size_t out_off[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        oy[k] = py0 + r0 + k - V;
        out_ok[k] = oz_ok && (r0 + k) >= V && oy[k] < a.ey;
        out_off[k] = !out_ok[k] ? 0
                     : CMP ? (size_t)oy[k] * a.ez + oz
                                 : (size_t)wrapi(a.y0 + oy[k], a.n1) * a.n2 + wrapi(a.z0 + oz, a.n2);
    }
    const int o = (r0 + 1) * RP + (tz + 1) + dz;     // first centre in a ring slot
    size_t d_yz[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) d_yz[k] = (size_t)wrapi(cy0 + r0 + k, a.n1) * a.n2 + wrapi(cz0 + tz, a.n2);
    float prev[2][NC];   // 2 x 2 centre sums of the previous plane, per output row
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int q = 0; q < NC; ++q) prev[k][q] = 0.f;
    for (int c = c_first; c <= c_last; ++c) {
        const float* P0 = ring + slot(c - 1) * SLOT;
        const float* P1 = ring + slot(c) * SLOT;
        const float* P2 = ring + slot(c + 1) * SLOT;
        float nxt2[LP];
        if (tma) {
            // plane c + 3 into the slot of plane c - 2, read before the last barrier
            if (threadIdx.x == 0 && c + 3 <= c_last + 1) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(c + 3);
            }
            ok = arrived(c + 1) && ok;
        } else {
            // plane c + 2 goes into the slot of plane c - 3 (read before the last
            // barrier); plane c + 3 is fetched into registers, a whole plane of
            // work ahead of its use
            if (c + 3 <= c_last + 1) fetch(c + 3, nxt2);
            if (c + 2 <= c_last + 1) put(slot(c + 2), nxt);
        }

        // the two stencils: rows r0 - 1 .. r0 + 2 of P1 at z - 1 .. z + 1, rows
        // r0 - 1 .. r0 + 2 of P0 and P2 at z, rows r0, r0 + 1 of P0 and P2 at z +- 1
        const int om = o - RP, o1 = o + RP, op = o + 2 * RP;
        const float a_m0 = P1[om - 1], a_m1 = P1[om], a_m2 = P1[om + 1];
        const float a_00 = P1[o - 1], a_01 = P1[o], a_02 = P1[o + 1];
        const float a_10 = P1[o1 - 1], a_11 = P1[o1], a_12 = P1[o1 + 1];
        const float a_p0 = P1[op - 1], a_p1 = P1[op], a_p2 = P1[op + 1];
        const float b_m = P0[om], b_0 = P0[o], b_1 = P0[o1], b_p = P0[op];
        const float b_0m = P0[o - 1], b_0p = P0[o + 1], b_1m = P0[o1 - 1], b_1p = P0[o1 + 1];
        const float c_m = P2[om], c_0 = P2[o], c_1 = P2[o1], c_p = P2[op];
        const float c_0m = P2[o - 1], c_0p = P2[o + 1], c_1m = P2[o1 - 1], c_1p = P2[o1 + 1];
        float dl[2] = {0.f, 0.f};
        if (a.delta) {
            const size_t base = (size_t)wrapi(c, a.n0) * a.n1 * a.n2;
            dl[0] = __ldg(a.delta + base + d_yz[0]);
            dl[1] = __ldg(a.delta + base + d_yz[1]);
        }
        float h[2][NC];
        // centre (r0, z): y neighbours rows r0 -+ 1
        centre_channels<KIND>(a_01, b_0, c_0, a_m1, a_11, a_00, a_02, c_1 - c_m, b_m - b_1, c_0p - c_0m, b_0m - b_0p,
                              a_12 - a_10, a_m0 - a_m2, dl[0], a.delta != nullptr, a, h[0]);
        // centre (r0 + 1, z): y neighbours rows r0, r0 + 2
        centre_channels<KIND>(a_11, b_1, c_1, a_01, a_p1, a_10, a_12, c_p - c_0, b_0 - b_p, c_1p - c_1m, b_1m - b_1p,
                              a_p2 - a_p0, a_00 - a_02, dl[1], a.delta != nullptr, a, h[1]);
        if (!ok) {
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int q = 0; q < NC; ++q) h[k][q] = __int_as_float(0x7fc00000);
        }

        float pz[2][NC];
        if constexpr (MODE == 0) {
            // z pairs: each centre and the one below it in z (the lane to the left)
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int q = 0; q < NC; ++q) pz[k][q] = h[k][q] + __shfl_up_sync(0xffffffffu, h[k][q], 1);
            if (w < NW - 1) {
#pragma unroll
                for (int q = 0; q < NC; ++q) sP[(c - c_first) & 1][q][threadIdx.x] = pz[1][q];
            }
        }
        // the plane that arrives next is in the ring and the second-row z pairs
        // of plane c are shared; the next iteration writes the other sP buffer
        // and a ring slot not read here
        __syncthreads();
        if constexpr (MODE == 0) {
            // vertex row r0 + 1: centre rows r0 and r0 + 1 (this thread); vertex
            // row r0: centre rows r0 - 1 (the warp above's second row) and r0
            float b[2][NC];
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                b[1][q] = pz[0][q] + pz[1][q];
                b[0][q] = w >= 1 ? pz[0][q] + sP[(c - c_first) & 1][q][threadIdx.x - 32] : 0.f;
            }
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (c > c_first && out_ok[k]) {
                    const size_t pt = out_plane<CMP>(a, c) + out_off[k];
                    if constexpr (KIND == 0) {
                        store_rec(a.rec + 2 * pt, (prev[k][0] + b[k][0]) * 0.125f, (prev[k][1] + b[k][1]) * 0.125f,
                                  (prev[k][2] + b[k][2]) * 0.125f, (prev[k][3] + b[k][3]) * 0.125f,
                                  (prev[k][4] + b[k][4]) * 0.125f, (prev[k][5] + b[k][5]) * 0.125f,
                                  (prev[k][6] + b[k][6]) * 0.125f);
                    } else {
                        a.rec[pt] = make_float4((prev[k][0] + b[k][0]) * 0.125f, (prev[k][1] + b[k][1]) * 0.125f,
                                                (prev[k][2] + b[k][2]) * 0.125f, (prev[k][3] + b[k][3]) * 0.125f);
                    }
                }
#pragma unroll
                for (int q = 0; q < NC; ++q) prev[k][q] = b[k][q];
            }
        } else {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (!out_ok[k]) continue;
                const size_t pt = out_plane<CMP>(a, c) + out_off[k];
                if constexpr (KIND == 0) {
                    store_rec(a.rec + 2 * pt, h[k][0], h[k][1], h[k][2], h[k][3], h[k][4], h[k][5], h[k][6]);
                } else {
                    a.rec[pt] = make_float4(h[k][0], h[k][1], h[k][2], h[k][3]);
                }
            }
        }
        if (!tma) {
#pragma unroll
            for (int k = 0; k < LP; ++k) nxt[k] = nxt2[k];
        }
    }
    if (tma && __syncthreads_or(!ok) && threadIdx.x == 0) {
        // a copy did not complete in time: wait (bounded) for every copy this
        // block issued before its shared memory is released
        for (int p = p0; p <= c_last + 1; ++p) mbar_wait(&mbar[slot(p)], (unsigned)(((p - p0) / NSLOT) & 1));
    }
}

// ---------------------------------------------------------------------------
// Transpose of the above: gradient records (8 FP64 channel sums per point, at
// vertices or centres) -> dL/dPhi
// (and dL/ddelta when delta was an independent input).
//   vertices: gH(c) = (1/8) sum of the gradient records of the 8 vertices of c
//             (the transpose of the 8-cell mean);
//   delta derived from tr(H): gH_aa += gdelta / (1.5 Omega_m (H0/c)^2);
//   dL/dPhi(m) += sum_ab (D_ab^T gH_ab)(m), and the central differences are
//             symmetric on the periodic grid, so D_ab^T = D_ab.
// One CTA handles 4 x 4 x 16 cells of the output box (the whole grid, or the
// cells within the stencils' reach of the points a trace can touch); each
// output cell is written by one thread.
// ---------------------------------------------------------------------------

constexpr int AX = 4, AY = 4, AZ = 16;

struct TidalAdjArgs {
    const double2* grad;
    float* dphi;
    float* ddelta;
    int n0, n1, n2;
    int x0, y0, z0;             // output box origin, each in [0, n)
    int ex, ey, ez;             // output box extents, each <= n
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

    // first output cell of the tile, relative to the box and unwrapped
    const int bx0 = blockIdx.z * AX, by0 = blockIdx.y * AY, bz0 = blockIdx.x * AZ;
    const int cx0 = a.x0 + bx0, cy0 = a.y0 + by0, cz0 = a.z0 + bz0;
    for (int i = threadIdx.x; i < NG; i += NT) {
        const int z = i % GZ, y = (i / GZ) % GY, x = i / (GZ * GY);
        const int gx = wrapi(cx0 - 1 + x, a.n0), gy = wrapi(cy0 - 1 + y, a.n1), gz = wrapi(cz0 - 1 + z, a.n2);
        const size_t p = ((size_t)gx * a.n1 + gy) * a.n2 + gz;
        // the FP64 sums of the 8 channels (see the gradient record layout in rr.h)
        const double2 g0 = __ldg(a.grad + 4 * p), g1 = __ldg(a.grad + 4 * p + 1);
        const double2 g2 = __ldg(a.grad + 4 * p + 2), g3 = __ldg(a.grad + 4 * p + 3);
        sg[0][i] = d2f_bits(g0.x); sg[1][i] = d2f_bits(g0.y); sg[2][i] = d2f_bits(g1.x); sg[3][i] = d2f_bits(g1.y);
        sg[4][i] = d2f_bits(g2.x); sg[5][i] = d2f_bits(g2.y); sg[6][i] = d2f_bits(g3.x);
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
        if (bx0 + x >= a.ex || by0 + y >= a.ey || bz0 + z >= a.ez) continue;
        const size_t p = ((size_t)wrapi(cx0 + x, a.n0) * a.n1 + wrapi(cy0 + y, a.n1)) * a.n2 + wrapi(cz0 + z, a.n2);
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

// Zero the 64-byte gradient records of the points of a box (periodic wrap):
// four 16-byte stores per point, z fastest.
__global__ void zero_records_box_kernel(float4* __restrict__ rec, int n0, int n1, int n2, int x0, int y0, int z0,
                                        int ex, int ey, int ez)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4LL * ex * ey * ez) return;
    const long long pt = i >> 2;
    const int z = (int)(pt % ez);
    const long long r = pt / ez;
    const int y = (int)(r % ey), x = (int)(r / ey);
    const size_t p = ((size_t)wrapi(x0 + x, n0) * n1 + wrapi(y0 + y, n1)) * n2 + wrapi(z0 + z, n2);
    rec[4 * p + (i & 3)] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Scalar-pair records (generic form): channel ch of the float2 record of each
// point = Q or its 8-cell vertex mean (Sec. 2.7), with Q = field, or (field -
// prev) * inv_dt (a finite-difference time derivative, e.g. of the potential
// for the ISW integral). One thread per point of the box, z fastest.
template <int MODE>
__global__ void scalar_records_kernel(const float* __restrict__ field, const float* __restrict__ prev, float inv_dt,
                                      int ch, float* __restrict__ rec, int n0, int n1, int n2, int x0, int y0,
                                      int z0, int ex, int ey, int ez)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)ex * ey * ez) return;
    const int z = (int)(i % ez), y = (int)((i / ez) % ey), x = (int)(i / ((long long)ez * ey));
    const int px = wrapi(x0 + x, n0), py = wrapi(y0 + y, n1), pz = wrapi(z0 + z, n2);
    auto q = [&](int cx, int cy, int cz) {
        const size_t c = ((size_t)cx * n1 + cy) * n2 + cz;
        const float f = __ldg(field + c);
        return prev ? (f - __ldg(prev + c)) * inv_dt : f;
    };
    float v;
    if (MODE == 0) {
        const int xm = wrapi(px - 1, n0), ym = wrapi(py - 1, n1), zm = wrapi(pz - 1, n2);
        v = ((q(xm, ym, zm) + q(xm, ym, pz)) + (q(xm, py, zm) + q(xm, py, pz))) +
            ((q(px, ym, zm) + q(px, ym, pz)) + (q(px, py, zm) + q(px, py, pz)));
        v *= 0.125f;
    } else {
        v = q(px, py, pz);
    }
    rec[2 * (((size_t)px * n1 + py) * n2 + pz) + ch] = v;
}

}  // namespace

cudaError_t launch_scalar_records(const rr_grid_desc& g, const float* field, const float* prev, float inv_dt,
                                  int channel, float* rec, int where, const int32_t* bbox, cudaStream_t s)
{
    int x0 = 0, y0 = 0, z0 = 0, ex = g.n[0], ey = g.n[1], ez = g.n[2];
    if (bbox) {
        x0 = ((bbox[0] % g.n[0]) + g.n[0]) % g.n[0]; ex = bbox[1] - bbox[0];
        y0 = ((bbox[2] % g.n[1]) + g.n[1]) % g.n[1]; ey = bbox[3] - bbox[2];
        z0 = ((bbox[4] % g.n[2]) + g.n[2]) % g.n[2]; ez = bbox[5] - bbox[4];
    }
    const long long npts = (long long)ex * ey * ez;
    const int nt = 256;
    const unsigned blocks = (unsigned)((npts + nt - 1) / nt);
    if (where == RR_AT_VERTICES)
        scalar_records_kernel<0><<<blocks, nt, 0, s>>>(field, prev, inv_dt, channel, rec, g.n[0], g.n[1], g.n[2], x0,
                                                       y0, z0, ex, ey, ez);
    else
        scalar_records_kernel<1><<<blocks, nt, 0, s>>>(field, prev, inv_dt, channel, rec, g.n[0], g.n[1], g.n[2], x0,
                                                       y0, z0, ex, ey, ez);
    return cudaGetLastError();
}

namespace {

// The driver's tensor-map encoder, looked up once through the runtime (the
// library links no driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Tensor map of the potential (dims z, y, x; box RP x PYR x 1 floats) for the
// tidal kernel's plane copies, when the rows are a multiple of 16 bytes, the
// grid is at least one box wide and the encoder is available.
bool phi_tensor_map(const rr_grid_desc& g, const float* phi, CUtensorMap* map)
{
    if (g.n[2] % 4 != 0 || g.n[2] < RP || g.n[1] < PYR || (reinterpret_cast<uintptr_t>(phi) & 15u)) return false;
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)g.n[2], (cuuint64_t)g.n[1], (cuuint64_t)g.n[0]};
    const cuuint64_t strides[2] = {(cuuint64_t)g.n[2] * 4, (cuuint64_t)g.n[2] * g.n[1] * 4};
    const cuuint32_t box[3] = {(cuuint32_t)RP, (cuuint32_t)PYR, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(phi), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

cudaError_t launch_tidal(const rr_grid_desc& g, const float* phi, const float* delta, float* rec, int where,
                         const int32_t* bbox, cudaStream_t s, int kind, bool compact)
{
    TidalArgs a;
    a.compact = compact && bbox ? 1 : 0;
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
    a.ih2h = (float)(0.5 / h);
    // planes per CTA: long marches on big boxes; short ones when the box has
    // few y-z tiles, so that every SM still gets a couple of CTAs
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            nsm = 152;
    }
    const int oy = where == RR_AT_VERTICES ? TY - 1 : TY, oz = where == RR_AT_VERTICES ? TZ - 1 : TZ;
    const long long tiles_yz = (long long)((a.ez + oz - 1) / oz) * ((a.ey + oy - 1) / oy);
    const long long want = (long long)a.ex * tiles_yz / (2LL * nsm);
    a.xchunk = (int)std::max(2LL, std::min((long long)XCHUNK_MAX, want));
    dim3 grid((a.ez + oz - 1) / oz, (a.ey + oy - 1) / oy, (a.ex + a.xchunk - 1) / a.xchunk);
    CUtensorMap map;
    const bool tma = phi_tensor_map(g, phi, &map);
    if (!tma) memset(&map, 0, sizeof(map));
#define RR_TIDAL_LAUNCH(M, K)                                                        \
    do {                                                                              \
        if (tma) tidal_kernel<M, K, true><<<grid, NT, 0, s>>>(a, map);                \
        else tidal_kernel<M, K, false><<<grid, NT, 0, s>>>(a, map);                  \
    } while (0)
    if (a.compact) {
        // box-local tidal records (the other kinds are whole-grid only)
        if (where == RR_AT_VERTICES) {
            if (tma) tidal_kernel<0, 0, true, true><<<grid, NT, 0, s>>>(a, map);
            else tidal_kernel<0, 0, false, true><<<grid, NT, 0, s>>>(a, map);
        } else {
            if (tma) tidal_kernel<1, 0, true, true><<<grid, NT, 0, s>>>(a, map);
            else tidal_kernel<1, 0, false, true><<<grid, NT, 0, s>>>(a, map);
        }
        return cudaGetLastError();
    }
    if (kind == 0) {
        if (where == RR_AT_VERTICES) RR_TIDAL_LAUNCH(0, 0);
        else RR_TIDAL_LAUNCH(1, 0);
    } else {
        if (where == RR_AT_VERTICES) RR_TIDAL_LAUNCH(0, 1);
        else RR_TIDAL_LAUNCH(1, 1);
    }
#undef RR_TIDAL_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_tidal_adjoint(const rr_grid_desc& g, const float* grad_rec, int where, float* dphi, float* ddelta,
                                 cudaStream_t s, const long long* box0, const long long* box1)
{
    TidalAdjArgs a;
    a.grad = reinterpret_cast<const double2*>(grad_rec);
    a.dphi = dphi;
    a.ddelta = ddelta;
    a.n0 = g.n[0]; a.n1 = g.n[1]; a.n2 = g.n[2];
    int o[3], e[3];
    for (int k = 0; k < 3; ++k) {
        if (box0 && box1 && box1[k] - box0[k] < g.n[k]) {
            o[k] = (int)(((box0[k] % g.n[k]) + g.n[k]) % g.n[k]);
            e[k] = (int)std::max(0LL, box1[k] - box0[k]);
        } else {
            o[k] = 0;
            e[k] = g.n[k];
        }
    }
    a.x0 = o[0]; a.y0 = o[1]; a.z0 = o[2];
    a.ex = e[0]; a.ey = e[1]; a.ez = e[2];
    const double h = g.box / g.n[0];
    a.ih2 = (float)(1.0 / (h * h));
    a.iq = (float)(0.25 / (h * h));
    a.dinv = (float)(1.0 / (1.5 * g.omega_m * kH0OverC * kH0OverC));
    if (a.ex == 0 || a.ey == 0 || a.ez == 0) return cudaSuccess;
    dim3 grid((a.ez + AZ - 1) / AZ, (a.ey + AY - 1) / AY, (a.ex + AX - 1) / AX);
    if (where == RR_AT_VERTICES)
        tidal_adjoint_kernel<0><<<grid, NT, 0, s>>>(a);
    else
        tidal_adjoint_kernel<1><<<grid, NT, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t zero_grad_records(const rr_grid_desc& g, float* grad_rec, const long long* box0, const long long* box1,
                              cudaStream_t s)
{
    long long o[3], e[3];
    bool whole = true;
    for (int k = 0; k < 3; ++k) {
        if (box1[k] - box0[k] < g.n[k]) {
            o[k] = ((box0[k] % g.n[k]) + g.n[k]) % g.n[k];
            e[k] = std::max(0LL, box1[k] - box0[k]);
            whole = false;
        } else {
            o[k] = 0;
            e[k] = g.n[k];
        }
    }
    if (whole) return cudaMemsetAsync(grad_rec, 0, (size_t)g.n[0] * g.n[1] * g.n[2] * 64, s);
    const long long n = 4 * e[0] * e[1] * e[2];
    if (n == 0) return cudaSuccess;
    zero_records_box_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        reinterpret_cast<float4*>(grad_rec), g.n[0], g.n[1], g.n[2], (int)o[0], (int)o[1], (int)o[2], (int)e[0],
        (int)e[1], (int)e[2]);
    return cudaGetLastError();
}

}  // namespace rr
