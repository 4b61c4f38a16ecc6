// Adaptive meshes: the mesh plan (built once per mesh on the host, then kept
// on the device) and the per-step kernels that turn the potential into
// per-leaf records (Secs. 2.7, 3.3).
//
// Per step (rr_amr_tidal):
//  1. amr_tidal_kernel, one launch per level, coarse to fine: d_a d_b Phi at
//     every cell by the central differences of Eq. (tidalexample) when the 18
//     same-level stencil neighbours exist, else the coarser level's values
//     interpolated trilinearly to the cell centre (the option Sec. 3.3
//     adopts; hence the level order); delta from tr(H) at a = 1.
//  2. amr_vertex_kernel: the value at every distinct lattice vertex the leaf
//     corners need, as the plan's weighted sum of up to 8 leaves (Sec. 2.7:
//     the mean of 8 same-level leaves, or Eqs. (alphac3d), (alphaf3d)).
//  3. amr_leafrec_kernel: per leaf corner the mean of its 1, 2 or 4 plan
//     vertices (2 or 4: a corner in the middle of a coarse edge or face),
//     8 corners x 8 floats = 256 bytes per leaf, read by the AMR trace kernel
//     as one contiguous block.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <new>
#include <thread>
#include <vector>

#include "rr_internal.h"

using namespace rr;

namespace {

// Host view of the mesh for the plan construction.
struct AmrHost {
    int n = 0, lmax = 0;
    double box = 0, omega_m = 0;
    std::vector<std::vector<int32_t>> octs;   // per level l >= 1: parent coords at level l-1
    std::vector<int64_t> base;                // first cell number of each level (lmax + 2 entries)
    std::vector<int32_t> refined;             // cell -> oct index at the next level, or -1
    std::vector<int64_t> leaf_cell;           // leaf id -> cell number
    int64_t ncells = 0;

    int64_t side(int l) const { return (int64_t)n << l; }
    static int64_t wrap(int64_t i, int64_t m)
    {
        const int64_t r = i % m;
        return r < 0 ? r + m : r;
    }
    // cell number of (l, i, j, k) (periodic) or -1 if that cell does not exist
    int64_t cell_at(int l, int64_t i, int64_t j, int64_t k) const
    {
        const int64_t m = side(l);
        i = wrap(i, m); j = wrap(j, m); k = wrap(k, m);
        int64_t c = ((i >> l) * n + (j >> l)) * n + (k >> l);
        for (int lv = 1; lv <= l; ++lv) {
            const int32_t o = refined[(size_t)c];
            if (o < 0) return -1;
            const int sh = l - lv;
            c = base[(size_t)lv] + 8 * (int64_t)o + ((i >> sh) & 1) + 2 * ((j >> sh) & 1) + 4 * ((k >> sh) & 1);
        }
        return c;
    }
    // level and integer coordinates of cell number c
    void coords(int64_t c, int& l, int64_t x[3]) const
    {
        l = 0;
        while (l < lmax && c >= base[(size_t)l + 1]) ++l;
        if (l == 0) {
            x[0] = c / ((int64_t)n * n); x[1] = (c / n) % n; x[2] = c % n;
            return;
        }
        const int64_t r = c - base[(size_t)l], o = r / 8, ch = r % 8;
        const int32_t* p = &octs[(size_t)l][(size_t)(3 * o)];
        x[0] = 2 * (int64_t)p[0] + (ch & 1);
        x[1] = 2 * (int64_t)p[1] + ((ch >> 1) & 1);
        x[2] = 2 * (int64_t)p[2] + ((ch >> 2) & 1);
    }
    // leaf containing the finest-lattice point V + s/2 (s in {-1, +1}^3): its
    // cell number, level in lvl
    int64_t leaf_near(const int64_t V[3], const int s[3], int& lvl) const
    {
        int64_t q[3];
        const int64_t M = side(lmax);
        for (int a = 0; a < 3; ++a) q[a] = wrap(s[a] > 0 ? V[a] : V[a] - 1, M);   // finest cell
        int64_t c = ((q[0] >> lmax) * n + (q[1] >> lmax)) * n + (q[2] >> lmax);
        int l = 0;
        while (l < lmax) {
            const int32_t o = refined[(size_t)c];
            if (o < 0) break;
            ++l;
            const int sh = lmax - l;
            c = base[(size_t)l] + 8 * (int64_t)o + ((q[0] >> sh) & 1) + 2 * ((q[1] >> sh) & 1) + 4 * ((q[2] >> sh) & 1);
        }
        lvl = l;
        return c;
    }
};

}  // namespace

struct rr_amr {
    AmrHost h;
    int64_t nleaves = 0, nverts = 0;
    int32_t* d_link = nullptr;      // per cell: leaf id, or -(first child) - 1
    int32_t* d_stencil = nullptr;   // per cell: 18 neighbour cells (FD) or 8 coarser cells (interpolation)
    int8_t* d_mode = nullptr;       // per cell: 0 FD, 1 interpolation
    float* d_frac = nullptr;        // per cell: interpolation fractions (x, y, z)
    int32_t* d_vcell = nullptr;     // per vertex: 8 leaf cells
    float* d_vw = nullptr;          // per vertex: 8 weights
    int32_t* d_corner = nullptr;    // per leaf corner: 4 vertex ids (-1: unused)
    int32_t* d_leaf_cell = nullptr; // per leaf: cell number
    int32_t* d_coarse = nullptr;    // per cell: its level-0 ancestor (cell number)
    float* d_H = nullptr;           // per cell: 8 floats (scratch)
    float* d_V = nullptr;           // per vertex: 8 floats (scratch)
    // per level, the first cell number / leaf id whose coarse x is >= i (n + 1
    // entries), when every level's cells are ordered by coarse x (octs listed
    // in lexicographic order); footprint launches then cover x-slabs only
    bool x_sorted = false;
    std::vector<std::vector<int64_t>> cell_x, leaf_x;
};

namespace {

constexpr int NTA = 256;

// A box of coarse cells {x0, x0 + wx) x ... (periodic), or all of them.
struct AmrBox {
    int n, all;
    int x0, wx, y0, wy, z0, wz;
};

__device__ __forceinline__ bool in_range(int i, int x0, int w, int m, int n)
{
    if (w + 2 * m >= n) return true;
    int d = (i - x0 + m) % n;
    if (d < 0) d += n;
    return d < w + 2 * m;
}

// Is coarse cell c0 within `margin` coarse cells of the box?
__device__ __forceinline__ bool in_box(const AmrBox& b, int c0, int margin)
{
    if (b.all) return true;
    const int i = c0 / (b.n * b.n), j = (c0 / b.n) % b.n, k = c0 % b.n;
    return in_range(i, b.x0, b.wx, margin, b.n) && in_range(j, b.y0, b.wy, margin, b.n) &&
           in_range(k, b.z0, b.wz, margin, b.n);
}

// Up to kMaxRanges index ranges [start, start + len) covered by one launch;
// pre[] holds their prefix sums (thread t serves range r with pre[r] <= t < pre[r + 1]).
constexpr int kMaxRanges = 2 * (kAmrMaxLevel + 1);
struct Ranges {
    int n;
    int64_t start[kMaxRanges];
    int64_t pre[kMaxRanges + 1];
};

__device__ __forceinline__ int64_t range_at(const Ranges& R, int64_t t)
{
    int r = 0;
    while (r + 1 < R.n && t >= R.pre[r + 1]) ++r;
    return R.start[r] + (t - R.pre[r]);
}

struct TidalAmrArgs {
    const float* phi;
    const int32_t* stencil;
    const int8_t* mode;
    const float* frac;
    const int32_t* coarse;
    float* H;
    Ranges cells;
    float ih2, iq, dinv;
    float ih2h;   // 1/(2h): gradient mode
    AmrBox box;
    int margin;
    int grad;     // Method A: {d_x Phi, d_y Phi, d_z Phi, 0}, {0, 0, delta, 0} in the same 8 channels
    // generic integrals: {Q0, Q1, 0, 0}, {0, 0, 0, 0} with Q_c = field_c or (field_c - prev_c) * idt_c
    const float* f0;
    const float* p0;
    const float* f1;
    const float* p1;
    float idt0, idt1;
    int scalar;
};

__global__ void __launch_bounds__(NTA) amr_tidal_kernel(const TidalAmrArgs a)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.cells.pre[a.cells.n]) return;
    const int c = (int)range_at(a.cells, t);
    if (!in_box(a.box, __ldg(a.coarse + c), a.margin)) return;
    if (a.scalar) {
        // the cell values themselves (no stencil, no fallback)
        float q0 = __ldg(a.f0 + c), q1 = 0.f;
        if (a.p0) q0 = (q0 - __ldg(a.p0 + c)) * a.idt0;
        if (a.f1) {
            q1 = __ldg(a.f1 + c);
            if (a.p1) q1 = (q1 - __ldg(a.p1 + c)) * a.idt1;
        }
        float4* out = reinterpret_cast<float4*>(a.H) + 2 * (int64_t)c;
        out[0] = make_float4(q0, q1, 0.f, 0.f);
        out[1] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const int32_t* s = a.stencil + 18 * (int64_t)c;
    float h[6];
    if (a.mode[c] == 0) {
        float v[18];
#pragma unroll
        for (int k = 0; k < 18; ++k) v[k] = __ldg(a.phi + s[k]);
        const float p0 = __ldg(a.phi + c);
        // differences of neighbouring values first: exact when they are within
        // a factor 2 of each other, so a smooth potential on a fine level keeps
        // its FP32 precision in the second differences
        h[0] = ((v[0] - p0) + (v[1] - p0)) * a.ih2;
        h[1] = ((v[2] - p0) + (v[3] - p0)) * a.ih2;
        h[2] = ((v[4] - p0) + (v[5] - p0)) * a.ih2;
        h[3] = ((v[6] - v[8]) + (v[7] - v[9])) * a.iq;
        h[4] = ((v[10] - v[12]) + (v[11] - v[13])) * a.iq;
        h[5] = ((v[14] - v[16]) + (v[15] - v[17])) * a.iq;
        if (a.grad) {
            // central first differences (x-, x+, y-, y+, z-, z+ are stencil entries 0-5)
            float4* out = reinterpret_cast<float4*>(a.H) + 2 * (int64_t)c;
            out[0] = make_float4((v[1] - v[0]) * a.ih2h, (v[3] - v[2]) * a.ih2h, (v[5] - v[4]) * a.ih2h, 0.f);
            out[1] = make_float4(0.f, 0.f, (h[0] + h[1] + h[2]) * a.dinv, 0.f);
            return;
        }
    } else if (a.grad) {
        // the coarser level's gradient and delta interpolated (Sec. 3.3's rule)
        const float fx = a.frac[3 * (int64_t)c], fy = a.frac[3 * (int64_t)c + 1], fz = a.frac[3 * (int64_t)c + 2];
        float g[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float w = ((k & 1) ? fx : 1.f - fx) * ((k & 2) ? fy : 1.f - fy) * ((k & 4) ? fz : 1.f - fz);
            const float4 lo = reinterpret_cast<const float4*>(a.H)[2 * (int64_t)s[k]];
            const float4 hi = reinterpret_cast<const float4*>(a.H)[2 * (int64_t)s[k] + 1];
            g[0] = fmaf(w, lo.x, g[0]); g[1] = fmaf(w, lo.y, g[1]);
            g[2] = fmaf(w, lo.z, g[2]); g[3] = fmaf(w, hi.z, g[3]);
        }
        float4* out = reinterpret_cast<float4*>(a.H) + 2 * (int64_t)c;
        out[0] = make_float4(g[0], g[1], g[2], 0.f);
        out[1] = make_float4(0.f, 0.f, g[3], 0.f);
        return;
    } else {
        // the coarser level was written by an earlier launch: plain loads
        const float fx = a.frac[3 * (int64_t)c], fy = a.frac[3 * (int64_t)c + 1], fz = a.frac[3 * (int64_t)c + 2];
#pragma unroll
        for (int q = 0; q < 6; ++q) h[q] = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float w = ((k & 1) ? fx : 1.f - fx) * ((k & 2) ? fy : 1.f - fy) * ((k & 4) ? fz : 1.f - fz);
            const float4 lo = reinterpret_cast<const float4*>(a.H)[2 * (int64_t)s[k]];
            const float4 hi = reinterpret_cast<const float4*>(a.H)[2 * (int64_t)s[k] + 1];
            h[0] = fmaf(w, lo.x, h[0]); h[1] = fmaf(w, lo.y, h[1]);
            h[2] = fmaf(w, lo.z, h[2]); h[3] = fmaf(w, lo.w, h[3]);
            h[4] = fmaf(w, hi.x, h[4]); h[5] = fmaf(w, hi.y, h[5]);
        }
    }
    float4* out = reinterpret_cast<float4*>(a.H) + 2 * (int64_t)c;
    out[0] = make_float4(h[0], h[1], h[2], h[3]);
    out[1] = make_float4(h[4], h[5], (h[0] + h[1] + h[2]) * a.dinv, 0.f);
}

// One thread per vertex slot (slot v belongs to leaf v, owner of its lower corner).
__global__ void __launch_bounds__(NTA) amr_vertex_kernel(const int32_t* __restrict__ vcell,
                                                         const float* __restrict__ vw, const float* __restrict__ H,
                                                         float* __restrict__ V, const Ranges slots,
                                                         const int32_t* __restrict__ leaf_cell,
                                                         const int32_t* __restrict__ coarse, const AmrBox box)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= slots.pre[slots.n]) return;
    const int v = (int)range_at(slots, t);
    if (!in_box(box, __ldg(coarse + __ldg(leaf_cell + v)), 2)) return;
    float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int32_t c = __ldg(vcell + 8 * (int64_t)v + k);
        const float w = __ldg(vw + 8 * (int64_t)v + k);
        const float4 lo = __ldg(reinterpret_cast<const float4*>(H) + 2 * (int64_t)c);
        const float4 hi = __ldg(reinterpret_cast<const float4*>(H) + 2 * (int64_t)c + 1);
        acc[0] = fmaf(w, lo.x, acc[0]); acc[1] = fmaf(w, lo.y, acc[1]);
        acc[2] = fmaf(w, lo.z, acc[2]); acc[3] = fmaf(w, lo.w, acc[3]);
        acc[4] = fmaf(w, hi.x, acc[4]); acc[5] = fmaf(w, hi.y, acc[5]);
        acc[6] = fmaf(w, hi.z, acc[6]);
    }
    float4* out = reinterpret_cast<float4*>(V) + 2 * (int64_t)v;
    out[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
    out[1] = make_float4(acc[4], acc[5], acc[6], 0.f);
}

// One thread per leaf corner: the mean of the corner's 1, 2 or 4 vertices.
__global__ void __launch_bounds__(NTA) amr_leafrec_kernel(const int32_t* __restrict__ corner,
                                                          const float* __restrict__ V, float* __restrict__ rec,
                                                          const Ranges corners, const int32_t* __restrict__ leaf_cell,
                                                          const int32_t* __restrict__ coarse, const AmrBox box)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= corners.pre[corners.n]) return;
    const int64_t t = range_at(corners, i);
    if (!in_box(box, __ldg(coarse + __ldg(leaf_cell + t / 8)), 0)) return;
    const int4 r = __ldg(reinterpret_cast<const int4*>(corner) + t);
    const int ids[4] = {r.x, r.y, r.z, r.w};
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = make_float4(0.f, 0.f, 0.f, 0.f);
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (ids[k] < 0) continue;
        const float4 x = __ldg(reinterpret_cast<const float4*>(V) + 2 * (int64_t)ids[k]);
        const float4 y = __ldg(reinterpret_cast<const float4*>(V) + 2 * (int64_t)ids[k] + 1);
        a.x += x.x; a.y += x.y; a.z += x.z; a.w += x.w;
        b.x += y.x; b.y += y.y; b.z += y.z;
        ++cnt;
    }
    const float inv = cnt == 4 ? 0.25f : (cnt == 2 ? 0.5f : 1.f);
    float4* out = reinterpret_cast<float4*>(rec) + 2 * t;
    out[0] = make_float4(a.x * inv, a.y * inv, a.z * inv, a.w * inv);
    out[1] = make_float4(b.x * inv, b.y * inv, b.z * inv, 0.f);
}

// One thread per leaf: its own cell record (centres, for NGP).
__global__ void __launch_bounds__(NTA) amr_leafcentre_kernel(const int32_t* __restrict__ leaf_cell,
                                                             const float* __restrict__ H, float* __restrict__ rec,
                                                             const Ranges leaves, const int32_t* __restrict__ coarse,
                                                             const AmrBox box)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= leaves.pre[leaves.n]) return;
    const int64_t t = range_at(leaves, i);
    const int64_t c = __ldg(leaf_cell + t);
    if (!in_box(box, __ldg(coarse + c), 0)) return;
    float4* out = reinterpret_cast<float4*>(rec) + 2 * t;
    out[0] = __ldg(reinterpret_cast<const float4*>(H) + 2 * c);
    out[1] = __ldg(reinterpret_cast<const float4*>(H) + 2 * c + 1);
}

// ------------------------------------------------------------ host plan

// f(begin, end) over [0, n) in chunks on all hardware threads (serial when
// n is small or no thread can be started).
template <class F>
void parallel_for(int64_t n, F&& f)
{
    unsigned nt = std::thread::hardware_concurrency();
    nt = std::max(1u, std::min(nt, 128u));
    constexpr int64_t kChunk = 4096;
    if (nt == 1 || n < 4 * kChunk) {
        f((int64_t)0, n);
        return;
    }
    std::atomic<int64_t> next{0};
    auto work = [&]() {
        for (;;) {
            const int64_t b = next.fetch_add(kChunk);
            if (b >= n) break;
            f(b, std::min(n, b + kChunk));
        }
    };
    std::vector<std::thread> pool;
    try {
        for (unsigned t = 1; t < nt; ++t) pool.emplace_back(work);
    } catch (...) {
        // fewer threads: the ones started and this one share the work
    }
    work();
    for (std::thread& t : pool) t.join();
}

// The value at lattice vertex V (finest units) as 8 (leaf cell, weight) terms
// when V is a corner of every leaf around it (returns 0); 1 when V lies in the
// middle of a coarse edge or face (odd[] then marks the axes along which it is
// off the coarse lattice, lc is the coarse level); -1 if the leaves around V
// differ by more than one level.
int vertex_terms(const AmrHost& h, const int64_t V[3], int32_t cells[8], float w[8], int odd[3], int& lc)
{
    int lv[8];
    int64_t cc[8];
    int lmin = 99, lmx = -1;
    for (int o = 0; o < 8; ++o) {
        const int s[3] = {(o & 1) ? 1 : -1, (o & 2) ? 1 : -1, (o & 4) ? 1 : -1};
        cc[o] = h.leaf_near(V, s, lv[o]);
        lmin = std::min(lmin, lv[o]);
        lmx = std::max(lmx, lv[o]);
    }
    lc = lmin;
    odd[0] = odd[1] = odd[2] = 0;
    if (lmx == lmin) {
        for (int o = 0; o < 8; ++o) { cells[o] = (int32_t)cc[o]; w[o] = 0.125f; }
        return 0;
    }
    if (lmx - lmin > 1) return -1;
    const int64_t cstep = (int64_t)1 << (h.lmax - lmin);
    int nodd = 0;
    for (int a = 0; a < 3; ++a) {
        odd[a] = (AmrHost::wrap(V[a], h.side(h.lmax)) % cstep) != 0;
        nodd += odd[a];
    }
    if (nodd > 0) return 1;
    // shared by coarse and fine leaves: Eqs. (alphac3d), (alphaf3d), with
    // N_fv of a fine leaf = its corners that touch a coarser leaf
    const int64_t fstep = (int64_t)1 << (h.lmax - lmx);
    int Nc = 0, nfv[8];
    double sum_fv = 0.0;
    for (int o = 0; o < 8; ++o) {
        nfv[o] = 0;
        if (lv[o] == lmin) { ++Nc; continue; }
        int l;
        int64_t x[3];
        h.coords(cc[o], l, x);
        for (int t = 0; t < 8; ++t) {
            const int64_t W[3] = {(x[0] + (t & 1)) * fstep, (x[1] + ((t >> 1) & 1)) * fstep,
                                  (x[2] + ((t >> 2) & 1)) * fstep};
            bool coarser = false;
            for (int q = 0; q < 8 && !coarser; ++q) {
                const int s[3] = {(q & 1) ? 1 : -1, (q & 2) ? 1 : -1, (q & 4) ? 1 : -1};
                int lq;
                h.leaf_near(W, s, lq);
                coarser = lq < lmx;
            }
            nfv[o] += coarser;
        }
        sum_fv += nfv[o];
    }
    const double ac = 1.0 / ((double)Nc + sum_fv / 8.0);
    for (int o = 0; o < 8; ++o) {
        cells[o] = (int32_t)cc[o];
        w[o] = (float)(lv[o] == lmin ? ac : ac * nfv[o] / 8.0);
    }
    return 0;
}

struct Plan {
    std::vector<int32_t> link, stencil, vcell, corner, leaf_cell, coarse;
    std::vector<int8_t> mode;
    std::vector<float> frac, vw;
};

rr_status build_plan(AmrHost& h, Plan& P, int64_t& nleaves, int64_t& nverts)
{
    const int L = h.lmax;
    h.base.assign((size_t)L + 2, 0);
    h.base[1] = (int64_t)h.n * h.n * h.n;
    for (int l = 1; l <= L; ++l)
        h.base[(size_t)l + 1] = h.base[(size_t)l] + 8 * (int64_t)(h.octs[(size_t)l].size() / 3);
    h.ncells = h.base[(size_t)L + 1];
    if (h.ncells > (int64_t)2147483647 - 8) return RR_ERR_ARG;   // cell numbers are int32 on the device
    h.refined.assign((size_t)h.ncells, -1);
    for (int l = 1; l <= L; ++l) {
        const std::vector<int32_t>& o = h.octs[(size_t)l];
        const int64_t m = (int64_t)o.size() / 3, side = h.side(l - 1);
        for (int64_t q = 0; q < m; ++q) {
            for (int a = 0; a < 3; ++a)
                if (o[3 * q + a] < 0 || o[3 * q + a] >= side) return RR_ERR_ARG;
            const int64_t c = h.cell_at(l - 1, o[3 * q], o[3 * q + 1], o[3 * q + 2]);
            if (c < 0 || h.refined[(size_t)c] >= 0) return RR_ERR_ARG;   // missing parent, or listed twice
            h.refined[(size_t)c] = (int32_t)q;
        }
    }
    // links and leaves
    P.link.assign((size_t)h.ncells, 0);
    h.leaf_cell.clear();
    for (int64_t c = 0; c < h.ncells; ++c) {
        const int32_t o = h.refined[(size_t)c];
        if (o >= 0) {
            int l;
            int64_t x[3];
            h.coords(c, l, x);
            P.link[(size_t)c] = -(int32_t)(h.base[(size_t)l + 1] + 8 * (int64_t)o) - 1;
        } else {
            P.link[(size_t)c] = (int32_t)h.leaf_cell.size();
            h.leaf_cell.push_back(c);
        }
    }
    nleaves = (int64_t)h.leaf_cell.size();
    P.leaf_cell.assign(h.leaf_cell.begin(), h.leaf_cell.end());
    P.coarse.assign((size_t)h.ncells, 0);
    parallel_for(h.ncells, [&](int64_t c0, int64_t c1) {
        for (int64_t c = c0; c < c1; ++c) {
            int l;
            int64_t x[3];
            h.coords(c, l, x);
            P.coarse[(size_t)c] = (int32_t)((((x[0] >> l) * h.n) + (x[1] >> l)) * h.n + (x[2] >> l));
        }
    });

    // per cell: 18 same-level stencil neighbours, or 8 coarser cells to interpolate from
    static const int offs[18][3] = {{-1, 0, 0}, {1, 0, 0},   {0, -1, 0}, {0, 1, 0},  {0, 0, -1}, {0, 0, 1},
                                    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1},
                                    {1, 0, -1}, {-1, 0, 1},  {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    P.stencil.assign((size_t)h.ncells * 18, 0);
    P.mode.assign((size_t)h.ncells, 0);
    P.frac.assign((size_t)h.ncells * 3, 0.f);
    std::atomic<int> bad{0};
    parallel_for(h.ncells, [&](int64_t c0, int64_t c1) {
        for (int64_t c = c0; c < c1; ++c) {
            int l;
            int64_t x[3];
            h.coords(c, l, x);
            bool ok = true;
            int32_t nb[18];
            for (int t = 0; t < 18 && ok; ++t) {
                const int64_t q = h.cell_at(l, x[0] + offs[t][0], x[1] + offs[t][1], x[2] + offs[t][2]);
                ok = q >= 0;
                nb[t] = (int32_t)q;
            }
            if (ok) {
                memcpy(&P.stencil[(size_t)c * 18], nb, sizeof(nb));
                continue;
            }
            if (l == 0) {
                bad = 1;
                continue;
            }
            // fine centre in coarse-centre units: x / 2 - 1/4
            P.mode[(size_t)c] = 1;
            int64_t lo[3];
            for (int a = 0; a < 3; ++a) {
                if (x[a] % 2 == 0) { lo[a] = x[a] / 2 - 1; P.frac[(size_t)c * 3 + a] = 0.75f; }
                else { lo[a] = (x[a] - 1) / 2; P.frac[(size_t)c * 3 + a] = 0.25f; }
            }
            for (int t = 0; t < 8; ++t) {
                const int64_t q = h.cell_at(l - 1, lo[0] + (t & 1), lo[1] + ((t >> 1) & 1), lo[2] + ((t >> 2) & 1));
                if (q < 0) bad = 1;   // not 2:1 balanced
                P.stencil[(size_t)c * 18 + t] = (int32_t)q;
            }
        }
    });
    if (bad) return RR_ERR_ARG;

    // Vertices. A lattice point V that is a corner of every leaf around it is
    // owned by the leaf just above it (the leaf containing V + (1/2, 1/2, 1/2)
    // finest cells), of which it is the lower corner; so the plan keeps one
    // vertex slot per leaf, for its lower corner, with zero weights when that
    // corner is hanging. Every other leaf corner lies in the middle of a
    // coarser leaf's edge or face and takes the mean of that edge's or face's
    // coarse vertices.
    const int64_t M = h.side(L);
    nverts = nleaves;
    P.vcell.assign((size_t)nleaves * 8, 0);
    P.vw.assign((size_t)nleaves * 8, 0.f);
    P.corner.assign((size_t)nleaves * 8 * 4, -1);
    std::vector<uint8_t> is_vertex((size_t)nleaves, 0);
    auto lower_corner = [&](int64_t leaf, int64_t V[3]) {
        int l;
        int64_t x[3];
        h.coords(h.leaf_cell[(size_t)leaf], l, x);
        for (int a = 0; a < 3; ++a) V[a] = x[a] << (L - l);
    };
    parallel_for(nleaves, [&](int64_t b, int64_t e) {
        for (int64_t lf = b; lf < e; ++lf) {
            int64_t V[3];
            lower_corner(lf, V);
            int32_t cells[8];
            float w[8];
            int odd[3], lc;
            const int rc = vertex_terms(h, V, cells, w, odd, lc);
            if (rc < 0) {
                bad = 1;
                continue;
            }
            if (rc == 0) {
                memcpy(&P.vcell[(size_t)lf * 8], cells, sizeof(cells));
                memcpy(&P.vw[(size_t)lf * 8], w, sizeof(w));
                is_vertex[(size_t)lf] = 1;
            } else {
                for (int k = 0; k < 8; ++k) P.vcell[(size_t)lf * 8 + k] = (int32_t)h.leaf_cell[(size_t)lf];
            }
        }
    });
    if (bad) return RR_ERR_ARG;
    // slot of the plan vertex at V, or -1 if V is not one
    auto vertex_at = [&](const int64_t V[3]) -> int32_t {
        static const int up[3] = {1, 1, 1};
        int lv;
        const int32_t owner = P.link[(size_t)h.leaf_near(V, up, lv)];
        int64_t W[3];
        lower_corner(owner, W);
        for (int a = 0; a < 3; ++a)
            if (W[a] != AmrHost::wrap(V[a], M)) return -1;
        return is_vertex[(size_t)owner] ? owner : -1;
    };
    parallel_for(nleaves, [&](int64_t b, int64_t e) {
        for (int64_t lf = b; lf < e; ++lf) {
            int l;
            int64_t x[3];
            h.coords(h.leaf_cell[(size_t)lf], l, x);
            const int64_t step = (int64_t)1 << (L - l);
            for (int t = 0; t < 8; ++t) {
                const int64_t V[3] = {(x[0] + (t & 1)) * step, (x[1] + ((t >> 1) & 1)) * step,
                                      (x[2] + ((t >> 2) & 1)) * step};
                int32_t* slot = &P.corner[((size_t)lf * 8 + t) * 4];
                const int32_t id = vertex_at(V);
                if (id >= 0) {
                    slot[0] = id;
                    continue;
                }
                // middle of a coarse edge or face: the mean of its 2 or 4 coarse vertices
                int32_t cells[8];
                float w[8];
                int odd[3], lc;
                const int nodd_rc = vertex_terms(h, V, cells, w, odd, lc);
                const int nodd = odd[0] + odd[1] + odd[2];
                if (nodd_rc != 1 || nodd == 3) {
                    bad = 1;
                    break;
                }
                const int64_t half = ((int64_t)1 << (L - lc)) / 2;
                for (int p = 0; p < (1 << nodd); ++p) {
                    int64_t W[3] = {V[0], V[1], V[2]};
                    int bit = 0;
                    for (int a = 0; a < 3; ++a)
                        if (odd[a]) {
                            W[a] += ((p >> bit) & 1) ? half : -half;
                            ++bit;
                        }
                    const int32_t wid = vertex_at(W);
                    if (wid < 0) bad = 1;   // a coarse vertex in the middle of a coarser edge: not balanced
                    slot[p] = wid;
                }
            }
        }
    });
    if (bad) return RR_ERR_ARG;
    return RR_OK;
}

void free_amr(rr_amr* A)
{
    if (!A) return;
    cudaFree(A->d_link);
    cudaFree(A->d_stencil);
    cudaFree(A->d_mode);
    cudaFree(A->d_frac);
    cudaFree(A->d_vcell);
    cudaFree(A->d_vw);
    cudaFree(A->d_corner);
    cudaFree(A->d_leaf_cell);
    cudaFree(A->d_coarse);
    cudaFree(A->d_H);
    cudaFree(A->d_V);
    delete A;
}

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& src)
{
    const size_t bytes = src.size() * sizeof(T);
    cudaError_t e = cudaMalloc((void**)dst, bytes > 0 ? bytes : 16);
    if (e == cudaSuccess && bytes) e = cudaMemcpy(*dst, src.data(), bytes, cudaMemcpyHostToDevice);
    return e;
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + NTA - 1) / NTA); }

// Per level, the first cell number and the first leaf id whose coarse x is >= i.
void build_x_tables(rr_amr* A, const Plan& P)
{
    const AmrHost& h = A->h;
    const int n = h.n, L = h.lmax;
    const int64_t nn = (int64_t)n * n;
    A->cell_x.assign((size_t)L + 1, std::vector<int64_t>());
    A->leaf_x.assign((size_t)L + 1, std::vector<int64_t>());
    A->x_sorted = true;
    // first index of each x in [first, last) of a sequence whose x never decreases
    auto table = [&](int64_t first, int64_t last, auto x_of, std::vector<int64_t>& tab) {
        std::vector<int64_t> cnt((size_t)n, 0);
        int prev = 0;
        for (int64_t i = first; i < last; ++i) {
            const int x = x_of(i);
            if (x < prev) return false;
            ++cnt[(size_t)x];
            prev = x;
        }
        tab.assign((size_t)n + 1, first);
        for (int i = 0; i < n; ++i) tab[(size_t)i + 1] = tab[(size_t)i] + cnt[(size_t)i];
        return true;
    };
    for (int l = 0; l <= L && A->x_sorted; ++l) {
        const int64_t c0 = h.base[(size_t)l], c1 = h.base[(size_t)l + 1];
        const int64_t f0 = std::lower_bound(h.leaf_cell.begin(), h.leaf_cell.end(), c0) - h.leaf_cell.begin();
        const int64_t f1 = std::lower_bound(h.leaf_cell.begin(), h.leaf_cell.end(), c1) - h.leaf_cell.begin();
        A->x_sorted = table(c0, c1, [&](int64_t c) { return (int)(P.coarse[(size_t)c] / nn); }, A->cell_x[(size_t)l]) &&
                      table(f0, f1, [&](int64_t f) { return (int)(P.coarse[(size_t)h.leaf_cell[(size_t)f]] / nn); },
                            A->leaf_x[(size_t)l]);
    }
}

// Add the part of table `tab` (n + 1 entries: first index with coarse x >= i)
// for x in [lo, lo + w) (periodic), times `mult`, to R.
void add_x_ranges(Ranges& R, const std::vector<int64_t>& tab, int lo, int w, int n, int64_t mult)
{
    auto push = [&](int64_t a, int64_t b) {
        if (b <= a || R.n >= kMaxRanges) return;
        R.start[R.n] = a * mult;
        R.pre[R.n + 1] = R.pre[R.n] + (b - a) * mult;
        ++R.n;
    };
    if (w >= n) {
        push(tab[0], tab[(size_t)n]);
        return;
    }
    lo = (int)AmrHost::wrap(lo, n);
    const int hi = lo + w;
    if (hi <= n) {
        push(tab[(size_t)lo], tab[(size_t)hi]);
    } else {
        push(tab[(size_t)lo], tab[(size_t)n]);
        push(tab[0], tab[(size_t)(hi - n)]);
    }
}

Ranges one_range(int64_t start, int64_t len)
{
    Ranges R;
    R.n = 0;
    R.pre[0] = 0;
    if (len > 0) {
        R.n = 1;
        R.start[0] = start;
        R.pre[1] = len;
    }
    return R;
}

}  // namespace

extern "C" {

rr_status rr_amr_create(const rr_amr_desc* desc, const int32_t* const* octs, const int64_t* noct, rr_amr** out)
{
    if (!desc || !out) return RR_ERR_ARG;
    *out = nullptr;
    if (desc->n < 2 || desc->n > 4096 || desc->lmax < 0 || desc->lmax > kAmrMaxLevel) return RR_ERR_ARG;
    if (!std::isfinite(desc->box) || !(desc->box > 0) || !std::isfinite(desc->omega_m) || !(desc->omega_m > 0))
        return RR_ERR_ARG;
    if (((int64_t)desc->n << desc->lmax) > ((int64_t)1 << 24)) return RR_ERR_ARG;
    if (desc->lmax > 0 && (!octs || !noct)) return RR_ERR_ARG;
    for (int l = 1; l <= desc->lmax; ++l)
        if (noct[l] < 0 || (noct[l] > 0 && !octs[l]) || noct[l] > ((int64_t)1 << 28)) return RR_ERR_ARG;
    rr_amr* A = new (std::nothrow) rr_amr();
    if (!A) return RR_ERR_OOM;
    A->h.n = desc->n;
    A->h.lmax = desc->lmax;
    A->h.box = desc->box;
    A->h.omega_m = desc->omega_m;
    A->h.octs.assign((size_t)desc->lmax + 1, std::vector<int32_t>());
    for (int l = 1; l <= desc->lmax; ++l) A->h.octs[(size_t)l].assign(octs[l], octs[l] + 3 * noct[l]);
    Plan P;
    rr_status st = build_plan(A->h, P, A->nleaves, A->nverts);
    if (st == RR_OK) {
        cudaError_t e = upload(&A->d_link, P.link);
        if (e == cudaSuccess) e = upload(&A->d_stencil, P.stencil);
        if (e == cudaSuccess) e = upload(&A->d_mode, P.mode);
        if (e == cudaSuccess) e = upload(&A->d_frac, P.frac);
        if (e == cudaSuccess) e = upload(&A->d_vcell, P.vcell);
        if (e == cudaSuccess) e = upload(&A->d_vw, P.vw);
        if (e == cudaSuccess) e = upload(&A->d_corner, P.corner);
        if (e == cudaSuccess) e = upload(&A->d_leaf_cell, P.leaf_cell);
        if (e == cudaSuccess) e = upload(&A->d_coarse, P.coarse);
        if (e == cudaSuccess) e = cudaMalloc((void**)&A->d_H, (size_t)A->h.ncells * 8 * sizeof(float));
        if (e == cudaSuccess)
            e = cudaMalloc((void**)&A->d_V, (size_t)std::max<int64_t>(A->nverts, 1) * 8 * sizeof(float));
        st = status_of_cuda(e);
    }
    if (st != RR_OK) {
        free_amr(A);
        return st;
    }
    build_x_tables(A, P);
    std::vector<int32_t>().swap(A->h.refined);   // the tables live on the device from here on
    *out = A;
    return RR_OK;
}

rr_status rr_amr_destroy(rr_amr* A)
{
    if (!A) return RR_ERR_ARG;
    cudaDeviceSynchronize();
    free_amr(A);
    return RR_OK;
}

rr_status rr_amr_sizes(rr_amr* A, int64_t* ncells, int64_t* nleaves, int64_t* nverts)
{
    if (!A) return RR_ERR_ARG;
    if (ncells) *ncells = A->h.ncells;
    if (nleaves) *nleaves = A->nleaves;
    if (nverts) *nverts = A->nverts;
    return RR_OK;
}

struct ScalarIn {
    const float* f0 = nullptr;
    const float* p0 = nullptr;
    const float* f1 = nullptr;
    const float* p1 = nullptr;
    float idt0 = 1.f, idt1 = 1.f;
};

static rr_status amr_records(rr_amr* A, const float* phi, int32_t where, float* leaf_rec, float* cell_tidal,
                              const int32_t* bbox, void* stream, int grad, const ScalarIn* sc = nullptr)
{
    if (!A || !phi || !leaf_rec || ((uintptr_t)leaf_rec & 15u)) return RR_ERR_ARG;
    if (cell_tidal && ((uintptr_t)cell_tidal & 15u)) return RR_ERR_ARG;
    if (where != RR_AT_VERTICES && where != RR_AT_CENTRES) return RR_ERR_ARG;
    const AmrHost& h = A->h;
    AmrBox box;
    box.n = h.n;
    box.all = bbox ? 0 : 1;
    box.x0 = box.y0 = box.z0 = 0;
    box.wx = box.wy = box.wz = h.n;
    if (bbox) {
        for (int a = 0; a < 3; ++a) {
            const int64_t w = (int64_t)bbox[2 * a + 1] - bbox[2 * a];
            if (w < 1 || w > h.n) return RR_ERR_ARG;
        }
        box.x0 = (int)AmrHost::wrap(bbox[0], h.n); box.wx = bbox[1] - bbox[0];
        box.y0 = (int)AmrHost::wrap(bbox[2], h.n); box.wy = bbox[3] - bbox[2];
        box.z0 = (int)AmrHost::wrap(bbox[4], h.n); box.wz = bbox[5] - bbox[4];
    }
    cudaStream_t s = (cudaStream_t)stream;
    float* H = cell_tidal ? cell_tidal : A->d_H;
    const double h0 = h.box / h.n;
    // index ranges of the cells / leaves a launch covers: x-slabs of the box
    // (plus the launch's margin) when the levels are ordered by coarse x
    const bool slabs = bbox && A->x_sorted;
    auto level_cells = [&](int l, int margin) {
        if (!slabs) return one_range(h.base[(size_t)l], h.base[(size_t)l + 1] - h.base[(size_t)l]);
        Ranges R;
        R.n = 0;
        R.pre[0] = 0;
        add_x_ranges(R, A->cell_x[(size_t)l], box.x0 - margin, box.wx + 2 * margin, h.n, 1);
        return R;
    };
    auto all_leaves = [&](int margin, int64_t mult) {
        if (!slabs) return one_range(0, A->nleaves * mult);
        Ranges R;
        R.n = 0;
        R.pre[0] = 0;
        for (int l = 0; l <= h.lmax; ++l)
            add_x_ranges(R, A->leaf_x[(size_t)l], box.x0 - margin, box.wx + 2 * margin, h.n, mult);
        return R;
    };
    for (int l = 0; l <= h.lmax; ++l) {
        const double hl = h0 / (double)((int64_t)1 << l);
        TidalAmrArgs a;
        a.phi = phi;
        a.stencil = A->d_stencil;
        a.mode = A->d_mode;
        a.frac = A->d_frac;
        a.coarse = A->d_coarse;
        a.H = H;
        a.ih2 = (float)(1.0 / (hl * hl));
        a.iq = (float)(0.25 / (hl * hl));
        a.dinv = (float)(1.0 / (1.5 * h.omega_m * kH0OverC * kH0OverC));
        a.ih2h = (float)(0.5 / hl);
        a.grad = grad;
        a.scalar = sc ? 1 : 0;
        a.f0 = sc ? sc->f0 : nullptr;
        a.p0 = sc ? sc->p0 : nullptr;
        a.f1 = sc ? sc->f1 : nullptr;
        a.p1 = sc ? sc->p1 : nullptr;
        a.idt0 = sc ? sc->idt0 : 1.f;
        a.idt1 = sc ? sc->idt1 : 1.f;
        a.box = box;
        // vertices read leaves up to 3 coarse cells outside the box; an
        // interpolated cell reads the coarser level one coarse cell further out
        a.margin = 3 + h.lmax - l;
        if (l == 0 && !grad && !sc && ((uintptr_t)H & 31u) == 0) {
            // the domain level is the regular coarse grid in row-major cell
            // order with every neighbour present: its second differences are
            // those of the uniform tidal kernel (same formulas, same order of
            // operations), which marches its planes by tensor copy; records at
            // the cell centres, over the box widened by the margin
            rr_grid_desc cg;
            cg.n[0] = cg.n[1] = cg.n[2] = h.n;
            cg.box = h.box;
            cg.omega_m = h.omega_m;
            int32_t cb[6];
            const int32_t* cbp = nullptr;
            if (!box.all) {
                const int b0[3] = {box.x0, box.y0, box.z0}, bw[3] = {box.wx, box.wy, box.wz};
                bool whole = true;
                for (int q = 0; q < 3; ++q) {
                    if (bw[q] + 2 * a.margin >= h.n) {
                        cb[2 * q] = 0;
                        cb[2 * q + 1] = h.n;
                    } else {
                        cb[2 * q] = b0[q] - a.margin;
                        cb[2 * q + 1] = b0[q] + bw[q] + a.margin;
                        whole = false;
                    }
                }
                if (!whole) cbp = cb;
            }
            const cudaError_t e = launch_tidal(cg, phi, nullptr, H, RR_AT_CENTRES, cbp, s, 0);
            if (e != cudaSuccess) return status_of_cuda(e);
            continue;
        }
        a.cells = level_cells(l, a.margin);
        const int64_t cnt = a.cells.pre[a.cells.n];
        if (cnt == 0) continue;
        amr_tidal_kernel<<<blocks_for(cnt), NTA, 0, s>>>(a);
    }
    if (where == RR_AT_VERTICES) {
        const Ranges slots = all_leaves(2, 1);
        if (slots.pre[slots.n] > 0)
            amr_vertex_kernel<<<blocks_for(slots.pre[slots.n]), NTA, 0, s>>>(A->d_vcell, A->d_vw, H, A->d_V, slots,
                                                                             A->d_leaf_cell, A->d_coarse, box);
        const Ranges corners = all_leaves(0, 8);
        if (corners.pre[corners.n] > 0)
            amr_leafrec_kernel<<<blocks_for(corners.pre[corners.n]), NTA, 0, s>>>(
                A->d_corner, A->d_V, leaf_rec, corners, A->d_leaf_cell, A->d_coarse, box);
    } else {
        const Ranges leaves = all_leaves(0, 1);
        if (leaves.pre[leaves.n] > 0)
            amr_leafcentre_kernel<<<blocks_for(leaves.pre[leaves.n]), NTA, 0, s>>>(A->d_leaf_cell, H, leaf_rec,
                                                                                   leaves, A->d_coarse, box);
    }
    return status_of_cuda(cudaGetLastError());
}

rr_status rr_amr_tidal(rr_amr* A, const float* phi, int32_t where, float* leaf_rec, float* cell_tidal,
                       const int32_t* bbox, void* stream)
{
    return amr_records(A, phi, where, leaf_rec, cell_tidal, bbox, stream, 0);
}

rr_status rr_amr_gradient(rr_amr* A, const float* phi, int32_t where, float* leaf_rec, float* cell_grad,
                          const int32_t* bbox, void* stream)
{
    return amr_records(A, phi, where, leaf_rec, cell_grad, bbox, stream, 1);
}

rr_status rr_amr_scalars(rr_amr* A, const float* field0, const float* prev0, double inv_dt0, const float* field1,
                         const float* prev1, double inv_dt1, int32_t where, float* leaf_rec, float* cell_buf,
                         const int32_t* bbox, void* stream)
{
    if (!field0 || !std::isfinite(inv_dt0) || !std::isfinite(inv_dt1)) return RR_ERR_ARG;
    ScalarIn sc;
    sc.f0 = field0;
    sc.p0 = prev0;
    sc.f1 = field1;
    sc.p1 = field1 ? prev1 : nullptr;
    sc.idt0 = (float)inv_dt0;
    sc.idt1 = (float)inv_dt1;
    return amr_records(A, field0, where, leaf_rec, cell_buf, bbox, stream, 0, &sc);
}

static TraceArgs amr_trace_args(rr_ctx* ctx, rr_amr* A, const float* leaf_rec, double chi_a, double chi_b,
                                double scale, double a_step)
{
    // the walk runs on the finest lattice: n 2^lmax cells of h_0 / 2^lmax
    rr_grid_desc fine;
    fine.n[0] = fine.n[1] = fine.n[2] = A->h.n << A->h.lmax;
    fine.box = A->h.box;
    fine.omega_m = A->h.omega_m;
    TraceArgs a = make_trace_args(ctx, &fine, leaf_rec, chi_a, chi_b, scale, a_step);
    // FP32 path variable: sub-steps of at most 256 finest cells (and 32 coarse
    // ones), so that an ulp of the path stays below 2e-5 of a finest cell; 64
    // finest cells gave maps within 1.2e-6 of the map rms of these and a 14 %
    // slower walk on the production mesh (the restarts' set-up and link descent)
    a.sub_len = (float)(std::min(32.0, 256.0 / (double)(1 << A->h.lmax)) * (A->h.box / A->h.n));
    return a;
}

rr_status rr_amr_trace_steps(rr_ctx* ctx, rr_amr* A, int32_t nsteps, const float* const* leaf_rec,
                             const double* chi_a, const double* chi_b, const double* scale, const double* a_step,
                             void* stream)
{
    if (!ctx || !A || nsteps < 0) return RR_ERR_ARG;
    if (nsteps == 0) return RR_OK;
    if (!leaf_rec || !chi_a || !chi_b || !scale || !a_step) return RR_ERR_ARG;
    if (ctx->bundle.flags & (RR_FP64_DDA | RR_PLAIN_SUMS | RR_SOURCE_MOMENTS)) {
        // the errors of rr_amr_trace_step, step by step
        for (int32_t i = 0; i < nsteps; ++i) {
            rr_status st = rr_amr_trace_step(ctx, A, leaf_rec[i], chi_a[i], chi_b[i], scale[i], a_step[i], stream);
            if (st != RR_OK) return st;
        }
        return RR_OK;
    }
    rr_grid_desc g;   // the coarse grid: argument and step-order checks
    g.n[0] = g.n[1] = g.n[2] = A->h.n;
    g.box = A->h.box;
    g.omega_m = A->h.omega_m;
    const size_t log0 = ctx->log.size();
    const bool reloc0 = ctx->relocated;
    for (int32_t i = 0; i < nsteps; ++i) {
        rr_status st = validate_step(ctx, &g, leaf_rec[i], chi_a[i], chi_b[i], scale[i], a_step[i]);
        if (st != RR_OK) {
            ctx->log.resize(log0);
            ctx->relocated = reloc0;
            return st;
        }
        StepRecord r = make_step_record(ctx, &g, chi_a[i], chi_b[i], scale[i], a_step[i]);
        r.amr = 1;
        ctx->log.push_back(r);
        ctx->relocated = false;
    }
    AmrDevice m;
    m.link = A->d_link;
    m.n = A->h.n;
    m.lmax = A->h.lmax;
    const TraceArgs a0 = amr_trace_args(ctx, A, leaf_rec[0], chi_a[0], chi_b[0], scale[0], a_step[0]);
    cudaError_t e = cudaSuccess;
    for (int32_t i = 0; i < nsteps && e == cudaSuccess;) {
        StepBlock blk{};
        blk.n = 0;
        while (i < nsteps && blk.n < kMaxStepBlock) {
            const TraceArgs a = amr_trace_args(ctx, A, leaf_rec[i], chi_a[i], chi_b[i], scale[i], a_step[i]);
            StepArgs& st = blk.s[blk.n++];
            st.rec = a.rec;
            st.chi_a = a.chi_a; st.chi_b = a.chi_b;
            st.cah = a.cah; st.cal = a.cal; st.Lf = a.Lf; st.D0f = a.D0f;
            st.sch = a.sch; st.scl = a.scl; st.bsh = a.bsh; st.bsl = a.bsl;
            ++i;
        }
        e = launch_trace_amr_steps(a0, m, blk, ctx->bundle.interp, (cudaStream_t)stream,
                                   (ctx->bundle.flags & RR_SHEAR)      ? kFormShear
                                   : (ctx->bundle.flags & RR_METHOD_A) ? kFormMethodA
                                   : (ctx->bundle.flags & RR_GENERIC)  ? kFormGeneric
                                                                       : kFormKahan);
    }
    return status_of_cuda(e);
}

rr_status rr_amr_trace_step(rr_ctx* ctx, rr_amr* A, const float* leaf_rec, double chi_a, double chi_b,
                            double scale, double a_step, void* stream)
{
    if (!ctx || !A) return RR_ERR_ARG;
    if (ctx->bundle.flags & (RR_FP64_DDA | RR_PLAIN_SUMS | RR_SOURCE_MOMENTS)) return RR_ERR_ARG;
    rr_grid_desc g;   // the coarse grid: argument and step-order checks
    g.n[0] = g.n[1] = g.n[2] = A->h.n;
    g.box = A->h.box;
    g.omega_m = A->h.omega_m;
    rr_status st = validate_step(ctx, &g, leaf_rec, chi_a, chi_b, scale, a_step);
    if (st != RR_OK) return st;
    TraceArgs a = amr_trace_args(ctx, A, leaf_rec, chi_a, chi_b, scale, a_step);
    AmrDevice m;
    m.link = A->d_link;
    m.n = A->h.n;
    m.lmax = A->h.lmax;
    const cudaError_t e =
        launch_trace_amr(a, m, ctx->bundle.interp, (cudaStream_t)stream,
                         (ctx->bundle.flags & RR_SHEAR)      ? kFormShear
                         : (ctx->bundle.flags & RR_METHOD_A) ? kFormMethodA
                         : (ctx->bundle.flags & RR_GENERIC)  ? kFormGeneric
                                                             : kFormKahan);
    if (e != cudaSuccess) return status_of_cuda(e);
    StepRecord r = make_step_record(ctx, &g, chi_a, chi_b, scale, a_step);
    r.amr = 1;
    ctx->log.push_back(r);
    ctx->relocated = false;
    return RR_OK;
}

}  // extern "C"
