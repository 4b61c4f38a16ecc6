// Device helpers of the cell walk shared by the uniform-grid and the
// adaptive-mesh trace kernels: ray tiles, record loads, the projection onto
// Q_kappa, the trilinear field on a line, float-float arithmetic, compensated
// sums, and the per-ray, per-step walk setup (see trace.cu for the method).
#pragma once

#include <math_constants.h>

#include "fpbits.cuh"
#include "rr_internal.h"

namespace rr {
namespace {

constexpr int NT_MAX = 256;       // largest block the tile configurations use

// Ray (ix, iy) handled by this thread in ray tile (tx, ty): a warp covers
// wx x (32/wx) neighbouring pixels (x fastest), a block bwx x bwy warps.
__device__ __forceinline__ void tile_ray(const TileCfg& t, int tx, int ty, int& ix, int& iy)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wy = 32 / t.wx;
    ix = tx * (t.wx * t.bwx) + (warp % t.bwx) * t.wx + (lane % t.wx);
    iy = ty * (wy * t.bwy) + (warp / t.bwx) * wy + (lane / t.wx);
}

// starts moving the line holding p into L2; the per-ray accumulators are
// read and written once, after the walk, so their fetch overlaps the walk
__device__ __forceinline__ void prefetch_l2(const void* p)
{
    asm volatile("prefetch.global.L2 [%0];" :: "l"(p));
}

// Blocks ahead (in launch order) whose rays' directions a block moves into L2
// before its own walk: about half of the blocks resident on the GPU at once
// (152 SMs x 4), so that a block started later finds the first loads of its
// set-up on chip instead of in DRAM (the per-ray state of a step is larger
// than L2). Measured insensitive between 152 and 1216 on the production trace.
constexpr int kPrefetchAhead = 304;

// The directions of this thread's ray in the block kPrefetchAhead blocks
// later into L2 (the uniform-grid walk; the adaptive-mesh walk and the adjoint
// measured no gain from it).
__device__ __forceinline__ void prefetch_ahead(const TraceArgs& A, const TileCfg& t)
{
    const int nb = blockIdx.y * gridDim.x + blockIdx.x + kPrefetchAhead;
    if (nb >= (int)(gridDim.x * gridDim.y)) return;
    int ix, iy;
    tile_ray(t, nb % gridDim.x, nb / gridDim.x, ix, iy);
    if (ix >= A.nx || iy >= A.ny) return;
    const long long r = (long long)iy * A.nx + ix;
    prefetch_l2(A.dirh + r);
    prefetch_l2(A.dirl + r);
}


__device__ __forceinline__ int wrap_once(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

// A ray's accumulators held in registers across the steps of one launch (the
// multi-step kernels): read from the ray state at the end of the first step,
// written back after the last.
struct RayAcc {
    float2 k, b;
    float2 x1, x2;   // the shear pair (gamma1, gamma2), or the B moments of kappa and Born kappa
    uint32_t n;
    bool loaded;
};

struct Rec {
    float4 a, b;
};

__device__ __forceinline__ Rec load_rec(const float4* __restrict__ rec, long long idx)
{
    Rec r;
    r.a = __ldg(rec + 2 * idx);
    r.b = __ldg(rec + 2 * idx + 1);
    return r;
}

// one 32-byte tidal record in a single 256-bit load (the record buffers are
// 32-byte aligned: the entry points check it); faster than two 16-byte loads
// in the flat-addressed walk, slower in the others
__device__ __forceinline__ Rec load_rec32(const float4* __restrict__ rec, long long idx)
{
    Rec r;
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(r.a.x), "=f"(r.a.y), "=f"(r.a.z), "=f"(r.a.w), "=f"(r.b.x), "=f"(r.b.y), "=f"(r.b.z), "=f"(r.b.w)
        : "l"(rec + 2 * idx));
    return r;
}

// A gradient record of Method A: one float4 {d_x Phi, d_y Phi, d_z Phi, delta}
// per point.
__device__ __forceinline__ float4 load_grad_rec(const float4* __restrict__ rec, long long idx)
{
    return __ldg(rec + idx);
}

// (n . grad Phi, delta) of a gradient record for the direction n
__device__ __forceinline__ float2 radial_pair(float4 n, float4 r)
{
    return make_float2(fmaf(n.x, r.x, fmaf(n.y, r.y, n.z * r.z)), r.w);
}

// Q_kappa = tr(H) - n^T H n = w . (xx, yy, zz, xy, xz, yz)
__device__ __forceinline__ float project(const float w[6], const Rec& r)
{
    float q = w[0] * r.a.x;
    q = fmaf(w[1], r.a.y, q);
    q = fmaf(w[2], r.a.z, q);
    q = fmaf(w[3], r.a.w, q);
    q = fmaf(w[4], r.b.x, q);
    q = fmaf(w[5], r.b.y, q);
    return q;
}

// Trilinear field on the line u(s) = u0 + v s as the cubic e0 + e1 s + e2 s^2
// + e3 s^3. q[i + 2j + 4k] is the value at the mirrored corner (i, j, k).
__device__ __forceinline__ void line_cubic(const float q[8], float u0, float u1, float u2, float v0, float v1,
                                           float v2, float e[4])
{
    float A[4], B[4];
#pragma unroll
    for (int jk = 0; jk < 4; ++jk) {
        const float lo = q[2 * jk], d = q[2 * jk + 1] - lo;
        A[jk] = fmaf(d, u0, lo);
        B[jk] = d * v0;
    }
    float M0[2], M1[2], M2[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float C = A[2 * k + 1] - A[2 * k], D = B[2 * k + 1] - B[2 * k];
        M0[k] = fmaf(C, u1, A[2 * k]);
        M1[k] = fmaf(C, v1, fmaf(D, u1, B[2 * k]));
        M2[k] = D * v1;
    }
    const float E0 = M0[1] - M0[0], E1 = M1[1] - M1[0], E2 = M2[1] - M2[0];
    e[0] = fmaf(E0, u2, M0[0]);
    e[1] = fmaf(E0, v2, fmaf(E1, u2, M1[0]));
    e[2] = fmaf(E1, v2, fmaf(E2, u2, M2[0]));
    e[3] = E2 * v2;
}

// ---- float-float helpers (error-free transformations) ----------------------

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e)
{
    p = a * b;
    e = fmaf(a, b, -p);
}

// acc (hi, lo) + (x_hi + x_lo) * (s_hi + s_lo)
__device__ __forceinline__ float2 ff_mul_add(float2 acc, float xh, float xl, float sh, float sl)
{
    float ph, pe;
    two_prod(xh, sh, ph, pe);
    const float pl = pe + fmaf(xh, sl, xl * sh);
    float s, e;
    two_sum(acc.x, ph, s, e);
    const float t = e + (acc.y + pl);
    const float hi = s + t;
    return make_float2(hi, t - (hi - s));
}

// ---- (kappa, delta) pairs on the packed FP32 pipe (FFMA2 / FADD2 / FMUL2) ---
// Each packed operation rounds each lane exactly as its scalar counterpart.

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }

// a - b as fma(b, -1, a): one rounding, the same result as a scalar subtraction
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// line_cubic on the pair channels: q[m] = (Q_kappa, delta) at mirrored corner m
__device__ __forceinline__ void line_cubic2(const float2 q[8], float2 u0, float2 u1, float2 u2, float2 v0,
                                            float2 v1, float2 v2, float2 e[4])
{
    float2 A[4], B[4];
#pragma unroll
    for (int jk = 0; jk < 4; ++jk) {
        const float2 lo = q[2 * jk], d = sub2(q[2 * jk + 1], lo);
        A[jk] = __ffma2_rn(d, u0, lo);
        B[jk] = __fmul2_rn(d, v0);
    }
    float2 M0[2], M1[2], M2[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float2 C = sub2(A[2 * k + 1], A[2 * k]), D = sub2(B[2 * k + 1], B[2 * k]);
        M0[k] = __ffma2_rn(C, u1, A[2 * k]);
        M1[k] = __ffma2_rn(C, v1, __ffma2_rn(D, u1, B[2 * k]));
        M2[k] = __fmul2_rn(D, v1);
    }
    const float2 E0 = sub2(M0[1], M0[0]), E1 = sub2(M1[1], M1[0]), E2 = sub2(M2[1], M2[0]);
    e[0] = __ffma2_rn(E0, u2, M0[0]);
    e[1] = __ffma2_rn(E0, v2, __ffma2_rn(E1, u2, M1[0]));
    e[2] = __ffma2_rn(E1, v2, __ffma2_rn(E2, u2, M2[0]));
    e[3] = __fmul2_rn(E2, v2);
}

// Kahan sums of both channels at once
struct Acc2 {
    float2 s = {0.f, 0.f}, c = {0.f, 0.f};
    __device__ __forceinline__ void add(float2 x)
    {
        const float2 y = sub2(x, c);
        const float2 t = __fadd2_rn(s, y);
        c = sub2(sub2(t, s), y);
        s = t;
    }
    __device__ __forceinline__ bool finite() const
    {
        return isfinite(s.x) && isfinite(c.x) && isfinite(s.y) && isfinite(c.y);
    }
};

// The segment integrals of the FP32 walk, (kappa, Born) as one pair. The
// segment starts at path sig of the sub-step (chi_A = chiA0 - sig, chi_s -
// chi_A = D0 + sig) and has length t; along it the lensing kernel is
// g(chi_A - s) = G0 + G1 s + G2 s^2.
//  trilinear: the field on the line is the cubic e_0..e_3 of line_cubic2
//             (corners q, mirrored entry point u, rates v) and the integral is
//             sum_N e_{N-1} J_N with J_N = int_0^t g s^(N-1) ds (Eq. Iclensing);
//  NGP:       the constant value times J_1 (Eq. Iclensing_ngp).
__device__ __forceinline__ void kernel_coeffs(float t, float sig, float chiA0, float D0, float chis, float ichis,
                                              float& G0, float& G1, float& G2)
{
    const float chiA = chiA0 - sig;
    G0 = (D0 + sig) * chiA * ichis;
    G1 = __fmul_rn(__fmaf_rn(2.f, chiA, -chis), ichis);
    G2 = -ichis;
}

// J_N = int_0^t (G0 + G1 s + G2 s^2) s^(N-1) ds = t^N (G0 / N + t (G1 / (N + 1)
// + t G2 / (N + 2))) for N = 1..4, every operation rounded as written (no
// contraction left to the compiler, so every kernel that inlines this gives
// the same values)
__device__ __forceinline__ void j_moments(float t, float G0, float G1, float G2, float J[4])
{
    const float t2 = __fmul_rn(t, t);
    const float tG2 = __fmul_rn(t, G2);
    J[0] = __fmul_rn(t, __fmaf_rn(t, __fmaf_rn(G1, 0.5f, __fmul_rn(tG2, 1.f / 3.f)), G0));
    J[1] = __fmul_rn(t2, __fmaf_rn(t, __fmaf_rn(G1, 1.f / 3.f, __fmul_rn(tG2, 0.25f)), __fmul_rn(G0, 0.5f)));
    J[2] = __fmul_rn(__fmul_rn(t2, t),
                     __fmaf_rn(t, __fmaf_rn(G1, 0.25f, __fmul_rn(tG2, 0.2f)), __fmul_rn(G0, 1.f / 3.f)));
    J[3] = __fmul_rn(__fmul_rn(t2, t2),
                     __fmaf_rn(t, __fmaf_rn(G1, 0.2f, __fmul_rn(tG2, 1.f / 6.f)), __fmul_rn(G0, 0.25f)));
}

// sum_N e_{N-1} J_N for the cubic e (pair channels) and the quadratic kernel
// G0 + G1 s + G2 s^2 over [0, t]
__device__ __forceinline__ float2 dot_kernel(const float2 e2[4], float t, float G0, float G1, float G2)
{
    float J[4];
    j_moments(t, G0, G1, G2, J);
    float2 x = __fmul2_rn(e2[0], bc2(J[0]));
    x = __ffma2_rn(e2[1], bc2(J[1]), x);
    x = __ffma2_rn(e2[2], bc2(J[2]), x);
    return __ffma2_rn(e2[3], bc2(J[3]), x);
}

__device__ __forceinline__ float2 segment_trilinear(const float2 q[8], float u0, float u1, float u2, float v0,
                                                    float v1, float v2, float t, float G0, float G1, float G2)
{
    float2 e2[4];
    line_cubic2(q, bc2(u0), bc2(u1), bc2(u2), bc2(v0), bc2(v1), bc2(v2), e2);
    return dot_kernel(e2, t, G0, G1, G2);
}

// Method A (Eq. kappa2): the pair (n . grad Phi, delta) with two kernels, the
// first channel with K = dg/dchi = 1 - 2 chi/chi_s, i.e. K(chi_A - s) = -G1 -
// 2 G2 s, the second (Born) with g itself: sum_N e_{N-1} (L_N, J_N), L_N =
// int_0^t K s^(N-1) ds.
__device__ __forceinline__ float2 dot_kernel_a(const float2 e2[4], float t, float G0, float G1, float G2)
{
    float J[4], Lk[4];
    j_moments(t, G0, G1, G2, J);
    j_moments(t, -G1, -2.f * G2, 0.f, Lk);   // K = dg/dchi: K0 = -G1, K1 = -2 G2
    float2 x = __fmul2_rn(e2[0], make_float2(Lk[0], J[0]));
    x = __ffma2_rn(e2[1], make_float2(Lk[1], J[1]), x);
    x = __ffma2_rn(e2[2], make_float2(Lk[2], J[2]), x);
    return __ffma2_rn(e2[3], make_float2(Lk[3], J[3]), x);
}

__device__ __forceinline__ float2 segment_trilinear_a(const float2 q[8], float u0, float u1, float u2, float v0,
                                                      float v1, float v2, float t, float G0, float G1, float G2)
{
    float2 e2[4];
    line_cubic2(q, bc2(u0), bc2(u1), bc2(u2), bc2(v0), bc2(v1), bc2(v2), e2);
    return dot_kernel_a(e2, t, G0, G1, G2);
}

__device__ __forceinline__ float2 segment_ngp_a(float2 q, float t, float G0, float G1, float G2)
{
    float J[4], Lk[4];
    j_moments(t, G0, G1, G2, J);
    j_moments(t, -G1, -2.f * G2, 0.f, Lk);
    return __fmul2_rn(q, make_float2(Lk[0], J[0]));
}

// Two channels with their own quadratic kernels, K_c(chi_A - s) = G0c + G1c s
// + G2c s^2 (the generic form): sum_N e_{N-1} (J_N(x), J_N(y)).
__device__ __forceinline__ float2 dot_kernel_pair(const float2 e2[4], float t, float2 G0, float2 G1, float2 G2)
{
    const float2 t1 = bc2(t), t2 = bc2(t * t);
    const float2 t3 = __fmul2_rn(t2, t1), t4 = __fmul2_rn(t2, t2);
    // J_N = t^N (G0 / N + t (G1 / (N+1) + t G2 / (N+2)))
    auto J = [&](float2 tn, float a, float b, float c) {
        const float2 in = __ffma2_rn(t1, __ffma2_rn(t1, __fmul2_rn(G2, bc2(c)), __fmul2_rn(G1, bc2(b))),
                                     __fmul2_rn(G0, bc2(a)));
        return __fmul2_rn(tn, in);
    };
    float2 x = __fmul2_rn(e2[0], J(t1, 1.f, 0.5f, 1.f / 3.f));
    x = __ffma2_rn(e2[1], J(t2, 0.5f, 1.f / 3.f, 0.25f), x);
    x = __ffma2_rn(e2[2], J(t3, 1.f / 3.f, 0.25f, 0.2f), x);
    return __ffma2_rn(e2[3], J(t4, 0.25f, 0.2f, 1.f / 6.f), x);
}

// First channel of the trilinear field of the mirrored corners q at the
// mirrored point u (the constant term of the line cubic there).
__device__ __forceinline__ float trilinear_x(const float2 q[8], float u0, float u1, float u2)
{
    float a[4];
#pragma unroll
    for (int jk = 0; jk < 4; ++jk) a[jk] = fmaf(q[2 * jk + 1].x - q[2 * jk].x, u0, q[2 * jk].x);
    const float b0 = fmaf(a[1] - a[0], u1, a[0]), b1 = fmaf(a[3] - a[2], u1, a[2]);
    return fmaf(b1 - b0, u2, b0);
}

__device__ __forceinline__ float2 segment_ngp(float2 q, float t, float G0, float G1, float G2)
{
    float J[4];
    j_moments(t, G0, G1, G2, J);
    return __fmul2_rn(q, bc2(J[0]));
}

// Q weights of the shear (Eqs. gamma1, gamma2) for the direction n = (sin th
// cos ph, sin th sin ph, cos th): with the transverse frame e_phi = (-sin ph,
// cos ph, 0), e_theta = (cos th cos ph, cos th sin ph, -sin th) (ph = 0 on the
// z axis), gamma1 takes Q = e_phi.H.e_phi - e_theta.H.e_theta = w1 . H and
// gamma2 Q = 2 e_phi.H.e_theta = w2 . H, H = (xx, yy, zz, xy, xz, yz).
// sin th = |(n_x, n_y)| and (cos ph, sin ph) = (n_x, n_y) / sin th keep full
// relative precision however close the ray is to the axis.
__device__ __forceinline__ void shear_weights(float4 n, float w1[6], float w2[6])
{
    const float st = sqrtf(fmaf(n.x, n.x, n.y * n.y));
    float cp = 1.f, sp = 0.f;
    if (st > 0.f) {
        cp = n.x / st;
        sp = n.y / st;
    }
    const float fx = -sp, fy = cp;                          // e_phi
    const float tx = n.z * cp, ty = n.z * sp, tz = -st;     // e_theta
    // (every sum of products rounded as written: no contraction left to the compiler)
    w1[0] = __fsub_rn(__fmul_rn(fx, fx), __fmul_rn(tx, tx));
    w1[1] = __fsub_rn(__fmul_rn(fy, fy), __fmul_rn(ty, ty));
    w1[2] = -tz * tz;
    w1[3] = 2.f * __fsub_rn(__fmul_rn(fx, fy), __fmul_rn(tx, ty));
    w1[4] = -2.f * tx * tz;
    w1[5] = -2.f * ty * tz;
    w2[0] = 2.f * fx * tx;
    w2[1] = 2.f * fy * ty;
    w2[2] = 0.f;
    w2[3] = 2.f * __fadd_rn(__fmul_rn(fx, ty), __fmul_rn(fy, tx));
    w2[4] = 2.f * fx * tz;
    w2[5] = 2.f * fy * tz;
}

// float of an integer in [0, 2^23) and back, exact, on the FP32/integer pipes
// (the bit pattern of 2^23 + i), instead of the conversion unit
__device__ __forceinline__ float i2f_exact(int i) { return __int_as_float(0x4B000000 | i) - 8388608.f; }
__device__ __forceinline__ int f2i_exact(float f) { return __float_as_int(f + 8388608.f) - 0x4B000000; }
// a float holding an integer of either sign to int: exact through the bit
// pattern of 1.5 * 2^23 + f for |f| < 2^22, the conversion unit otherwise
__device__ __forceinline__ int f2i_signed(float f)
{
    return fabsf(f) < 4194304.f ? __float_as_int(f + 12582912.f) - 0x4B400000 : (int)f;
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float x)
{
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

template <class R>
struct Acc;

template <>
struct Acc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) { kahan_add(s, c, x); }
    __device__ __forceinline__ bool finite() const { return isfinite(s) && isfinite(c); }
    // the compensated sum s - c as a float-float pair
    __device__ __forceinline__ void pair(float& hi, float& lo) const { two_sum(s, -c, hi, lo); }
};

template <>
struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ bool finite() const { return isfinite(s); }
    __device__ __forceinline__ void pair(float& hi, float& lo) const
    {
        hi = (float)s;
        lo = (float)(s - (double)hi);
    }
};

// Per-ray, per-step state of the cell walk (everything the loop needs).
template <class R>
struct Walk {
    int c[3], sgn[3], k[3];      // cell, motion sign per axis (+1: +axis), crossings so far
    int vlo[3], vhi[3];          // vertex indices of the mirrored faces 0 (entry) and 1 (exit)
    R T0[3], td[3], v[3], cu[3];
    R L, chiA0, D0;
    float w[6];                  // Q_kappa = w . H
    int max_iter;
};

// The part [lo, hi] of the step [chi_b, chi_a] that ray `rid` traverses: all
// of it with periodic wrap; clipped to the box in FP64 otherwise. chi_hi is
// also given as a float-float pair, with hi - lo and chi_s - hi in FP32.
struct RayRange {
    float ch, cl, Lf, D0f;
    double hi, lo;
};

__device__ __forceinline__ bool ray_range(const TraceArgs& A, long long rid, RayRange& g)
{
    g.ch = A.cah; g.cl = A.cal; g.Lf = A.Lf; g.D0f = A.D0f;
    g.hi = A.chi_a; g.lo = A.chi_b;
    if (!A.periodic) {
        const int nn[3] = {A.n0, A.n1, A.n2};
        const double nd[3] = {A.dir[3 * rid], A.dir[3 * rid + 1], A.dir[3 * rid + 2]};
        const double obs[3] = {A.obs0, A.obs1, A.obs2};
        double hi = g.hi, lo = g.lo;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double ext = nn[a] * A.h;
            if (nd[a] == 0.0) {
                if (obs[a] < 0.0 || obs[a] > ext) hi = lo;
            } else {
                const double c0 = -obs[a] / nd[a], c1 = (ext - obs[a]) / nd[a];
                hi = fmin(hi, fmax(c0, c1));
                lo = fmax(lo, fmin(c0, c1));
            }
        }
        if (!(hi > lo)) return false;
        g.hi = hi;
        g.lo = lo;
        g.ch = (float)hi;
        g.cl = (float)(hi - (double)g.ch);
        g.Lf = (float)(hi - lo);
        g.D0f = (float)(A.chi_s - hi);
    }
    return true;
}

// Sub-step j of nsub equal pieces of the FP32 walk: start (bh + bl) =
// chi_hi - j dsub as a float-float pair (exact: TwoProd and TwoSum), length,
// and chi_s - start. Consecutive sub-steps meet at the same point. EXACT:
// integers become floats through the exact bit pattern instead of the
// conversion unit (same values; measured faster in the adaptive-mesh walk,
// slower in the uniform one, where the conversions are rare).
template <bool EXACT = false>
__device__ __forceinline__ void sub_step(const RayRange& g, int j, int nsub, float dsub, float& bh, float& bl,
                                         float& L, float& D0)
{
    if (nsub == 1) {
        bh = g.ch; bl = g.cl; L = g.Lf; D0 = g.D0f;
        return;
    }
    float p, pe;
    const float fj = EXACT ? i2f_exact(j) : (float)j;
    two_prod(fj, dsub, p, pe);
    float s, t;
    two_sum(g.ch, -p, s, t);
    const float lo = t + (g.cl - pe);
    bh = s + lo;
    bl = lo - (bh - s);
    L = (j == nsub - 1) ? fmaf(-(EXACT ? i2f_exact(nsub - 1) : (float)(nsub - 1)), dsub, g.Lf) : dsub;
    D0 = fmaf(fj, dsub, g.D0f);
}

// Start point (bh + bl, or hi in FP64), start cell and crossing distances of
// ray `rid` for a walk of length Lf (see the file comment). EXACT: as for
// sub_step (the start cell through the exact bit pattern, the periodic wrap
// only for cells outside [0, n)).
template <class R, bool EXACT = false>
__device__ __forceinline__ void walk_setup(const TraceArgs& A, long long rid, float ch, float cl, float Lf,
                                           float D0f, double hi, double lo, Walk<R>& W)
{
    constexpr bool F64 = sizeof(R) == 8;
    const int nn[3] = {A.n0, A.n1, A.n2};
    const float4 nh4 = A.dirh[rid];
    const float nh[3] = {nh4.x, nh4.y, nh4.z};

    // Start cell; distances (in cells) from the start point to the lower and
    // upper face on each axis.
    int* c = W.c; int* sgn = W.sgn; int* k = W.k;
    R* T0 = W.T0; R* td = W.td; R* v = W.v; R* cu = W.cu;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R flo, fhi;   // distance to the lower / upper face
        long long cell;
        if constexpr (F64) {
            const double na = A.dir[3 * rid + a];
            const double oa = a == 0 ? A.obs0 : (a == 1 ? A.obs1 : A.obs2);
            const double ua = fma(hi, na, oa) * A.inv_h;
            double fl = floor(ua);
            double f = ua - fl, g = (fl + 1.0) - ua;
            // exactly on a face while moving toward -a: the cell below
            if (na > 0.0 && f == 0.0) { fl -= 1.0; f = 1.0; g = 0.0; }
            cell = (long long)fl;
            flo = f;
            fhi = g;
        } else {
            const float4 nl4 = A.dirl[rid];
            const float nl = a == 0 ? nl4.x : (a == 1 ? nl4.y : nl4.z);
            // x = obs + chi n in float-float
            float ph, pe;
            two_prod(ch, nh[a], ph, pe);
            const float pl = pe + fmaf(ch, nl, cl * nh[a]);
            float xs, xe;
            two_sum(A.oh[a], ph, xs, xe);
            const float xl = xe + (A.ol[a] + pl);
            // u = x / h
            float uh, ue;
            two_prod(xs, A.ihh, uh, ue);
            float ul = ue + fmaf(xs, A.ihl, xl * A.ihh);
            const float un = uh + ul;
            ul = ul - (un - uh);
            uh = un;
            float fl = floorf(uh);
            float f, g;
            if (uh == fl && ul < 0.f) {
                fl -= 1.f;
                f = 1.f + ul;
                g = -ul;
            } else {
                f = (uh - fl) + ul;
                g = ((fl + 1.f) - uh) - ul;
            }
            // exactly on a face while moving toward -a: the cell below
            if (nh[a] > 0.f && f == 0.f) { fl -= 1.f; f = 1.f; g = 0.f; }
            if constexpr (EXACT) cell = f2i_signed(fl);
            else cell = (long long)fl;
            flo = f;
            fhi = g;
        }
        int ci = (int)cell;
        if (A.periodic) {
            // (the division of the wrap only for a cell outside [0, n))
            if ((unsigned)ci >= (unsigned)nn[a]) {
                ci %= nn[a];
                if (ci < 0) ci += nn[a];
            }
        } else if (ci < 0) {
            ci = 0; flo = (R)0; fhi = (R)1;
        } else if (ci >= nn[a]) {
            ci = nn[a] - 1; flo = (R)1; fhi = (R)0;
        }
        c[a] = ci;
        sgn[a] = nh[a] > 0.f ? -1 : 1;   // motion along a is -n_a
        const R u0 = sgn[a] > 0 ? flo : fhi;      // mirrored: grows along the motion
        const R e0 = sgn[a] > 0 ? fhi : flo;      // distance to the exit face
        R va;
        if constexpr (F64) va = (R)(fabs(A.dir[3 * rid + a]) * A.inv_h);
        else va = fabsf(nh[a]) * A.inv_hf;
        v[a] = va;
        k[a] = 0;
        if (va > (R)0) {
            // path to the k-th face crossing on this axis: T0 + k td (one rounding)
            td[a] = (R)1 / va;
            T0[a] = e0 * td[a];
            cu[a] = (R)1;
        } else {
            T0[a] = (R)1e30;   // never crosses; u stays u0
            td[a] = (R)0;
            cu[a] = u0;
        }
    }
    // vertex indices of the mirrored faces 0 (entry side) and 1 (exit side)
    int* vlo = W.vlo; int* vhi = W.vhi;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int up = c[a] + 1 == nn[a] ? 0 : c[a] + 1;
        vlo[a] = sgn[a] > 0 ? c[a] : up;
        vhi[a] = sgn[a] > 0 ? up : c[a];
    }
    float* w = W.w;
    // (sums of products rounded as written: every kernel gets the same weights)
    w[0] = __fadd_rn(__fmul_rn(nh[1], nh[1]), __fmul_rn(nh[2], nh[2]));
    w[1] = __fadd_rn(__fmul_rn(nh[0], nh[0]), __fmul_rn(nh[2], nh[2]));
    w[2] = __fadd_rn(__fmul_rn(nh[0], nh[0]), __fmul_rn(nh[1], nh[1]));
    w[3] = -2.f * nh[0] * nh[1];
    w[4] = -2.f * nh[0] * nh[2];
    w[5] = -2.f * nh[1] * nh[2];

    W.L = F64 ? (R)(hi - lo) : (R)Lf;
    W.chiA0 = F64 ? (R)hi : (R)ch;
    W.D0 = F64 ? (R)(A.chi_s - hi) : (R)D0f;
    const float cap = ceilf(Lf * (fabsf(nh[0]) + fabsf(nh[1]) + fabsf(nh[2])) * A.inv_hf * 1.0001f);
    if constexpr (EXACT) W.max_iter = cap < 4194304.f ? f2i_signed(cap) + 8 : 0x3fffffff;
    else W.max_iter = (int)cap + 8;
}

}  // namespace
}  // namespace rr
