// Adjoint of the cell-by-cell integration (the transpose of rr_trace_step).
//
// kappa and Born kappa are linear in the records, so the gradient of a loss
// with respect to the records is the transpose of the forward map: the walk
// of a logged step is replayed (geometry only) and every segment's weights
// dI/dq of its 8 corners (or its centre) are scattered back, scaled by the
// per-ray dL/dkappa and dL/dkappa_born.
#include "walk.cuh"

namespace rr {
namespace {

// Transpose of line_cubic: given the weights J_N of the cubic's coefficients
// e_{N-1} in the segment integral, the weight of each corner value q[m].
__device__ __forceinline__ void line_cubic_adjoint(const float J[4], float u0, float u1, float u2, float v0,
                                                   float v1, float v2, float W[8])
{
    const float E0 = J[0] * u2 + J[1] * v2;
    const float E1 = J[1] * u2 + J[2] * v2;
    const float E2 = J[2] * u2 + J[3] * v2;
    const float M0[2] = {J[0] - E0, E0};
    const float M1[2] = {J[1] - E1, E1};
    const float M2[2] = {J[2] - E2, E2};
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        const float C = fmaf(M0[kk], u1, M1[kk] * v1);
        const float D = fmaf(M1[kk], u1, M2[kk] * v1);
        const float A0 = M0[kk] - C, A1 = C;
        const float B0 = M1[kk] - D, B1 = D;
        // x-step for the pairs jk = 2 kk (j = 0) and 2 kk + 1 (j = 1)
        const float d0 = fmaf(A0, u0, B0 * v0);
        const float d1 = fmaf(A1, u0, B1 * v0);
        W[4 * kk + 0] = A0 - d0;
        W[4 * kk + 1] = d0;
        W[4 * kk + 2] = A1 - d1;
        W[4 * kk + 3] = d1;
    }
}

// Add S * (gk w, gb) to the gradient record of point idx: 8 FP64 sums, one
// per record channel {Hxx, Hyy, Hzz, Hxy, Hxz, Hyz, delta, 0} (64 B), for the
// lanes in `lanes` (the others take no part).
//
// For each distinct point of those lanes the warp sums their contributions in
// one reduce-scatter butterfly (every lane takes part, lanes flushing another
// point with zeros; each of the first three exchanges halves the channels a
// lane keeps: 4 + 2 + 1 + 1 + 1 shuffles instead of 5 per channel), after
// which lane 4c holds the point's total of channel c and adds it to the
// record with an FP64 atomic whose value is not used: a reduction, with no
// round trip for the lane. FP64 sums keep their accuracy where thousands of
// contributions of both signs meet; the 32-term warp sums are plain FP32 (a
// relative error of a few ulp per flush). A warp with inactive lanes adds
// every lane's channels on its own.
__device__ __forceinline__ void flush_grad(double* __restrict__ grad, long long idx, float S, float gk, float gb,
                                           const float* w, unsigned lanes = 0xffffffffu)
{
    constexpr unsigned FULL = 0xffffffffu;
    const float a = gk * S;
    const float x[8] = {a * w[0], a * w[1], a * w[2], a * w[3], a * w[4], a * w[5], gb * S, 0.f};
    const unsigned active = __activemask();
    if (active != FULL) {
        if (S != 0.f) {
            double* p = grad + 8 * idx;
#pragma unroll
            for (int c = 0; c < 7; ++c) atomicAdd(p + c, (double)x[c]);
        }
        return;
    }
    const int lane = threadIdx.x & 31;
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    const int ch = lane >> 2;
    const bool part = (lanes >> lane) & 1;
    unsigned todo = lanes;
    while (todo) {   // one pass per distinct point (todo is the same in every lane)
        const long long key = __shfl_sync(FULL, idx, __ffs(todo) - 1);
        const bool mine = part && idx == key;
        todo &= ~__ballot_sync(FULL, mine);
        float y[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) y[i] = mine ? x[i] : 0.f;
        // xor 16: keep channels 4 b4 .. 4 b4 + 3
        float k4[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float sx = b4 ? y[i] : y[4 + i];
            k4[i] = (b4 ? y[4 + i] : y[i]) + __shfl_xor_sync(FULL, sx, 16);
        }
        // xor 8: keep 2 of the 4
        float k2[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const float sx = b3 ? k4[i] : k4[2 + i];
            k2[i] = (b3 ? k4[2 + i] : k4[i]) + __shfl_xor_sync(FULL, sx, 8);
        }
        // xor 4: keep 1 of the 2; xor 2, xor 1: the warp's total of channel (lane >> 2)
        float v = (b2 ? k2[1] : k2[0]) + __shfl_xor_sync(FULL, b2 ? k2[0] : k2[1], 4);
        v += __shfl_xor_sync(FULL, v, 2);
        v += __shfl_xor_sync(FULL, v, 1);
        if ((lane & 3) == 0 && ch < 7 && v != 0.f) atomicAdd(grad + 8 * key + ch, (double)v);
    }
}

// Warps per block of the adjoint launch (the default ray tile) and the floats
// of one lane's row in the face-flush staging area: 4 corners x 8 channels,
// padded so that the lanes' 16-byte stores and the column reads below each
// take the minimum of four shared-memory wavefronts.
constexpr int kAdjWarps = 4;
constexpr int kRow = 36;

// One round of the face flush: corner r's channel values of the lanes with
// bit r of `in` set (zeros for the others) summed over the warp through
// shared memory and added to point K[r], for each corner r with bit r of
// `valid` set. Each lane stores its 4 x 8 values as a row; lane l then sums
// 8 rows (l >> 3 selects which) of columns 4 (l & 7) .. + 3, and two shuffle
// exchanges leave lane l with the warp's total of corner (l & 7) >> 1,
// channel 4 ((l & 7) & 1) + ((l >> 3) & 3), which it adds to the record with
// one FP64 reduction.
__device__ __forceinline__ void face_round(double* __restrict__ grad, const long long K[4], unsigned valid,
                                           unsigned in, const float F[4], float gk, float gb, const float* w,
                                           float* __restrict__ sm)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float* row = sm + lane * kRow;
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const float S = (in >> r & 1) ? F[r] : 0.f;
        const float a = gk * S;
        *reinterpret_cast<float4*>(row + 8 * r) = make_float4(a * w[0], a * w[1], a * w[2], a * w[3]);
        *reinterpret_cast<float4*>(row + 8 * r + 4) = make_float4(a * w[4], a * w[5], gb * S, 0.f);
    }
    __syncwarp();
    const int g = lane >> 3, c = lane & 7;
    const float* col = sm + 8 * g * kRow + 4 * c;
    float4 acc = *reinterpret_cast<const float4*>(col);
#pragma unroll
    for (int j = 1; j < 8; ++j) {
        const float4 v = *reinterpret_cast<const float4*>(col + j * kRow);
        acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
    // lanes c, c + 8, c + 16, c + 24 hold the 4 row groups' partial sums of
    // columns 4c .. 4c + 3: reduce-scatter them
    const bool b4 = lane & 16, b3 = lane & 8;
    const float k0 = (b4 ? acc.z : acc.x) + __shfl_xor_sync(FULL, b4 ? acc.x : acc.z, 16);
    const float k1 = (b4 ? acc.w : acc.y) + __shfl_xor_sync(FULL, b4 ? acc.y : acc.w, 16);
    const float v = (b3 ? k1 : k0) + __shfl_xor_sync(FULL, b3 ? k0 : k1, 8);
    const int r = c >> 1, ch = 4 * (c & 1) + 2 * b4 + b3;
    const long long p = r == 0 ? K[0] : (r == 1 ? K[1] : (r == 2 ? K[2] : K[3]));
    if ((valid >> r & 1) && ch < 7 && v != 0.f) atomicAdd(grad + 8 * p + ch, (double)v);
}

// Flush the 4 corners of the face a crossing leaves (F[r]: the ray's sum of
// dI/dq for point P[r]). Neighbouring rays of a warp are far closer together
// than a cell, so at a crossing the lanes mostly flush the same 4 points, or,
// while the warp straddles a cell plane, two points per corner (one on each
// side). Per corner, group A is the lanes flushing lane 0's point and group B
// those flushing the point of the first lane outside A; one round sums group
// A of all four corners, a second round group B where a corner has one, and
// the lanes of any further point go through flush_grad. A partial warp adds
// per lane.
__device__ __forceinline__ void flush_face(double* __restrict__ grad, const long long P[4], const float F[4], float gk,
                                           float gb, const float* w, float* __restrict__ sm)
{
    constexpr unsigned FULL = 0xffffffffu;
    if (__activemask() != FULL) {
#pragma unroll
        for (int r = 0; r < 4; ++r) flush_grad(grad, P[r], F[r], gk, gb, w);
        return;
    }
    long long K[4];
    unsigned inA = 0, multi = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        K[r] = __shfl_sync(FULL, P[r], 0);
        const bool a = P[r] == K[r];
        if (a) inA |= 1u << r;
        if (__ballot_sync(FULL, a) != FULL) multi |= 1u << r;
    }
    face_round(grad, K, 0xfu, inA, F, gk, gb, w, sm);
    if (multi) {
        unsigned inB = 0, rest[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const unsigned outA = ~__ballot_sync(FULL, inA >> r & 1);
            K[r] = __shfl_sync(FULL, P[r], outA ? __ffs(outA) - 1 : 0);
            const bool b = !(inA >> r & 1) && P[r] == K[r];
            if (b) inB |= 1u << r;
            rest[r] = outA & ~__ballot_sync(FULL, b);
        }
        face_round(grad, K, multi, inB, F, gk, gb, w, sm);
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (rest[r]) flush_grad(grad, P[r], F[r], gk, gb, w, rest[r]);
    }
}

// Adjoint of one step: replays the walk and, for every point the ray's
// segments read (the 8 vertices of each cell, or its centre), accumulates
// dI/dq of the segment integrals (the transpose of the forward map) while the
// point stays in the ray's current cell; a point is flushed into the
// gradient records once per residency, as gk * S * w (the six tidal channels
// through Q_kappa = w . H) and gb * S (delta), summed over the warp and added
// in FP64 (flush_grad).
// The FP32 trilinear form is capped at 128 registers (4 blocks of kAdjWarps
// warps per SM): uncapped it takes more and runs slower, and at 96 registers
// (5 blocks) its spills cost more than the occupancy gains.
template <int INTERP, class R>
__global__ void __launch_bounds__(32 * kAdjWarps, (INTERP == RR_TRILINEAR && sizeof(R) == 4) ? 4 : 1)
    trace_adjoint_kernel(const TraceArgs A, const AdjArgs B, const TileCfg tc)
{
    constexpr bool F64 = sizeof(R) == 8;
    __shared__ __align__(16) float stage[INTERP == RR_TRILINEAR ? kAdjWarps * 32 * kRow : 1];
    float* sm = stage + (INTERP == RR_TRILINEAR ? (threadIdx.x >> 5) * 32 * kRow : 0);
    int ix, iy;
    tile_ray(tc, blockIdx.x, blockIdx.y, ix, iy);
    if (ix >= A.nx || iy >= A.ny) return;
    const long long rid = (long long)iy * A.nx + ix;
    const float gk = B.dkappa ? (float)(B.dkappa[rid] * B.kscale) : 0.f;
    const float gb = B.dkborn ? (float)(B.dkborn[rid] * B.bscale) : 0.f;
    if (gk == 0.f && gb == 0.f) return;
    const int nn[3] = {A.n0, A.n1, A.n2};
    RayRange rg;
    if (!ray_range(A, rid, rg)) return;
    const R chis = (R)A.chi_s;
    const R ichis = F64 ? (R)(1.0 / A.chi_s) : (R)A.inv_chi_s_f;
    const long long sx = (long long)A.n1 * A.n2, sy = A.n2;
    const R eps_rel = F64 ? (R)1.4551915228366852e-11 : (R)4.76837158203125e-07;
    const int nsub = F64 ? 1 : max(1, (int)ceilf(rg.Lf / A.sub_len));
    const float dsub = rg.Lf / (float)nsub;
    bool overflow = false;
    for (int j = 0; j < nsub && !overflow; ++j) {
    float bh, bl, Lj, D0j;
    sub_step(rg, j, nsub, dsub, bh, bl, Lj, D0j);
    Walk<R> W;
    walk_setup<R>(A, rid, bh, bl, Lj, D0j, rg.hi, rg.lo, W);
    int* c = W.c;
    const int* sgn = W.sgn;
    int* k = W.k;
    int* vlo = W.vlo;
    int* vhi = W.vhi;
    const float* w = W.w;
    const R L = W.L, chiA0 = W.chiA0, D0 = W.D0;
    const R eps_end = L * eps_rel;

    float S[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    // point index of the cell's entry corner (vertex vlo on every axis) and
    // the index step from vlo to vhi per axis (periodic wrap included)
    const long long st[3] = {sx, sy, 1};
    long long P0 = vlo[0] * sx + vlo[1] * sy + vlo[2];
    long long Dv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) Dv[a] = (long long)(vhi[a] - vlo[a]) * st[a];
    R sig = 0;
    R T[3] = {W.T0[0], W.T0[1], W.T0[2]};
    int iter = 0;
    while (true) {
        R tend = T[0];
        int e = 0;
        if (T[1] < tend) { tend = T[1]; e = 1; }
        if (T[2] < tend) { tend = T[2]; e = 2; }
        const bool last = !(tend < L - eps_end);
        if (last) tend = L;
        const R t = tend - sig;
        if (t > tend * eps_rel) {
            R u[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) u[a] = fmin(fmax(fma(sig - T[a], W.v[a], W.cu[a]), (R)0), (R)1);
            const R chiA = chiA0 - sig;
            const R G0 = (D0 + sig) * chiA * ichis;
            const R G1 = (2 * chiA - chis) * ichis;
            const R G2 = -ichis;
            const R t2 = t * t;
            const R J1 = t * (G0 + t * (G1 * (R)0.5 + t * G2 * (R)(1.0 / 3.0)));
            if (INTERP == RR_TRILINEAR) {
                const float J[4] = {(float)J1,
                                    (float)(t2 * (G0 * (R)0.5 + t * (G1 * (R)(1.0 / 3.0) + t * G2 * (R)0.25))),
                                    (float)(t2 * t * (G0 * (R)(1.0 / 3.0) + t * (G1 * (R)0.25 + t * G2 * (R)0.2))),
                                    (float)(t2 * t2 * (G0 * (R)0.25 + t * (G1 * (R)0.2 + t * G2 * (R)(1.0 / 6.0))))};
                float Wm[8];
                line_cubic_adjoint(J, (float)u[0], (float)u[1], (float)u[2], (float)W.v[0], (float)W.v[1],
                                   (float)W.v[2], Wm);
#pragma unroll
                for (int m = 0; m < 8; ++m) S[m] += Wm[m];
            } else {
                S[0] += (float)J1;
            }
        }
        sig = tend;
        if (last) break;

        int nvhi = 0, ncell = 0, ne = 1;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (a == e) {
                nvhi = wrap_once(vhi[a] + sgn[a], nn[a]);
                ncell = c[a] + sgn[a];
                ne = nn[a];
            }
        if (INTERP == RR_TRILINEAR) {
            // the 4 corners on the entry face along e leave the ray's cell:
            // corner m of the cell has bit a set when it lies on vhi along
            // axis a; r = 0..3 runs over the face's corners, the first of
            // the two other axes (a < b) as bit 0
            const bool e0 = e == 0, e1 = e == 1, e2 = e == 2;
            const float F[4] = {S[0], e0 ? S[2] : S[1], e2 ? S[2] : S[4], e0 ? S[6] : (e1 ? S[5] : S[3])};
            const long long Da = e0 ? Dv[1] : Dv[0], Db = e2 ? Dv[1] : Dv[2];
            const long long P[4] = {P0, P0 + Da, P0 + Db, P0 + Da + Db};
            flush_face(B.grad, P, F, gk, gb, w, sm);
            // the exit face's sums become the entry face's
            const float s1 = S[1], s2 = S[2], s3 = S[3], s4 = S[4], s5 = S[5], s6 = S[6], s7 = S[7];
            S[0] = e0 ? s1 : (e1 ? s2 : s4);
            S[1] = e0 ? 0.f : (e1 ? s3 : s5);
            S[2] = e0 ? s3 : (e1 ? 0.f : s6);
            S[3] = e2 ? s7 : 0.f;
            S[4] = e0 ? s5 : (e1 ? s6 : 0.f);
            S[5] = e1 ? s7 : 0.f;
            S[6] = e0 ? s7 : 0.f;
            S[7] = 0.f;
        } else {
            flush_grad(B.grad, c[0] * sx + c[1] * sy + c[2], S[0], gk, gb, w);
            S[0] = 0.f;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (a == e) {
                c[a] = wrap_once(ncell, nn[a]);
                P0 += Dv[a];
                Dv[a] = (long long)(nvhi - vhi[a]) * st[a];
                vlo[a] = vhi[a];
                vhi[a] = nvhi;
                k[a] += 1;
                T[a] = fma((R)k[a], W.td[a], W.T0[a]);
            }
        // the ray left the box (no wrap): the corners still pending are
        // flushed below
        if (!A.periodic && (ncell < 0 || ncell >= ne)) break;
        if (++iter > W.max_iter) {
            overflow = true;
            break;
        }
    }
    // flush everything still pending
    if (INTERP == RR_TRILINEAR) {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int gx = (m & 1) ? vhi[0] : vlo[0];
            const int gy = (m & 2) ? vhi[1] : vlo[1];
            const int gz = (m & 4) ? vhi[2] : vlo[2];
            flush_grad(B.grad, gx * sx + gy * sy + gz, S[m], gk, gb, w);
        }
    } else {
        flush_grad(B.grad, c[0] * sx + c[1] * sy + c[2], S[0], gk, gb, w);
    }
    }
    if (overflow) atomicOr(A.err, kErrStepLimit);
}

}  // namespace

cudaError_t launch_trace_adjoint(const TraceArgs& a, const AdjArgs& b, int interp, bool fp64_dda, cudaStream_t s)
{
    const TileCfg t{};
    const dim3 grid = tile_grid(t, a.nx, a.ny);
    const int nt = 32 * t.bwx * t.bwy;
    if (nt > 32 * kAdjWarps) return cudaErrorInvalidConfiguration;   // the face-flush staging holds kAdjWarps warps
    if (interp == RR_TRILINEAR) {
        if (fp64_dda)
            trace_adjoint_kernel<RR_TRILINEAR, double><<<grid, nt, 0, s>>>(a, b, t);
        else
            trace_adjoint_kernel<RR_TRILINEAR, float><<<grid, nt, 0, s>>>(a, b, t);
    } else {
        if (fp64_dda)
            trace_adjoint_kernel<RR_NGP, double><<<grid, nt, 0, s>>>(a, b, t);
        else
            trace_adjoint_kernel<RR_NGP, float><<<grid, nt, 0, s>>>(a, b, t);
    }
    return cudaGetLastError();
}

}  // namespace rr
