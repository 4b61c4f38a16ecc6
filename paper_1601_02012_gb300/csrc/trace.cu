// Cell-by-cell line-of-sight integration over one step (Secs. 2.5-2.6, 3.2).
//
// One thread owns one ray; a warp owns an 8 x 4 tile of neighbouring pixels,
// so that its rays sit in the same or adjacent cells at every chi and the
// record gathers of a warp mostly hit the same 128-byte lines (served by L1).
//
// Per ray and step:
//  * Setup: the start point obs + chi_a n (Eq. raypos) and its cell. In the
//    FP32 form this is float-float arithmetic (chi_a, n, obs and 1/h carried
//    as pairs of floats, ~2^-46 relative), because GB300 issues FP64 at a
//    small fraction of the FP32 rate; the plain form uses FP64. The distances
//    from the start point to the cell's two faces on each axis are both
//    obtained with full relative precision.
//  * The walk runs in cell-local "mirrored" coordinates u_a in [0, 1] that
//    grow along the motion (-n). The path to the k-th face crossing on axis a
//    is T0_a + k td_a (one rounding, no drift); the nearest crossing picks the
//    exit face (the exit-plane rule of Sec. 2.5.1, Eq. disttocross), ties go
//    to the lowest axis. The step ends when the path reaches chi_a - chi_b.
//  * Trilinear mode keeps the projected values of the cell's 8 vertices in
//    registers; crossing a face keeps the 4 shared vertices and gathers the 4
//    new ones (2 x 16-byte loads each), issued before the current segment's
//    arithmetic.
//  * Along the segment, chi = chi_A - s for s in [0, t]; the trilinear field
//    restricted to the line is a cubic in s (the d_N of Appendix B, written
//    about the entry point) and the lensing kernel is the quadratic
//    g(chi_A - s); the segment integral (Eq. Iclensing) is the exact
//    sum_N e_N J_N with J_N = int_0^t g(chi_A - s) s^(N-1) ds.
//  * Sums over the segments of a step are compensated FP32 (Kahan); the step
//    total times the step's scale is added to the ray's float-float
//    accumulator (~48 bits).
#include <type_traits>

#include "walk.cuh"

namespace rr {
namespace {

// Crossing face e of the mirrored cell: the 4 corners on the exit side become
// the entry side and the 4 new corner values p come in on the exit side.
// SEL: the same moves as selects on e (no divergent branches), slot by slot
// the value it takes for e = 0, 1, 2. Selects are used everywhere: faster in
// the shear and Method A forms and in the multi-step kernels (2 % on the
// production pass), the same as the branches for one default step per launch.
template <bool SEL = true>
__device__ __forceinline__ void shift_corners(float2 q[8], const float2 p[4], int e)
{
    if constexpr (SEL) {
        const bool e0 = e == 0, e1 = e == 1;
        float2 n[8];
        n[0] = e0 ? q[1] : (e1 ? q[2] : q[4]);
        n[1] = e0 ? p[0] : (e1 ? q[3] : q[5]);
        n[2] = e0 ? q[3] : (e1 ? p[0] : q[6]);
        n[3] = (e0 || e1) ? p[1] : q[7];
        n[4] = e0 ? q[5] : (e1 ? q[6] : p[0]);
        n[5] = e0 ? p[2] : (e1 ? q[7] : p[1]);
        n[6] = e0 ? q[7] : p[2];
        n[7] = p[3];
#pragma unroll
        for (int i = 0; i < 8; ++i) q[i] = n[i];
    } else if (e == 0) {
        q[0] = q[1]; q[2] = q[3]; q[4] = q[5]; q[6] = q[7];
        q[1] = p[0]; q[3] = p[1]; q[5] = p[2]; q[7] = p[3];
    } else if (e == 1) {
        q[0] = q[2]; q[1] = q[3]; q[4] = q[6]; q[5] = q[7];
        q[2] = p[0]; q[3] = p[1]; q[6] = p[2]; q[7] = p[3];
    } else {
        q[0] = q[4]; q[1] = q[5]; q[2] = q[6]; q[3] = q[7];
        q[4] = p[0]; q[5] = p[1]; q[6] = p[2]; q[7] = p[3];
    }
}

// One ray over one step. INTERP: RR_NGP or RR_TRILINEAR. R: float
// (compensated FP32 walk) or double (plain FP64 walk). FORM (FP32 only):
// kFormKahan (default), kFormPlain (uncompensated FP32 sums within and across
// steps, for comparison), kFormMoments (the moments A = int chi Q and
// B = int chi^2 Q of Eq. Isources instead of kappa: the kernel g becomes chi
// and chi^2, i.e. (G0, G1, G2) = (chi_A, -1, 0) and (chi_A^2, -2 chi_A, 1)) or
// kFormShear (kappa and Born kappa, and the shear pair (gamma1, gamma2) of Eqs.
// gamma1, gamma2 from a second projection of the same records, carried as a
// second packed pair through the same segments) or kFormMethodA (Method A,
// Eq. kappa2, on gradient records {grad Phi, delta}: the first channel
// integrates n . grad Phi with the kernel dg/dchi and adds the step's surface
// terms -g n.grad Phi at the start and +g n.grad Phi at the end of the traced
// interval (Eq. 2nterm); the second is the Born term as in the other forms) or
// kFormGeneric (two scalar fields from float2 records, each with its own
// quadratic kernel K(chi): the generic integrals of Eqs. Ic, Icfinal).
// ADDR: how the trilinear walk addresses its records.
//  kAddrIndex:  vertex indices per axis, with periodic wrap (any grid).
//  kAddrPlanes: the 64-bit record offsets of the mirrored cell's two vertex
//               planes per axis (entry and exit side), with wrap, so that a
//               record's offset is two additions (6.5 % faster than indices
//               on the production workload). The persistent batch kernel,
//               which also holds its staged arguments, and the forms with
//               more per-segment state (moments, shear, Method A, generic)
//               measured 1.5-4 % slower with them and keep indices.
//  kAddrFlat:   no wrap: a 32-bit point index B of the mirrored cell's entry
//               corner and a constant signed stride d_a per axis (the next
//               vertex plane along the motion), so the 8 corners are B plus
//               sums of the d_a and a crossing of face e is B += d_e. Valid
//               when no ray of the step comes within a cell of the periodic
//               seam and the grid has fewer than 2^31 points: the host checks
//               the step's footprint box; each sub-step checks its own cell
//               range first and, outside it, flags kErrRange and reads nothing.
template <int INTERP, class R, int FORM = kFormKahan, int ADDR = kAddrPlanes, bool REGACC = false>
__device__ __forceinline__ void trace_ray(const TraceArgs& A, int ix, int iy, RayAcc* acc = nullptr)
{
    static_assert(!REGACC || (FORM != kFormPlain && sizeof(R) == 4), "register accumulators: FP32 compensated forms");
    using OT = unsigned long long;
    constexpr bool PLANES = ADDR == kAddrPlanes;
    constexpr bool FLAT = ADDR == kAddrFlat;
    static_assert(!FLAT || (INTERP == RR_TRILINEAR && sizeof(R) == 4), "flat addressing: FP32 trilinear walk");
    constexpr bool F64 = sizeof(R) == 8;
    constexpr bool SH = !F64 && FORM == kFormShear;
    constexpr bool MA = !F64 && FORM == kFormMethodA;
    constexpr bool GEN = !F64 && FORM == kFormGeneric;
    // one record per point: 2 float4 of the tidal tensor, 1 gradient float4
    // (Method A) or a float2 scalar pair (generic form)
    using PR = typename std::conditional<MA, float4, typename std::conditional<GEN, float2, Rec>::type>::type;
    const long long rid = (long long)iy * A.nx + ix;
    const int nn[3] = {A.n0, A.n1, A.n2};
    RayRange rg;
    if (!ray_range(A, rid, rg)) return;
    if (!REGACC || !acc->loaded) {
        prefetch_l2(A.kacc + rid);
        prefetch_l2(A.bacc + rid);
        prefetch_l2(A.nseg + rid);
        if constexpr (SH) {
            prefetch_l2(A.g1acc + rid);
            prefetch_l2(A.g2acc + rid);
        }
    }
    const R chis = (R)A.chi_s;
    const R ichis = F64 ? (R)(1.0 / A.chi_s) : (R)A.inv_chi_s_f;
    const long long sx = (long long)A.n1 * A.n2, sy = A.n2;
    // FP32: sub-steps of at most sub_len, so that the path variable stays small
    const int nsub = F64 ? 1 : max(1, (int)ceilf(rg.Lf / A.sub_len));
    const float dsub = rg.Lf / (float)nsub;

    // per-step sums of (kappa, Born kappa): packed Kahan pairs (FP32) or FP64
    Acc2 s2;
    Acc2 s2m;   // moments form: the B moments; shear form: (gamma1, gamma2)
    float w1[6], w2[6];   // shear form: the Q weights of gamma1, gamma2
    if constexpr (SH) shear_weights(A.dirh[rid], w1, w2);
    float4 nd;            // Method A: the direction, for n . grad Phi
    if constexpr (MA) nd = A.dirh[rid];
    // Method A: n . grad Phi and g at the start and at the end of the interval
    float qa = 0.f, ga = 0.f, qb = 0.f, gb = 0.f;
    Acc<R> sk, sb;
    uint32_t cnt = 0;
    int iter = 0;
    bool overflow = false;
    int pc0 = -1, pc1 = -1, pc2 = -1;   // cell where the previous sub-step ended
    int pB = -1;                        // FLAT: entry corner where the previous sub-step ended
    for (int j = 0; j < nsub && !overflow; ++j) {
    float bh, bl, Lj, D0j;
    sub_step(rg, j, nsub, dsub, bh, bl, Lj, D0j);
    Walk<R> W;
    walk_setup<R>(A, rid, bh, bl, Lj, D0j, rg.hi, rg.lo, W);
    int* c = W.c;
    const int* sgn = W.sgn;
    int* k = W.k;
    // offsets of the entry-side (plo) and exit-side (phi) vertex planes per
    // axis (PLANES), or the vertex indices themselves
    const OT st[3] = {(OT)A.n1 * (OT)A.n2, (OT)A.n2, (OT)1};
    OT plo[3], phi[3];
    int* vlo = W.vlo;
    int* vhi = W.vhi;
    if constexpr (PLANES) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            plo[a] = (OT)vlo[a] * st[a];
            phi[a] = (OT)vhi[a] * st[a];
        }
    }
    const R* T0 = W.T0;
    const R* td = W.td;
    const R* v = W.v;
    const R* cu = W.cu;
    const float* w = W.w;
    const R L = W.L, chiA0 = W.chiA0, D0 = W.D0;
    const int max_iter = W.max_iter;
    // FLAT: entry corner B, strides d, crossing counts as floats
    int fB = 0, fd[3] = {0, 0, 0};
    float kf[3] = {0.f, 0.f, 0.f};
    if constexpr (FLAT) {
        bool inside = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            // box-local vertex and cell coordinates (the records' box starts
            // at fo, periodically)
            const int sa = a == 0 ? A.fs0 : (a == 1 ? A.fs1 : 1);
            int vl = vlo[a] - A.fo[a];
            if (vl < 0) vl += nn[a];
            int cl = c[a] - A.fo[a];
            if (cl < 0) cl += nn[a];
            fB += vl * sa;
            fd[a] = sgn[a] * sa;
            // crossings this sub-step can make on axis a (2 more than the path
            // allows, for rounding); cells c .. c + sgn K, vertex planes one further
            int K = 0;
            if (T0[a] < L) {
                const float x = (L - T0[a]) * v[a];
                if (x < 4194304.f) K = f2i_exact(x) + 2;
                else inside = false;
            }
            const int lo = sgn[a] > 0 ? cl : cl - K, hi = sgn[a] > 0 ? cl + K + 1 : cl + 1;
            if (lo < 0 || hi > A.fe[a] - 1) inside = false;
        }
        if (!inside) {
            atomicOr(A.err, kErrRange);
            break;
        }
    }
    auto fetch = [&](long long i) -> PR {
        if constexpr (MA) return load_grad_rec(A.rec, i);
        else if constexpr (GEN) return __ldg(reinterpret_cast<const float2*>(A.rec) + i);
        else if constexpr (FLAT) return load_rec32(A.rec, i);
        else return load_rec(A.rec, i);
    };
    // (the channel pair the walk integrates) of a record
    auto pair = [&](const PR& r) -> float2 {
        if constexpr (MA) return radial_pair(nd, r);
        else if constexpr (GEN) return r;
        else return make_float2(project(w, r), r.b.z);
    };
    // a sub-step that resumes inside the previous one's last cell does not
    // start a new cell segment
    bool resume;
    if constexpr (FLAT) resume = j > 0 && fB == pB;
    else resume = j > 0 && c[0] == pc0 && c[1] == pc1 && c[2] == pc2;
    iter = 0;

    // Field cache: (projected kappa value, delta) at the 8 mirrored corners
    // (trilinear) or at the cell centre (NGP); the shear form also keeps
    // (gamma1, gamma2) values there.
    float2 q2[8];
    float2 g2[SH ? 8 : 1];
    if (INTERP == RR_TRILINEAR) {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            long long o;
            if constexpr (FLAT) {
                o = (unsigned)(fB + ((m & 1) ? fd[0] : 0) + ((m & 2) ? fd[1] : 0) + ((m & 4) ? fd[2] : 0));
            } else if constexpr (PLANES) {
                o = (long long)(((m & 1) ? phi[0] : plo[0]) + ((m & 2) ? phi[1] : plo[1]) +
                                ((m & 4) ? phi[2] : plo[2]));
            } else {
                const int gx = (m & 1) ? vhi[0] : vlo[0];
                const int gy = (m & 2) ? vhi[1] : vlo[1];
                const int gz = (m & 4) ? vhi[2] : vlo[2];
                o = gx * sx + gy * sy + gz;
            }
            const PR r = fetch(o);
            q2[m] = pair(r);
            if constexpr (SH) g2[m] = make_float2(project(w1, r), project(w2, r));
        }
    } else {
        const PR r = fetch(c[0] * sx + c[1] * sy + c[2]);
        q2[0] = pair(r);
        if constexpr (SH) g2[0] = make_float2(project(w1, r), project(w2, r));
    }

    R sig = 0;                       // path from the sub-step start to the segment entry
    R T[3] = {T0[0], T0[1], T0[2]};  // path to the next face crossing per axis
    // Crossings closer together than the walk resolves are one crossing: a
    // crossing within eps_rel * L of the step's end, and a segment shorter
    // than eps_rel * (its end), are rounding slivers at an edge or corner the
    // ray passes through; they are neither integrated nor counted. FP32: 4 ulp
    // of the path. FP64: 2^-36, above the error the FP64 start point carries
    // into a crossing distance (ulp(|p|) / |n_a|) for rays 1e-4 rad off an axis.
    const R eps_rel = F64 ? (R)1.4551915228366852e-11 : (R)4.76837158203125e-07;
    const R eps_end = L * eps_rel;
    while (true) {
        // exit plane: the nearest face crossing (lowest axis on ties)
        R tend = T[0];
        int e = 0;
        if (T[1] < tend) { tend = T[1]; e = 1; }
        if (T[2] < tend) { tend = T[2]; e = 2; }
        const bool last = !(tend < L - eps_end);
        if (last) tend = L;
        const R t = tend - sig;
        // mirrored entry point of this segment
        R u[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if constexpr (FLAT) u[a] = __saturatef(fmaf(sig - T[a], v[a], cu[a]));
            else u[a] = fmin(fmax(fma(sig - T[a], v[a], cu[a]), (R)0), (R)1);
        }

        // Prefetch the next cell's new records before this segment's arithmetic.
        // (register arrays are indexed only through unrolled loops, never by e)
        int ncell = 0, ne = 1;
        OT nph = 0;     // offset of the vertex plane beyond the exit face (PLANES)
        int nvhi = 0;   // its vertex index (otherwise)
        PR nr[4];
        // FLAT: the stride along the exit axis
        const int fde = e == 0 ? fd[0] : (e == 1 ? fd[1] : fd[2]);
        if (FLAT && !last) {
            // the new exit-side corners: B + 2 d_e plus 0, d_A, d_B, d_A + d_B
            // over the other two axes A < B
            const int P = fB + 2 * fde;
            const int dA = e == 0 ? fd[1] : fd[0];
            const int dB = e == 2 ? fd[1] : fd[2];
            nr[0] = fetch((unsigned)P);
            nr[1] = fetch((unsigned)(P + dA));
            nr[2] = fetch((unsigned)(P + dB));
            nr[3] = fetch((unsigned)(P + dA + dB));
        } else if (!last) {
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if (a == e) {
                    ncell = c[a] + sgn[a];
                    ne = nn[a];
                    // the exit-side plane one vertex further along the motion, with wrap
                    if constexpr (PLANES) {
                        const OT span = st[a] * (OT)nn[a];
                        if (sgn[a] > 0) nph = phi[a] + st[a] == span ? (OT)0 : phi[a] + st[a];
                        else nph = phi[a] == 0 ? span - st[a] : phi[a] - st[a];
                    } else {
                        nvhi = wrap_once(vhi[a] + sgn[a], nn[a]);
                    }
                }
            if (INTERP == RR_TRILINEAR) {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int pb = r & 1, qb2 = r >> 1;
                    if constexpr (PLANES) {
                        const OT ox = e == 0 ? nph : (pb ? phi[0] : plo[0]);
                        const OT oy = e == 1 ? nph : (e == 0 ? (pb ? phi[1] : plo[1]) : (qb2 ? phi[1] : plo[1]));
                        const OT oz = e == 2 ? nph : (qb2 ? phi[2] : plo[2]);
                        nr[r] = fetch((long long)(ox + oy + oz));
                    } else {
                        const int gx = e == 0 ? nvhi : (pb ? vhi[0] : vlo[0]);
                        const int gy = e == 1 ? nvhi : (e == 0 ? (pb ? vhi[1] : vlo[1]) : (qb2 ? vhi[1] : vlo[1]));
                        const int gz = e == 2 ? nvhi : (qb2 ? vhi[2] : vlo[2]);
                        nr[r] = fetch(gx * sx + gy * sy + gz);
                    }
                }
            } else {
                const int cx = e == 0 ? wrap_once(ncell, nn[0]) : c[0];
                const int cy = e == 1 ? wrap_once(ncell, nn[1]) : c[1];
                const int cz = e == 2 ? wrap_once(ncell, nn[2]) : c[2];
                nr[0] = fetch(cx * sx + cy * sy + cz);
            }
        }
        if constexpr (MA) {
            // the surface terms of Eq. (2nterm): n . grad Phi and g at the start
            // of the traced interval (the first segment's entry) and at its end
            // (the exit of the segment that ends the interval: the last one,
            // or, without wrap, the one leaving the box)
            if (j == 0 && iter == 0) {
                qa = INTERP == RR_TRILINEAR ? trilinear_x(q2, u[0], u[1], u[2]) : q2[0].x;
                ga = D0 * chiA0 * ichis;
            }
            if (last || (!A.periodic && (ncell < 0 || ncell >= ne))) {
                if (INTERP == RR_TRILINEAR) {
                    float ue[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) ue[a] = fminf(fmaxf(fmaf(t, v[a], u[a]), 0.f), 1.f);
                    qb = trilinear_x(q2, ue[0], ue[1], ue[2]);
                } else {
                    qb = q2[0].x;
                }
                float G0, G1, G2;
                kernel_coeffs(t, sig, chiA0, D0, chis, ichis, G0, G1, G2);
                gb = fmaf(t, fmaf(t, G2, G1), G0);
            }
        }

        if (t > tend * eps_rel) {
            if constexpr (!F64 && FORM == kFormMoments) {
                const float chiA = chiA0 - sig;
                if (INTERP == RR_TRILINEAR) {
                    float2 e2[4];
                    line_cubic2(q2, bc2(u[0]), bc2(u[1]), bc2(u[2]), bc2(v[0]), bc2(v[1]), bc2(v[2]), e2);
                    s2.add(dot_kernel(e2, t, chiA, -1.f, 0.f));
                    s2m.add(dot_kernel(e2, t, chiA * chiA, -2.f * chiA, 1.f));
                } else {
                    s2.add(segment_ngp(q2[0], t, chiA, -1.f, 0.f));
                    s2m.add(segment_ngp(q2[0], t, chiA * chiA, -2.f * chiA, 1.f));
                }
            } else if constexpr (GEN) {
                // each channel's kernel about the entry point: K(chi_A - s) =
                // K(chi_A) - K'(chi_A) s + k2 s^2
                const float chiA = chiA0 - sig;
                const float2 G0 = make_float2(fmaf(chiA, fmaf(chiA, A.kq[2], A.kq[1]), A.kq[0]),
                                              fmaf(chiA, fmaf(chiA, A.kq[5], A.kq[4]), A.kq[3]));
                const float2 G1 = make_float2(-fmaf(2.f * A.kq[2], chiA, A.kq[1]), -fmaf(2.f * A.kq[5], chiA, A.kq[4]));
                const float2 G2 = make_float2(A.kq[2], A.kq[5]);
                if (INTERP == RR_TRILINEAR) {
                    float2 e2[4];
                    line_cubic2(q2, bc2(u[0]), bc2(u[1]), bc2(u[2]), bc2(v[0]), bc2(v[1]), bc2(v[2]), e2);
                    s2.add(dot_kernel_pair(e2, t, G0, G1, G2));
                } else {
                    const float2 tt = bc2(t);
                    const float2 J1 = __fmul2_rn(tt, __ffma2_rn(tt, __ffma2_rn(tt, __fmul2_rn(G2, bc2(1.f / 3.f)),
                                                                              __fmul2_rn(G1, bc2(0.5f))), G0));
                    s2.add(__fmul2_rn(q2[0], J1));
                }
            } else if constexpr (MA) {
                float G0, G1, G2;
                kernel_coeffs(t, sig, chiA0, D0, chis, ichis, G0, G1, G2);
                s2.add(INTERP == RR_TRILINEAR
                           ? segment_trilinear_a(q2, u[0], u[1], u[2], v[0], v[1], v[2], t, G0, G1, G2)
                           : segment_ngp_a(q2[0], t, G0, G1, G2));
            } else if constexpr (!F64) {
                float G0, G1, G2;
                kernel_coeffs(t, sig, chiA0, D0, chis, ichis, G0, G1, G2);
                const float2 x = INTERP == RR_TRILINEAR
                                     ? segment_trilinear(q2, u[0], u[1], u[2], v[0], v[1], v[2], t, G0, G1, G2)
                                     : segment_ngp(q2[0], t, G0, G1, G2);
                if constexpr (FORM == kFormPlain) s2.s = __fadd2_rn(s2.s, x);
                else s2.add(x);
                if constexpr (SH)
                    s2m.add(INTERP == RR_TRILINEAR
                                ? segment_trilinear(g2, u[0], u[1], u[2], v[0], v[1], v[2], t, G0, G1, G2)
                                : segment_ngp(g2[0], t, G0, G1, G2));
            } else {
                // lensing kernel g(chi_A - s) = G0 + G1 s + G2 s^2 about the entry
                // point; J_N and the sums rounded as written (the single-launch and
                // the batch kernels must give the same values)
                const double chiA = chiA0 - sig;
                const double G0 = (D0 + sig) * chiA * ichis;
                const double G1 = __dmul_rn(__fma_rn(2.0, chiA, -(double)chis), ichis);
                const double G2 = -ichis;
                const double t2 = __dmul_rn(t, t);
                const double tn[4] = {t, t2, __dmul_rn(t2, t), __dmul_rn(t2, t2)};
                const double ca[4] = {1.0, 0.5, 1.0 / 3.0, 0.25};
                const double cb[4] = {0.5, 1.0 / 3.0, 0.25, 0.2};
                const double cc[4] = {1.0 / 3.0, 0.25, 0.2, 1.0 / 6.0};
                double J[4];
#pragma unroll
                for (int n = 0; n < 4; ++n)
                    J[n] = __dmul_rn(tn[n], __fma_rn(t, __fma_rn(t, __dmul_rn(G2, cc[n]), __dmul_rn(G1, cb[n])),
                                                   __dmul_rn(G0, ca[n])));
                if (INTERP == RR_TRILINEAR) {
                    float2 e2[4];
                    line_cubic2(q2, bc2((float)u[0]), bc2((float)u[1]), bc2((float)u[2]), bc2((float)v[0]),
                                bc2((float)v[1]), bc2((float)v[2]), e2);
                    double xk = __dmul_rn((double)e2[0].x, J[0]), xb = __dmul_rn((double)e2[0].y, J[0]);
#pragma unroll
                    for (int n = 1; n < 4; ++n) {
                        xk = __fma_rn((double)e2[n].x, J[n], xk);
                        xb = __fma_rn((double)e2[n].y, J[n], xb);
                    }
                    sk.add((R)xk);
                    sb.add((R)xb);
                } else {
                    sk.add((R)__dmul_rn((double)q2[0].x, J[0]));
                    sb.add((R)__dmul_rn((double)q2[0].y, J[0]));
                }
            }
            if (resume) resume = false;
            else ++cnt;
        }
        sig = tend;
        if (last) break;

        // cross the exit face e
        resume = false;
        if constexpr (FLAT) {
            fB += fde;
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if (a == e) {
                    kf[a] += 1.f;
                    T[a] = fmaf(kf[a], td[a], T0[a]);
                }
        } else {
        if (!A.periodic && (ncell < 0 || ncell >= ne)) break;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (a == e) {
                c[a] = wrap_once(ncell, nn[a]);
                if constexpr (PLANES) {
                    plo[a] = phi[a];
                    phi[a] = nph;
                } else {
                    vlo[a] = vhi[a];
                    vhi[a] = nvhi;
                }
                k[a] += 1;
                if constexpr (F64) T[a] = fma((R)k[a], td[a], T0[a]);
                else T[a] = fmaf(i2f_exact(k[a]), td[a], T0[a]);
            }
        }
        if (INTERP == RR_TRILINEAR) {
            float2 p2[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) p2[r] = pair(nr[r]);
            shift_corners(q2, p2, e);
            if constexpr (SH) {
#pragma unroll
                for (int r = 0; r < 4; ++r) p2[r] = make_float2(project(w1, nr[r]), project(w2, nr[r]));
                shift_corners<true>(g2, p2, e);
            }
        } else {
            q2[0] = pair(nr[0]);
            if constexpr (SH) g2[0] = make_float2(project(w1, nr[0]), project(w2, nr[0]));
        }
        if (++iter > max_iter) {
            overflow = true;
            break;
        }
    }
    pc0 = c[0]; pc1 = c[1]; pc2 = c[2];
    pB = fB;
    }

    if constexpr (MA) {
        s2.add(make_float2(-ga * qa, 0.f));
        s2.add(make_float2(gb * qb, 0.f));
    }
    if constexpr (!F64) {
        sk.s = s2.s.x; sk.c = s2.c.x;
        sb.s = s2.s.y; sb.c = s2.c.y;
    }
    if (overflow) atomicOr(A.err, kErrStepLimit);
    if (!sk.finite() || !sb.finite()) atomicOr(A.err, kErrNonFinite);
    if constexpr (REGACC) {
        // the first step of the launch: the ray's state from memory
        if (!acc->loaded) {
            acc->k = A.kacc[rid];
            acc->b = A.bacc[rid];
            acc->n = A.nseg[rid];
            if constexpr (SH) {
                acc->x1 = A.g1acc[rid];
                acc->x2 = A.g2acc[rid];
            }
            if constexpr (FORM == kFormMoments) {
                acc->x1 = A.kmom[rid];
                acc->x2 = A.bmom[rid];
            }
            acc->loaded = true;
        }
    }
    if constexpr (SH) {
        float gh, gl;
        if (!s2m.finite()) atomicOr(A.err, kErrNonFinite);
        two_sum(s2m.s.x, -s2m.c.x, gh, gl);
        if constexpr (REGACC) acc->x1 = ff_mul_add(acc->x1, gh, gl, A.sch, A.scl);
        else A.g1acc[rid] = ff_mul_add(A.g1acc[rid], gh, gl, A.sch, A.scl);
        two_sum(s2m.s.y, -s2m.c.y, gh, gl);
        if constexpr (REGACC) acc->x2 = ff_mul_add(acc->x2, gh, gl, A.sch, A.scl);
        else A.g2acc[rid] = ff_mul_add(A.g2acc[rid], gh, gl, A.sch, A.scl);
    }
    if constexpr (FORM == kFormMoments) {
        float mh, ml;
        if (!s2m.finite()) atomicOr(A.err, kErrNonFinite);
        two_sum(s2m.s.x, -s2m.c.x, mh, ml);
        if constexpr (REGACC) acc->x1 = ff_mul_add(acc->x1, mh, ml, A.sch, A.scl);
        else A.kmom[rid] = ff_mul_add(A.kmom[rid], mh, ml, A.sch, A.scl);
        two_sum(s2m.s.y, -s2m.c.y, mh, ml);
        if constexpr (REGACC) acc->x2 = ff_mul_add(acc->x2, mh, ml, A.bsh, A.bsl);
        else A.bmom[rid] = ff_mul_add(A.bmom[rid], mh, ml, A.bsh, A.bsl);
    }
    if constexpr (FORM == kFormPlain) {
        // plain FP32 across steps too: the high word only
        A.kacc[rid] = make_float2(fmaf(sk.s, A.sch, A.kacc[rid].x), 0.f);
        A.bacc[rid] = make_float2(fmaf(sb.s, A.bsh, A.bacc[rid].x), 0.f);
        A.nseg[rid] += cnt;
        return;
    }
    float kh, kl, bh, bl;
    sk.pair(kh, kl);
    sb.pair(bh, bl);
    if constexpr (REGACC) {
        acc->k = ff_mul_add(acc->k, kh, kl, A.sch, A.scl);
        acc->b = ff_mul_add(acc->b, bh, bl, A.bsh, A.bsl);
        acc->n += cnt;
        return;
    }
    A.kacc[rid] = ff_mul_add(A.kacc[rid], kh, kl, A.sch, A.scl);
    A.bacc[rid] = ff_mul_add(A.bacc[rid], bh, bl, A.bsh, A.bsl);
    A.nseg[rid] += cnt;
}


template <int INTERP, class R, int FORM = kFormKahan, int ADDR = (FORM == kFormKahan ? kAddrPlanes : kAddrIndex)>
__global__ void __launch_bounds__(NT_MAX, 2) trace_kernel(const TraceArgs A, const TileCfg t)
{
    prefetch_ahead(A, t);
    int ix, iy;
    tile_ray(t, blockIdx.x, blockIdx.y, ix, iy);
    if (ix < A.nx && iy < A.ny) trace_ray<INTERP, R, FORM, ADDR>(A, ix, iy);
}

// Consecutive steps of one bundle in one launch (the default FP32 form): each
// thread walks its ray through the steps in order, every step reading its own
// records with its own interval and scales, the ray's accumulators kept in
// registers in between. Per step the arithmetic is that of trace_kernel, so
// the result equals one trace_kernel launch per step bit for bit; what goes
// is the per-launch and per-step traffic of the ray state (directions,
// accumulators) and all launches but one.
template <int INTERP, int ADDR, int FORM>
__global__ void __launch_bounds__(NT_MAX, 2)
    trace_steps_kernel(const TraceArgs A, const __grid_constant__ StepBlock S, const TileCfg t)
{
    prefetch_ahead(A, t);
    int ix, iy;
    tile_ray(t, blockIdx.x, blockIdx.y, ix, iy);
    if (ix >= A.nx || iy >= A.ny) return;
    RayAcc acc;
    acc.loaded = false;
    for (int g = 0; g < S.n; ++g) {
        const StepArgs& st = S.s[g];
        TraceArgs As = A;
        As.rec = st.rec;
        As.chi_a = st.chi_a; As.chi_b = st.chi_b;
        As.cah = st.cah; As.cal = st.cal;
        As.Lf = st.Lf; As.D0f = st.D0f;
        As.sch = st.sch; As.scl = st.scl;
        As.bsh = st.bsh; As.bsl = st.bsl;
        As.fo[0] = st.fo[0]; As.fo[1] = st.fo[1]; As.fo[2] = st.fo[2];
        As.fe[0] = st.fe[0]; As.fe[1] = st.fe[1]; As.fe[2] = st.fe[2];
        As.fs0 = st.fs0; As.fs1 = st.fs1;
        trace_ray<INTERP, float, FORM, ADDR, true>(As, ix, iy, &acc);
    }
    if (acc.loaded) {
        const long long rid = (long long)iy * A.nx + ix;
        A.kacc[rid] = acc.k;
        A.bacc[rid] = acc.b;
        A.nseg[rid] = acc.n;
        if constexpr (FORM == kFormShear) {
            A.g1acc[rid] = acc.x1;
            A.g2acc[rid] = acc.x2;
        }
        if constexpr (FORM == kFormMoments) {
            A.kmom[rid] = acc.x1;
            A.bmom[rid] = acc.x2;
        }
    }
}

// Persistent work queue over the ray tiles of many bundles (lightcones): each
// block takes `chunk` consecutive tiles from a global counter (monotonic, no
// waiting), finds the bundle by binary search in the tile offsets, stages that
// bundle's arguments in shared memory and traces the tile.
template <int INTERP, class R>
__global__ void __launch_bounds__(NT_MAX, 2) trace_batch_kernel(const BatchArgs B)
{
    __shared__ TraceArgs sA;
    __shared__ int s_item, s_cone;
    const int total = B.tile_start[B.ncones];
    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(B.counter, B.chunk);
        __syncthreads();
        const int item0 = s_item;
        __syncthreads();
        if (item0 >= total) break;
        for (int c = 0; c < B.chunk; ++c) {
            const int item = item0 + c;
            if (item >= total) break;
            if (threadIdx.x == 0) {
                int lo = 0, hi = B.ncones - 1;   // last cone with tile_start <= item
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (B.tile_start[mid] <= item) lo = mid;
                    else hi = mid - 1;
                }
                s_cone = lo;
            }
            __syncthreads();
            const int cone = s_cone;
            {
                const int* src = reinterpret_cast<const int*>(B.cones + cone);
                int* dst = reinterpret_cast<int*>(&sA);
                for (int i = threadIdx.x; i < (int)(sizeof(TraceArgs) / sizeof(int)); i += blockDim.x)
                    dst[i] = __ldg(src + i);
            }
            __syncthreads();
            const int local = item - B.tile_start[cone];
            const int ntx = B.tiles_x[cone];
            int ix, iy;
            tile_ray(B.tile, local % ntx, local / ntx, ix, iy);
            if (ix < sA.nx && iy < sA.ny) trace_ray<INTERP, R, kFormKahan, kAddrIndex>(sA, ix, iy);
            __syncthreads();
        }
    }
}

}  // namespace

dim3 tile_grid(const TileCfg& t, int nx, int ny)
{
    const int bx = t.wx * t.bwx, by = (32 / t.wx) * t.bwy;
    return dim3((unsigned)((nx + bx - 1) / bx), (unsigned)((ny + by - 1) / by));
}

bool tile_ok(const TileCfg& t)
{
    return (t.wx == 1 || t.wx == 2 || t.wx == 4 || t.wx == 8 || t.wx == 16 || t.wx == 32) && t.bwx >= 1 &&
           t.bwy >= 1 && t.bwx * t.bwy * 32 <= NT_MAX;
}

namespace {

template <int INTERP, class R, int FORM>
cudaError_t launch_one(const TraceArgs& a, const dim3& grid, int nt, cudaStream_t s, const TileCfg& t)
{
    trace_kernel<INTERP, R, FORM><<<grid, nt, 0, s>>>(a, t);
    return cudaGetLastError();
}

template <int FORM>
cudaError_t launch_form(const TraceArgs& a, int interp, const dim3& grid, int nt, cudaStream_t s, const TileCfg& t)
{
    return interp == RR_TRILINEAR ? launch_one<RR_TRILINEAR, float, FORM>(a, grid, nt, s, t)
                                  : launch_one<RR_NGP, float, FORM>(a, grid, nt, s, t);
}

}  // namespace

cudaError_t launch_trace(const TraceArgs& a, int interp, bool fp64_dda, cudaStream_t s, const TileCfg& t,
                         int form, bool flat)
{
    if (!tile_ok(t)) return cudaErrorInvalidValue;
    const dim3 grid = tile_grid(t, a.nx, a.ny);
    const int nt = 32 * t.bwx * t.bwy;
    if (flat && !fp64_dda && interp == RR_TRILINEAR && a.periodic) {
        switch (form) {
        case kFormPlain: trace_kernel<RR_TRILINEAR, float, kFormPlain, kAddrFlat><<<grid, nt, 0, s>>>(a, t); break;
        case kFormMoments: trace_kernel<RR_TRILINEAR, float, kFormMoments, kAddrFlat><<<grid, nt, 0, s>>>(a, t); break;
        case kFormGeneric: trace_kernel<RR_TRILINEAR, float, kFormGeneric, kAddrFlat><<<grid, nt, 0, s>>>(a, t); break;
        case kFormMethodA: trace_kernel<RR_TRILINEAR, float, kFormMethodA, kAddrFlat><<<grid, nt, 0, s>>>(a, t); break;
        case kFormShear: trace_kernel<RR_TRILINEAR, float, kFormShear, kAddrFlat><<<grid, nt, 0, s>>>(a, t); break;
        default: trace_kernel<RR_TRILINEAR, float, kFormKahan, kAddrFlat><<<grid, nt, 0, s>>>(a, t); break;
        }
        return cudaGetLastError();
    }
    if (fp64_dda)
        return interp == RR_TRILINEAR ? launch_one<RR_TRILINEAR, double, kFormKahan>(a, grid, nt, s, t)
                                      : launch_one<RR_NGP, double, kFormKahan>(a, grid, nt, s, t);
    switch (form) {
    case kFormPlain: return launch_form<kFormPlain>(a, interp, grid, nt, s, t);
    case kFormMoments: return launch_form<kFormMoments>(a, interp, grid, nt, s, t);
    case kFormGeneric: return launch_form<kFormGeneric>(a, interp, grid, nt, s, t);
    case kFormMethodA: return launch_form<kFormMethodA>(a, interp, grid, nt, s, t);
    // (the shear form's 128-register cap of two resident blocks spills a few
    // bytes; 168 registers without spills measured 2 % slower)
    case kFormShear: return launch_form<kFormShear>(a, interp, grid, nt, s, t);
    default: return launch_form<kFormKahan>(a, interp, grid, nt, s, t);
    }
}

template <int FORM>
static void launch_steps_form(const TraceArgs& a, const StepBlock& b, int interp, bool flat, dim3 grid, int nt,
                              const TileCfg& t, cudaStream_t s)
{
    // the addressing of each form's single-step kernel: flat for trilinear
    // steps clear of the seam (or box-local records); otherwise vertex-plane
    // offsets for the default form and vertex indices for the others
    constexpr int ADDR = FORM == kFormKahan ? kAddrPlanes : kAddrIndex;
    if (interp == RR_TRILINEAR) {
        if (flat && a.periodic) trace_steps_kernel<RR_TRILINEAR, kAddrFlat, FORM><<<grid, nt, 0, s>>>(a, b, t);
        else trace_steps_kernel<RR_TRILINEAR, ADDR, FORM><<<grid, nt, 0, s>>>(a, b, t);
    } else {
        trace_steps_kernel<RR_NGP, ADDR, FORM><<<grid, nt, 0, s>>>(a, b, t);
    }
}

cudaError_t launch_trace_steps(const TraceArgs& a, const StepBlock& b, int interp, bool flat, cudaStream_t s,
                               int form)
{
    const TileCfg t{};
    if (b.n < 1 || b.n > kMaxStepBlock) return cudaErrorInvalidValue;
    const dim3 grid = tile_grid(t, a.nx, a.ny);
    const int nt = 32 * t.bwx * t.bwy;
    switch (form) {
    case kFormKahan: launch_steps_form<kFormKahan>(a, b, interp, flat, grid, nt, t, s); break;
    case kFormShear: launch_steps_form<kFormShear>(a, b, interp, flat, grid, nt, t, s); break;
    case kFormMoments: launch_steps_form<kFormMoments>(a, b, interp, flat, grid, nt, t, s); break;
    case kFormMethodA: launch_steps_form<kFormMethodA>(a, b, interp, flat, grid, nt, t, s); break;
    case kFormGeneric: launch_steps_form<kFormGeneric>(a, b, interp, flat, grid, nt, t, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_trace(const TraceArgs& a, int interp, bool fp64_dda, cudaStream_t s)
{
    return launch_trace(a, interp, fp64_dda, s, TileCfg{});
}

cudaError_t launch_trace_batch(const BatchArgs& b, int interp, bool fp64_dda, int blocks, cudaStream_t s)
{
    if (!tile_ok(b.tile) || b.chunk < 1 || blocks < 1) return cudaErrorInvalidValue;
    const int nt = 32 * b.tile.bwx * b.tile.bwy;
    if (interp == RR_TRILINEAR) {
        if (fp64_dda)
            trace_batch_kernel<RR_TRILINEAR, double><<<blocks, nt, 0, s>>>(b);
        else
            trace_batch_kernel<RR_TRILINEAR, float><<<blocks, nt, 0, s>>>(b);
    } else {
        if (fp64_dda)
            trace_batch_kernel<RR_NGP, double><<<blocks, nt, 0, s>>>(b);
        else
            trace_batch_kernel<RR_NGP, float><<<blocks, nt, 0, s>>>(b);
    }
    return cudaGetLastError();
}

int batch_blocks_per_sm(int interp, bool fp64_dda, const TileCfg& t)
{
    const int nt = 32 * t.bwx * t.bwy;
    int n = 0;
    cudaError_t e;
    if (interp == RR_TRILINEAR)
        e = fp64_dda ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, trace_batch_kernel<RR_TRILINEAR, double>, nt, 0)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, trace_batch_kernel<RR_TRILINEAR, float>, nt, 0);
    else
        e = fp64_dda ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, trace_batch_kernel<RR_NGP, double>, nt, 0)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, trace_batch_kernel<RR_NGP, float>, nt, 0);
    return (e == cudaSuccess && n > 0) ? n : 1;
}
}  // namespace rr

