// Line-of-sight integration over an adaptive mesh (Secs. 2.5.1, 2.7, 3.3).
//
// The ray walks the finest lattice (side n 2^lmax) with the parametric
// crossings of the uniform walk -- the k-th finest-face crossing on axis a at
// path T0_a + k td_a, one rounding, float-float start point per sub-step --
// but stops only where it leaves a leaf: a leaf of level l spans 2^(lmax - l)
// finest cells per axis, so from the current finest cell q its exit on axis a
// is a known number m_a of crossings ahead, and the nearest of the three exits
// ends the segment (lowest axis on ties). After the exit the other axes catch
// up: their crossing counters advance to the first crossing at or after the
// exit point, which moves q along them. The leaf of q is found by descending
// the refinement links from the coarse cell (at most lmax dependent loads).
//
// Inside a leaf the field is the trilinear interpolation of the leaf's 8
// corner values (one contiguous 256-byte record) or, for NGP, the leaf's own
// value; the segment integral is that of the uniform walk with the leaf's own
// cell size. Consecutive segments in the same leaf (separated only by a
// rounding sliver at an edge or corner) are one leaf segment, so the segment
// count is the number of leaf segments. FORM kFormShear: also the shear
// (gamma1, gamma2) of Eqs. gamma1, gamma2, a second projection of the same
// corner records carried through the same segment integrals. kFormMethodA:
// Method A (Eq. kappa2) on gradient records (rr_amr_gradient): n . grad Phi
// with the kernel dg/dchi, the density term with g, and the step's surface
// terms at the two ends of the traced interval (Eq. 2nterm). kFormGeneric: two
// scalar channels (rr_amr_scalars records) with their own quadratic kernels.
#include "walk.cuh"

namespace rr {
namespace {

// Leaf containing the finest cell q (each in [0, n 2^lmax)): its id, or -1 if
// the links are inconsistent; its level in lev.
__device__ __forceinline__ int coarse_link(const AmrDevice& M, const int q[3])
{
    const int L = M.lmax;
    return __ldg(M.link + ((q[0] >> L) * M.n + (q[1] >> L)) * M.n + (q[2] >> L));
}

// The leaf holding finest cell q, descending from its coarse cell's link
// value v (coarse_link).
__device__ __forceinline__ int amr_locate(const AmrDevice& M, const int q[3], int v, int& lev)
{
    const int L = M.lmax;
    int l = 0;
    while (v < 0 && l < L) {
        ++l;
        const int sh = L - l;
        v = __ldg(M.link + (-v - 1) + ((q[0] >> sh) & 1) + 2 * ((q[1] >> sh) & 1) + 4 * ((q[2] >> sh) & 1));
    }
    lev = l;
    return v < 0 ? -1 : v;
}

template <int INTERP, int FORM, bool REGACC = false>
__device__ __forceinline__ void trace_ray_amr(const TraceArgs& A, const AmrDevice& M, int ix, int iy,
                                              RayAcc* acc = nullptr)
{
    static_assert(!REGACC || FORM == kFormKahan || FORM == kFormShear || FORM == kFormMethodA ||
                      FORM == kFormGeneric,
                  "register accumulators: the compensated forms of the adaptive-mesh walk");
    constexpr bool SH = FORM == kFormShear;
    constexpr bool MA = FORM == kFormMethodA;
    constexpr bool GEN = FORM == kFormGeneric;
    // AHEAD: advance to the next cell before integrating the current one and
    // load its coarse link then, so that the load overlaps the segment's
    // arithmetic (faster for the shear and Method A walks, whose segments
    // carry more arithmetic; slower for the default and generic ones)
    constexpr bool AHEAD = SH || MA;
    const long long rid = (long long)iy * A.nx + ix;
    const int NF = A.n0;   // finest cells per side
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
    const float chis = (float)A.chi_s;
    const float ichis = A.inv_chi_s_f;
    const int nsub = max(1, f2i_signed(fminf(ceilf(rg.Lf / A.sub_len), 4194303.f)));
    const float dsub = rg.Lf / i2f_exact(nsub);
    const int L = M.lmax;
    // slivers: as in the uniform walk, 4 ulp of the path
    const float eps_rel = 4.76837158203125e-07f;

    Acc2 s2;   // (kappa, Born kappa) Kahan pairs
    Acc2 sg;   // (gamma1, gamma2), shear only
    float w1[6], w2[6];
    if constexpr (SH) shear_weights(A.dirh[rid], w1, w2);
    float4 nd;   // Method A: the direction
    if constexpr (MA) nd = A.dirh[rid];
    float qa = 0.f, ga = 0.f, qb = 0.f, gb = 0.f;   // Method A: n . grad Phi and g at the two ends
    uint32_t cnt = 0;
    bool overflow = false;
    int prev_leaf = -1;   // leaf of the last integrated segment
    for (int j = 0; j < nsub && !overflow; ++j) {
        float bh, bl, Lj, D0j;
        sub_step<true>(rg, j, nsub, dsub, bh, bl, Lj, D0j);
        Walk<float> W;
        walk_setup<float, true>(A, rid, bh, bl, Lj, D0j, rg.hi, rg.lo, W);
        const float Ls = W.L, chiA0 = W.chiA0, D0 = W.D0;
        const float eps_end = Ls * eps_rel;
        int q[3] = {W.c[0], W.c[1], W.c[2]};   // finest cell of the current point
        float K[3] = {0.f, 0.f, 0.f};           // finest-face crossings so far, per axis (exact integers)
        const int flip = (W.sgn[0] < 0 ? 1 : 0) | (W.sgn[1] < 0 ? 2 : 0) | (W.sgn[2] < 0 ? 4 : 0);
        float sig = 0.f;                        // path from the sub-step start to the segment entry
        int iter = 0;
        int link0 = AHEAD ? coarse_link(M, q) : 0;   // AHEAD: the current cell's coarse link
        while (true) {
            int lev;
            const int leaf = amr_locate(M, q, AHEAD ? link0 : coarse_link(M, q), lev);
            if (leaf < 0) {
                overflow = true;
                break;
            }
            const int sh = L - lev;
            const int span = 1 << sh;
            const float inv_span = __int_as_float((127 - sh) << 23);   // 2^-sh
            // crossings to the leaf's exit face (m), mirrored finest position in the
            // leaf (jp) and path to the exit (Tx), per axis
            int m[3], jp[3];
            float mf[3], Tx[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int pos = q[a] & (span - 1);
                m[a] = W.sgn[a] > 0 ? span - pos : pos + 1;
                jp[a] = W.sgn[a] > 0 ? pos : span - 1 - pos;
                mf[a] = i2f_exact(m[a]);
                Tx[a] = W.v[a] > 0.f ? fmaf(K[a] + (mf[a] - 1.f), W.td[a], W.T0[a]) : 1e30f;
            }
            float tend = Tx[0];
            int e = 0;
            if (Tx[1] < tend) { tend = Tx[1]; e = 1; }
            if (Tx[2] < tend) { tend = Tx[2]; e = 2; }
            const bool last = !(tend < Ls - eps_end);
            if (last) tend = Ls;
            const float t = tend - sig;
            const bool integrate = t > tend * eps_rel;
            // Method A: the first piece of the interval and the one that ends it
            // (the last, or the one leaving a bounded box) give the surface terms
            bool first = false, ends = false;
            if constexpr (MA) {
                first = j == 0 && iter == 0;
                ends = last;
                if (!A.periodic && !last) {
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        if (a == e) {
                            const int nq = q[a] + W.sgn[a] * m[a];
                            ends = nq < 0 || nq >= NF;
                        }
                }
            }

            // leave through axis e; the other axes advance to their first
            // crossing at or after the exit point (never past their own exit).
            // Returns whether the exit leaves the box.
            auto advance = [&]() -> bool {
                bool out = false;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (a == e) {
                        K[a] += mf[a];
                        const int nq = q[a] + W.sgn[a] * m[a];
                        out = nq < 0 || nq >= NF;
                        q[a] = wrap_once(nq, NF);
                    } else if (W.v[a] > 0.f) {
                        // counters are exact integers in float: the first crossing at or
                        // after tend (those before sig are counted already; the axis's own
                        // exit, kmax, is not before tend). Nearly always zero or one more
                        // crossing: tested one at a time; beyond that the closed form.
                        const float kmax = K[a] + (mf[a] - 1.f);
                        float k = K[a];
                        if (k < kmax && fmaf(k, W.td[a], W.T0[a]) < tend) {
                            k += 1.f;
                            if (k < kmax && fmaf(k, W.td[a], W.T0[a]) < tend) {
                                k = fminf(fmaxf(ceilf((tend - W.T0[a]) * W.v[a]), k + 1.f), kmax);
                                while (k > K[a] + 2.f && fmaf(k - 1.f, W.td[a], W.T0[a]) >= tend) k -= 1.f;
                                while (k < kmax && fmaf(k, W.td[a], W.T0[a]) < tend) k += 1.f;
                            }
                            q[a] = wrap_once(q[a] + W.sgn[a] * f2i_exact(k - K[a]), NF);
                            K[a] = k;
                        }
                    }
                }
                return out;
            };
            bool outside = false;
            if constexpr (AHEAD) {
                // nothing below reads q or K
                if (!last) {
                    outside = advance();
                    link0 = coarse_link(M, q);
                }
            }

            if (integrate || first || ends) {
                float2 q2[8];   // (Q_kappa, delta) at the mirrored corners, or the leaf's own value
                float2 g2[SH ? 8 : 1];   // (Q_gamma1, Q_gamma2) there
                if (INTERP == RR_TRILINEAR) {
                    const float4* r = A.rec + 16 * (long long)leaf;
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        // (two 16-byte loads: one 32-byte load per corner measured 3 % slower here)
                        const int rc = c ^ flip;
                        Rec x;
                        x.a = __ldg(r + 2 * rc);
                        x.b = __ldg(r + 2 * rc + 1);
                        q2[c] = MA ? radial_pair(nd, x.a) : make_float2(project(W.w, x), x.b.z);
                        if constexpr (MA) q2[c].y = x.b.z;
                        if constexpr (GEN) q2[c] = make_float2(x.a.x, x.a.y);
                        if constexpr (SH) g2[c] = make_float2(project(w1, x), project(w2, x));
                    }
                } else {
                    const Rec x = load_rec(A.rec, leaf);
                    q2[0] = MA ? make_float2(radial_pair(nd, x.a).x, x.b.z) : make_float2(project(W.w, x), x.b.z);
                    if constexpr (GEN) q2[0] = make_float2(x.a.x, x.a.y);
                    if constexpr (SH) g2[0] = make_float2(project(w1, x), project(w2, x));
                }
                float G0, G1, G2;
                kernel_coeffs(t, sig, chiA0, D0, chis, ichis, G0, G1, G2);
                // generic form: each channel's kernel about the entry point
                float2 K0, K1, K2;
                if constexpr (GEN) {
                    const float chiA = chiA0 - sig;
                    K0 = make_float2(fmaf(chiA, fmaf(chiA, A.kq[2], A.kq[1]), A.kq[0]),
                                     fmaf(chiA, fmaf(chiA, A.kq[5], A.kq[4]), A.kq[3]));
                    K1 = make_float2(-fmaf(2.f * A.kq[2], chiA, A.kq[1]), -fmaf(2.f * A.kq[5], chiA, A.kq[4]));
                    K2 = make_float2(A.kq[2], A.kq[5]);
                }
                if (INTERP == RR_TRILINEAR) {
                    float u[3], vl[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        vl[a] = W.v[a] * inv_span;
                        u[a] = W.v[a] > 0.f ? fminf(fmaxf(fmaf(sig - Tx[a], vl[a], 1.f), 0.f), 1.f)
                                            : (i2f_exact(jp[a]) + W.cu[a]) * inv_span;
                    }
                    if (integrate) {
                        if constexpr (GEN) {
                            float2 e2[4];
                            line_cubic2(q2, bc2(u[0]), bc2(u[1]), bc2(u[2]), bc2(vl[0]), bc2(vl[1]), bc2(vl[2]), e2);
                            s2.add(dot_kernel_pair(e2, t, K0, K1, K2));
                        } else if constexpr (MA)
                            s2.add(segment_trilinear_a(q2, u[0], u[1], u[2], vl[0], vl[1], vl[2], t, G0, G1, G2));
                        else
                            s2.add(segment_trilinear(q2, u[0], u[1], u[2], vl[0], vl[1], vl[2], t, G0, G1, G2));
                        if constexpr (SH)
                            sg.add(segment_trilinear(g2, u[0], u[1], u[2], vl[0], vl[1], vl[2], t, G0, G1, G2));
                    }
                    if constexpr (MA) {
                        if (first) {
                            qa = trilinear_x(q2, u[0], u[1], u[2]);
                            ga = D0 * chiA0 * ichis;
                        }
                        if (ends) {
                            float ue[3];
#pragma unroll
                            for (int a = 0; a < 3; ++a) ue[a] = fminf(fmaxf(fmaf(t, vl[a], u[a]), 0.f), 1.f);
                            qb = trilinear_x(q2, ue[0], ue[1], ue[2]);
                            gb = fmaf(t, fmaf(t, G2, G1), G0);
                        }
                    }
                } else {
                    if (integrate) {
                        if constexpr (GEN) {
                            const float2 tt = bc2(t);
                            const float2 J1 = __fmul2_rn(
                                tt, __ffma2_rn(tt, __ffma2_rn(tt, __fmul2_rn(K2, bc2(1.f / 3.f)), __fmul2_rn(K1, bc2(0.5f))),
                                               K0));
                            s2.add(__fmul2_rn(q2[0], J1));
                        } else if constexpr (MA) s2.add(segment_ngp_a(q2[0], t, G0, G1, G2));
                        else s2.add(segment_ngp(q2[0], t, G0, G1, G2));
                        if constexpr (SH) sg.add(segment_ngp(g2[0], t, G0, G1, G2));
                    }
                    if constexpr (MA) {
                        if (first) {
                            qa = q2[0].x;
                            ga = D0 * chiA0 * ichis;
                        }
                        if (ends) {
                            qb = q2[0].x;
                            gb = fmaf(t, fmaf(t, G2, G1), G0);
                        }
                    }
                }
                if (integrate) {
                    if (leaf != prev_leaf) ++cnt;
                    prev_leaf = leaf;
                }
            }
            sig = tend;
            if (last) break;
            if constexpr (!AHEAD) outside = advance();
            if (!A.periodic && outside) break;
            if (++iter > W.max_iter) {
                overflow = true;
                break;
            }
        }
    }

    if constexpr (MA) {
        s2.add(make_float2(-ga * qa, 0.f));
        s2.add(make_float2(gb * qb, 0.f));
    }
    if (overflow) atomicOr(A.err, kErrStepLimit);
    if (!s2.finite()) atomicOr(A.err, kErrNonFinite);
    float kh, kl, bh, bl;
    two_sum(s2.s.x, -s2.c.x, kh, kl);
    two_sum(s2.s.y, -s2.c.y, bh, bl);
    if constexpr (REGACC) {
        if (!acc->loaded) {
            acc->k = A.kacc[rid];
            acc->b = A.bacc[rid];
            acc->n = A.nseg[rid];
            if constexpr (SH) {
                acc->x1 = A.g1acc[rid];
                acc->x2 = A.g2acc[rid];
            }
            acc->loaded = true;
        }
        acc->k = ff_mul_add(acc->k, kh, kl, A.sch, A.scl);
        acc->b = ff_mul_add(acc->b, bh, bl, A.bsh, A.bsl);
        acc->n += cnt;
        if constexpr (SH) {
            if (!sg.finite()) atomicOr(A.err, kErrNonFinite);
            float gh, gl;
            two_sum(sg.s.x, -sg.c.x, gh, gl);
            acc->x1 = ff_mul_add(acc->x1, gh, gl, A.sch, A.scl);
            two_sum(sg.s.y, -sg.c.y, gh, gl);
            acc->x2 = ff_mul_add(acc->x2, gh, gl, A.sch, A.scl);
        }
        return;
    }
    A.kacc[rid] = ff_mul_add(A.kacc[rid], kh, kl, A.sch, A.scl);
    A.bacc[rid] = ff_mul_add(A.bacc[rid], bh, bl, A.bsh, A.bsl);
    A.nseg[rid] += cnt;
    if constexpr (SH) {
        if (!sg.finite()) atomicOr(A.err, kErrNonFinite);
        float gh, gl;
        two_sum(sg.s.x, -sg.c.x, gh, gl);
        A.g1acc[rid] = ff_mul_add(A.g1acc[rid], gh, gl, A.sch, A.scl);
        two_sum(sg.s.y, -sg.c.y, gh, gl);
        A.g2acc[rid] = ff_mul_add(A.g2acc[rid], gh, gl, A.sch, A.scl);
    }
}

template <int INTERP, int FORM>
__global__ void __launch_bounds__(NT_MAX, 2) trace_amr_kernel(const TraceArgs A, const AmrDevice M, const TileCfg t)
{
    int ix, iy;
    tile_ray(t, blockIdx.x, blockIdx.y, ix, iy);
    if (ix < A.nx && iy < A.ny) trace_ray_amr<INTERP, FORM>(A, M, ix, iy);
}

// Consecutive steps over the adaptive mesh in one launch, as
// trace_steps_kernel does on the uniform grid: every step its own leaf
// records, interval and scales, the ray's sums (and its shear pair) in
// registers in between; per step the arithmetic of trace_amr_kernel, so the
// same results bit for bit.
template <int INTERP, int FORM>
__global__ void __launch_bounds__(NT_MAX, 2)
    trace_amr_steps_kernel(const TraceArgs A, const AmrDevice M, const __grid_constant__ StepBlock S, const TileCfg t)
{
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
        trace_ray_amr<INTERP, FORM, true>(As, M, ix, iy, &acc);
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
    }
}

}  // namespace

cudaError_t launch_trace_amr_steps(const TraceArgs& a, const AmrDevice& m, const StepBlock& b, int interp,
                                   cudaStream_t s, int form)
{
    if (b.n < 1 || b.n > kMaxStepBlock) return cudaErrorInvalidValue;
    const TileCfg t;
    const dim3 grid = tile_grid(t, a.nx, a.ny);
    const dim3 block(32 * t.bwx * t.bwy);
    const bool tri = interp == RR_TRILINEAR;
#define RR_AMR_STEPS(F)                                                                              \
    do {                                                                                              \
        if (tri) trace_amr_steps_kernel<RR_TRILINEAR, F><<<grid, block, 0, s>>>(a, m, b, t);          \
        else trace_amr_steps_kernel<RR_NGP, F><<<grid, block, 0, s>>>(a, m, b, t);                   \
    } while (0)
    switch (form) {
    case kFormKahan: RR_AMR_STEPS(kFormKahan); break;
    case kFormShear: RR_AMR_STEPS(kFormShear); break;
    case kFormMethodA: RR_AMR_STEPS(kFormMethodA); break;
    case kFormGeneric: RR_AMR_STEPS(kFormGeneric); break;
    default: return cudaErrorInvalidValue;
    }
#undef RR_AMR_STEPS
    return cudaGetLastError();
}

cudaError_t launch_trace_amr(const TraceArgs& a, const AmrDevice& m, int interp, cudaStream_t s, int form)
{
    const TileCfg t;
    const dim3 grid = tile_grid(t, a.nx, a.ny);
    const dim3 block(32 * t.bwx * t.bwy);
    const bool tri = interp == RR_TRILINEAR;
    if (form == kFormShear) {
        if (tri) trace_amr_kernel<RR_TRILINEAR, kFormShear><<<grid, block, 0, s>>>(a, m, t);
        else trace_amr_kernel<RR_NGP, kFormShear><<<grid, block, 0, s>>>(a, m, t);
    } else if (form == kFormGeneric) {
        if (tri) trace_amr_kernel<RR_TRILINEAR, kFormGeneric><<<grid, block, 0, s>>>(a, m, t);
        else trace_amr_kernel<RR_NGP, kFormGeneric><<<grid, block, 0, s>>>(a, m, t);
    } else if (form == kFormMethodA) {
        if (tri) trace_amr_kernel<RR_TRILINEAR, kFormMethodA><<<grid, block, 0, s>>>(a, m, t);
        else trace_amr_kernel<RR_NGP, kFormMethodA><<<grid, block, 0, s>>>(a, m, t);
    } else {
        if (tri) trace_amr_kernel<RR_TRILINEAR, kFormKahan><<<grid, block, 0, s>>>(a, m, t);
        else trace_amr_kernel<RR_NGP, kFormKahan><<<grid, block, 0, s>>>(a, m, t);
    }
    return cudaGetLastError();
}

}  // namespace rr
