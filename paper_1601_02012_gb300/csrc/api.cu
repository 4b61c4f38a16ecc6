// C ABI: argument validation, contexts, stream plumbing, the step log.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>

#include "rr_internal.h"

using namespace rr;

namespace {

bool is_finite(double x) { return std::isfinite(x); }

bool is_aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
// tidal records (32 B per point) are read and written with 32-byte vector accesses
bool is_aligned32(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 31u) == 0; }

rr_status from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return RR_OK;
    if (e == cudaErrorMemoryAllocation) return RR_ERR_OOM;
    return RR_ERR_CUDA;
}

rr_status status_from_word(uint32_t w)
{
    if (w & kErrStepLimit) return RR_ERR_STEP_LIMIT;
    if (w & kErrNonFinite) return RR_ERR_NONFINITE;
    if (w & kErrRange) return RR_ERR_RANGE;
    return RR_OK;
}

void free_state(RayState& s)
{
    cudaFree(s.dir);
    cudaFree(s.dirh);
    cudaFree(s.dirl);
    cudaFree(s.kacc);
    cudaFree(s.bacc);
    cudaFree(s.kmom);
    cudaFree(s.bmom);
    cudaFree(s.g1acc);
    cudaFree(s.g2acc);
    cudaFree(s.nseg);
    cudaFree(s.err);
    cudaFree(s.total);
    s = RayState{};
}


}  // namespace

namespace rr {

rr_status check_bundle(const rr_bundle_desc* b)
{
    if (!b) return RR_ERR_ARG;
    if (b->nx < 1 || b->ny < 1 || (long long)b->nx * b->ny > (1LL << 30)) return RR_ERR_ARG;
    if (!is_finite(b->fov_x) || !is_finite(b->fov_y) || b->fov_x < 0 || b->fov_y < 0 || b->fov_x >= M_PI ||
        b->fov_y >= M_PI)
        return RR_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!is_finite(b->obs[a])) return RR_ERR_ARG;
    if (!is_finite(b->chi_s) || !(b->chi_s > 0)) return RR_ERR_ARG;
    if (b->interp != RR_NGP && b->interp != RR_TRILINEAR) return RR_ERR_ARG;
    if (b->flags &
        ~(RR_PERIODIC | RR_FP64_DDA | RR_PLAIN_SUMS | RR_SOURCE_MOMENTS | RR_SHEAR | RR_METHOD_A | RR_GENERIC))
        return RR_ERR_ARG;
    if ((b->flags & RR_PLAIN_SUMS) && (b->flags & (RR_FP64_DDA | RR_SOURCE_MOMENTS))) return RR_ERR_ARG;
    if ((b->flags & RR_SOURCE_MOMENTS) && (b->flags & RR_FP64_DDA)) return RR_ERR_ARG;
    if ((b->flags & RR_SHEAR) && (b->flags & (RR_FP64_DDA | RR_PLAIN_SUMS | RR_SOURCE_MOMENTS))) return RR_ERR_ARG;
    if ((b->flags & RR_METHOD_A) && (b->flags & (RR_FP64_DDA | RR_PLAIN_SUMS | RR_SOURCE_MOMENTS | RR_SHEAR)))
        return RR_ERR_ARG;
    if ((b->flags & RR_GENERIC) &&
        (b->flags & (RR_FP64_DDA | RR_PLAIN_SUMS | RR_SOURCE_MOMENTS | RR_SHEAR | RR_METHOD_A)))
        return RR_ERR_ARG;
    return RR_OK;
}

rr_status check_grid(const rr_grid_desc* g)
{
    if (!g) return RR_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (g->n[a] < 2 || g->n[a] > 4096) return RR_ERR_ARG;
    if (!is_finite(g->box) || !(g->box > 0)) return RR_ERR_ARG;
    if (!is_finite(g->omega_m) || !(g->omega_m > 0)) return RR_ERR_ARG;
    return RR_OK;
}

// The step geometry and a bundle's per-ray state pointers, as the kernels take them.
TraceArgs make_trace_args(const rr_bundle_desc& b, const RayState& st, const rr_grid_desc* grid, const float* rec,
                          double chi_a, double chi_b, double scale, double a_step, const double* obs,
                          const double* kq)
{
    if (!obs) obs = b.obs;
    TraceArgs a{};
    a.rec = reinterpret_cast<const float4*>(rec);
    a.n0 = grid->n[0]; a.n1 = grid->n[1]; a.n2 = grid->n[2];
    a.h = grid->box / grid->n[0];
    a.inv_h = 1.0 / a.h;
    a.inv_hf = (float)a.inv_h;
    split_ff(a.inv_h, a.ihh, a.ihl);
    a.nx = b.nx; a.ny = b.ny;
    a.obs0 = obs[0]; a.obs1 = obs[1]; a.obs2 = obs[2];
    for (int i = 0; i < 3; ++i) split_ff(obs[i], a.oh[i], a.ol[i]);
    a.chi_s = b.chi_s;
    a.chi_a = chi_a;
    a.chi_b = chi_b;
    split_ff(chi_a, a.cah, a.cal);
    a.Lf = (float)(chi_a - chi_b);
    a.D0f = (float)(b.chi_s - chi_a);
    a.inv_chi_s_f = (float)(1.0 / b.chi_s);
    a.sub_len = (float)(32.0 * a.h);
    a.periodic = (b.flags & RR_PERIODIC) ? 1 : 0;
    // flat addressing over the whole grid's records
    for (int i = 0; i < 3; ++i) {
        a.fo[i] = 0;
        a.fe[i] = grid->n[i];
    }
    a.fs0 = grid->n[1] * grid->n[2];
    a.fs1 = grid->n[2];
    a.dir = st.dir;
    a.dirh = st.dirh;
    a.dirl = st.dirl;
    a.kacc = st.kacc;
    a.bacc = st.bacc;
    a.kmom = st.kmom;
    a.bmom = st.bmom;
    a.g1acc = st.g1acc;
    a.g2acc = st.g2acc;
    a.nseg = st.nseg;
    a.err = st.err;
    split_ff(scale, a.sch, a.scl);
    if (b.flags & RR_GENERIC) {
        // both channels are plain integrals times the step's scale
        a.bsh = a.sch;
        a.bsl = a.scl;
    } else {
        split_ff(scale * 1.5 * grid->omega_m * kH0OverC * kH0OverC / a_step, a.bsh, a.bsl);
    }
    // the generic form's kernels (default: the lensing kernel g = chi - chi^2 / chi_s on both channels)
    const double kg[6] = {0.0, 1.0, -1.0 / b.chi_s, 0.0, 1.0, -1.0 / b.chi_s};
    if (!kq) kq = kg;
    for (int i = 0; i < 6; ++i) a.kq[i] = (float)kq[i];
    return a;
}

// The step geometry and the context's state pointers, as the kernels take them.
TraceArgs make_trace_args(rr_ctx* ctx, const rr_grid_desc* grid, const float* rec, double chi_a, double chi_b,
                          double scale, double a_step, const double* obs)
{
    return make_trace_args(ctx->bundle, ctx->st, grid, rec, chi_a, chi_b, scale, a_step, obs, ctx->kq);
}

StepRecord make_step_record(const rr_ctx* ctx, const rr_grid_desc* grid, double chi_a, double chi_b, double scale,
                            double a_step)
{
    StepRecord r{*grid, chi_a, chi_b, scale, a_step};
    for (int i = 0; i < 3; ++i) r.obs[i] = ctx->bundle.obs[i];
    return r;
}


rr_status validate_step(rr_ctx* ctx, const rr_grid_desc* grid, const float* rec, double chi_a, double chi_b,
                        double scale, double a_step)
{
    if (!ctx) return RR_ERR_ARG;
    rr_status st = check_grid(grid);
    if (st != RR_OK) return st;
    // tidal records (every form but Method A's gradient and the generic scalar records): 32-byte aligned
    const bool tidal = !(ctx->bundle.flags & (RR_METHOD_A | RR_GENERIC));
    if (!rec || !is_aligned16(rec) || (tidal && !is_aligned32(rec))) return RR_ERR_ARG;
    if (!is_finite(chi_a) || !is_finite(chi_b) || !is_finite(scale) || !is_finite(a_step) || !(a_step > 0))
        return RR_ERR_ARG;
    if (!(chi_a > chi_b) || chi_b < 0 || chi_a > ctx->bundle.chi_s * (1.0 + 1e-12)) return RR_ERR_ARG;
    if (!ctx->log.empty() && !ctx->relocated) {
        const double prev = ctx->log.back().chi_b;
        if (fabs(prev - chi_a) > 1e-12 * std::max(1.0, fabs(chi_a))) return RR_ERR_STATE;
    }
    return RR_OK;
}

rr_status status_of_cuda(cudaError_t e) { return from_cuda(e); }

}  // namespace rr

namespace rr {

// Bounds [lo, hi] per axis of the positions obs + chi n of the bundle's rays
// for chi in [chi_b, chi_a]. n_x = theta_x sinc(theta) lies in
// [-sin(U_x/2), sin(U_x/2)] because sinc decreases on [0, pi); n_z = cos(theta)
// lies in [cos(theta_max), 1]; a position is linear in chi, so its extremes
// are at the ends of the interval.
static void position_bounds(const rr_bundle_desc& b, const double obs[3], double chi_a, double chi_b,
                            double lo[3], double hi[3])
{
    const double hx = b.nx > 1 ? 0.5 * b.fov_x : 0.0, hy = b.ny > 1 ? 0.5 * b.fov_y : 0.0;
    const double thmax = sqrt(hx * hx + hy * hy);
    const double nlo[3] = {-sin(hx), -sin(hy), cos(thmax)};
    const double nhi[3] = {sin(hx), sin(hy), 1.0};
    for (int a = 0; a < 3; ++a) {
        const double c1 = chi_a * nlo[a], c2 = chi_b * nlo[a], c3 = chi_a * nhi[a], c4 = chi_b * nhi[a];
        lo[a] = obs[a] + std::min(std::min(c1, c2), std::min(c3, c4));
        hi[a] = obs[a] + std::max(std::max(c1, c2), std::max(c3, c4));
    }
}

void footprint_box(const rr_bundle_desc& b, const double obs[3], const rr_grid_desc& g, double chi_a,
                   double chi_b, long long i0[3], long long i1[3])
{
    double lo[3], hi[3];
    position_bounds(b, obs, chi_a, chi_b, lo, hi);
    const double h = g.box / g.n[0];
    for (int a = 0; a < 3; ++a) {
        const double f0 = floor(lo[a] / h), f1 = floor(hi[a] / h);
        // (saturated far outside any grid; the callers compare against [0, n])
        i0[a] = (f0 > -1e15 ? (long long)f0 : -1000000000000000LL) - 1;
        i1[a] = (f1 < 1e15 ? (long long)f1 : 1000000000000000LL) + 3;
    }
}

bool flat_ok(const rr_bundle_desc& b, const double obs[3], const rr_grid_desc& g, double chi_a, double chi_b)
{
    if (!(b.flags & RR_PERIODIC) || b.interp != RR_TRILINEAR) return false;
    if ((long long)g.n[0] * g.n[1] * g.n[2] >= (1LL << 31)) return false;
    // every position of the step inside [2 h, (n - 3) h) per axis: the walk's
    // cells then lie in 2 .. n - 4, and each sub-step's own check (up to 2
    // crossings more than its path allows, planes one further) stays in
    // [0, n - 1]: no vertex plane across the periodic seam
    double lo[3], hi[3];
    position_bounds(b, obs, chi_a, chi_b, lo, hi);
    const double h = g.box / g.n[0];
    for (int a = 0; a < 3; ++a)
        if (!(lo[a] >= 2.0 * h) || !(hi[a] < (g.n[a] - 3) * h)) return false;
    return true;
}

}  // namespace rr

extern "C" {

const char* rr_status_string(rr_status s)
{
    switch (s) {
    case RR_OK: return "RR_OK";
    case RR_ERR_ARG: return "RR_ERR_ARG: invalid argument";
    case RR_ERR_CUDA: return "RR_ERR_CUDA: a CUDA runtime call failed";
    case RR_ERR_OOM: return "RR_ERR_OOM: device allocation failed";
    case RR_ERR_STEP_LIMIT: return "RR_ERR_STEP_LIMIT: a ray exceeded its per-step iteration cap";
    case RR_ERR_STATE: return "RR_ERR_STATE: calls out of order";
    case RR_ERR_NONFINITE: return "RR_ERR_NONFINITE: a per-ray sum is not finite";
    case RR_ERR_CAPACITY: return "RR_ERR_CAPACITY: more rays than the fixed no-allocation scratch holds";
    case RR_ERR_RANGE: return "RR_ERR_RANGE: a ray left the index range its step's record addressing covers";
    }
    return "unknown rr_status";
}

static rr_status create_context(const rr_bundle_desc* bundle, int32_t y0, int32_t y1, rr_ctx** out)
{
    if (!out) return RR_ERR_ARG;
    *out = nullptr;
    rr_status st = check_bundle(bundle);
    if (st != RR_OK) return st;
    if (y0 < 0 || y1 > bundle->ny || !(y0 < y1)) return RR_ERR_ARG;
    rr_ctx* ctx = new (std::nothrow) rr_ctx();
    if (!ctx) return RR_ERR_OOM;
    ctx->bundle = *bundle;
    ctx->bundle.ny = y1 - y0;
    ctx->row0 = y0;
    ctx->ny_full = bundle->ny;
    // generic form: both kernels start as the lensing kernel g = chi - chi^2 / chi_s
    for (int c = 0; c < 2; ++c) {
        ctx->kq[3 * c] = 0.0;
        ctx->kq[3 * c + 1] = 1.0;
        ctx->kq[3 * c + 2] = -1.0 / bundle->chi_s;
    }
    cudaGetDevice(&ctx->device);
    const size_t nr = (size_t)bundle->nx * (size_t)(y1 - y0);
    cudaError_t e = cudaSuccess;
    RayState& s = ctx->st;
    if (e == cudaSuccess) e = cudaMalloc(&s.dir, 3 * nr * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&s.dirh, nr * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&s.dirl, nr * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&s.kacc, nr * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&s.bacc, nr * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&s.nseg, nr * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&s.err, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&s.total, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->host_err, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->host_total, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(s.kacc, 0, nr * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemset(s.bacc, 0, nr * sizeof(float2));
    if (bundle->flags & RR_SOURCE_MOMENTS) {
        if (e == cudaSuccess) e = cudaMalloc(&s.kmom, nr * sizeof(float2));
        if (e == cudaSuccess) e = cudaMalloc(&s.bmom, nr * sizeof(float2));
        if (e == cudaSuccess) e = cudaMemset(s.kmom, 0, nr * sizeof(float2));
        if (e == cudaSuccess) e = cudaMemset(s.bmom, 0, nr * sizeof(float2));
    }
    if (bundle->flags & RR_SHEAR) {
        if (e == cudaSuccess) e = cudaMalloc(&s.g1acc, nr * sizeof(float2));
        if (e == cudaSuccess) e = cudaMalloc(&s.g2acc, nr * sizeof(float2));
        if (e == cudaSuccess) e = cudaMemset(s.g1acc, 0, nr * sizeof(float2));
        if (e == cudaSuccess) e = cudaMemset(s.g2acc, 0, nr * sizeof(float2));
    }
    if (e == cudaSuccess) e = cudaMemset(s.nseg, 0, nr * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(s.err, 0, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(s.total, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = launch_init_directions(*bundle, s.dir, s.dirh, s.dirl, 0, y0, y1 - y0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_state(s);
        if (ctx->host_err) cudaFreeHost(ctx->host_err);
        if (ctx->host_total) cudaFreeHost(ctx->host_total);
        delete ctx;
        return from_cuda(e);
    }
    *out = ctx;
    return RR_OK;
}

rr_status rr_create(const rr_bundle_desc* bundle, rr_ctx** out)
{
    return create_context(bundle, 0, bundle ? bundle->ny : 0, out);
}

rr_status rr_create_band(const rr_bundle_desc* bundle, int32_t y0, int32_t y1, rr_ctx** out)
{
    return create_context(bundle, y0, y1, out);
}

rr_status rr_destroy(rr_ctx* ctx)
{
    if (!ctx) return RR_ERR_ARG;
    cudaDeviceSynchronize();
    free_state(ctx->st);
    cudaFreeHost(ctx->host_err);
    cudaFreeHost(ctx->host_total);
    delete ctx;
    return RR_OK;
}

rr_status rr_reset(rr_ctx* ctx, void* stream)
{
    if (!ctx) return RR_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nr = (size_t)ctx->bundle.nx * ctx->bundle.ny;
    cudaError_t e = cudaMemsetAsync(ctx->st.kacc, 0, nr * sizeof(float2), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->st.bacc, 0, nr * sizeof(float2), s);
    if (e == cudaSuccess && ctx->st.kmom) e = cudaMemsetAsync(ctx->st.kmom, 0, nr * sizeof(float2), s);
    if (e == cudaSuccess && ctx->st.bmom) e = cudaMemsetAsync(ctx->st.bmom, 0, nr * sizeof(float2), s);
    if (e == cudaSuccess && ctx->st.g1acc) e = cudaMemsetAsync(ctx->st.g1acc, 0, nr * sizeof(float2), s);
    if (e == cudaSuccess && ctx->st.g2acc) e = cudaMemsetAsync(ctx->st.g2acc, 0, nr * sizeof(float2), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->st.nseg, 0, nr * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->st.err, 0, sizeof(uint32_t), s);
    ctx->log.clear();
    ctx->last_total = 0;
    return from_cuda(e);
}

static rr_status point_records(const rr_grid_desc* grid, const float* phi, const float* delta, float* rec,
                               int32_t where, const int32_t* bbox, void* stream, int kind)
{
    rr_status st = check_grid(grid);
    if (st != RR_OK) return st;
    if (!phi || !rec || !is_aligned16(rec) || (kind == 0 && !is_aligned32(rec))) return RR_ERR_ARG;
    if (where != RR_AT_VERTICES && where != RR_AT_CENTRES) return RR_ERR_ARG;
    if (bbox) {
        for (int a = 0; a < 3; ++a) {
            const long long ext = (long long)bbox[2 * a + 1] - bbox[2 * a];
            if (ext < 1 || ext > grid->n[a]) return RR_ERR_ARG;
            if (bbox[2 * a] < -(1 << 20) || bbox[2 * a + 1] > (1 << 20)) return RR_ERR_ARG;
        }
    }
    return from_cuda(launch_tidal(*grid, phi, delta, rec, where, bbox, (cudaStream_t)stream, kind));
}

rr_status rr_tidal_tensor(const rr_grid_desc* grid, const float* phi, const float* delta, float* rec,
                          int32_t where, const int32_t* bbox, void* stream)
{
    return point_records(grid, phi, delta, rec, where, bbox, stream, 0);
}

rr_status rr_tidal_tensor_box(const rr_grid_desc* grid, const float* phi, const float* delta, float* rec,
                              int32_t where, const int32_t* bbox, void* stream)
{
    rr_status st = check_grid(grid);
    if (st != RR_OK) return st;
    if (!phi || !rec || !bbox || !is_aligned32(rec)) return RR_ERR_ARG;
    if (where != RR_AT_VERTICES && where != RR_AT_CENTRES) return RR_ERR_ARG;
    long long npts = 1;
    for (int a = 0; a < 3; ++a) {
        const long long ext = (long long)bbox[2 * a + 1] - bbox[2 * a];
        if (ext < 1 || ext > grid->n[a]) return RR_ERR_ARG;
        if (bbox[2 * a] < -(1 << 20) || bbox[2 * a + 1] > (1 << 20)) return RR_ERR_ARG;
        npts *= ext;
    }
    if (npts >= (1LL << 31)) return RR_ERR_ARG;
    return from_cuda(launch_tidal(*grid, phi, delta, rec, where, bbox, (cudaStream_t)stream, 0, true));
}

rr_status rr_scalar_records(const rr_grid_desc* grid, const float* field, const float* field_prev, double inv_dt,
                            int32_t channel, float* rec, int32_t where, const int32_t* bbox, void* stream)
{
    rr_status st = check_grid(grid);
    if (st != RR_OK) return st;
    if (!field || !rec || !is_aligned16(rec) || (channel != 0 && channel != 1) || !is_finite(inv_dt))
        return RR_ERR_ARG;
    if (where != RR_AT_VERTICES && where != RR_AT_CENTRES) return RR_ERR_ARG;
    if (bbox) {
        for (int a = 0; a < 3; ++a) {
            const long long ext = (long long)bbox[2 * a + 1] - bbox[2 * a];
            if (ext < 1 || ext > grid->n[a]) return RR_ERR_ARG;
            if (bbox[2 * a] < -(1 << 20) || bbox[2 * a + 1] > (1 << 20)) return RR_ERR_ARG;
        }
    }
    return from_cuda(launch_scalar_records(*grid, field, field_prev, (float)inv_dt, channel, rec, where, bbox,
                                           (cudaStream_t)stream));
}

rr_status rr_upload_box(const rr_grid_desc* grid, const float* host, float* dev, const int32_t* bbox,
                        int64_t* bytes, void* stream)
{
    rr_status st = check_grid(grid);
    if (st != RR_OK) return st;
    if (!host || !dev) return RR_ERR_ARG;
    const int* n = grid->n;
    const cudaStream_t s = (cudaStream_t)stream;
    if (!bbox) {
        const size_t all = sizeof(float) * (size_t)n[0] * n[1] * n[2];
        if (bytes) *bytes = (int64_t)all;
        return from_cuda(cudaMemcpyAsync(dev, host, all, cudaMemcpyHostToDevice, s));
    }
    // per axis: the widened range as at most two runs of indices in [0, n)
    int r0[3][2], rw[3][2], nr[3];
    for (int a = 0; a < 3; ++a) {
        const long long ext = (long long)bbox[2 * a + 1] - bbox[2 * a];
        if (ext < 1 || ext > n[a]) return RR_ERR_ARG;
        if (bbox[2 * a] < -(1 << 20) || bbox[2 * a + 1] > (1 << 20)) return RR_ERR_ARG;
        const long long w = ext + 4;
        if (w >= n[a]) {
            nr[a] = 1; r0[a][0] = 0; rw[a][0] = n[a];
            continue;
        }
        const int lo = (int)(((long long)bbox[2 * a] - 2) % n[a] + n[a]) % n[a];
        if (lo + w <= n[a]) {
            nr[a] = 1; r0[a][0] = lo; rw[a][0] = (int)w;
        } else {
            nr[a] = 2;
            r0[a][0] = lo; rw[a][0] = n[a] - lo;
            r0[a][1] = 0;  rw[a][1] = (int)(lo + w - n[a]);
        }
    }
    const size_t pitch = sizeof(float) * (size_t)n[2];
    int64_t total = 0;
    for (int i = 0; i < nr[0]; ++i)
        for (int j = 0; j < nr[1]; ++j)
            for (int k = 0; k < nr[2]; ++k) {
                cudaMemcpy3DParms p;
                memset(&p, 0, sizeof(p));
                p.srcPtr = make_cudaPitchedPtr(const_cast<float*>(host), pitch, n[2], n[1]);
                p.dstPtr = make_cudaPitchedPtr(dev, pitch, n[2], n[1]);
                p.srcPos = make_cudaPos(sizeof(float) * (size_t)r0[2][k], r0[1][j], r0[0][i]);
                p.dstPos = p.srcPos;
                p.extent = make_cudaExtent(sizeof(float) * (size_t)rw[2][k], rw[1][j], rw[0][i]);
                p.kind = cudaMemcpyHostToDevice;
                const cudaError_t e = cudaMemcpy3DAsync(&p, s);
                if (e != cudaSuccess) return from_cuda(e);
                total += (int64_t)sizeof(float) * rw[2][k] * rw[1][j] * rw[0][i];
            }
    if (bytes) *bytes = total;
    return RR_OK;
}

rr_status rr_set_kernels(rr_ctx* ctx, const double k[6])
{
    if (!ctx || !k) return RR_ERR_ARG;
    if (!(ctx->bundle.flags & RR_GENERIC)) return RR_ERR_STATE;
    for (int i = 0; i < 6; ++i)
        if (!is_finite(k[i])) return RR_ERR_ARG;
    for (int i = 0; i < 6; ++i) ctx->kq[i] = k[i];
    return RR_OK;
}

rr_status rr_set_observer(rr_ctx* ctx, const double obs[3])
{
    if (!ctx || !obs) return RR_ERR_ARG;
    for (int i = 0; i < 3; ++i)
        if (!is_finite(obs[i])) return RR_ERR_ARG;
    for (int i = 0; i < 3; ++i) ctx->bundle.obs[i] = obs[i];
    ctx->relocated = true;
    return RR_OK;
}

rr_status rr_gradient_records(const rr_grid_desc* grid, const float* phi, const float* delta, float* rec,
                              int32_t where, const int32_t* bbox, void* stream)
{
    return point_records(grid, phi, delta, rec, where, bbox, stream, 1);
}

rr_status rr_footprint_bbox(const rr_bundle_desc* b, const rr_grid_desc* g, double chi_a, double chi_b,
                            int32_t bbox[6])
{
    rr_status st = check_bundle(b);
    if (st != RR_OK) return st;
    st = check_grid(g);
    if (st != RR_OK) return st;
    if (!bbox || !is_finite(chi_a) || !is_finite(chi_b) || !(chi_a >= chi_b) || chi_b < 0) return RR_ERR_ARG;
    long long b0[3], b1[3];
    footprint_box(*b, b->obs, *g, chi_a, chi_b, b0, b1);
    for (int a = 0; a < 3; ++a) {
        long long i0 = b0[a], i1 = b1[a];
        if (i1 - i0 >= g->n[a] || i0 < -(1 << 20) || i1 > (1 << 20)) {
            i0 = 0;
            i1 = g->n[a];
        }
        bbox[2 * a] = (int32_t)i0;
        bbox[2 * a + 1] = (int32_t)i1;
    }
    return RR_OK;
}

rr_status rr_trace_step(rr_ctx* ctx, const rr_grid_desc* grid, const float* rec, double chi_a, double chi_b,
                        double scale, double a_step, void* stream)
{
    rr_status st = validate_step(ctx, grid, rec, chi_a, chi_b, scale, a_step);
    if (st != RR_OK) return st;
    const rr_bundle_desc& b = ctx->bundle;
    TraceArgs a = make_trace_args(ctx, grid, rec, chi_a, chi_b, scale, a_step);
    const int form = (b.flags & RR_SOURCE_MOMENTS) ? kFormMoments
                     : (b.flags & RR_PLAIN_SUMS)   ? kFormPlain
                     : (b.flags & RR_SHEAR)        ? kFormShear
                     : (b.flags & RR_METHOD_A)     ? kFormMethodA
                     : (b.flags & RR_GENERIC)      ? kFormGeneric
                                                   : kFormKahan;
    // (the footprint of the whole bundle holds the footprint of a band of it)
    rr_bundle_desc whole = b;
    whole.ny = ctx->ny_full;
    const bool flat = !(b.flags & RR_FP64_DDA) && flat_ok(whole, b.obs, *grid, chi_a, chi_b);
    cudaError_t e =
        launch_trace(a, b.interp, (b.flags & RR_FP64_DDA) != 0, (cudaStream_t)stream, TileCfg{}, form, flat);
    if (e != cudaSuccess) return from_cuda(e);
    ctx->log.push_back(make_step_record(ctx, grid, chi_a, chi_b, scale, a_step));
    ctx->relocated = false;
    return RR_OK;
}

// Does the box [bb[2a], bb[2a + 1]) per axis (periodically) hold the points
// [f0[a], f1[a])?
static bool box_holds(const int32_t* bb, const long long f0[3], const long long f1[3], const rr_grid_desc& g)
{
    for (int a = 0; a < 3; ++a) {
        const long long n = g.n[a], b0 = bb[2 * a], b1 = bb[2 * a + 1];
        if (f1[a] - f0[a] > b1 - b0) return false;
        // the box's periodic image that starts at or below f0, within a period
        const long long d = f0[a] - b0;
        const long long m = d >= 0 ? d / n : -((-d + n - 1) / n);
        if (f1[a] > b1 + m * n) return false;
    }
    return true;
}

rr_status rr_trace_steps(rr_ctx* ctx, const rr_grid_desc* grid, int32_t nsteps, const float* const* rec,
                         const int32_t* boxes, const double* chi_a, const double* chi_b, const double* scale,
                         const double* a_step, void* stream)
{
    if (!ctx || nsteps < 0) return RR_ERR_ARG;
    if (nsteps == 0) return RR_OK;
    if (!rec || !chi_a || !chi_b || !scale || !a_step) return RR_ERR_ARG;
    const rr_bundle_desc& b = ctx->bundle;
    const bool fused = !(b.flags & (RR_FP64_DDA | RR_PLAIN_SUMS));
    const int form = (b.flags & RR_SOURCE_MOMENTS) ? kFormMoments
                     : (b.flags & RR_SHEAR)        ? kFormShear
                     : (b.flags & RR_METHOD_A)     ? kFormMethodA
                     : (b.flags & RR_GENERIC)      ? kFormGeneric
                                                   : kFormKahan;
    rr_bundle_desc whole = b;
    whole.ny = ctx->ny_full;
    if (boxes) {
        // records of each step's box only: the flat walk over them (trilinear,
        // periodic, a form that reads tidal records); each box must hold the
        // step's footprint
        if (!fused || form == kFormMethodA || form == kFormGeneric || b.interp != RR_TRILINEAR ||
            !(b.flags & RR_PERIODIC))
            return RR_ERR_ARG;
        rr_status st = check_grid(grid);
        if (st != RR_OK) return st;
        for (int32_t i = 0; i < nsteps; ++i) {
            const int32_t* bb = boxes + 6 * (size_t)i;
            long long npts = 1;
            for (int a = 0; a < 3; ++a) {
                const long long ext = (long long)bb[2 * a + 1] - bb[2 * a];
                if (ext < 1 || ext > grid->n[a] || bb[2 * a] < -(1 << 20) || bb[2 * a + 1] > (1 << 20))
                    return RR_ERR_ARG;
                npts *= ext;
            }
            if (npts >= (1LL << 31) || !is_finite(chi_a[i]) || !is_finite(chi_b[i])) return RR_ERR_ARG;
            // the footprint box widened by one point per side: the flat walk
            // checks one vertex plane beyond the footprint's reach
            long long f0[3], f1[3];
            footprint_box(whole, b.obs, *grid, chi_a[i], chi_b[i], f0, f1);
            for (int a = 0; a < 3; ++a) {
                f0[a] -= 1;
                f1[a] += 1;
            }
            if (!box_holds(bb, f0, f1, *grid)) return RR_ERR_ARG;
        }
    }
    if (!fused) {
        // other forms: one launch per step (the same results)
        for (int32_t i = 0; i < nsteps; ++i) {
            rr_status st = rr_trace_step(ctx, grid, rec[i], chi_a[i], chi_b[i], scale[i], a_step[i], stream);
            if (st != RR_OK) return st;
        }
        return RR_OK;
    }
    // validate every step in order (each continuing the previous one) before
    // anything is launched; the log takes them only if all pass
    const size_t log0 = ctx->log.size();
    const bool reloc0 = ctx->relocated;
    for (int32_t i = 0; i < nsteps; ++i) {
        rr_status st = validate_step(ctx, grid, rec[i], chi_a[i], chi_b[i], scale[i], a_step[i]);
        if (st != RR_OK) {
            ctx->log.resize(log0);
            ctx->relocated = reloc0;
            return st;
        }
        ctx->log.push_back(make_step_record(ctx, grid, chi_a[i], chi_b[i], scale[i], a_step[i]));
        ctx->relocated = false;
    }
    const TraceArgs a0 = make_trace_args(ctx, grid, rec[0], chi_a[0], chi_b[0], scale[0], a_step[0]);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    // blocks of up to kMaxStepBlock steps that all take the flat addressing
    // (trilinear) or any steps (NGP) go to one launch each; a trilinear step
    // outside the flat range is launched on its own
    int32_t i = 0;
    while (i < nsteps && e == cudaSuccess) {
        const bool tri = b.interp == RR_TRILINEAR;
        auto flat_at = [&](int32_t k) { return boxes || flat_ok(whole, b.obs, *grid, chi_a[k], chi_b[k]); };
        if (tri && !flat_at(i)) {
            const TraceArgs a = make_trace_args(ctx, grid, rec[i], chi_a[i], chi_b[i], scale[i], a_step[i]);
            e = launch_trace(a, b.interp, false, s, TileCfg{}, form, false);
            ++i;
            continue;
        }
        StepBlock blk{};
        blk.n = 0;
        while (i < nsteps && blk.n < kMaxStepBlock && (!tri || flat_at(i))) {
            const TraceArgs a = make_trace_args(ctx, grid, rec[i], chi_a[i], chi_b[i], scale[i], a_step[i]);
            StepArgs& st = blk.s[blk.n++];
            st.rec = a.rec;
            st.chi_a = a.chi_a; st.chi_b = a.chi_b;
            st.cah = a.cah; st.cal = a.cal; st.Lf = a.Lf; st.D0f = a.D0f;
            st.sch = a.sch; st.scl = a.scl; st.bsh = a.bsh; st.bsl = a.bsl;
            for (int q = 0; q < 3; ++q) {
                st.fo[q] = a.fo[q];
                st.fe[q] = a.fe[q];
            }
            st.fs0 = a.fs0;
            st.fs1 = a.fs1;
            if (boxes) {
                const int32_t* bb = boxes + 6 * (size_t)i;
                for (int q = 0; q < 3; ++q) {
                    st.fo[q] = (int)(((bb[2 * q] % grid->n[q]) + grid->n[q]) % grid->n[q]);
                    st.fe[q] = bb[2 * q + 1] - bb[2 * q];
                }
                st.fs0 = st.fe[1] * st.fe[2];
                st.fs1 = st.fe[2];
            }
            ++i;
        }
        e = launch_trace_steps(a0, blk, b.interp, tri, s, form);
    }
    return from_cuda(e);
}

rr_status rr_sync_status(rr_ctx* ctx, void* stream)
{
    if (!ctx) return RR_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(ctx->host_err, ctx->st.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return from_cuda(e);
    return status_from_word(*ctx->host_err);
}

rr_status rr_finalize(rr_ctx* ctx, double* kappa, double* kappa_born, void* stream)
{
    if (!ctx || !kappa) return RR_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int nr = ctx->bundle.nx * ctx->bundle.ny;
    cudaError_t e = launch_finalize(nr, ctx->st.kacc, ctx->st.bacc, ctx->st.nseg, kappa, kappa_born,
                                    ctx->st.total, s, ctx->st.kmom, ctx->st.bmom, ctx->bundle.chi_s,
                                    (ctx->bundle.flags & RR_METHOD_A) != 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->host_total, ctx->st.total, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return from_cuda(e);
    rr_status st = rr_sync_status(ctx, stream);
    ctx->last_total = *ctx->host_total;
    return st;
}

rr_status rr_segment_count(rr_ctx* ctx, uint64_t* total, uint32_t* per_ray, void* stream)
{
    if (!ctx) return RR_ERR_ARG;
    if (total) *total = ctx->last_total;
    if (per_ray) {
        const size_t nr = (size_t)ctx->bundle.nx * ctx->bundle.ny;
        return from_cuda(cudaMemcpyAsync(per_ray, ctx->st.nseg, nr * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                                         (cudaStream_t)stream));
    }
    return RR_OK;
}

rr_status rr_moments(rr_ctx* ctx, double* out, void* stream)
{
    if (!ctx || !out) return RR_ERR_ARG;
    if (!ctx->st.kmom) return RR_ERR_STATE;
    const int nr = ctx->bundle.nx * ctx->bundle.ny;
    return from_cuda(launch_moments(nr, ctx->st.kacc, ctx->st.kmom, ctx->st.bacc, ctx->st.bmom, out,
                                    (cudaStream_t)stream));
}

rr_status rr_shear(rr_ctx* ctx, double* gamma1, double* gamma2, void* stream)
{
    if (!ctx || !gamma1 || !gamma2) return RR_ERR_ARG;
    if (!ctx->st.g1acc) return RR_ERR_STATE;
    const int nr = ctx->bundle.nx * ctx->bundle.ny;
    return from_cuda(launch_shear_out(nr, ctx->st.g1acc, ctx->st.g2acc, gamma1, gamma2, (cudaStream_t)stream));
}

rr_status rr_source_kappa(const double* m_end, const double* m_k, int64_t nrays, double chi_k, double* kappa,
                          double* kappa_born, void* stream)
{
    if (!m_end || !kappa || nrays < 1 || !is_finite(chi_k) || !(chi_k > 0)) return RR_ERR_ARG;
    return from_cuda(launch_source_kappa(m_end, m_k, (long long)nrays, chi_k, kappa, kappa_born,
                                         (cudaStream_t)stream));
}

rr_status rr_step_count(rr_ctx* ctx, int32_t* n)
{
    if (!ctx || !n) return RR_ERR_ARG;
    *n = (int32_t)ctx->log.size();
    return RR_OK;
}

rr_status rr_trace_step_adjoint(rr_ctx* ctx, int32_t step, const double* dL_dkappa, const double* dL_dkborn,
                                float* grad_rec, void* stream)
{
    if (!ctx || !grad_rec || !is_aligned16(grad_rec)) return RR_ERR_ARG;
    if (!dL_dkappa && !dL_dkborn) return RR_ERR_ARG;
    if (step < 0 || step >= (int32_t)ctx->log.size()) return RR_ERR_STATE;
    const StepRecord& r = ctx->log[(size_t)step];
    if (r.amr || (ctx->bundle.flags & (RR_SOURCE_MOMENTS | RR_METHOD_A | RR_GENERIC))) return RR_ERR_STATE;
    // the records pointer is not read by the adjoint (it needs geometry only);
    // the step is replayed from the observer it was traced from
    TraceArgs a = make_trace_args(ctx, &r.grid, grad_rec, r.chi_a, r.chi_b, r.scale, r.a_step, r.obs);
    AdjArgs g;
    g.dkappa = dL_dkappa;
    g.dkborn = dL_dkborn;
    g.grad = reinterpret_cast<double*>(grad_rec);
    g.kscale = r.scale;
    g.bscale = r.scale * 1.5 * r.grid.omega_m * kH0OverC * kH0OverC / r.a_step;
    return from_cuda(launch_trace_adjoint(a, g, ctx->bundle.interp, (ctx->bundle.flags & RR_FP64_DDA) != 0,
                                          (cudaStream_t)stream));
}

rr_status rr_tidal_tensor_adjoint(const rr_grid_desc* grid, const float* grad_rec, int32_t where, float* dL_dphi,
                                  float* dL_ddelta, void* stream)
{
    rr_status st = check_grid(grid);
    if (st != RR_OK) return st;
    if (!grad_rec || !is_aligned16(grad_rec) || !dL_dphi) return RR_ERR_ARG;
    if (where != RR_AT_VERTICES && where != RR_AT_CENTRES) return RR_ERR_ARG;
    return from_cuda(launch_tidal_adjoint(*grid, grad_rec, where, dL_dphi, dL_ddelta, (cudaStream_t)stream));
}

rr_status rr_trace_backward(rr_ctx* ctx, const double* dL_dkappa, const double* dL_dkborn, float* grad_rec,
                            float* dL_dphi, float* dL_ddelta, void* stream)
{
    if (!ctx || !grad_rec || !dL_dphi) return RR_ERR_ARG;
    if (!dL_dkappa && !dL_dkborn) return RR_ERR_ARG;
    if (ctx->log.empty()) return RR_ERR_STATE;
    const rr_grid_desc& g = ctx->log.front().grid;
    for (const StepRecord& r : ctx->log)
        if (r.amr || r.grid.n[0] != g.n[0] || r.grid.n[1] != g.n[1] || r.grid.n[2] != g.n[2] || r.grid.box != g.box ||
            r.grid.omega_m != g.omega_m)
            return RR_ERR_STATE;
    if (!is_aligned16(grad_rec)) return RR_ERR_ARG;
    // The adjoint of a step adds only to the points its rays' cells touch,
    // which lie in the step's footprint box (the box the forward computes its
    // records over), so only the union U of those boxes is non-zero and only
    // the cells within the stencils' reach of U get a gradient. Vertices: a
    // cell's dL/dPhi reads the records of the points m - 1 .. m + 2 per axis
    // (the 8-vertex mean, then the +-1 central differences), so the output
    // box is U widened by 2 below and 1 above, and the records it reads (all
    // zeroed here) U widened by 3 on both sides; centres: 1 and 1, 2 and 2.
    rr_bundle_desc whole = ctx->bundle;
    whole.ny = ctx->ny_full;
    long long u0[3], u1[3];
    for (size_t k = 0; k < ctx->log.size(); ++k) {
        const StepRecord& r = ctx->log[k];
        long long b0[3], b1[3];
        footprint_box(whole, r.obs, r.grid, r.chi_a, r.chi_b, b0, b1);
        for (int a = 0; a < 3; ++a) {
            u0[a] = k ? std::min(u0[a], b0[a]) : b0[a];
            u1[a] = k ? std::max(u1[a], b1[a]) : b1[a];
        }
    }
    const bool vert = ctx->bundle.interp == RR_TRILINEAR;
    long long z0[3], z1[3], o0[3], o1[3];
    for (int a = 0; a < 3; ++a) {
        z0[a] = u0[a] - (vert ? 3 : 2);
        z1[a] = u1[a] + (vert ? 3 : 2);
        o0[a] = u0[a] - (vert ? 2 : 1);
        o1[a] = u1[a] + 1;
    }
    cudaError_t e = zero_grad_records(g, grad_rec, z0, z1, (cudaStream_t)stream);
    if (e != cudaSuccess) return from_cuda(e);
    for (int32_t k = 0; k < (int32_t)ctx->log.size(); ++k) {
        rr_status st = rr_trace_step_adjoint(ctx, k, dL_dkappa, dL_dkborn, grad_rec, stream);
        if (st != RR_OK) return st;
    }
    return from_cuda(launch_tidal_adjoint(g, grad_rec, vert ? RR_AT_VERTICES : RR_AT_CENTRES, dL_dphi, dL_ddelta,
                                          (cudaStream_t)stream, o0, o1));
}

}  // extern "C"
