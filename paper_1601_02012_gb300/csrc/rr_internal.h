// Internal declarations shared by the translation units of librr.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "rr.h"

namespace rr {

constexpr double kH0OverC = 1.0 / 2997.92458;  // h/Mpc

// Bits of the device error word.
// kErrRange: a ray of a step launched with flat (no-wrap) record addressing
// would have left the index range that addressing covers; it read nothing.
enum : uint32_t { kErrStepLimit = 1u, kErrNonFinite = 2u, kErrRange = 4u };

// Per-ray state, structure of arrays, indexed by ray id (Eq. rayid).
struct RayState {
    double* dir = nullptr;      // 3 per ray: n_hat (Eq. raypos), FP64
    float4* dirh = nullptr;     // n_hat rounded to FP32 (x, y, z, 0)
    float4* dirl = nullptr;     // n_hat - dirh rounded to FP32 (float-float low parts)
    float2* kacc = nullptr;     // kappa accumulated across steps, float-float (hi, lo); A moment (moments form)
    float2* bacc = nullptr;     // Born kappa, float-float; Born A moment (moments form)
    float2* kmom = nullptr;     // moments form only: B moment of kappa, float-float
    float2* bmom = nullptr;     // moments form only: B moment of Born kappa
    float2* g1acc = nullptr;    // shear form only: gamma1, float-float
    float2* g2acc = nullptr;    // shear form only: gamma2, float-float
    uint32_t* nseg = nullptr;   // non-empty segments since reset
    uint32_t* err = nullptr;    // device error word
    unsigned long long* total = nullptr;  // segment total written by finalize
};

struct StepRecord {
    rr_grid_desc grid;
    double chi_a, chi_b, scale, a_step;
    int amr = 0;                // traced over an adaptive mesh (no adjoint)
    double obs[3] = {0, 0, 0};  // the observer the step was traced from
};

constexpr int kAmrMaxLevel = 8;

// Adaptive mesh as the trace kernel reads it. link[cell] >= 0: the cell is a
// leaf with that id; link[cell] < 0: refined, its 8 children are the cells
// -link - 1 + (dx + 2 dy + 4 dz).
struct AmrDevice {
    const int32_t* link;
    int n;                      // coarse cells per side
    int lmax;
};

// Geometry of one step, handed to the trace kernels by value. Doubles are
// also given as float-float pairs (hi = (float)x, lo = (float)(x - hi)).
struct TraceArgs {
    const float4* rec;          // 2 float4 per point
    int n0, n1, n2;
    double h;                   // cell size
    double inv_h;
    float inv_hf;               // 1/h rounded to FP32
    float ihh, ihl;             // 1/h as float-float
    int nx, ny;                 // rays
    double obs0, obs1, obs2;
    float oh[3], ol[3];         // observer as float-float
    double chi_s, chi_a, chi_b;
    float cah, cal;             // chi_a as float-float
    float Lf;                   // chi_a - chi_b rounded to FP32
    float D0f;                  // chi_s - chi_a rounded to FP32
    float inv_chi_s_f;          // 1/chi_s rounded to FP32
    float sub_len;              // FP32 walk: longest sub-step (32 cell sizes)
    int periodic;
    const double* dir;
    const float4* dirh;
    const float4* dirl;
    float2* kacc;
    float2* bacc;
    float2* kmom;               // B moments (moments form), else unused
    float2* bmom;
    float2* g1acc;              // gamma1, gamma2 (shear form), else unused
    float2* g2acc;
    float kq[6];                // generic form: K_c(chi) = kq[3c] + kq[3c+1] chi + kq[3c+2] chi^2
    uint32_t* nseg;
    uint32_t* err;
    float sch, scl;             // scale (multiplies the kappa step sum), float-float
    float bsh, bsl;             // scale * 1.5 Omega_m (H0/c)^2 / a_step, float-float
    // flat record addressing: the records cover the box of points fo .. fo +
    // fe - 1 per axis (fo in [0, n), periodic), point (i, j, k) of the box at
    // i fs0 + j fs1 + k; the whole grid: fo = 0, fe = n, fs0 = n1 n2, fs1 = n2
    int fo[3], fe[3];
    int fs0, fs1;
};

// The per-step fields of TraceArgs for a launch over several consecutive
// steps (trace_steps_kernel); the other fields are shared.
struct StepArgs {
    const float4* rec;
    double chi_a, chi_b;
    float cah, cal, Lf, D0f;
    float sch, scl, bsh, bsl;
    int fo[3], fe[3];
    int fs0, fs1;
};
constexpr int kMaxStepBlock = 16;
struct StepBlock {
    int n;
    StepArgs s[kMaxStepBlock];
};

// Adjoint of one step: per-ray derivatives of the loss and the gradient
// records (8 FP64 sums per point, in the channel order of the records).
struct AdjArgs {
    const double* dkappa;       // dL/dkappa per ray, or NULL
    const double* dkborn;       // dL/dkappa_born per ray, or NULL
    double* grad;
    double kscale;              // the step's scale
    double bscale;              // scale * 1.5 Omega_m (H0/c)^2 / a_step
};

// Ray-tile shape: a warp covers wx x (32/wx) pixels, a block bwx x bwy warps.
struct TileCfg {
    int wx = 8, bwx = 2, bwy = 2;
};

// Arguments of the persistent batched trace (device pointers).
struct BatchArgs {
    const TraceArgs* cones;     // per bundle
    const int* tile_start;      // ncones + 1 prefix offsets of the ray tiles
    const int* tiles_x;         // tiles along x per bundle
    int ncones;
    int* counter;               // work counter, zeroed before each launch
    int chunk;                  // tiles taken per counter increment
    TileCfg tile;
};

// Launchers (one per translation unit).
// Directions of the rows [row0, row0 + nrows) of bundle b (all rows: nrows < 0).
cudaError_t launch_init_directions(const rr_bundle_desc& b, double* dir, float4* dirh, float4* dirl, cudaStream_t s,
                                   int row0 = 0, int nrows = -1);
// kind 0: tidal records (2 float4 per point); kind 1: gradient records (1 float4)
// compact (with a bbox): the records stored box-local, point (i, j, k) of the
// box at (i ey + j) ez + k
cudaError_t launch_tidal(const rr_grid_desc& g, const float* phi, const float* delta, float* rec, int where,
                         const int32_t* bbox, cudaStream_t s, int kind = 0, bool compact = false);
cudaError_t launch_trace(const TraceArgs& a, int interp, bool fp64_dda, cudaStream_t s);
// Forms of the FP32 walk's sums.
enum { kFormKahan = 0, kFormPlain = 1, kFormMoments = 2, kFormShear = 3, kFormMethodA = 4, kFormGeneric = 5 };
// Record addressing of the trilinear walk (see trace.cu).
enum { kAddrIndex = 0, kAddrPlanes = 1, kAddrFlat = 2 };
// flat: the caller has checked that no ray of the step comes within a cell of
// the periodic seam and that the grid has fewer than 2^31 points (used by the
// default FP32 trilinear periodic form only; ignored otherwise).
cudaError_t launch_trace(const TraceArgs& a, int interp, bool fp64_dda, cudaStream_t s, const TileCfg& t,
                         int form = kFormKahan, bool flat = false);
cudaError_t launch_trace_batch(const BatchArgs& b, int interp, bool fp64_dda, int blocks, cudaStream_t s);
// Steps b.s[0 .. b.n) of an FP32 compensated form (kFormKahan, kFormShear,
// kFormMoments, kFormMethodA, kFormGeneric) in one launch; a holds the shared
// fields. flat: every step passed the flat-addressing check (trilinear).
cudaError_t launch_trace_steps(const TraceArgs& a, const StepBlock& b, int interp, bool flat, cudaStream_t s,
                               int form = kFormKahan);
int batch_blocks_per_sm(int interp, bool fp64_dda, const TileCfg& t);
dim3 tile_grid(const TileCfg& t, int nx, int ny);
bool tile_ok(const TileCfg& t);
// form: kFormKahan, kFormShear (also gamma1, gamma2 into g1acc, g2acc) or kFormMethodA
cudaError_t launch_trace_amr(const TraceArgs& a, const AmrDevice& m, int interp, cudaStream_t s, int form = 0);
// Steps b.s[0 .. b.n) over the adaptive mesh in one launch (kFormKahan,
// kFormShear, kFormMethodA, kFormGeneric)
cudaError_t launch_trace_amr_steps(const TraceArgs& a, const AmrDevice& m, const StepBlock& b, int interp,
                                   cudaStream_t s, int form = kFormKahan);
cudaError_t launch_trace_adjoint(const TraceArgs& a, const AdjArgs& b, int interp, bool fp64_dda, cudaStream_t s);
// The transposed stencils over the output box [box0, box1) per axis (point
// indices, unwrapped; an axis whose extent reaches n, or no box, is whole):
// dL/dPhi is accumulated only there.
cudaError_t launch_tidal_adjoint(const rr_grid_desc& g, const float* grad_rec, int where, float* dphi, float* ddelta,
                                 cudaStream_t s, const long long* box0 = nullptr, const long long* box1 = nullptr);
// Zero the gradient records (64 B per point) of the points in [box0, box1)
// per axis (unwrapped point indices; an axis whose extent reaches n is whole).
cudaError_t zero_grad_records(const rr_grid_desc& g, float* grad_rec, const long long* box0, const long long* box1,
                              cudaStream_t s);
cudaError_t launch_finalize(int nrays, const float2* kacc, const float2* bacc, const uint32_t* nseg,
                            double* out_kappa, double* out_kborn, unsigned long long* total, cudaStream_t s,
                            const float2* kmom = nullptr, const float2* bmom = nullptr, double chi_s = 0.0,
                            bool add_born = false);
cudaError_t launch_moments(int nrays, const float2* kacc, const float2* kmom, const float2* bacc, const float2* bmom,
                           double* out, cudaStream_t s);
cudaError_t launch_shear_out(int nrays, const float2* g1acc, const float2* g2acc, double* gamma1, double* gamma2,
                             cudaStream_t s);
// Scalar-pair records of the generic form: channel `channel` (0 or 1) of the
// float2 records = field, or (field - prev) * inv_dt, at vertices or centres.
cudaError_t launch_scalar_records(const rr_grid_desc& g, const float* field, const float* prev, float inv_dt,
                                  int channel, float* rec, int where, const int32_t* bbox, cudaStream_t s);
cudaError_t launch_source_kappa(const double* m_end, const double* m_k, long long nrays, double chi_k, double* kappa,
                                double* kborn, cudaStream_t s);

// The step geometry and a context's state pointers as the kernels take them.
// (obs: the observer to trace from; NULL: the context's current one)
TraceArgs make_trace_args(rr_ctx* ctx, const rr_grid_desc* grid, const float* rec, double chi_a, double chi_b,
                          double scale, double a_step, const double* obs = nullptr);
// The same for a bundle and per-ray state held outside a context (kq: the
// generic form's six kernel coefficients, or NULL for the lensing kernel g).
TraceArgs make_trace_args(const rr_bundle_desc& b, const RayState& st, const rr_grid_desc* grid, const float* rec,
                          double chi_a, double chi_b, double scale, double a_step, const double* obs,
                          const double* kq);
// Index box [i0, i1) per axis of the cells the rays of bundle b (observer
// obs) can reach between chi_b and chi_a, widened by 1 cell below and 2
// above, without any wrap or clamp (the values may lie outside [0, n)).
void footprint_box(const rr_bundle_desc& b, const double obs[3], const rr_grid_desc& g, double chi_a,
                   double chi_b, long long i0[3], long long i1[3]);
// Whether a step of bundle b (observer obs) on grid g can use flat record
// addressing: periodic trilinear FP32 walk, fewer than 2^31 points, and every
// position the rays take in the step at least 2 cells from the periodic seam
// below and 3 above on every axis (no vertex plane the walk reads lies
// across the seam).
bool flat_ok(const rr_bundle_desc& b, const double obs[3], const rr_grid_desc& g, double chi_a, double chi_b);
// Argument checks of a bundle and a grid description (RR_OK or RR_ERR_ARG).
rr_status check_bundle(const rr_bundle_desc* b);
rr_status check_grid(const rr_grid_desc* g);
// The log entry of a step traced now from the context's current observer.
StepRecord make_step_record(const rr_ctx* ctx, const rr_grid_desc* grid, double chi_a, double chi_b, double scale,
                            double a_step);
// Argument and step-order checks of rr_trace_step.
rr_status validate_step(rr_ctx* ctx, const rr_grid_desc* grid, const float* rec, double chi_a, double chi_b,
                        double scale, double a_step);
rr_status status_of_cuda(cudaError_t e);

// hi = (float)x, lo = (float)(x - hi)
inline void split_ff(double x, float& hi, float& lo)
{
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

}  // namespace rr

struct rr_ctx {
    // The context's own rays: rows [row0, row0 + bundle.ny) of a bundle of
    // ny_full rows (rr_create_band; rr_create: row0 = 0, ny_full = bundle.ny).
    // Sizes and kernels use bundle.ny; directions and footprints use ny_full.
    rr_bundle_desc bundle;
    int row0 = 0;
    int ny_full = 0;
    rr::RayState st;
    int device = 0;
    std::vector<rr::StepRecord> log;
    unsigned long long last_total = 0;
    uint32_t* host_err = nullptr;             // pinned
    unsigned long long* host_total = nullptr; // pinned
    bool relocated = false;                   // observer moved since the last step: no continuity check
    double kq[6] = {0, 1, 0, 0, 1, 0};        // generic form kernels (set at create and by rr_set_kernels)
};
