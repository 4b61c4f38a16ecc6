// Internal declarations shared by the translation units of librr.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "rr.h"

namespace rr {

constexpr double kH0OverC = 1.0 / 2997.92458;  // h/Mpc

// Bits of the device error word.
enum : uint32_t { kErrStepLimit = 1u, kErrNonFinite = 2u };

// Per-ray state, structure of arrays, indexed by ray id (Eq. rayid).
struct RayState {
    double* dir = nullptr;      // 3 per ray: n_hat (Eq. raypos), FP64
    double* kappa = nullptr;    // FP64 accumulators across steps
    double* kborn = nullptr;
    uint32_t* nseg = nullptr;   // non-empty segments since reset
    uint32_t* err = nullptr;    // device error word
    unsigned long long* total = nullptr;  // segment total written by finalize
};

struct StepRecord {
    rr_grid_desc grid;
    double chi_a, chi_b, scale, a_step;
};

// Geometry of one step, handed to the trace kernels by value.
struct TraceArgs {
    const float4* rec;          // 2 float4 per point
    int n0, n1, n2;
    double h;                   // cell size
    double inv_h;
    int nx, ny;                 // rays
    double obs0, obs1, obs2;
    double chi_s, chi_a, chi_b;
    int periodic;
    const double* dir;
    double* kappa;
    double* kborn;
    uint32_t* nseg;
    uint32_t* err;
    double scale;               // multiplies kappa and born sums
    double born_pref;           // 1.5 Omega_m (H0/c)^2 / a_step
};

// Launchers (one per translation unit).
cudaError_t launch_init_directions(const rr_bundle_desc& b, double* dir, cudaStream_t s);
cudaError_t launch_tidal(const rr_grid_desc& g, const float* phi, const float* delta, float* rec, int where,
                         const int32_t* bbox, cudaStream_t s);
cudaError_t launch_trace(const TraceArgs& a, int interp, bool fp64_dda, cudaStream_t s);
cudaError_t launch_finalize(int nrays, const double* kappa, const double* kborn, const uint32_t* nseg,
                            double* out_kappa, double* out_kborn, unsigned long long* total, cudaStream_t s);

}  // namespace rr

struct rr_ctx {
    rr_bundle_desc bundle;
    rr::RayState st;
    int device = 0;
    std::vector<rr::StepRecord> log;
    unsigned long long last_total = 0;
    uint32_t* host_err = nullptr;             // pinned
    unsigned long long* host_total = nullptr; // pinned
};
