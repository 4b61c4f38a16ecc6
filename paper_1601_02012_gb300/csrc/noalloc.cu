// rr_trace_step_noalloc: one trace step whose scratch lives in a fixed device
// array of this library instead of memory the library allocates.
//
// The regular path (rr_create + rr_trace_step + rr_finalize) keeps the per-ray
// state in device memory it obtains with cudaMalloc. Some callers cannot let a
// library allocate: a host framework may already own the whole device memory
// pool through its own allocator, or the caller may be in a section where the
// implicit device synchronisation of cudaMalloc/cudaFree is not acceptable, or
// a plugin host may forbid driver allocations outright. For them this entry
// point uses a file-scope __device__ array (kNoAllocBytes, a few MB, held by
// every GPU that loads the library until the process exits) for the per-ray
// directions, accumulators, segment counters and error word.
#include <cmath>
#include <mutex>

#include "rr_internal.h"

using namespace rr;

namespace {

constexpr size_t kMaxRays = RR_NOALLOC_MAX_RAYS;
constexpr size_t kSlot = 256;  // every sub-array starts on a 256-byte boundary

constexpr size_t align_up(size_t x) { return (x + kSlot - 1) / kSlot * kSlot; }

// byte offsets of the sub-arrays inside the scratch
constexpr size_t kOffErr = 0;
constexpr size_t kOffTotal = kOffErr + kSlot;
constexpr size_t kOffDir = kOffTotal + kSlot;
constexpr size_t kOffDirh = kOffDir + align_up(kMaxRays * 3 * sizeof(double));
constexpr size_t kOffDirl = kOffDirh + align_up(kMaxRays * sizeof(float4));
constexpr size_t kOffKacc = kOffDirl + align_up(kMaxRays * sizeof(float4));
constexpr size_t kOffBacc = kOffKacc + align_up(kMaxRays * sizeof(float2));
constexpr size_t kOffNseg = kOffBacc + align_up(kMaxRays * sizeof(float2));
constexpr size_t kNoAllocBytes = kOffNseg + align_up(kMaxRays * sizeof(uint32_t));

// The scratch. In host code this name is only a host-side stand-in for the
// device symbol, never a device address: the address kernels need comes from
// cudaGetSymbolAddress below, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device (set up on the first
// call on that device).
cudaError_t scratch_on_current_device(unsigned char** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

rr_status to_status(cudaError_t e)
{
    return e == cudaSuccess ? RR_OK : RR_ERR_CUDA;
}

}  // namespace

extern "C" rr_status rr_trace_step_noalloc(const rr_bundle_desc* bundle, const rr_grid_desc* grid,
                                           const float* rec, double chi_a, double chi_b, double scale,
                                           double a_step, double* kappa, double* kappa_born, void* stream)
{
    // the argument checks of rr_create and rr_trace_step, without the step-order check
    if (!kappa) return RR_ERR_ARG;
    rr_status st = check_bundle(bundle);
    if (st == RR_OK) st = check_grid(grid);
    if (st != RR_OK) return st;
    if (bundle->flags & ~(RR_PERIODIC | RR_FP64_DDA)) return RR_ERR_ARG;
    if ((size_t)bundle->nx * (size_t)bundle->ny > kMaxRays) return RR_ERR_CAPACITY;
    if (!rec || ((uintptr_t)rec & 31u) != 0) return RR_ERR_ARG;
    if (!std::isfinite(chi_a) || !std::isfinite(chi_b) || !std::isfinite(scale) || !std::isfinite(a_step) ||
        !(a_step > 0))
        return RR_ERR_ARG;
    if (!(chi_a > chi_b) || !(chi_b >= 0) || chi_a > bundle->chi_s * (1.0 + 1e-12)) return RR_ERR_ARG;

    unsigned char* base = nullptr;
    cudaError_t e = scratch_on_current_device(&base);
    if (e != cudaSuccess) return to_status(e);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nr = (size_t)bundle->nx * bundle->ny;
    uint32_t* err = reinterpret_cast<uint32_t*>(base + kOffErr);
    unsigned long long* total = reinterpret_cast<unsigned long long*>(base + kOffTotal);
    double* dir = reinterpret_cast<double*>(base + kOffDir);
    float4* dirh = reinterpret_cast<float4*>(base + kOffDirh);
    float4* dirl = reinterpret_cast<float4*>(base + kOffDirl);
    float2* kacc = reinterpret_cast<float2*>(base + kOffKacc);
    float2* bacc = reinterpret_cast<float2*>(base + kOffBacc);
    uint32_t* nseg = reinterpret_cast<uint32_t*>(base + kOffNseg);

    // The array keeps the previous call's contents: clear what accumulates.
    e = cudaMemsetAsync(err, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(kacc, 0, nr * sizeof(float2), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bacc, 0, nr * sizeof(float2), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(nseg, 0, nr * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = launch_init_directions(*bundle, dir, dirh, dirl, s);
    if (e != cudaSuccess) return to_status(e);

    RayState rs;
    rs.dir = dir;
    rs.dirh = dirh;
    rs.dirl = dirl;
    rs.kacc = kacc;
    rs.bacc = bacc;
    rs.nseg = nseg;
    rs.err = err;
    rs.total = total;
    const TraceArgs a = make_trace_args(*bundle, rs, grid, rec, chi_a, chi_b, scale, a_step, nullptr, nullptr);
    e = launch_trace(a, bundle->interp, (bundle->flags & RR_FP64_DDA) != 0, s);
    if (e == cudaSuccess) e = launch_finalize((int)nr, kacc, bacc, nseg, kappa, kappa_born, total, s);
    if (e != cudaSuccess) return to_status(e);

    uint32_t word = 0;
    e = cudaMemcpyAsync(&word, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return to_status(e);
    if (word & kErrStepLimit) return RR_ERR_STEP_LIMIT;
    if (word & kErrNonFinite) return RR_ERR_NONFINITE;
    if (word & kErrRange) return RR_ERR_RANGE;
    return RR_OK;
}
