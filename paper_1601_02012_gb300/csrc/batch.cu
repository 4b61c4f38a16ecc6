// Many bundles (lightcones) in one persistent launch, and the autotuner that
// picks its ray-tile shape, block size and queue chunk.
//
// Each bundle keeps its own rr_ctx (per-ray state, step log). A step of the
// batch is staged on the host (rr_batch_set_step for every bundle), copied to
// the device as one table of kernel arguments (rr_batch_upload), and traced by
// one persistent launch whose blocks pull ray tiles of all bundles from a
// device counter (rr_batch_trace). Upload, trace and finalize only enqueue
// work on the stream (no synchronisation), so a caller can capture them, and
// the tidal calls of the bundles, in one CUDA graph and replay it.
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "rr_internal.h"

using namespace rr;

struct rr_batch {
    std::vector<rr_ctx*> cones;
    int interp = RR_TRILINEAR;
    bool fp64 = false;
    TileCfg tile;
    int chunk = 1;
    int blocks_per_sm = 0;       // 0: as many as fit (occupancy)
    int sms = 1;
    std::vector<bool> staged;
    // host staging (pinned) and its device copy
    TraceArgs* h_args = nullptr;
    int* h_tiles = nullptr;      // tile_start[n+1] then tiles_x[n]
    TraceArgs* d_args = nullptr;
    int* d_tiles = nullptr;
    int* d_counter = nullptr;
    int total_tiles = 0;
};

namespace {

void free_batch(rr_batch* b)
{
    for (rr_ctx* c : b->cones)
        if (c) rr_destroy(c);
    cudaFreeHost(b->h_args);
    cudaFreeHost(b->h_tiles);
    cudaFree(b->d_args);
    cudaFree(b->d_tiles);
    cudaFree(b->d_counter);
    delete b;
}

// Fill the tile tables for the current tile shape.
void build_tiles(rr_batch* b)
{
    const int n = (int)b->cones.size();
    int acc = 0;
    for (int i = 0; i < n; ++i) {
        const dim3 g = tile_grid(b->tile, b->cones[i]->bundle.nx, b->cones[i]->bundle.ny);
        b->h_tiles[i] = acc;
        b->h_tiles[n + 1 + i] = (int)g.x;
        acc += (int)(g.x * g.y);
    }
    b->h_tiles[n] = acc;
    b->total_tiles = acc;
}

int grid_blocks(const rr_batch* b)
{
    const int per_sm = b->blocks_per_sm > 0 ? b->blocks_per_sm : batch_blocks_per_sm(b->interp, b->fp64, b->tile);
    long long blocks = (long long)per_sm * b->sms;
    if (blocks > b->total_tiles) blocks = b->total_tiles;
    return blocks < 1 ? 1 : (int)blocks;
}

}  // namespace

extern "C" {

rr_status rr_batch_create(int32_t n, const rr_bundle_desc* bundles, rr_batch** out)
{
    if (!out || !bundles || n < 1 || n > (1 << 16)) return RR_ERR_ARG;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (bundles[i].interp != bundles[0].interp) return RR_ERR_ARG;
        if ((bundles[i].flags & RR_FP64_DDA) != (bundles[0].flags & RR_FP64_DDA)) return RR_ERR_ARG;
        if (bundles[i].flags & (RR_PLAIN_SUMS | RR_SOURCE_MOMENTS | RR_SHEAR | RR_METHOD_A | RR_GENERIC))
            return RR_ERR_ARG;
    }
    rr_batch* b = new (std::nothrow) rr_batch();
    if (!b) return RR_ERR_OOM;
    b->interp = bundles[0].interp;
    b->fp64 = (bundles[0].flags & RR_FP64_DDA) != 0;
    b->cones.assign((size_t)n, nullptr);
    b->staged.assign((size_t)n, false);
    for (int i = 0; i < n; ++i) {
        rr_status st = rr_create(&bundles[i], &b->cones[(size_t)i]);
        if (st != RR_OK) {
            free_batch(b);
            return st;
        }
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (b->sms < 1) b->sms = 1;
    cudaError_t e = cudaMallocHost(&b->h_args, sizeof(TraceArgs) * (size_t)n);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_tiles, sizeof(int) * (size_t)(2 * n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_args, sizeof(TraceArgs) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tiles, sizeof(int) * (size_t)(2 * n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(int));
    if (e != cudaSuccess) {
        free_batch(b);
        return status_of_cuda(e);
    }
    memset(b->h_args, 0, sizeof(TraceArgs) * (size_t)n);
    build_tiles(b);
    *out = b;
    return RR_OK;
}

rr_status rr_batch_destroy(rr_batch* b)
{
    if (!b) return RR_ERR_ARG;
    cudaDeviceSynchronize();
    free_batch(b);
    return RR_OK;
}

rr_status rr_batch_size(rr_batch* b, int32_t* n)
{
    if (!b || !n) return RR_ERR_ARG;
    *n = (int32_t)b->cones.size();
    return RR_OK;
}

rr_status rr_batch_context(rr_batch* b, int32_t i, rr_ctx** ctx)
{
    if (!b || !ctx || i < 0 || i >= (int32_t)b->cones.size()) return RR_ERR_ARG;
    *ctx = b->cones[(size_t)i];
    return RR_OK;
}

rr_status rr_batch_reset(rr_batch* b, void* stream)
{
    if (!b) return RR_ERR_ARG;
    for (size_t i = 0; i < b->cones.size(); ++i) {
        rr_status st = rr_reset(b->cones[i], stream);
        if (st != RR_OK) return st;
        b->staged[i] = false;
    }
    return RR_OK;
}

rr_status rr_batch_clear(rr_batch* b, void* stream)
{
    if (!b) return RR_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    for (rr_ctx* c : b->cones) {
        const size_t nr = (size_t)c->bundle.nx * c->bundle.ny;
        cudaError_t e = cudaMemsetAsync(c->st.kacc, 0, nr * sizeof(float2), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->st.bacc, 0, nr * sizeof(float2), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->st.nseg, 0, nr * sizeof(uint32_t), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->st.err, 0, sizeof(uint32_t), s);
        if (e != cudaSuccess) return status_of_cuda(e);
    }
    return RR_OK;
}

rr_status rr_batch_set_step(rr_batch* b, int32_t i, const rr_grid_desc* grid, const float* rec, double chi_a,
                            double chi_b, double scale, double a_step)
{
    if (!b || i < 0 || i >= (int32_t)b->cones.size()) return RR_ERR_ARG;
    rr_ctx* c = b->cones[(size_t)i];
    rr_status st = validate_step(c, grid, rec, chi_a, chi_b, scale, a_step);
    if (st != RR_OK) return st;
    b->h_args[i] = make_trace_args(c, grid, rec, chi_a, chi_b, scale, a_step);
    c->log.push_back(make_step_record(c, grid, chi_a, chi_b, scale, a_step));
    b->staged[(size_t)i] = true;
    return RR_OK;
}

rr_status rr_batch_upload(rr_batch* b, void* stream)
{
    if (!b) return RR_ERR_ARG;
    for (size_t i = 0; i < b->staged.size(); ++i)
        if (!b->staged[i]) return RR_ERR_STATE;
    const int n = (int)b->cones.size();
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(b->d_args, b->h_args, sizeof(TraceArgs) * (size_t)n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_tiles, b->h_tiles, sizeof(int) * (size_t)(2 * n + 1), cudaMemcpyHostToDevice, s);
    return status_of_cuda(e);
}

rr_status rr_batch_trace(rr_batch* b, void* stream)
{
    if (!b) return RR_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)b->cones.size();
    cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return status_of_cuda(e);
    BatchArgs a;
    a.cones = b->d_args;
    a.tile_start = b->d_tiles;
    a.tiles_x = b->d_tiles + n + 1;
    a.ncones = n;
    a.counter = b->d_counter;
    a.chunk = b->chunk;
    a.tile = b->tile;
    return status_of_cuda(launch_trace_batch(a, b->interp, b->fp64, grid_blocks(b), s));
}

rr_status rr_batch_finalize(rr_batch* b, double* const* kappa, double* const* kappa_born, void* stream)
{
    if (!b || !kappa) return RR_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    for (size_t i = 0; i < b->cones.size(); ++i) {
        rr_ctx* c = b->cones[i];
        if (!kappa[i]) return RR_ERR_ARG;
        const int nr = c->bundle.nx * c->bundle.ny;
        cudaError_t e = launch_finalize(nr, c->st.kacc, c->st.bacc, c->st.nseg, kappa[i],
                                        kappa_born ? kappa_born[i] : nullptr, c->st.total, s);
        if (e != cudaSuccess) return status_of_cuda(e);
    }
    return RR_OK;
}

rr_status rr_batch_sync_status(rr_batch* b, uint64_t* total_segments, void* stream)
{
    if (!b) return RR_ERR_ARG;
    rr_status worst = RR_OK;
    uint64_t tot = 0;
    for (rr_ctx* c : b->cones) {
        cudaError_t e = cudaMemcpyAsync(c->host_total, c->st.total, sizeof(unsigned long long),
                                        cudaMemcpyDeviceToHost, (cudaStream_t)stream);
        if (e != cudaSuccess) return status_of_cuda(e);
        rr_status st = rr_sync_status(c, stream);
        c->last_total = *c->host_total;
        tot += c->last_total;
        if (st != RR_OK && worst == RR_OK) worst = st;
    }
    if (total_segments) *total_segments = tot;
    return worst;
}

rr_status rr_batch_set_tuning(rr_batch* b, int32_t wx, int32_t bwx, int32_t bwy, int32_t chunk,
                              int32_t blocks_per_sm)
{
    if (!b) return RR_ERR_ARG;
    TileCfg t;
    t.wx = wx;
    t.bwx = bwx;
    t.bwy = bwy;
    if (!tile_ok(t) || chunk < 1 || chunk > 64 || blocks_per_sm < 0 || blocks_per_sm > 64) return RR_ERR_ARG;
    b->tile = t;
    b->chunk = chunk;
    b->blocks_per_sm = blocks_per_sm;
    build_tiles(b);
    return RR_OK;
}

rr_status rr_batch_get_tuning(rr_batch* b, int32_t out[5])
{
    if (!b || !out) return RR_ERR_ARG;
    out[0] = b->tile.wx;
    out[1] = b->tile.bwx;
    out[2] = b->tile.bwy;
    out[3] = b->chunk;
    out[4] = b->blocks_per_sm;
    return RR_OK;
}

rr_status rr_batch_autotune(rr_batch* b, int32_t reps, float* best_ms, void* stream)
{
    if (!b || reps < 1) return RR_ERR_ARG;
    for (size_t i = 0; i < b->staged.size(); ++i)
        if (!b->staged[i]) return RR_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    static const int kWx[] = {4, 8, 16, 32};
    static const int kWarps[][2] = {{1, 2}, {2, 1}, {2, 2}, {1, 4}, {4, 1}, {2, 4}, {4, 2}};
    static const int kChunk[] = {1, 2, 4};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return RR_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return RR_ERR_CUDA;
    }
    const TileCfg keep_t = b->tile;
    const int keep_chunk = b->chunk;
    TileCfg best_t = keep_t;
    int best_chunk = keep_chunk;
    float best = 3.4e38f;
    rr_status st = RR_OK;
    for (int wx : kWx)
        for (const auto& wp : kWarps)
            for (int ch : kChunk) {
                if (st != RR_OK) break;
                if (rr_batch_set_tuning(b, wx, wp[0], wp[1], ch, 0) != RR_OK) continue;
                st = rr_batch_upload(b, s);
                if (st == RR_OK) st = rr_batch_trace(b, s);   // warm-up
                if (st != RR_OK) break;
                cudaEventRecord(e0, s);
                for (int r = 0; r < reps && st == RR_OK; ++r) st = rr_batch_trace(b, s);
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) st = RR_ERR_CUDA;
                if (st != RR_OK) break;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= reps;
                if (ms < best) {
                    best = ms;
                    best_t = b->tile;
                    best_chunk = b->chunk;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    rr_batch_set_tuning(b, best_t.wx, best_t.bwx, best_t.bwy, best_chunk, 0);
    if (st != RR_OK) return st;
    // the timing runs accumulated into the bundles' sums: clear them and keep
    // the staged step (and its log entry) so that the caller can trace it
    st = rr_batch_clear(b, stream);
    if (st != RR_OK) return st;
    if (best_ms) *best_ms = best;
    return rr_batch_upload(b, s);
}

}  // extern "C"
