/*
 * rr.h -- C ABI of the GB300 line-of-sight convergence tracer.
 *
 * The library integrates the weak-lensing convergence kappa (Eq. kappa of
 * Barreira, Llinares, Bose & Li 2016, "RAY-RAMSES", arXiv:1601.02012) and the
 * density-based Born convergence (first term of Eq. kappa2) cell by cell
 * along straight rays through a periodic uniform grid (Secs. 2.4-2.6, 3.2-3.4).
 *
 * Conventions for every call:
 *  - Units: lengths in comoving Mpc/h; the potential is Phi/c^2, so that
 *    kappa = int g(chi_s, chi) Q dchi with g = (chi_s - chi) chi / chi_s.
 *  - 3D arrays are row-major [ix][iy][iz] (z fastest), cell (i,j,k) spans
 *    [ih, (i+1)h) x ...; vertex (i,j,k) sits at (ih, jh, kh); indices wrap
 *    periodically (vertex n is vertex 0).
 *  - Device pointers are caller-owned (allocated by the caller, e.g. torch);
 *    the library never frees or reallocates them. The only memory the
 *    library allocates itself is the per-ray state owned by an rr_ctx.
 *  - Calls that take a stream enqueue their work on it asynchronously and
 *    return at once, except where stated. `stream` is a cudaStream_t passed
 *    as void* (NULL = the legacy default stream).
 *  - Errors are returned as rr_status codes; nothing is thrown across the
 *    ABI. Device-side failures (iteration cap, non-finite sums) are recorded
 *    in a per-context error word and reported by rr_finalize / rr_sync_status.
 *  - A context is not thread-safe: one host thread drives it at a time.
 */
#ifndef RR_H
#define RR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RR_OK = 0,
    RR_ERR_ARG = -1,        /* invalid argument (null pointer, size, interval) */
    RR_ERR_CUDA = -2,       /* a CUDA runtime call failed */
    RR_ERR_OOM = -3,        /* device allocation failed */
    RR_ERR_STEP_LIMIT = -4, /* a ray exceeded its per-step iteration cap */
    RR_ERR_STATE = -5,      /* calls out of order (e.g. a gap between steps) */
    RR_ERR_NONFINITE = -6,  /* a per-ray sum became NaN or infinite */
    RR_ERR_CAPACITY = -7,   /* more rays than rr_trace_step_noalloc's fixed scratch holds */
    RR_ERR_RANGE = -8       /* internal check: a ray of a step traced with flat (no-wrap) record
                               addressing would have left the index range it covers; that ray read
                               nothing and its step contributes nothing */
} rr_status;

/* rr_bundle_desc.interp: how Q varies inside a cell (Sec. 2.6). */
enum { RR_NGP = 0,          /* constant centre value, Eq. (Icngp) / (Iclensing_ngp) */
       RR_TRILINEAR = 1 };  /* trilinear from the 8 vertices, Eq. (Icfinal) / (Iclensing) */

/* rr_bundle_desc.flags */
enum { RR_PERIODIC = 1,     /* wrap cell indices; else a ray stops at the box faces */
       RR_FP64_DDA = 2,     /* plain form: cell walk, kernel integrals and per-step
                               sums in FP64 (default: FP32 walk in cell-local
                               coordinates with compensated FP32 sums) */
       RR_PLAIN_SUMS = 4,   /* the FP32 walk with uncompensated FP32 sums, within and
                               across steps: only to measure what the compensation
                               buys (rr_create / rr_trace_step only; not with
                               RR_FP64_DDA, batches, AMR or the no-allocation call) */
       RR_SOURCE_MOMENTS = 8,   /* rays accumulate the two moments of Eq. (Isources),
                               A = int chi Q dchi and B = int chi^2 Q dchi (for kappa
                               and Born kappa) instead of kappa itself, so that kappa
                               for any source distance chi_k <= chi_s follows from one
                               pass (rr_moments, rr_source_kappa); FP32 walk with
                               compensated sums; rr_create / rr_trace_step only */
       RR_SHEAR = 16,       /* rays also accumulate the shear gamma1, gamma2 (Eqs.
                               gamma1, gamma2) in the same walk as kappa (rr_shear);
                               FP32 walk with compensated sums; rr_create /
                               rr_trace_step / rr_amr_trace_step; not with
                               RR_FP64_DDA, RR_PLAIN_SUMS or RR_SOURCE_MOMENTS */
       RR_METHOD_A = 32,    /* Method A (Eq. kappa2): rr_trace_step reads gradient
                               records (rr_gradient_records) and accumulates the
                               density term (kappa_born) and, separately, the
                               integral of (1 - 2 chi/chi_s) n.grad(Phi) plus each
                               step's surface term g n.grad(Phi) |_end - |_start
                               of the traced interval (Eq. 2nterm); rr_finalize
                               writes kappa = the sum of the three terms and
                               kappa_born = the density term. FP32 walk with
                               compensated sums; rr_create / rr_trace_step /
                               rr_amr_trace_step (records of rr_amr_gradient);
                               no adjoint; not with the other optional flags */
       RR_GENERIC = 64 };   /* generic integrals (Eqs. Ic, Icngp, Icfinal): rr_trace_step
                               reads scalar-pair records (rr_scalar_records) and
                               accumulates int K_c(chi) Q_c dchi for the two channels,
                               K_c quadratic in chi (rr_set_kernels; default: the
                               lensing kernel g for both); rr_finalize writes channel
                               0 into kappa and channel 1 into kappa_born. FP32 walk
                               with compensated sums; rr_create / rr_trace_step /
                               rr_amr_trace_step (records of rr_amr_scalars); no
                               adjoint; not with the other optional flags */

/* rr_tidal_tensor: where the records are evaluated. */
enum { RR_AT_VERTICES = 0,  /* mean of the 8 cells sharing each vertex (Sec. 2.7); trilinear */
       RR_AT_CENTRES = 1 }; /* the cell-centre values themselves; NGP */

/*
 * A light bundle (Sec. 2.4): N_x x N_y rays at the angles of Eq. (txty),
 *   theta_a = Upsilon_a / (N_a - 1) * (i_a - 1) - Upsilon_a / 2,
 * read on the flat sky as theta = sqrt(theta_x^2 + theta_y^2),
 * phi = atan2(theta_y, theta_x), direction n = (sin th cos ph, sin th sin ph,
 * cos th) (Eq. raypos); N_a = 1 puts the single ray at theta_a = 0. The ray
 * of pixel (i_x, i_y) has id (i_y - 1) N_x + (i_x - 1) (Eq. rayid, x fastest).
 * Light travels from chi_s towards the observer, i.e. along -n.
 */
typedef struct {
    int32_t nx, ny;       /* rays per side, >= 1 */
    double fov_x, fov_y;  /* Upsilon_x, Upsilon_y in radians, [0, pi) */
    double obs[3];        /* observer position in box coordinates, Mpc/h */
    double chi_s;         /* comoving distance of the sources, > 0 */
    int32_t interp;       /* RR_NGP or RR_TRILINEAR */
    int32_t flags;        /* RR_PERIODIC | RR_FP64_DDA | RR_PLAIN_SUMS | RR_SOURCE_MOMENTS | RR_SHEAR |
                             RR_METHOD_A | RR_GENERIC */
} rr_bundle_desc;

/* A uniform grid of n[0] x n[1] x n[2] cubic cells of size h = box / n[0]. */
typedef struct {
    int32_t n[3];         /* each in [2, 4096] */
    double box;           /* extent along x in Mpc/h, > 0 */
    double omega_m;       /* matter density parameter, for the Born prefactor and derived delta */
} rr_grid_desc;

typedef struct rr_ctx rr_ctx;

/* Human-readable name of a status code (static string, never NULL). */
const char* rr_status_string(rr_status s);

/*
 * Create a tracing context for one bundle on the current CUDA device: device
 * per-ray state (direction, float-float accumulators of kappa and Born kappa,
 * segment counter) and an error word, all zeroed. Synchronous. *out receives the
 * handle. RR_ERR_ARG on an invalid bundle, RR_ERR_OOM if the state does not
 * fit. Initialising the ray directions (Eq. txty, raypos) runs on the device.
 */
rr_status rr_create(const rr_bundle_desc* bundle, rr_ctx** out);

/*
 * A context for the rows [y0, y1) of `bundle` only: the rays of pixels
 * (i_x, i_y) with y0 <= i_y < y1, directions from Eq. (txty) with the whole
 * bundle's N_y, ids counted from row y0 (Eq. rayid restricted to the band).
 * Rays are independent (Secs. 2.3-2.5: the paper exchanges rays between
 * processes only because it splits the volume), so a bundle traced on several
 * GPUs gives each one a band of rows: every call below then works on the
 * band's (y1 - y0) x nx rays, rr_finalize writes rows y0 .. y1 - 1 of the
 * whole map, and the whole map is the bands' maps concatenated in row order;
 * the adjoint of the whole bundle is the sum over the bands of their
 * rr_trace_backward results, each given its own rows of dL/dkappa. Footprint
 * boxes (rr_footprint_bbox) of the whole bundle hold those of every band.
 * Synchronous, as rr_create. RR_ERR_ARG unless 0 <= y0 < y1 <= ny.
 */
rr_status rr_create_band(const rr_bundle_desc* bundle, int32_t y0, int32_t y1, rr_ctx** out);

/* Free the context and its device state (synchronises the device first). */
rr_status rr_destroy(rr_ctx* ctx);

/* Zero the accumulators, the error word and the step log so that a new
 * sequence of steps can start (asynchronous on `stream`). */
rr_status rr_reset(rr_ctx* ctx, void* stream);

/*
 * Tidal tensor d_a d_b Phi by the central differences of Eq. (tidalexample)
 * at the cell centres (periodic), then records at the vertices (mean of the
 * 8 cells sharing a vertex, Sec. 2.7) or at the centres.
 *   phi    device, n0*n1*n2 floats, Phi/c^2 at cell centres.
 *   delta  device, n0*n1*n2 floats, or NULL: the density contrast. When NULL
 *          it is derived from the same stencils through the comoving Poisson
 *          equation at a = 1: delta = tr(H) / (1.5 Omega_m (H0/c)^2).
 *   rec    device, n0*n1*n2 records of 8 floats (32 bytes, 32-byte aligned:
 *          each record is written and read with one 32-byte access):
 *          {Hxx, Hyy, Hzz, Hxy}, {Hxz, Hyz, delta, 0}, H in (h/Mpc)^2.
 *   where  RR_AT_VERTICES or RR_AT_CENTRES.
 *   bbox   NULL for the whole grid, else 6 ints {x0, x1, y0, y1, z0, z1}:
 *          only points with x0 <= i < x1 (etc.) are written, indices taken
 *          modulo n (x0 may be negative); x1 - x0 must lie in [1, n0].
 * RR_ERR_ARG on a null/misaligned pointer or a bad box.
 */
rr_status rr_tidal_tensor(const rr_grid_desc* grid, const float* phi, const float* delta, float* rec,
                          int32_t where, const int32_t* bbox, void* stream);

/*
 * rr_tidal_tensor over the box bbox (required: 6 int32 {x0, x1, y0, y1, z0,
 * z1}, each extent in [1, n], periodic) with the records stored box-local:
 * point (x0 + i, y0 + j, z0 + k) (wrapped) at record (i ey + j) ez + k, ex ey ez
 * records of 32 bytes in all (fewer than 2^31; rec 32-byte aligned). A box
 * that holds a step's footprint (rr_footprint_bbox) widened by one point per
 * side is all rr_trace_steps needs of that step's records. RR_ERR_ARG as rr_tidal_tensor, and for a NULL
 * bbox.
 */
rr_status rr_tidal_tensor_box(const rr_grid_desc* grid, const float* phi, const float* delta, float* rec,
                              int32_t where, const int32_t* bbox, void* stream);

/*
 * Gradient records of Method A (Eq. kappa2, Sec. 3.5): d_a Phi by central
 * differences (Phi_{+1} - Phi_{-1}) / (2h) at the cell centres (periodic),
 * then records at the vertices (mean of the 8 cells, Sec. 2.7) or at the
 * centres. Arguments as for rr_tidal_tensor, except
 *   rec    device, n0*n1*n2 records of 4 floats (16 bytes, 16-byte aligned):
 *          {d_x Phi, d_y Phi, d_z Phi, delta}, grad Phi in h/Mpc; delta given,
 *          or (NULL) derived from the 7-point Laplacian as rr_tidal_tensor does.
 * These are the records rr_trace_step reads for an RR_METHOD_A context.
 */
rr_status rr_gradient_records(const rr_grid_desc* grid, const float* phi, const float* delta, float* rec,
                              int32_t where, const int32_t* bbox, void* stream);

/*
 * Scalar-pair records of the generic integrals (RR_GENERIC; Eqs. Ic, Icngp,
 * Icfinal, Sec. 2.6): writes channel `channel` (0 or 1) of each point's
 * float2 record, leaving the other channel as it was.
 *   field       device, n0*n1*n2 floats at cell centres.
 *   field_prev  device, n0*n1*n2 floats, or NULL. When given, the channel is
 *               the finite-difference time derivative (field - field_prev) *
 *               inv_dt (the ISW integrand of Sec. 6 for a potential); else the
 *               field itself.
 *   rec         device, n0*n1*n2 records of 2 floats (8 bytes; 16-byte aligned
 *               base), at the vertices (mean of the 8 cells sharing a vertex,
 *               Sec. 2.7) or at the centres (where).
 *   bbox        as for rr_tidal_tensor.
 * RR_ERR_ARG on a null/misaligned pointer, a channel other than 0/1, a
 * non-finite inv_dt or a bad box.
 */
rr_status rr_scalar_records(const rr_grid_desc* grid, const float* field, const float* field_prev, double inv_dt,
                            int32_t channel, float* rec, int32_t where, const int32_t* bbox, void* stream);

/*
 * Kernels of an RR_GENERIC context, used by the steps traced after the call:
 * K_c(chi) = k[3c] + k[3c+1] chi + k[3c+2] chi^2 for channel c = 0, 1 (chi in
 * Mpc/h; the lensing kernel g(chi_s, chi) is {0, 1, -1/chi_s}, its derivative
 * dg/dchi {1, -2/chi_s, 0}, a plain line integral {1, 0, 0}). Host-side only.
 * RR_ERR_ARG on a null pointer or a non-finite coefficient, RR_ERR_STATE for
 * a context without RR_GENERIC.
 */
rr_status rr_set_kernels(rr_ctx* ctx, const double k[6]);

/*
 * Move the observer (box coordinates, Mpc/h) for the steps traced after the
 * call, keeping the ray directions: the tiling of Sec. 2.2, where each box of
 * a tile is traced from the observer's position relative to that box's origin
 * (with RR_PERIODIC off a ray is then traced only while it is inside the box),
 * or the re-use of one box with a relocated observer (Sec. 6). The next step
 * may start at any chi_a <= chi_s (the continuity check with the previous step
 * is waived once); the step log keeps each step's observer, so the adjoint
 * replays every step from the observer it was traced from. Host-side only.
 * RR_ERR_ARG on a null pointer or a non-finite coordinate.
 */
rr_status rr_set_observer(rr_ctx* ctx, const double obs[3]);

/*
 * Copy, from host memory into the same positions of a device array, the cells
 * of a cell-centred field (the potential Phi, delta, a scalar channel) that a
 * boxed rr_tidal_tensor, rr_gradient_records or rr_scalar_records call reads:
 * the box widened by 2 cells on each side (the stencils of Eq. (tidalexample)
 * and the 8-cell vertex mean of Sec. 2.7 reach 2 cells below a vertex box and
 * 1 above), indices modulo n. A step of the walk reads records only inside its
 * footprint (rr_footprint_bbox), so streaming each step's footprint replaces
 * copying the whole field. Cells outside the widened box are left as they were.
 *   host   host, n0*n1*n2 floats in the grid's [ix][iy][iz] order (z fastest);
 *          page-locked for a copy that is asynchronous to the host.
 *   dev    device, n0*n1*n2 floats, same order.
 *   bbox   6 ints as for rr_tidal_tensor, or NULL for the whole field.
 *   bytes  out (may be NULL): the bytes the call enqueued.
 * At most 8 three-dimensional copies (the wrapped pieces of the box) are
 * enqueued on `stream`; the call does not wait for them.
 * RR_ERR_ARG on a null pointer or a bad box; RR_ERR_CUDA if a copy is refused.
 */
rr_status rr_upload_box(const rr_grid_desc* grid, const float* host, float* dev, const int32_t* bbox,
                        int64_t* bytes, void* stream);

/*
 * Host helper: a conservative box of vertex (or centre) indices {x0, x1, y0,
 * y1, z0, z1} that contains every point the bundle's rays can read while
 * tracing [chi_b, chi_a] (the footprint of one step, used to restrict
 * rr_tidal_tensor). Pure host arithmetic, no device work.
 */
rr_status rr_footprint_bbox(const rr_bundle_desc* bundle, const rr_grid_desc* grid, double chi_a,
                            double chi_b, int32_t bbox[6]);

/*
 * Advance every ray of the bundle from chi_a down to chi_b (one N-body step,
 * Sec. 2.5.2), integrating cell by cell (Sec. 2.5.1, 2.6):
 *   kappa      += scale * sum_cells I_c with Q = n1n1 + n2n2 (Eqs. n1n1, n2n2,
 *                 Iclensing or Iclensing_ngp),
 *   kappa_born += scale * sum_cells I_c with Q = 1.5 Omega_m (H0/c)^2 delta / a_step
 *                 (first term of Eq. kappa2, a held constant over the step).
 *   rec      records from rr_tidal_tensor (vertices for RR_TRILINEAR,
 *            centres for RR_NGP; 32-byte aligned) covering every point the
 *            step reads; for an RR_METHOD_A context, records from
 *            rr_gradient_records (the kappa channel then follows Method A,
 *            see RR_METHOD_A; 16-byte aligned), for an RR_GENERIC one, from
 *            rr_scalar_records (16-byte aligned).
 *   scale    multiplies every channel of the records (the field of this step
 *            is scale * stored field).
 * Requires chi_s >= chi_a > chi_b >= 0 and, after the first step since
 * create/reset, chi_a equal to the previous step's chi_b (RR_ERR_STATE
 * otherwise). The step is appended to the context's step log.
 */
rr_status rr_trace_step(rr_ctx* ctx, const rr_grid_desc* grid, const float* rec, double chi_a,
                        double chi_b, double scale, double a_step, void* stream);

/*
 * Write the maps in rayid order (x fastest): kappa[ny*nx] and, if not NULL,
 * kappa_born[ny*nx], both device FP64. Also totals the per-ray segment
 * counters. Synchronises `stream` and returns the context's error word:
 * RR_ERR_STEP_LIMIT, RR_ERR_NONFINITE or RR_ERR_RANGE if a device-side check
 * failed during any step since create/reset, else RR_OK.
 */
rr_status rr_finalize(rr_ctx* ctx, double* kappa, double* kappa_born, void* stream);

/*
 * Source-redshift moments (contexts created with RR_SOURCE_MOMENTS; Eqs.
 * Isources, Isources1). kappa(chi_s) = int_0^chi_s (chi - chi^2/chi_s) Q dchi =
 * A(chi_s) - B(chi_s)/chi_s with A(X) = int_0^X chi Q dchi and B(X) = int_0^X
 * chi^2 Q dchi, where chi_s appears only as the upper limit and in the factor
 * of B. Rays integrate from the sources towards the observer, so the moments
 * accumulated down to chi_k are the parts above chi_k: A(chi_k) = A_end -
 * A_k with A_k taken once the steps down to chi_k are traced (same for B).
 * rr_finalize of such a context writes kappa for the context's own chi_s.
 */

/* The moments accumulated since create/reset: out = device FP64 [4][ny*nx],
 * rows A_kappa, B_kappa, A_born, B_born in rayid order, each summed over the
 * traced steps as scale * int chi^k Q dchi (Born: with the prefactor of Eq.
 * kappa2). Asynchronous. RR_ERR_STATE for a context without RR_SOURCE_MOMENTS. */
rr_status rr_moments(rr_ctx* ctx, double* out, void* stream);

/* kappa and Born kappa for sources at chi_k from two moment snapshots of
 * rr_moments: m_end after the last step (down to the observer), m_k after the
 * steps down to chi_k (NULL when chi_k is the context's chi_s: nothing traced
 * above it); kappa = (A_end - A_k) - (B_end - B_k) / chi_k per channel.
 * nrays entries per row; kappa_born may be NULL. Asynchronous; RR_ERR_ARG on
 * null pointers, nrays < 1 or chi_k <= 0. */
rr_status rr_source_kappa(const double* m_end, const double* m_k, int64_t nrays, double chi_k, double* kappa,
                          double* kappa_born, void* stream);

/*
 * Shear (contexts created with RR_SHEAR; Eqs. gamma1, gamma2, Sec. 3.4). Per
 * ray, in the transverse frame e_phi = (-sin phi, cos phi, 0), e_theta =
 * (cos theta cos phi, cos theta sin phi, -sin theta) of its direction (phi = 0
 * for the ray along the z axis), the walk integrates the lensing kernel times
 * Q1 = e_phi.H.e_phi - e_theta.H.e_theta (gamma1) and Q2 = 2 e_phi.H.e_theta
 * (gamma2, Eq. n1n2 read in that orthonormal frame), H the tidal tensor of the
 * records, with the field and kernel integrals of kappa (NGP or trilinear).
 * gamma1 and gamma2 = device FP64 [ny*nx] each, rayid order, summed over the
 * steps since create/reset with each step's scale (the kappa sum's factor).
 * Asynchronous; RR_ERR_ARG on null pointers, RR_ERR_STATE for a context
 * without RR_SHEAR.
 */
rr_status rr_shear(rr_ctx* ctx, double* gamma1, double* gamma2, void* stream);

/*
 * Steps i = 0 .. nsteps - 1 in order, each as rr_trace_step(ctx, grid, rec[i],
 * chi_a[i], chi_b[i], scale[i], a_step[i], stream) would trace it: the same
 * checks (every step continues the previous one), the same step log and the
 * same results bit for bit. rec, chi_a, chi_b, scale, a_step: host arrays of
 * nsteps entries; rec[i] are device record buffers (the same buffer may serve
 * several steps) that must all stay valid until the stream reaches the end of
 * the call. boxes: NULL (every rec[i] holds the whole grid's records, as for
 * rr_trace_step), or a host array of 6 int32 per step: rec[i] then holds only
 * the records of box i, in the box-local layout of rr_tidal_tensor_box, and
 * box i (periodically) must hold the step's footprint box (rr_footprint_bbox
 * of the whole bundle) widened by one point on each side, since the walk
 * checks one vertex plane beyond it; boxes need a periodic trilinear bundle
 * whose form reads tidal records (not RR_METHOD_A or RR_GENERIC; RR_ERR_ARG
 * otherwise, or for a box that misses the footprint). A step's records then
 * take its footprint's memory only, so that the records of many steps can be
 * resident at once. In the FP32 compensated forms (not RR_FP64_DDA or
 * RR_PLAIN_SUMS) up to 16 consecutive steps are traced by one launch: each
 * ray walks them in turn with its sums (and its shear pair or B moments)
 * held on chip, instead of reading and writing its state at every step (Sec.
 * 2.5.2 moves all rays to the end of one time step before the next; with the
 * records of several steps resident, one ray is moved through them). Steps
 * whose footprint reaches the periodic seam (trilinear, whole-grid records),
 * and the other forms, get one launch each. A moments snapshot (rr_moments)
 * between steps needs a call boundary there. If a step fails its checks nothing is launched and
 * the log is unchanged (RR_ERR_ARG / RR_ERR_STATE as rr_trace_step);
 * asynchronous otherwise. nsteps == 0: no-op.
 */
rr_status rr_trace_steps(rr_ctx* ctx, const rr_grid_desc* grid, int32_t nsteps, const float* const* rec,
                         const int32_t* boxes, const double* chi_a, const double* chi_b, const double* scale,
                         const double* a_step, void* stream);

/* Synchronise `stream` and return the error word (as rr_finalize does),
 * without writing maps. */
rr_status rr_sync_status(rr_ctx* ctx, void* stream);

/*
 * Number of non-empty cell segments traversed by all rays since
 * create/reset, as totalled by the last rr_finalize (host value). If
 * per_ray is not NULL it is a device uint32[ny*nx] that receives the per-ray
 * counts (asynchronous on `stream`).
 */
rr_status rr_segment_count(rr_ctx* ctx, uint64_t* total, uint32_t* per_ray, void* stream);

/* Number of steps in the context's step log (since create/reset). */
rr_status rr_step_count(rr_ctx* ctx, int32_t* n);

/*
 * Adjoint of logged step `step` (0-based, in call order): adds to grad_rec
 * the gradient of L with respect to the records that step read,
 *   grad_rec[p] += sum over rays and segments of dL/dI * dI/dq_p,
 * where q_p is the record at point p (vertices for RR_TRILINEAR, centres for
 * RR_NGP) and I the step's contribution to kappa (scale * Eq. Iclensing /
 * Iclensing_ngp through Q = n1n1 + n2n2) and to kappa_born (scale * first term
 * of Eq. kappa2). The map is linear in the records, so this is its exact
 * transpose; it needs the geometry only, not the records.
 *   dL_dkappa, dL_dkborn  device FP64 [ny*nx] in rayid order (either may be NULL).
 *   grad_rec              device, n0*n1*n2 gradient records of 64 B each
 *                         (16-byte aligned; passed as float*, 16 floats per
 *                         point): 8 FP64 sums, one per record channel
 *                         {Hxx,Hyy,Hzz,Hxy,Hxz,Hyz,delta,0}, accumulated with
 *                         FP64 atomic additions of warp-summed FP32
 *                         contributions (the order of additions is not
 *                         deterministic; the value is, to rounding).
 */
rr_status rr_trace_step_adjoint(rr_ctx* ctx, int32_t step, const double* dL_dkappa, const double* dL_dkborn,
                                float* grad_rec, void* stream);

/*
 * Transpose of rr_tidal_tensor: from gradient records (64 B per point, as
 * written by rr_trace_step_adjoint; at vertices or centres) to dL/dPhi at the
 * cell centres, accumulated (+=) into dL_dphi (device,
 * n0*n1*n2 floats). If dL_ddelta is NULL, delta is taken as derived from the
 * potential (rr_tidal_tensor with delta == NULL) and its gradient flows into
 * dL_dphi; otherwise dL/ddelta is accumulated into dL_ddelta.
 */
rr_status rr_tidal_tensor_adjoint(const rr_grid_desc* grid, const float* grad_rec, int32_t where, float* dL_dphi,
                                  float* dL_ddelta, void* stream);

/*
 * dL/dPhi for maps traced from one potential: all logged steps must share one
 * grid and their records must come from the same phi (each step's field being
 * scale_k * that phi). grad_rec is caller scratch (n0*n1*n2 gradient records of
 * 64 B, 16-byte aligned). The call zeroes the records of the points the logged
 * steps can reach (the union of their footprint boxes, rr_footprint_bbox of the
 * whole bundle, widened by the stencils' reach; the whole grid when that union
 * spans it), adds the adjoint of every logged step, then applies
 * rr_tidal_tensor_adjoint over the cells within the stencils' reach of that
 * union (every other cell's gradient is zero) into dL_dphi (accumulated) /
 * dL_ddelta (NULL: delta derived from phi). Records outside the zeroed box are
 * neither read nor written. RR_ERR_STATE if no step was traced or the grids
 * differ.
 */
rr_status rr_trace_backward(rr_ctx* ctx, const double* dL_dkappa, const double* dL_dkborn, float* grad_rec,
                            float* dL_dphi, float* dL_ddelta, void* stream);

/*
 * Batches: many bundles (lightcones) with their own grids, fields, ray counts
 * and source distances, traced by one persistent launch whose blocks take ray
 * tiles of all bundles from a device work counter (a counter that only
 * increments: no block waits on another). All bundles of a batch share
 * `interp` and the RR_FP64_DDA flag. Each bundle has its own rr_ctx
 * (rr_batch_context), so rr_trace_step_adjoint / rr_trace_backward work on
 * the bundles of a batch as on single contexts.
 *
 * Per step: rr_batch_set_step for every bundle (host-side: checks, step log,
 * staging of the kernel arguments in pinned host memory), then
 * rr_batch_upload (copies the staged table to the device), rr_batch_trace
 * (zeroes the work counter, one persistent launch), and after the last step
 * rr_batch_finalize (maps). Upload, trace and finalize only enqueue work on
 * `stream`, so they can be captured in a CUDA graph together with the
 * bundles' rr_tidal_tensor calls; a replay of that graph re-reads the staged
 * table, so restaging between replays (after the previous replay finished)
 * changes the steps. rr_batch_sync_status synchronises and reports.
 */
typedef struct rr_batch rr_batch;

/* n bundles; RR_ERR_ARG if n < 1 or the bundles mix interp / RR_FP64_DDA. */
rr_status rr_batch_create(int32_t n, const rr_bundle_desc* bundles, rr_batch** out);
rr_status rr_batch_destroy(rr_batch* b);
rr_status rr_batch_size(rr_batch* b, int32_t* n);
/* The context of bundle i (owned by the batch; do not destroy it). */
rr_status rr_batch_context(rr_batch* b, int32_t i, rr_ctx** ctx);
/* rr_reset of every bundle; clears the staged steps. */
rr_status rr_batch_reset(rr_batch* b, void* stream);
/* Zero every bundle's accumulators, segment counters and error word (device
 * memsets only: the step logs and the staged steps stay), e.g. at the start of
 * a captured graph that re-traces the same steps. */
rr_status rr_batch_clear(rr_batch* b, void* stream);
/* Stage one step of bundle i (arguments and checks as rr_trace_step). */
rr_status rr_batch_set_step(rr_batch* b, int32_t i, const rr_grid_desc* grid, const float* rec, double chi_a,
                            double chi_b, double scale, double a_step);
/* Copy the staged table to the device. RR_ERR_STATE if a bundle has no staged step. */
rr_status rr_batch_upload(rr_batch* b, void* stream);
/* Trace the uploaded step of every bundle in one persistent launch. */
rr_status rr_batch_trace(rr_batch* b, void* stream);
/* Maps of every bundle: kappa[i], kappa_born[i] (host arrays of device FP64
 * pointers; kappa_born may be NULL). Does not synchronise. */
rr_status rr_batch_finalize(rr_batch* b, double* const* kappa, double* const* kappa_born, void* stream);
/* Synchronise `stream`; *total_segments (may be NULL) = segments of all
 * bundles since reset; returns the first non-OK error word of a bundle. */
rr_status rr_batch_sync_status(rr_batch* b, uint64_t* total_segments, void* stream);
/*
 * Launch shape: a warp covers wx x (32/wx) pixels (wx in 1..32, a power of
 * two), a block bwx x bwy warps (at most 8), each counter increment takes
 * `chunk` tiles (1..64), blocks_per_sm persistent blocks per SM (0: as many as
 * the occupancy calculator allows). Results do not depend on the shape.
 */
rr_status rr_batch_set_tuning(rr_batch* b, int32_t wx, int32_t bwx, int32_t bwy, int32_t chunk,
                              int32_t blocks_per_sm);
/* out = {wx, bwx, bwy, chunk, blocks_per_sm}. */
rr_status rr_batch_get_tuning(rr_batch* b, int32_t out[5]);
/*
 * Autotuner: times `reps` traces of the staged step for every candidate
 * shape (wx in {4, 8, 16, 32}; 2, 4 or 8 warps per block in several
 * arrangements; chunk in {1, 2, 4}) with CUDA events and keeps the fastest
 * (*best_ms = its mean time). Synchronises. The timing runs accumulate into
 * the bundles' sums, so it clears every bundle's accumulators and counters
 * afterwards and re-uploads the staged step: call it right after staging the
 * first step, before tracing anything that must be kept.
 */
rr_status rr_batch_autotune(rr_batch* b, int32_t reps, float* best_ms, void* stream);

/*
 * Adaptive meshes (Secs. 2.5.1, 2.7, 3.3). A periodic n^3 coarse grid (level
 * 0, cell size h_0 = box / n) whose cells may be refined into octs of 8
 * children of half the size, down to level lmax <= 8, 2:1 balanced: the 26
 * level-(l-1) neighbours of the parent of every level-l oct exist. A cell that
 * is not refined is a leaf. Coordinates of a level-l cell are integers in
 * [0, n 2^l); the finest lattice has side n 2^lmax <= 2^24.
 *
 * Cells are numbered level after level: level 0 row-major (z fastest), then
 * for each level l >= 1 oct after oct in the order given to rr_amr_create,
 * 8 children per oct, child (dx, dy, dz) at 8 o + dx + 2 dy + 4 dz. Leaves are
 * numbered in the order of their cell numbers.
 *
 * rr_amr_create builds the mesh plan on the host and copies it to the current
 * device (synchronous; the host part runs on all hardware threads): per cell
 * its refinement link and either its 18 same-level stencil neighbours or the 8
 * coarser cells it interpolates from; per lattice vertex a leaf needs, its
 * value as a weighted sum of up to 8 leaves; per leaf corner the 1, 2 or 4
 * vertices whose mean it is.
 *   octs[l]  (l = 1..lmax) host int32 [noct[l] x 3]: the level-(l-1) cells
 *            refined into level-l octs, each listed once; octs[0] and
 *            noct[0] are ignored.
 * RR_ERR_ARG on a bad description, a parent that does not exist, a mesh that
 * is not 2:1 balanced, or more than 2^31 - 1 cells; RR_ERR_OOM if the plan does
 * not fit in device memory.
 */
typedef struct rr_amr rr_amr;

typedef struct {
    int32_t n;            /* coarse cells per side, [2, 4096] */
    int32_t lmax;         /* finest level, [0, 8] */
    double box;           /* extent in Mpc/h, > 0 */
    double omega_m;       /* for the Born prefactor and the derived delta */
} rr_amr_desc;

rr_status rr_amr_create(const rr_amr_desc* desc, const int32_t* const* octs, const int64_t* noct, rr_amr** out);
/* Free the plan (synchronises the device first). */
rr_status rr_amr_destroy(rr_amr* mesh);
/* Cells of all levels, leaves, and vertex slots of the plan (one per leaf: the
 * leaf's lower corner, which owns the lattice vertex there unless it is hanging)
 * (any may be NULL). */
rr_status rr_amr_sizes(rr_amr* mesh, int64_t* ncells, int64_t* nleaves, int64_t* nverts);

/*
 * Leaf records from the potential at every cell centre of every level:
 *   1. d_a d_b Phi at every cell, level by level: the central differences of
 *      Eq. (tidalexample) with the level's own spacing when all 18 stencil
 *      neighbours exist at that level; otherwise the coarser level's values
 *      interpolated trilinearly to the cell centre (Sec. 3.3); delta from
 *      tr(H) by the comoving Poisson equation at a = 1.
 *   2. RR_AT_VERTICES: the value at each leaf corner (Sec. 2.7) -- the mean of
 *      the 8 same-level leaves around a vertex; Eqs. (alphac3d), (alphaf3d)
 *      at a vertex shared by coarse and fine leaves; the mean of the 2 or 4
 *      vertices of the coarse edge or face in whose middle a corner lies.
 *      RR_AT_CENTRES: the leaf's own cell value.
 *   phi         device float [ncells], Phi/c^2 at cell centres in cell order.
 *   where       RR_AT_VERTICES (for RR_TRILINEAR) or RR_AT_CENTRES (RR_NGP).
 *   leaf_rec    device, 16-byte aligned (32-byte aligned for the tidal records
 *               that rr_amr_trace_step reads): RR_AT_VERTICES 64 floats per leaf
 *               (8 corners, corner dx + 2 dy + 4 dz, 8 floats each as in
 *               rr_tidal_tensor's records); RR_AT_CENTRES 8 floats per leaf.
 *   cell_tidal  device float [ncells x 8] or NULL: also receives step 1's
 *               per-cell records {Hxx, Hyy, Hzz, Hxy}, {Hxz, Hyz, delta, 0}.
 *   bbox        NULL for the whole mesh, else 6 ints {x0, x1, y0, y1, z0, z1}
 *               of coarse cells (as rr_footprint_bbox gives them for the
 *               coarse grid, indices modulo n, x1 - x0 in [1, n]): only the
 *               records of leaves inside that box are written (and the cell
 *               and vertex values they need, within lmax + 3 coarse cells).
 * Asynchronous on `stream` (lmax + 3 launches).
 */
rr_status rr_amr_tidal(rr_amr* mesh, const float* phi, int32_t where, float* leaf_rec, float* cell_tidal,
                       const int32_t* bbox, void* stream);

/*
 * The records of Method A (Eq. kappa2) over the adaptive mesh, in the layout
 * and with the arguments of rr_amr_tidal: per cell of every level d_a Phi by
 * central differences where the same-level stencil of rr_amr_tidal is
 * complete, else the coarser level's gradient interpolated trilinearly to the
 * cell centre (the Sec. 3.3 rule), and delta as rr_amr_tidal derives it; the
 * 8 channels hold {d_x Phi, d_y Phi, d_z Phi, 0}, {0, 0, delta, 0}, and the
 * vertex values and leaf records follow from them as for the tidal records.
 * These are the records rr_amr_trace_step reads for an RR_METHOD_A context.
 */
rr_status rr_amr_gradient(rr_amr* mesh, const float* phi, int32_t where, float* leaf_rec, float* cell_grad,
                          const int32_t* bbox, void* stream);

/*
 * The records of the generic integrals (RR_GENERIC; Eqs. Ic, Icngp, Icfinal)
 * over the adaptive mesh, in the layout and with the box and output arguments
 * of rr_amr_tidal: per cell Q0 and Q1, each its field's cell value or, when
 * its prev is given, (field - prev) * inv_dt (the ISW integrand of Sec. 6 for
 * a potential); the 8 channels hold {Q0, Q1, 0, 0}, {0, 0, 0, 0}, and vertex
 * values and leaf records follow as for the tidal records. field0: device,
 * one float per cell in cell order (as phi); field1 may be NULL (Q1 = 0).
 * RR_ERR_ARG on a null field0, a non-finite inv_dt or as rr_amr_tidal.
 */
rr_status rr_amr_scalars(rr_amr* mesh, const float* field0, const float* prev0, double inv_dt0, const float* field1,
                         const float* prev1, double inv_dt1, int32_t where, float* leaf_rec, float* cell_buf,
                         const int32_t* bbox, void* stream);

/*
 * rr_trace_step over an adaptive mesh: each ray advances leaf by leaf (the
 * crossings of the finest lattice grouped per leaf, Sec. 2.5.1) and adds the
 * integrals of rr_trace_step with each leaf's own cell size. `leaf_rec` from
 * rr_amr_tidal with RR_AT_VERTICES for RR_TRILINEAR bundles, RR_AT_CENTRES for
 * RR_NGP. Segment counts count leaf segments. An RR_SHEAR context also
 * accumulates the shear (rr_shear); an RR_METHOD_A context reads the records
 * of rr_amr_gradient and follows Method A as rr_trace_step does; an
 * RR_GENERIC context reads the records of rr_amr_scalars. RR_ERR_ARG for
 * RR_FP64_DDA bundles (the AMR walk is the FP32 float-float form only) and for
 * RR_PLAIN_SUMS and RR_SOURCE_MOMENTS; other checks and the step log as
 * rr_trace_step. Steps traced this way have no adjoint:
 * rr_trace_step_adjoint and rr_trace_backward return RR_ERR_STATE for them.
 */
rr_status rr_amr_trace_step(rr_ctx* ctx, rr_amr* mesh, const float* leaf_rec, double chi_a, double chi_b,
                            double scale, double a_step, void* stream);

/*
 * Steps i = 0 .. nsteps - 1 over the adaptive mesh, each as
 * rr_amr_trace_step(ctx, mesh, leaf_rec[i], chi_a[i], chi_b[i], scale[i],
 * a_step[i], stream) would trace it (the same checks, step log and results bit
 * for bit); host arrays of nsteps entries, leaf_rec[i] device leaf-record
 * buffers (the same buffer may serve several steps) that must stay valid until
 * the stream reaches the end of the call. Up to 16 consecutive steps are
 * traced by one launch, each ray walking them in turn with its sums (and its
 * shear pair) held on chip, as rr_trace_steps does. If a step fails its checks
 * nothing is launched and the log is unchanged (RR_ERR_ARG for the forms
 * rr_amr_trace_step refuses). nsteps == 0: no-op.
 */
rr_status rr_amr_trace_steps(rr_ctx* ctx, rr_amr* mesh, int32_t nsteps, const float* const* leaf_rec,
                             const double* chi_a, const double* chi_b, const double* scale, const double* a_step,
                             void* stream);

/*
 * One trace step that allocates nothing -- for callers that cannot let a
 * library allocate device memory: a host framework that already owns the
 * device memory pool through its own allocator, code that cannot afford the
 * device-wide synchronisation cudaMalloc/cudaFree imply, or a plugin host that
 * forbids driver allocations. The paper has no counterpart; it is an
 * alternative to rr_create + rr_trace_step + rr_finalize for a single step.
 *
 * It traces every ray of `bundle` from chi_a down to chi_b exactly as
 * rr_trace_step does (same kernels, same arguments and meaning) and writes
 * kappa and (if not NULL) kappa_born, device FP64 [ny*nx] in rayid order,
 * holding scale * the step's integrals. Every call then copies the device
 * error word to the host and waits for `stream` to finish
 * (cudaStreamSynchronize) before it returns, so it blocks the calling thread
 * until the step's work is done, and returns that word as rr_finalize does.
 *
 * Scratch: instead of memory the library allocates, the per-ray directions,
 * accumulators, segment counters and error word live in one fixed array in
 * the library's device memory, sized for RR_NOALLOC_MAX_RAYS rays (about
 * 4.8 MB). Every GPU that loads the library holds that array until the
 * process exits. The caller still provides `rec` and the output maps. The
 * first call on a device looks up the array's device address (once per
 * device, with that device current). Every call reuses the same array and
 * clears what it accumulates
 * into at the start; calls whose work overlaps on the GPU (two streams, or
 * two host threads, at once) race on it and must be serialised by the caller.
 * Returns RR_ERR_CAPACITY if nx * ny > RR_NOALLOC_MAX_RAYS, RR_ERR_ARG for
 * the argument errors rr_create and rr_trace_step reject (a field of view of
 * pi or more, non-finite observer, distances, scale or grid sizes, ...; no
 * step-order check: each call is independent) and for flags other than
 * RR_PERIODIC and RR_FP64_DDA.
 */
#define RR_NOALLOC_MAX_RAYS 65536
rr_status rr_trace_step_noalloc(const rr_bundle_desc* bundle, const rr_grid_desc* grid, const float* rec,
                                double chi_a, double chi_b, double scale, double a_step, double* kappa,
                                double* kappa_born, void* stream);

/*
 * Measurement helper (the paper has no counterpart): launches an FP32 FMA
 * throughput kernel on `stream`, `blocks` x `threads` threads, each running
 * independent fused multiply-add chains for `iters` iterations (packed != 0:
 * the packed two-lane FFMA2 form). *fmas receives the number of FMAs the
 * launch performs (lane operations; an FFMA2 counts two). Time the launch
 * with events on `stream`: FMAs / time is the FP32 FMA rate that the cell
 * walk's arithmetic roofline is reported against. `out` (device, >= blocks
 * floats) is never written for these arguments; it keeps the chains live.
 * Asynchronous. RR_ERR_ARG for bad sizes or null pointers.
 */
rr_status rr_fp32_peak(int32_t packed, int32_t blocks, int32_t threads, int32_t iters, float* out,
                       int64_t* fmas, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RR_H */
