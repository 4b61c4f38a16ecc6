/*
 * FP64 CPU oracle for the cell-by-cell line-of-sight convergence integral of
 * RAY-RAMSES (Barreira, Llinares, Bose & Li 2016, arXiv:1601.02012).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the independent reference that the
 * CUDA path is checked against. Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it. It shares no code, header, table
 * or helper with the CUDA library, and the library never calls it.
 *
 * What it computes, all in double precision, plainly and slowly:
 *   - d_a d_b Phi at cell centres by the central-difference stencils of
 *     Eq. (tidalexample), periodic indexing (Sec. 3.3);
 *   - vertex values as the mean of the 8 cells sharing the vertex
 *     (Sec. 2.7, regular-mesh vertices), evaluated on the fly;
 *   - ray directions from Eq. (txty) with theta = sqrt(tx^2 + ty^2),
 *     phi = atan2(ty, tx), i.e. (cos phi, sin phi) = (tx, ty) / theta
 *     (flat-sky polar reading of Eq. raypos);
 *   - the cells a ray crosses between chi_a and chi_b by merging the
 *     per-axis lists of face-crossing distances (the cell-by-cell walk of
 *     Sec. 2.5.1, written as an exact FP64 crossing list);
 *   - per cell: Q = n1n1 + n2n2 from Eqs. (n1n1), (n2n2); the NGP integral
 *     Eq. (Iclensing_ngp) or the trilinear integral Eq. (Iclensing) with the
 *     alpha_i of Eq. (trilinear_coef) and the d_N of Appendix B;
 *   - the density-based Born convergence, the first term of Eq. (kappa2),
 *     with a held constant over the step;
 *   - the shear (Eqs. gamma1, gamma2) by the same walk and integrals with
 *     Q = n1n1 - n2n2 and Q = 2 n1n2 (Eq. n1n2 in its orthonormal reading);
 *   - generic integrals int K Q dchi of two scalar fields with quadratic
 *     kernels K(chi) (Eqs. Ic, Icngp, Icfinal; the ISW integral of Sec. 6);
 *   - Method A (Eq. kappa2): d_a Phi at centres by central differences,
 *     the integral of (1 - 2 chi/chi_s) n.grad(Phi) by Eq. (Icfinal) with
 *     that kernel, and each step's surface term g n.grad(Phi) at the ends of
 *     the traced interval (Eq. 2nterm);
 *   - Neumaier-compensated per-ray sums;
 *   - the exact adjoint of all of the above (the transpose of a linear map),
 *     built segment by segment from unit-vector evaluations of the same
 *     closed forms.
 *
 * Layout: every 3D array is [ix][iy][iz] with z fastest. Cell (i,j,k) spans
 * [i h, (i+1) h) etc.; vertex (i,j,k) sits at (i h, j h, k h).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_H0_OVER_C (1.0 / 2997.92458) /* h/Mpc */

/* ------------------------------------------------------------------------- */
/* plain data                                                                */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t nx, ny;       /* rays per side (Eq. txty) */
    double fov_x, fov_y;  /* Upsilon_x, Upsilon_y in radians */
    double obs[3];        /* observer position in box coordinates */
    double chi_s;         /* source comoving distance */
    int32_t interp;       /* 0 = NGP (Eq. Icngp), 1 = trilinear (Eq. Icfinal) */
    int32_t periodic;     /* 1 = wrap cell indices, 0 = stop at the box faces */
} ora_bundle;

typedef struct {
    int32_t n[3];
    double box;           /* h = box / n[0] */
    double omega_m;
} ora_grid;

typedef struct { double sum, comp; } neu_t;

static void neu_add(neu_t* s, double x)
{
    double t = s->sum + x;
    if (fabs(s->sum) >= fabs(x)) s->comp += (s->sum - t) + x;
    else s->comp += (x - t) + s->sum;
    s->sum = t;
}

static double neu_val(const neu_t* s) { return s->sum + s->comp; }

static long wrap(long i, long n)
{
    long r = i % n;
    return r < 0 ? r + n : r;
}

static size_t cell_index(const ora_grid* g, long i, long j, long k)
{
    return ((size_t)wrap(i, g->n[0]) * (size_t)g->n[1] + (size_t)wrap(j, g->n[1])) * (size_t)g->n[2]
           + (size_t)wrap(k, g->n[2]);
}

static double grid_h(const ora_grid* g) { return g->box / (double)g->n[0]; }

/* ------------------------------------------------------------------------- */
/* Sec. 3.3, Eq. (tidalexample): d_a d_b Phi at cell centres                 */
/* ------------------------------------------------------------------------- */

/* H receives 6 values per cell in the order xx, yy, zz, xy, xz, yz. */
int ora_tidal_centres(const ora_grid* g, const double* phi, double* H)
{
    const double h = grid_h(g);
    const double ih2 = 1.0 / (h * h);
    for (long i = 0; i < g->n[0]; ++i)
        for (long j = 0; j < g->n[1]; ++j)
            for (long k = 0; k < g->n[2]; ++k) {
                double* out = H + 6 * cell_index(g, i, j, k);
                double p0 = phi[cell_index(g, i, j, k)];
                /* diagonal: (Phi_{-1} - 2 Phi_0 + Phi_{+1}) / h^2 */
                out[0] = (phi[cell_index(g, i - 1, j, k)] - 2.0 * p0 + phi[cell_index(g, i + 1, j, k)]) * ih2;
                out[1] = (phi[cell_index(g, i, j - 1, k)] - 2.0 * p0 + phi[cell_index(g, i, j + 1, k)]) * ih2;
                out[2] = (phi[cell_index(g, i, j, k - 1)] - 2.0 * p0 + phi[cell_index(g, i, j, k + 1)]) * ih2;
                /* mixed: (Phi_{++} + Phi_{--} - Phi_{+-} - Phi_{-+}) / (4 h^2) */
                out[3] = (phi[cell_index(g, i + 1, j + 1, k)] + phi[cell_index(g, i - 1, j - 1, k)]
                          - phi[cell_index(g, i + 1, j - 1, k)] - phi[cell_index(g, i - 1, j + 1, k)]) * 0.25 * ih2;
                out[4] = (phi[cell_index(g, i + 1, j, k + 1)] + phi[cell_index(g, i - 1, j, k - 1)]
                          - phi[cell_index(g, i + 1, j, k - 1)] - phi[cell_index(g, i - 1, j, k + 1)]) * 0.25 * ih2;
                out[5] = (phi[cell_index(g, i, j + 1, k + 1)] + phi[cell_index(g, i, j - 1, k - 1)]
                          - phi[cell_index(g, i, j + 1, k - 1)] - phi[cell_index(g, i, j - 1, k + 1)]) * 0.25 * ih2;
            }
    return 0;
}

/* Density contrast implied by the potential through the comoving Poisson
 * equation at a = 1: delta = (Hxx + Hyy + Hzz) / (1.5 Omega_m (H0/c)^2). */
int ora_delta_from_tidal(const ora_grid* g, const double* H, double* delta)
{
    const double inv = 1.0 / (1.5 * g->omega_m * ORA_H0_OVER_C * ORA_H0_OVER_C);
    size_t nc = (size_t)g->n[0] * g->n[1] * g->n[2];
    for (size_t c = 0; c < nc; ++c) delta[c] = (H[6 * c] + H[6 * c + 1] + H[6 * c + 2]) * inv;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Sec. 2.7: value at a regular-mesh vertex = mean of the 8 cells sharing it */
/* ------------------------------------------------------------------------- */

/* 7 channels: H (6) then delta. Vertex (i,j,k) is shared by the cells
 * (i-1..i, j-1..j, k-1..k). */
static void vertex_value(const ora_grid* g, const double* H, const double* delta,
                         long vi, long vj, long vk, double out[7])
{
    for (int c = 0; c < 7; ++c) out[c] = 0.0;
    for (int di = -1; di <= 0; ++di)
        for (int dj = -1; dj <= 0; ++dj)
            for (int dk = -1; dk <= 0; ++dk) {
                size_t ci = cell_index(g, vi + di, vj + dj, vk + dk);
                if (H)
                    for (int c = 0; c < 6; ++c) out[c] += H[6 * ci + c];
                if (delta) out[6] += delta[ci];
            }
    for (int c = 0; c < 7; ++c) out[c] *= 0.125;
}

/* All vertex values (for checking a stored vertex field). */
int ora_vertex_field(const ora_grid* g, const double* H, const double* delta, double* V)
{
    for (long i = 0; i < g->n[0]; ++i)
        for (long j = 0; j < g->n[1]; ++j)
            for (long k = 0; k < g->n[2]; ++k)
                vertex_value(g, H, delta, i, j, k, V + 7 * cell_index(g, i, j, k));
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Ray geometry: Eq. (txty), Eq. (rayid), Eq. (raypos)                       */
/* ------------------------------------------------------------------------- */

/* Eq. (txty) for 0-based ix = i_x - 1, written as (2 ix - (N - 1)) U / (2 (N - 1))
 * so that the central pixel of an odd row sits at theta_a = 0 exactly. */
static double pixel_angle(double fov, long n, long i)
{
    return n > 1 ? (double)(2 * i - (n - 1)) * (fov / (2.0 * (double)(n - 1))) : 0.0;
}

/* theta = sqrt(tx^2 + ty^2) and the polar angle phi = atan2(ty, tx), returned as
 * (sin phi, cos phi) = (ty, tx) / theta (phi = 0 at theta = 0). */
static void ray_angles(const ora_bundle* b, long ix, long iy, double* theta, double* sphi, double* cphi)
{
    double tx = pixel_angle(b->fov_x, b->nx, ix);
    double ty = pixel_angle(b->fov_y, b->ny, iy);
    *theta = sqrt(tx * tx + ty * ty);
    *sphi = (*theta > 0.0) ? ty / *theta : 0.0;
    *cphi = (*theta > 0.0) ? tx / *theta : 1.0;
}

/* Eq. (n1n1) + Eq. (n2n2): the transverse Laplacian seen by a ray with
 * direction angles (theta, phi). H = {xx, yy, zz, xy, xz, yz}. */
static void kappa_weights(double th, double sp, double cp, double w[6])
{
    double st = sin(th), ct = cos(th);
    double s2p = 2.0 * sp * cp, s2t = sin(2.0 * th);
    /* n1n1 = sin^2(ph) xx + cos^2(ph) yy - sin(2ph) xy */
    /* n2n2 = cos^2(ph) cos^2(th) xx + sin^2(ph) cos^2(th) yy + sin^2(th) zz
     *        + sin(2ph) cos^2(th) xy - sin(ph) sin(2th) yz - cos(ph) sin(2th) xz */
    w[0] = sp * sp + cp * cp * ct * ct;
    w[1] = cp * cp + sp * sp * ct * ct;
    w[2] = st * st;
    w[3] = -s2p + s2p * ct * ct;
    w[4] = -cp * s2t;
    w[5] = -sp * s2t;
}

/* Shear (Eqs. gamma1, gamma2). gamma1 takes Q = n1n1 - n2n2 with the printed
 * Eqs. (n1n1), (n2n2). gamma2 takes Q = 2 n1n2; the printed Eq. (n1n2) equals
 * e_phi^T H e_theta / sin(theta) for the orthonormal e_phi = (-sin ph, cos ph,
 * 0), e_theta = (cos th cos ph, cos th sin ph, -sin th) that Eqs. (n1n1),
 * (n2n2) use, and diverges at theta -> 0; the reading taken is the orthonormal
 * one, Eq. (n1n2) times sin(theta):
 *   n1n2 = cos th [cos ph sin ph (yy - xx) + (cos^2 ph - sin^2 ph) xy]
 *          + sin th (sin ph xz - cos ph yz). */
static void gamma1_weights(double th, double sp, double cp, double w[6])
{
    double st = sin(th), ct = cos(th);
    double s2p = 2.0 * sp * cp, s2t = sin(2.0 * th);
    w[0] = sp * sp - cp * cp * ct * ct;
    w[1] = cp * cp - sp * sp * ct * ct;
    w[2] = -st * st;
    w[3] = -s2p - s2p * ct * ct;
    w[4] = cp * s2t;
    w[5] = sp * s2t;
}

static void gamma2_weights(double th, double sp, double cp, double w[6])
{
    double st = sin(th), ct = cos(th);
    w[0] = -2.0 * ct * cp * sp;
    w[1] = 2.0 * ct * cp * sp;
    w[2] = 0.0;
    w[3] = 2.0 * ct * (cp * cp - sp * sp);
    w[4] = 2.0 * st * sp;
    w[5] = -2.0 * st * cp;
}

static double project(const double w[6], const double* Hc)
{
    return w[0] * Hc[0] + w[1] * Hc[1] + w[2] * Hc[2] + w[3] * Hc[3] + w[4] * Hc[4] + w[5] * Hc[5];
}

/* ------------------------------------------------------------------------- */
/* The cell walk (Sec. 2.5.1) as an exact list of face crossings             */
/* ------------------------------------------------------------------------- */

static int cmp_desc(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x < y) - (x > y);
}

/* Distances chi in (lo, hi) at which the ray o + chi n crosses a face x = m h
 * of any axis, plus lo and hi, sorted in decreasing order. */
static double* crossing_list(const double o[3], const double n[3], double h, double lo, double hi, long* count)
{
    long cap = 2;
    for (int a = 0; a < 3; ++a)
        if (n[a] != 0.0) cap += (long)(fabs(n[a]) * (hi - lo) / h) + 3;
    double* L = (double*)malloc(sizeof(double) * (size_t)cap);
    long m = 0;
    L[m++] = hi;
    L[m++] = lo;
    for (int a = 0; a < 3; ++a) {
        if (n[a] == 0.0) continue;
        double x0 = o[a] + lo * n[a], x1 = o[a] + hi * n[a];
        double xmin = fmin(x0, x1), xmax = fmax(x0, x1);
        for (long f = (long)floor(xmin / h) + 1; (double)f * h < xmax; ++f) {
            double c = ((double)f * h - o[a]) / n[a];
            if (c > lo && c < hi && m < cap) L[m++] = c;
        }
    }
    qsort(L, (size_t)m, sizeof(double), cmp_desc);
    *count = m;
    return L;
}

/* Part of [lo, hi] where the ray stays inside the box [0, n_a h] (stop
 * condition (ii) of Sec. 2.4 when the box is not periodic). */
static int clip_to_box(const ora_grid* g, const double o[3], const double n[3], double* lo, double* hi)
{
    const double h = grid_h(g);
    for (int a = 0; a < 3; ++a) {
        double ext = (double)g->n[a] * h;
        if (n[a] == 0.0) {
            if (o[a] < 0.0 || o[a] > ext) return 0;
            continue;
        }
        double c0 = (0.0 - o[a]) / n[a], c1 = (ext - o[a]) / n[a];
        double cmin = fmin(c0, c1), cmax = fmax(c0, c1);
        if (cmin > *lo) *lo = cmin;
        if (cmax < *hi) *hi = cmax;
    }
    return *hi > *lo;
}

/* ------------------------------------------------------------------------- */
/* Per-cell integrals (Sec. 2.6, Sec. 3.2, Appendix B)                       */
/* ------------------------------------------------------------------------- */

/* Eq. (Iclensing_ngp): Q_c / chi_s [chi_s/2 (chiA^2 - chiB^2) - (chiA^3 - chiB^3)/3] */
static double ic_ngp(double Qc, double chiA, double chiB, double chis)
{
    return Qc / chis * (0.5 * chis * (chiA * chiA - chiB * chiB) - (chiA * chiA * chiA - chiB * chiB * chiB) / 3.0);
}

/* The d_N of Eq. (Qcompact) (Appendix B) for the trilinear field of the
 * vertex values Q[0..7] = Q_1..Q_8 at P_1..P_8, P_{1 + i + 2j + 4k} = P_1 +
 * (i, j, k) h, along the ray from A, (a, b, c) = A - P_1; st, ct, sp, cp are
 * the ray's sin/cos of theta, phi. */
static void dn_coeffs(const double Q[8], double a, double b, double c, double h,
                      double st, double ct, double sp, double cp, double d[4])
{
    /* Eq. (trilinear_coef) */
    double al1 = Q[0];
    double al2 = Q[1] - Q[0];
    double al3 = Q[2] - Q[0];
    double al4 = Q[4] - Q[0];
    double al5 = Q[3] - Q[2] - Q[1] + Q[0];
    double al6 = Q[6] - Q[4] - Q[2] + Q[0];
    double al7 = Q[5] - Q[4] - Q[1] + Q[0];
    double al8 = Q[7] - Q[6] - Q[5] - Q[3] + Q[1] + Q[4] + Q[2] - Q[0];
    double h2 = h * h, h3 = h2 * h;
    double nx = st * cp, ny = st * sp, nz = ct;
    /* Appendix B, the d_N of Eq. (Qcompact) */
    d[0] = al1 + (al2 * a + al3 * b + al4 * c) / h + (al5 * a * b + al6 * b * c + al7 * a * c) / h2
           + al8 * a * b * c / h3;
    d[1] = (al2 * nx + al3 * ny + al4 * nz) / h
           + ((al6 * c + al5 * a) * ny + (al7 * c + al5 * b) * nx + (al7 * a + al6 * b) * nz) / h2
           + (al8 * b * c * nx + al8 * a * b * nz + al8 * a * c * ny) / h3;
    d[2] = (al5 * nx * ny + al7 * nx * nz + al6 * ny * nz) / h2
           + (al8 * a * ny * nz + al8 * b * nx * nz + al8 * c * nx * ny) / h3;
    d[3] = al8 / h3 * nx * ny * nz;
}

/* Eq. (Iclensing) for the trilinear field given by the vertex values
 * Q[0..7] = Q_1..Q_8 at P_1..P_8, P_{1 + i + 2j + 4k} = P_1 + (i, j, k) h.
 * (a, b, c) = A - P_1; st, ct, sp, cp are the ray's sin/cos of theta, phi. */
static double ic_trilinear(const double Q[8], double a, double b, double c, double h,
                           double st, double ct, double sp, double cp,
                           double chiA, double chiB, double chis)
{
    double d[4];
    dn_coeffs(Q, a, b, c, h, st, ct, sp, cp, d);
    /* Eq. (Iclensing), R = chi_B - chi_A */
    double R = chiB - chiA;
    double sum = 0.0;
    for (int N = 1; N <= 4; ++N) {
        double RN = pow(R, N);
        sum += d[N - 1] * (RN / N * (chiA - chis) * chiA + RN * R / (N + 1) * (2.0 * chiA - chis)
                           + RN * R * R / (N + 2));
    }
    return sum / chis;
}

/* ------------------------------------------------------------------------- */
/* Tracing                                                                   */
/* ------------------------------------------------------------------------- */

/* A ray's geometry. */
typedef struct {
    double th, st, ct, sp, cp;
    double n[3];
    double w[6];      /* Q weights of the first channel: kappa, or gamma1 */
    double w2[6];     /* second channel when it is a shear: gamma2 */
    int shear;        /* 0: (kappa, Born); 1: (gamma1, gamma2) */
} ray_geo;

static void make_ray(const ora_bundle* b, long ix, long iy, ray_geo* r)
{
    ray_angles(b, ix, iy, &r->th, &r->sp, &r->cp);
    r->st = sin(r->th); r->ct = cos(r->th);
    /* Eq. (raypos) */
    r->n[0] = r->st * r->cp;
    r->n[1] = r->st * r->sp;
    r->n[2] = r->ct;
    kappa_weights(r->th, r->sp, r->cp, r->w);
    r->shear = 0;
}

static void make_shear_ray(const ora_bundle* b, long ix, long iy, ray_geo* r)
{
    make_ray(b, ix, iy, r);
    gamma1_weights(r->th, r->sp, r->cp, r->w);
    gamma2_weights(r->th, r->sp, r->cp, r->w2);
    r->shear = 1;
}

/* Callback-free walk: for each non-empty segment, evaluate the two integrands
 * (kappa, Born) and optionally the 8 (or 1) coefficients dI/dQ_i. */
typedef struct {
    const ora_grid* g;
    const ora_bundle* b;
    const double* H;      /* centres, 6 per cell */
    const double* delta;  /* centres */
} field_t;

/* Per-segment geometry. */
typedef struct {
    long cell[3];         /* unwrapped cell index */
    double chiA, chiB;
    double a, b, c;       /* A - P_1 */
} segment_t;

static long walk(const field_t* F, const ray_geo* r, double chi_a, double chi_b,
                 segment_t** out_segs)
{
    const ora_grid* g = F->g;
    const double h = grid_h(g);
    double lo = chi_b, hi = chi_a;
    *out_segs = NULL;
    if (!F->b->periodic && !clip_to_box(g, F->b->obs, r->n, &lo, &hi)) return 0;
    if (!(hi > lo)) return 0;
    long m;
    double* L = crossing_list(F->b->obs, r->n, h, lo, hi, &m);
    segment_t* S = (segment_t*)malloc(sizeof(segment_t) * (size_t)(m > 0 ? m : 1));
    long ns = 0;
    for (long s = 0; s + 1 < m; ++s) {
        double A = L[s], B = L[s + 1];
        /* Coincident crossings (the ray passes through a cell edge or corner)
         * leave an empty segment, or a sliver of rounding size between the two
         * crossings; neither is a cell the ray traverses, so it is skipped and
         * not counted. */
        if (!(A - B > 1e-12 * fmax(A, h))) continue;
        double mid = 0.5 * (A + B);
        segment_t* sg = &S[ns++];
        for (int a = 0; a < 3; ++a) sg->cell[a] = (long)floor((F->b->obs[a] + mid * r->n[a]) / h);
        sg->chiA = A;
        sg->chiB = B;
        sg->a = F->b->obs[0] + A * r->n[0] - (double)sg->cell[0] * h;
        sg->b = F->b->obs[1] + A * r->n[1] - (double)sg->cell[1] * h;
        sg->c = F->b->obs[2] + A * r->n[2] - (double)sg->cell[2] * h;
    }
    free(L);
    *out_segs = S;
    return ns;
}

/* Q_kappa and Q_Born at the 8 vertices P_1..P_8 of a cell. */
static void cell_vertex_Q(const field_t* F, const ray_geo* r, const long cell[3],
                          double bpref, double Qk[8], double Qb[8])
{
    for (int v = 0; v < 8; ++v) {
        double val[7];
        vertex_value(F->g, F->H, F->delta, cell[0] + (v & 1), cell[1] + ((v >> 1) & 1),
                     cell[2] + ((v >> 2) & 1), val);
        Qk[v] = project(r->w, val);
        Qb[v] = r->shear ? project(r->w2, val) : bpref * val[6];
    }
}

/*
 * One step [chi_b, chi_a) for every ray. The step's field is scale * (stored
 * field); the Born term uses Q = 1.5 Omega_m (H0/c)^2 delta / a_step
 * (first term of Eq. kappa2, a constant during the step).
 * kappa, kborn, sum_r are accumulated (+=); nseg is accumulated.
 */
static int trace_step(const ora_bundle* b, const ora_grid* g, const double* H, const double* delta,
                      double chi_a, double chi_b, double scale, double a_step,
                      double* kappa, double* kborn, int64_t* nseg, double* sum_r, int nthreads,
                      const int64_t* rids, long nrids, int shear);

int ora_trace_step(const ora_bundle* b, const ora_grid* g, const double* H, const double* delta,
                   double chi_a, double chi_b, double scale, double a_step,
                   double* kappa, double* kborn, int64_t* nseg, double* sum_r, int nthreads,
                   const int64_t* rids, long nrids)
{
    return trace_step(b, g, H, delta, chi_a, chi_b, scale, a_step, kappa, kborn, nseg, sum_r, nthreads, rids,
                      nrids, 0);
}

/* The shear (Eqs. gamma1, gamma2) of one step: gamma1 and gamma2 are
 * accumulated like kappa, with Q = n1n1 - n2n2 and Q = 2 n1n2 (see
 * gamma2_weights for the reading of Eq. n1n2). */
int ora_trace_step_shear(const ora_bundle* b, const ora_grid* g, const double* H, double chi_a, double chi_b,
                         double scale, double* gamma1, double* gamma2, int nthreads, const int64_t* rids,
                         long nrids)
{
    return trace_step(b, g, H, NULL, chi_a, chi_b, scale, 1.0, gamma1, gamma2, NULL, NULL, nthreads, rids, nrids, 1);
}

static int trace_step(const ora_bundle* b, const ora_grid* g, const double* H, const double* delta,
                      double chi_a, double chi_b, double scale, double a_step,
                      double* kappa, double* kborn, int64_t* nseg, double* sum_r, int nthreads,
                      const int64_t* rids, long nrids, int shear)
{
    if (!(chi_a > chi_b) || chi_b < 0.0) return -1;
    field_t F = {g, b, H, delta};
    const double bpref = 1.5 * g->omega_m * ORA_H0_OVER_C * ORA_H0_OVER_C / a_step;
    const double h = grid_h(g);
    /* all rays, or only the listed ray ids (outputs then follow the list) */
    const long nr = rids ? nrids : (long)b->nx * b->ny;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (long slot = 0; slot < nr; ++slot) {
        const long rid = rids ? (long)rids[slot] : slot;
        ray_geo r;
        if (shear) make_shear_ray(b, rid % b->nx, rid / b->nx, &r);
        else make_ray(b, rid % b->nx, rid / b->nx, &r); /* Eq. (rayid), x fastest */
        segment_t* S;
        long ns = walk(&F, &r, chi_a, chi_b, &S);
        neu_t sk = {0, 0}, sb = {0, 0}, sr = {0, 0};
        for (long s = 0; s < ns; ++s) {
            const segment_t* sg = &S[s];
            double ik, ib;
            if (b->interp == 0) {
                size_t ci = cell_index(g, sg->cell[0], sg->cell[1], sg->cell[2]);
                double qk = project(r.w, H + 6 * ci);
                double qb = shear ? project(r.w2, H + 6 * ci) : bpref * delta[ci];
                ik = ic_ngp(qk, sg->chiA, sg->chiB, b->chi_s);
                ib = ic_ngp(qb, sg->chiA, sg->chiB, b->chi_s);
            } else {
                double Qk[8], Qb[8];
                cell_vertex_Q(&F, &r, sg->cell, bpref, Qk, Qb);
                ik = ic_trilinear(Qk, sg->a, sg->b, sg->c, h, r.st, r.ct, r.sp, r.cp, sg->chiA, sg->chiB, b->chi_s);
                ib = ic_trilinear(Qb, sg->a, sg->b, sg->c, h, r.st, r.ct, r.sp, r.cp, sg->chiA, sg->chiB, b->chi_s);
            }
            neu_add(&sk, ik);
            neu_add(&sb, ib);
            neu_add(&sr, sg->chiA - sg->chiB);
        }
        free(S);
        kappa[slot] += scale * neu_val(&sk);
        kborn[slot] += scale * neu_val(&sb);
        if (nseg) nseg[slot] += ns;
        if (sum_r) sum_r[slot] += neu_val(&sr);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Method A (Sec. 3.5, Eq. kappa2): the gradient and surface terms           */
/* ------------------------------------------------------------------------- */

/* d_a Phi at cell centres by central differences, (Phi_{+1} - Phi_{-1}) / (2h)
 * along each axis, periodic indexing (the field whose negative is the force
 * of the N-body code). G: 3 per cell, (x, y, z). */
int ora_fields_grad(const ora_grid* g, const double* phi, double* G)
{
    const double ih = 1.0 / grid_h(g);
    for (long i = 0; i < g->n[0]; ++i)
        for (long j = 0; j < g->n[1]; ++j)
            for (long k = 0; k < g->n[2]; ++k) {
                double* out = G + 3 * cell_index(g, i, j, k);
                out[0] = 0.5 * ih * (phi[cell_index(g, i + 1, j, k)] - phi[cell_index(g, i - 1, j, k)]);
                out[1] = 0.5 * ih * (phi[cell_index(g, i, j + 1, k)] - phi[cell_index(g, i, j - 1, k)]);
                out[2] = 0.5 * ih * (phi[cell_index(g, i, j, k + 1)] - phi[cell_index(g, i, j, k - 1)]);
            }
    return 0;
}

/* Q = n . grad Phi (the radial derivative of Eq. kappa2) at vertex (vi, vj,
 * vk): the mean of the 8 cells sharing it (Sec. 2.7). */
static double vertex_radial_grad(const ora_grid* g, const double* G, const double n[3], long vi, long vj, long vk)
{
    double v[3] = {0.0, 0.0, 0.0};
    for (int di = -1; di <= 0; ++di)
        for (int dj = -1; dj <= 0; ++dj)
            for (int dk = -1; dk <= 0; ++dk) {
                const double* gc = G + 3 * cell_index(g, vi + di, vj + dj, vk + dk);
                for (int a = 0; a < 3; ++a) v[a] += gc[a];
            }
    return 0.125 * (n[0] * v[0] + n[1] * v[1] + n[2] * v[2]);
}

/* Eq. (Icfinal) with the kernel K = d g / d chi = 1 - 2 chi / chi_s: with
 * R = chi_B - chi_A, int_{chi_B}^{chi_A} K (chi - chi_A)^{N-1} dchi =
 * -(1 - 2 chi_A / chi_s) R^N / N + (2 / chi_s) R^{N+1} / (N + 1). */
static double ic_dg_trilinear(const double d[4], double chiA, double chiB, double chis)
{
    double R = chiB - chiA;
    double sum = 0.0;
    for (int N = 1; N <= 4; ++N) {
        double RN = pow(R, N);
        sum += d[N - 1] * (-(1.0 - 2.0 * chiA / chis) * RN / N + 2.0 / chis * RN * R / (N + 1));
    }
    return sum;
}

/* Eq. (Icngp) with K = 1 - 2 chi / chi_s: Q_c [(chi_A - chi_B) - (chi_A^2 - chi_B^2) / chi_s] */
static double ic_dg_ngp(double Qc, double chiA, double chiB, double chis)
{
    return Qc * ((chiA - chiB) - (chiA * chiA - chiB * chiB) / chis);
}

static double lensing_g(double chi, double chis) { return (chis - chi) * chi / chis; }

/*
 * Method A's step terms for every ray: the second term of Eq. (kappa2),
 * int K n.grad(Phi) dchi with K = 1 - 2 chi / chi_s, and the step's part of
 * the surface term, g n.grad(Phi) evaluated at the start (chi_i) and the end
 * (chi_f) of the part of the ray traced in the step (Eq. 2nterm), entering
 * with a minus sign: kgrad += scale * (sum of cell integrals - [g Q](chi_i)
 * + [g Q](chi_f)). The first term (density, Born) is accumulated into kborn as
 * in ora_trace_step; the full Method A convergence is kgrad + kborn (the
 * d/dt term is dropped, as in the paper). The field at the two end points:
 * trilinear, the cubic of Eq. (Qcompact) of the first (last) cell at its own
 * start (at the end point); NGP, that cell's centre value.
 */
int ora_trace_step_method_a(const ora_bundle* b, const ora_grid* g, const double* G, const double* delta,
                            double chi_a, double chi_b, double scale, double a_step,
                            double* kgrad, double* kborn, int nthreads, const int64_t* rids, long nrids)
{
    if (!(chi_a > chi_b) || chi_b < 0.0) return -1;
    field_t F = {g, b, NULL, delta};
    const double bpref = 1.5 * g->omega_m * ORA_H0_OVER_C * ORA_H0_OVER_C / a_step;
    const double h = grid_h(g);
    const double chis = b->chi_s;
    const long nr = rids ? nrids : (long)b->nx * b->ny;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (long slot = 0; slot < nr; ++slot) {
        const long rid = rids ? (long)rids[slot] : slot;
        ray_geo r;
        make_ray(b, rid % b->nx, rid / b->nx, &r);
        segment_t* S;
        long ns = walk(&F, &r, chi_a, chi_b, &S);
        neu_t sg_sum = {0, 0}, sb = {0, 0};
        double q_start = 0.0, q_end = 0.0;
        for (long s = 0; s < ns; ++s) {
            const segment_t* sg = &S[s];
            double ig, ib;
            if (b->interp == 0) {
                size_t ci = cell_index(g, sg->cell[0], sg->cell[1], sg->cell[2]);
                const double* gc = G + 3 * ci;
                double qc = r.n[0] * gc[0] + r.n[1] * gc[1] + r.n[2] * gc[2];
                ig = ic_dg_ngp(qc, sg->chiA, sg->chiB, chis);
                ib = ic_ngp(bpref * delta[ci], sg->chiA, sg->chiB, chis);
                if (s == 0) q_start = qc;
                if (s == ns - 1) q_end = qc;
            } else {
                double Qg[8], Qb[8], d[4];
                for (int v = 0; v < 8; ++v) {
                    long vi = sg->cell[0] + (v & 1), vj = sg->cell[1] + ((v >> 1) & 1), vk = sg->cell[2] + ((v >> 2) & 1);
                    Qg[v] = vertex_radial_grad(g, G, r.n, vi, vj, vk);
                    double val[7];
                    vertex_value(g, NULL, delta, vi, vj, vk, val);
                    Qb[v] = bpref * val[6];
                }
                dn_coeffs(Qg, sg->a, sg->b, sg->c, h, r.st, r.ct, r.sp, r.cp, d);
                ig = ic_dg_trilinear(d, sg->chiA, sg->chiB, chis);
                ib = ic_trilinear(Qb, sg->a, sg->b, sg->c, h, r.st, r.ct, r.sp, r.cp, sg->chiA, sg->chiB, chis);
                if (s == 0) q_start = d[0];
                if (s == ns - 1) {
                    double R = S[ns - 1].chiB - sg->chiA;
                    q_end = d[0] + R * (d[1] + R * (d[2] + R * d[3]));
                }
            }
            neu_add(&sg_sum, ig);
            neu_add(&sb, ib);
        }
        if (ns > 0) {
            neu_add(&sg_sum, -lensing_g(S[0].chiA, chis) * q_start);
            neu_add(&sg_sum, lensing_g(S[ns - 1].chiB, chis) * q_end);
        }
        free(S);
        kgrad[slot] += scale * neu_val(&sg_sum);
        kborn[slot] += scale * neu_val(&sb);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Generic integrals I = int K(chi) Q dchi (Eqs. Ic, Icngp, Icfinal; Sec. 6)   */
/* ------------------------------------------------------------------------- */

/* Value of a scalar field at vertex (vi, vj, vk): the mean of the 8 cells
 * sharing it (Sec. 2.7). */
static double vertex_scalar(const ora_grid* g, const double* F, long vi, long vj, long vk)
{
    double v = 0.0;
    for (int di = -1; di <= 0; ++di)
        for (int dj = -1; dj <= 0; ++dj)
            for (int dk = -1; dk <= 0; ++dk) v += F[cell_index(g, vi + di, vj + dj, vk + dk)];
    return 0.125 * v;
}

/* Eq. (Icfinal) with a quadratic kernel K(chi) = k0 + k1 chi + k2 chi^2.
 * About chi_A, K = c0 + c1 s + c2 s^2 with s = chi - chi_A, c0 = K(chi_A),
 * c1 = k1 + 2 k2 chi_A, c2 = k2, and with R = chi_B - chi_A
 * int_{chi_B}^{chi_A} K s^{N-1} dchi = -(c0 R^N / N + c1 R^{N+1} / (N+1) + c2 R^{N+2} / (N+2)). */
static double ic_poly_trilinear(const double d[4], const double k[3], double chiA, double chiB)
{
    const double c0 = k[0] + chiA * (k[1] + chiA * k[2]), c1 = k[1] + 2.0 * k[2] * chiA, c2 = k[2];
    const double R = chiB - chiA;
    double sum = 0.0;
    for (int N = 1; N <= 4; ++N) {
        double RN = pow(R, N);
        sum -= d[N - 1] * (c0 * RN / N + c1 * RN * R / (N + 1) + c2 * RN * R * R / (N + 2));
    }
    return sum;
}

/* Eq. (Icngp) with the same kernel: Q_c [P(chi_A) - P(chi_B)], P' = K. */
static double ic_poly_ngp(double Qc, const double k[3], double chiA, double chiB)
{
    double PA = chiA * (k[0] + chiA * (k[1] / 2.0 + chiA * k[2] / 3.0));
    double PB = chiB * (k[0] + chiB * (k[1] / 2.0 + chiB * k[2] / 3.0));
    return Qc * (PA - PB);
}

/*
 * Two generic line-of-sight integrals per ray over one step: out_c +=
 * scale * sum over the crossed cells of int K_c(chi) Q_c dchi, with Q_c a
 * scalar field at cell centres (Q2 may be NULL: zero), taken at the centre
 * (NGP) or trilinear from the vertex means (Sec. 2.7), and K_c(chi) = k[3c] +
 * k[3c+1] chi + k[3c+2] chi^2. With Q = (Phi_curr - Phi_prev) / dt this is the
 * ISW integral of Sec. 6; with Q = delta and K = the lensing kernel, the
 * density term of Eq. (kappa2).
 */
int ora_trace_step_kq(const ora_bundle* b, const ora_grid* g, const double* Q1, const double* Q2,
                      double chi_a, double chi_b, double scale, const double* k, double* out1, double* out2,
                      int nthreads, const int64_t* rids, long nrids)
{
    if (!(chi_a > chi_b) || chi_b < 0.0) return -1;
    field_t F = {g, b, NULL, NULL};
    const double h = grid_h(g);
    const long nr = rids ? nrids : (long)b->nx * b->ny;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (long slot = 0; slot < nr; ++slot) {
        const long rid = rids ? (long)rids[slot] : slot;
        ray_geo r;
        make_ray(b, rid % b->nx, rid / b->nx, &r);
        segment_t* S;
        long ns = walk(&F, &r, chi_a, chi_b, &S);
        neu_t s1 = {0, 0}, s2 = {0, 0};
        for (long s = 0; s < ns; ++s) {
            const segment_t* sg = &S[s];
            double i1, i2 = 0.0;
            if (b->interp == 0) {
                size_t ci = cell_index(g, sg->cell[0], sg->cell[1], sg->cell[2]);
                i1 = ic_poly_ngp(Q1[ci], k, sg->chiA, sg->chiB);
                if (Q2) i2 = ic_poly_ngp(Q2[ci], k + 3, sg->chiA, sg->chiB);
            } else {
                double V1[8], V2[8], d[4];
                for (int v = 0; v < 8; ++v) {
                    long vi = sg->cell[0] + (v & 1), vj = sg->cell[1] + ((v >> 1) & 1), vk = sg->cell[2] + ((v >> 2) & 1);
                    V1[v] = vertex_scalar(g, Q1, vi, vj, vk);
                    V2[v] = Q2 ? vertex_scalar(g, Q2, vi, vj, vk) : 0.0;
                }
                dn_coeffs(V1, sg->a, sg->b, sg->c, h, r.st, r.ct, r.sp, r.cp, d);
                i1 = ic_poly_trilinear(d, k, sg->chiA, sg->chiB);
                if (Q2) {
                    dn_coeffs(V2, sg->a, sg->b, sg->c, h, r.st, r.ct, r.sp, r.cp, d);
                    i2 = ic_poly_trilinear(d, k + 3, sg->chiA, sg->chiB);
                }
            }
            neu_add(&s1, i1);
            neu_add(&s2, i2);
        }
        free(S);
        out1[slot] += scale * neu_val(&s1);
        out2[slot] += scale * neu_val(&s2);
    }
    return 0;
}

/* Segment list of one ray (for tests that integrate the field by brute force):
 * writes up to cap rows of (chiA, chiB, cell_x, cell_y, cell_z) and returns
 * the number of segments. */
long ora_ray_segments(const ora_bundle* b, const ora_grid* g, long rid, double chi_a, double chi_b,
                      double* rows, long cap)
{
    field_t F = {g, b, NULL, NULL};
    ray_geo r;
    make_ray(b, rid % b->nx, rid / b->nx, &r);
    segment_t* S;
    long ns = walk(&F, &r, chi_a, chi_b, &S);
    for (long s = 0; s < ns && s < cap; ++s) {
        rows[5 * s + 0] = S[s].chiA;
        rows[5 * s + 1] = S[s].chiB;
        rows[5 * s + 2] = (double)S[s].cell[0];
        rows[5 * s + 3] = (double)S[s].cell[1];
        rows[5 * s + 4] = (double)S[s].cell[2];
    }
    free(S);
    return ns;
}

/* Unit vector n of ray rid (Eq. raypos) and its projection weights. */
int ora_ray_direction(const ora_bundle* b, long rid, double n[3], double w[6])
{
    ray_geo r;
    make_ray(b, rid % b->nx, rid / b->nx, &r);
    for (int a = 0; a < 3; ++a) n[a] = r.n[a];
    for (int c = 0; c < 6; ++c) w[c] = r.w[c];
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Adjoint                                                                   */
/* ------------------------------------------------------------------------- */

/*
 * Gradient of L with respect to the centre fields, given dL/dkappa and
 * dL/dkborn per ray, for one step. Because kappa and kborn are linear in the
 * field, the gradient is the transpose of the forward map:
 *   1. per segment, dI/dQ_i (i over the 8 vertices, or the cell for NGP) by
 *      evaluating the same closed form on unit vectors;
 *   2. dQ_kappa/dH = the weights of Eq. (n1n1) + (n2n2); dQ_B/ddelta = bpref;
 *   3. the transpose of the 8-cell vertex mean.
 * Outputs (accumulated, +=): gH (6 per cell) and gdelta (1 per cell).
 * Runs on one thread: the scatter is the plain serial loop.
 */
int ora_trace_step_adjoint(const ora_bundle* b, const ora_grid* g,
                           double chi_a, double chi_b, double scale, double a_step,
                           const double* dL_dkappa, const double* dL_dkborn,
                           double* gH, double* gdelta)
{
    if (!(chi_a > chi_b) || chi_b < 0.0) return -1;
    field_t F = {g, b, NULL, NULL};
    const double bpref = 1.5 * g->omega_m * ORA_H0_OVER_C * ORA_H0_OVER_C / a_step;
    const double h = grid_h(g);
    const long nr = (long)b->nx * b->ny;
    for (long rid = 0; rid < nr; ++rid) {
        double gk = dL_dkappa ? dL_dkappa[rid] * scale : 0.0;
        double gb = dL_dkborn ? dL_dkborn[rid] * scale : 0.0;
        if (gk == 0.0 && gb == 0.0) continue;
        ray_geo r;
        make_ray(b, rid % b->nx, rid / b->nx, &r);
        segment_t* S;
        long ns = walk(&F, &r, chi_a, chi_b, &S);
        for (long s = 0; s < ns; ++s) {
            const segment_t* sg = &S[s];
            if (b->interp == 0) {
                double coef = ic_ngp(1.0, sg->chiA, sg->chiB, b->chi_s);
                size_t ci = cell_index(g, sg->cell[0], sg->cell[1], sg->cell[2]);
                for (int c = 0; c < 6; ++c) gH[6 * ci + c] += gk * coef * r.w[c];
                gdelta[ci] += gb * coef * bpref;
            } else {
                for (int v = 0; v < 8; ++v) {
                    double e[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                    e[v] = 1.0;
                    double coef = ic_trilinear(e, sg->a, sg->b, sg->c, h, r.st, r.ct, r.sp, r.cp,
                                               sg->chiA, sg->chiB, b->chi_s);
                    long vi = sg->cell[0] + (v & 1), vj = sg->cell[1] + ((v >> 1) & 1),
                         vk = sg->cell[2] + ((v >> 2) & 1);
                    /* transpose of the vertex mean: each of the 8 cells gets 1/8 */
                    for (int di = -1; di <= 0; ++di)
                        for (int dj = -1; dj <= 0; ++dj)
                            for (int dk = -1; dk <= 0; ++dk) {
                                size_t ci = cell_index(g, vi + di, vj + dj, vk + dk);
                                for (int c = 0; c < 6; ++c) gH[6 * ci + c] += 0.125 * gk * coef * r.w[c];
                                gdelta[ci] += 0.125 * gb * coef * bpref;
                            }
                }
            }
        }
        free(S);
    }
    return 0;
}

/* Transpose of ora_delta_from_tidal: gH_{xx,yy,zz} += gdelta / (1.5 Om (H0/c)^2). */
int ora_delta_from_tidal_adjoint(const ora_grid* g, const double* gdelta, double* gH)
{
    const double inv = 1.0 / (1.5 * g->omega_m * ORA_H0_OVER_C * ORA_H0_OVER_C);
    size_t nc = (size_t)g->n[0] * g->n[1] * g->n[2];
    for (size_t c = 0; c < nc; ++c)
        for (int k = 0; k < 3; ++k) gH[6 * c + k] += gdelta[c] * inv;
    return 0;
}

/* Transpose of ora_tidal_centres: scatter each stencil tap (accumulates). */
int ora_tidal_centres_adjoint(const ora_grid* g, const double* gH, double* gphi)
{
    const double h = grid_h(g);
    const double ih2 = 1.0 / (h * h), q = 0.25 * ih2;
    for (long i = 0; i < g->n[0]; ++i)
        for (long j = 0; j < g->n[1]; ++j)
            for (long k = 0; k < g->n[2]; ++k) {
                const double* G = gH + 6 * cell_index(g, i, j, k);
                gphi[cell_index(g, i - 1, j, k)] += G[0] * ih2;
                gphi[cell_index(g, i, j, k)] -= 2.0 * G[0] * ih2;
                gphi[cell_index(g, i + 1, j, k)] += G[0] * ih2;
                gphi[cell_index(g, i, j - 1, k)] += G[1] * ih2;
                gphi[cell_index(g, i, j, k)] -= 2.0 * G[1] * ih2;
                gphi[cell_index(g, i, j + 1, k)] += G[1] * ih2;
                gphi[cell_index(g, i, j, k - 1)] += G[2] * ih2;
                gphi[cell_index(g, i, j, k)] -= 2.0 * G[2] * ih2;
                gphi[cell_index(g, i, j, k + 1)] += G[2] * ih2;
                gphi[cell_index(g, i + 1, j + 1, k)] += G[3] * q;
                gphi[cell_index(g, i - 1, j - 1, k)] += G[3] * q;
                gphi[cell_index(g, i + 1, j - 1, k)] -= G[3] * q;
                gphi[cell_index(g, i - 1, j + 1, k)] -= G[3] * q;
                gphi[cell_index(g, i + 1, j, k + 1)] += G[4] * q;
                gphi[cell_index(g, i - 1, j, k - 1)] += G[4] * q;
                gphi[cell_index(g, i + 1, j, k - 1)] -= G[4] * q;
                gphi[cell_index(g, i - 1, j, k + 1)] -= G[4] * q;
                gphi[cell_index(g, i, j + 1, k + 1)] += G[5] * q;
                gphi[cell_index(g, i, j - 1, k - 1)] += G[5] * q;
                gphi[cell_index(g, i, j + 1, k - 1)] -= G[5] * q;
                gphi[cell_index(g, i, j - 1, k + 1)] -= G[5] * q;
            }
    return 0;
}
