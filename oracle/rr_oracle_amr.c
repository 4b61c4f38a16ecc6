/*
 * FP64 CPU oracle, adaptive-mesh part (RAY-RAMSES, Barreira et al. 2016).
 *
 * TEST INFRASTRUCTURE ONLY, like rr_oracle.c: only the tests, the smoke
 * check and the benchmark's CPU baseline load it; it shares nothing with the
 * CUDA library.
 *
 * The mesh: a periodic n^3 coarse grid (level 0) whose cells may be refined
 * into octs of 8 children, down to level lmax, 2:1 balanced. Levels are
 * described by the sorted list of refined parent cells (octs) and the
 * potential at every cell centre of every level. Everything here is computed
 * plainly and on demand:
 *   - point location: descend from the coarse cell while the cell is refined
 *     (a refined cell is found by binary search in the sorted oct list);
 *   - d_a d_b Phi at a cell (Sec. 3.3): the central differences of Eq.
 *     (tidalexample) when all 18 same-level stencil neighbours exist,
 *     otherwise the coarse level's d_a d_b Phi interpolated (trilinearly, from
 *     the 8 nearest coarse centres) to the cell centre -- the second option of
 *     Sec. 3.3, which the paper adopts;
 *   - the value at a leaf vertex (Sec. 2.7): the mean of the 8 same-level
 *     leaves around it; at a vertex shared by coarse and fine leaves the
 *     weights of Eqs. (alphac3d), (alphaf3d), with N_fv,i the number of
 *     vertices of fine leaf i on the coarse-fine interface (hanging ones
 *     included); at a vertex in the middle of a coarse edge or face the mean
 *     of the 2 or 4 coarse vertices of that edge or face;
 *   - the walk: every face of the finest lattice crossed by the ray, merged
 *     over the three axes; consecutive pieces in the same leaf form one leaf
 *     segment; per leaf segment the integrals of rr_oracle.c with the leaf's
 *     own size h;
 *   - the shear (Eqs. gamma1, gamma2) by the same walk with the weights of
 *     rr_oracle.c's shear (printed Eqs. n1n1 - n2n2; Eq. n1n2 read in the
 *     orthonormal frame);
 *   - Method A (Eq. kappa2): d_a Phi per cell by central differences (the
 *     coarse level's interpolated where the same-level stencil is incomplete,
 *     as for the tidal tensor), vertex values by the same rules, the integral
 *     of (1 - 2 chi/chi_s) n.grad(Phi) per leaf segment and the step's
 *     surface terms at the ends of the traced interval (Eq. 2nterm);
 *   - generic integrals int K(chi) Q dchi of a scalar field with a quadratic
 *     kernel (Eqs. Ic, Icngp, Icfinal), its vertex values by the same rules.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define AMR_LMAX 8
#define ORA_H0_OVER_C_A (1.0 / 2997.92458)

typedef struct {
    int32_t n, lmax;
    double box, omega_m;
    const int32_t* octs[AMR_LMAX + 1];  /* octs[l]: m_l x 3 parent coords at level l-1, sorted */
    int64_t noct[AMR_LMAX + 1];
    const double* phi[AMR_LMAX + 1];     /* level 0: n^3; level l >= 1: m_l x 8 */
} ora_amr_desc;

typedef struct {
    int32_t nx, ny;
    double fov_x, fov_y, obs[3], chi_s;
    int32_t interp, periodic;
} ora_amr_bundle;

typedef struct {
    const ora_amr_desc* d;
    int64_t* keys[AMR_LMAX + 1];
    double* H[AMR_LMAX + 1];   /* 7 channels per cell of each level */
    int64_t ncell[AMR_LMAX + 1];
    int grad;                  /* channels 0-2 hold d_a Phi instead of d_a d_a Phi (Method A) */
    int scalar;                /* channel 0 holds the cell value itself (generic integrals) */
} amr_t;

/* ---------------------------------------------------------------- lookup */

static int64_t side(const amr_t* A, int l) { return (int64_t)A->d->n << l; }

static int64_t wrapa(int64_t i, int64_t m)
{
    int64_t r = i % m;
    return r < 0 ? r + m : r;
}

static int64_t key3(int64_t i, int64_t j, int64_t k, int64_t m) { return (i * m + j) * m + k; }

/* index of the oct at level l whose parent is level-(l-1) cell (i,j,k), or -1 */
static int64_t oct_find(const amr_t* A, int l, int64_t i, int64_t j, int64_t k)
{
    if (l < 1 || l > A->d->lmax) return -1;
    const int64_t m = side(A, l - 1);
    const int64_t key = key3(wrapa(i, m), wrapa(j, m), wrapa(k, m), m);
    int64_t lo = 0, hi = A->d->noct[l] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        int64_t km = A->keys[l][mid];
        if (km == key) return mid;
        if (km < key) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

/* flat index of cell (l, i, j, k) within its level, or -1 if it does not exist */
static int64_t cell_find(const amr_t* A, int l, int64_t i, int64_t j, int64_t k)
{
    const int64_t m = side(A, l);
    i = wrapa(i, m); j = wrapa(j, m); k = wrapa(k, m);
    if (l == 0) return key3(i, j, k, m);
    int64_t o = oct_find(A, l, i >> 1, j >> 1, k >> 1);
    if (o < 0) return -1;
    return o * 8 + (i & 1) + 2 * (j & 1) + 4 * (k & 1);
}

static int is_refined(const amr_t* A, int l, int64_t i, int64_t j, int64_t k)
{
    return l < A->d->lmax && oct_find(A, l + 1, i, j, k) >= 0;
}

/* leaf containing the finest-lattice point (2 X + s) / 2 (half-integer
 * finest coordinates: X a lattice point, s in {-1, +1}^3); level in *lvl,
 * integer cell coords at that level in c[3] */
static void leaf_of_half(const amr_t* A, const int64_t X[3], const int s[3], int* lvl, int64_t c[3])
{
    const int L = A->d->lmax;
    int l = 0;
    for (;;) {
        for (int a = 0; a < 3; ++a) {
            /* floor((2X + s) / 2^(L - l + 1)) */
            int64_t num = 2 * X[a] + s[a];
            int64_t den = (int64_t)1 << (L - l + 1);
            int64_t q = num / den;
            if (num % den != 0 && num < 0) q -= 1;
            c[a] = wrapa(q, side(A, l));
        }
        if (!is_refined(A, l, c[0], c[1], c[2])) break;
        ++l;
    }
    *lvl = l;
}

/* leaf containing the point p (box coordinates) */
static void leaf_of_point(const amr_t* A, const double p[3], int* lvl, int64_t c[3])
{
    int l = 0;
    const double h0 = A->d->box / A->d->n;
    for (;;) {
        const double hl = h0 / (double)((int64_t)1 << l);
        for (int a = 0; a < 3; ++a) c[a] = wrapa((int64_t)floor(p[a] / hl), side(A, l));
        if (!is_refined(A, l, c[0], c[1], c[2])) break;
        ++l;
    }
    *lvl = l;
}

/* ------------------------------------------------------- tidal per cell */

static double phi_at(const amr_t* A, int l, int64_t idx) { return A->d->phi[l][idx]; }

static int tidal_at(amr_t* A, int l, int64_t i, int64_t j, int64_t k, double out[7]);

/* Eq. (tidalexample) if the 18 same-level neighbours exist; returns 0 if not */
static int tidal_fd(const amr_t* A, int l, int64_t i, int64_t j, int64_t k, double out[7])
{
    static const int offs[18][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1},
                                    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
                                    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    double v[18];
    for (int t = 0; t < 18; ++t) {
        int64_t idx = cell_find(A, l, i + offs[t][0], j + offs[t][1], k + offs[t][2]);
        if (idx < 0) return 0;
        v[t] = phi_at(A, l, idx);
    }
    const double p0 = phi_at(A, l, cell_find(A, l, i, j, k));
    const double h = A->d->box / A->d->n / (double)((int64_t)1 << l);
    const double ih2 = 1.0 / (h * h), q = 0.25 * ih2;
    out[0] = (v[0] - 2.0 * p0 + v[1]) * ih2;
    out[1] = (v[2] - 2.0 * p0 + v[3]) * ih2;
    out[2] = (v[4] - 2.0 * p0 + v[5]) * ih2;
    out[3] = (v[6] + v[7] - v[8] - v[9]) * q;
    out[4] = (v[10] + v[11] - v[12] - v[13]) * q;
    out[5] = (v[14] + v[15] - v[16] - v[17]) * q;
    if (A->grad) {
        /* Method A: the central first differences, with delta from the
         * Laplacian of the second differences (as for the tidal tensor) */
        const double lap = out[0] + out[1] + out[2];
        out[0] = 0.5 * (v[1] - v[0]) / h;
        out[1] = 0.5 * (v[3] - v[2]) / h;
        out[2] = 0.5 * (v[5] - v[4]) / h;
        out[3] = out[4] = 0.0;
        out[5] = lap;   /* moved to channel 6 by tidal_at */
    }
    return 1;
}

static int tidal_at(amr_t* A, int l, int64_t i, int64_t j, int64_t k, double out[7])
{
    int64_t idx = cell_find(A, l, i, j, k);
    if (idx < 0) return -1;
    double* memo = A->H[l] + 8 * idx;
    if (memo[7] == 1.0) {
        for (int c = 0; c < 7; ++c) out[c] = memo[c];
        return 0;
    }
    if (A->scalar) {
        /* generic integrals: the field's own cell value */
        for (int c = 0; c < 7; ++c) out[c] = 0.0;
        out[0] = phi_at(A, l, idx);
        for (int c = 0; c < 7; ++c) memo[c] = out[c];
        memo[7] = 1.0;
        return 0;
    }
    const double pref = 1.5 * A->d->omega_m * ORA_H0_OVER_C_A * ORA_H0_OVER_C_A;
    double delta;   /* Method A: delta of the cell */
    if (tidal_fd(A, l, i, j, k, out)) {
        delta = out[5] / pref;   /* (grad mode: channel 5 holds the Laplacian) */
    } else {
        /* coarse d_a d_b Phi interpolated to the fine centre (Sec. 3.3):
         * fine centre in coarse units = i/2 - 1/4 */
        int64_t c0[3];
        double f[3];
        const int64_t ii[3] = {wrapa(i, side(A, l)), wrapa(j, side(A, l)), wrapa(k, side(A, l))};
        for (int a = 0; a < 3; ++a) {
            if (ii[a] % 2 == 0) { c0[a] = ii[a] / 2 - 1; f[a] = 0.75; }
            else { c0[a] = (ii[a] - 1) / 2; f[a] = 0.25; }
        }
        double lap = 0.0;
        for (int c = 0; c < 6; ++c) out[c] = 0.0;
        for (int t = 0; t < 8; ++t) {
            const int dx = t & 1, dy = (t >> 1) & 1, dz = (t >> 2) & 1;
            double hc[7];
            if (tidal_at(A, l - 1, c0[0] + dx, c0[1] + dy, c0[2] + dz, hc) != 0) return -1;
            const double wgt = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
            for (int c = 0; c < 6; ++c) out[c] += wgt * hc[c];
            lap += wgt * hc[6];
        }
        delta = lap;   /* Method A: the coarse delta interpolated like the gradient */
    }
    if (A->grad) {
        out[5] = 0.0;
        out[6] = delta;
    } else {
        /* delta from the comoving Poisson equation at a = 1 */
        out[6] = (out[0] + out[1] + out[2]) / pref;
    }
    for (int c = 0; c < 7; ++c) memo[c] = out[c];
    memo[7] = 1.0;
    return 0;
}

/* ---------------------------------------------------- vertex values (2.7) */

typedef struct {
    int n;
    int cap;
    int lvl[64];
    int64_t c[64][3];
    double w[64];
} combo_t;

static void combo_add(combo_t* cb, int lvl, const int64_t c[3], double w)
{
    for (int t = 0; t < cb->n; ++t)
        if (cb->lvl[t] == lvl && cb->c[t][0] == c[0] && cb->c[t][1] == c[1] && cb->c[t][2] == c[2]) {
            cb->w[t] += w;
            return;
        }
    if (cb->n < 64) {
        cb->lvl[cb->n] = lvl;
        cb->c[cb->n][0] = c[0]; cb->c[cb->n][1] = c[1]; cb->c[cb->n][2] = c[2];
        cb->w[cb->n] = w;
        cb->n++;
    }
}

/* does some leaf around lattice point W have a level below lf? */
static int touches_coarser(const amr_t* A, const int64_t W[3], int lf)
{
    for (int o = 0; o < 8; ++o) {
        int s[3] = {(o & 1) ? 1 : -1, (o & 2) ? 1 : -1, (o & 4) ? 1 : -1};
        int lv;
        int64_t c[3];
        leaf_of_half(A, W, s, &lv, c);
        if (lv < lf) return 1;
    }
    return 0;
}

/* The vertex value at finest-lattice point V as a combination of leaf values. */
static int vertex_combo(const amr_t* A, const int64_t Vin[3], double scale, combo_t* out)
{
    const int L = A->d->lmax;
    const int64_t M = side(A, L);
    int64_t V[3] = {wrapa(Vin[0], M), wrapa(Vin[1], M), wrapa(Vin[2], M)};
    int lv[8];
    int64_t cc[8][3];
    int lmin = 99, lmx = -1;
    for (int o = 0; o < 8; ++o) {
        int s[3] = {(o & 1) ? 1 : -1, (o & 2) ? 1 : -1, (o & 4) ? 1 : -1};
        leaf_of_half(A, V, s, &lv[o], cc[o]);
        if (lv[o] < lmin) lmin = lv[o];
        if (lv[o] > lmx) lmx = lv[o];
    }
    if (lmx == lmin) {
        /* 8 cells of one level around a vertex: their mean */
        for (int o = 0; o < 8; ++o) combo_add(out, lv[o], cc[o], scale * 0.125);
        return 0;
    }
    if (lmx - lmin > 1) return -1; /* not 2:1 balanced */
    const int64_t cstep = (int64_t)1 << (L - lmin); /* coarse lattice spacing in finest units */
    const int64_t fstep = (int64_t)1 << (L - lmx);
    int odd[3], nodd = 0;
    for (int a = 0; a < 3; ++a) {
        odd[a] = (V[a] % cstep) != 0;
        nodd += odd[a];
    }
    if (nodd == 0) {
        /* vertex shared by coarse and fine leaves: Eqs. (alphac3d), (alphaf3d) */
        int Nc = 0;
        double sum_fv = 0.0;
        int nfv[8];
        for (int o = 0; o < 8; ++o) {
            nfv[o] = 0;
            if (lv[o] == lmin) { ++Nc; continue; }
            /* N_fv: vertices of this fine leaf on the coarse-fine interface */
            for (int t = 0; t < 8; ++t) {
                int64_t W[3];
                const int64_t d3[3] = {t & 1, (t >> 1) & 1, (t >> 2) & 1};
                for (int a = 0; a < 3; ++a) W[a] = (cc[o][a] + d3[a]) * fstep;
                nfv[o] += touches_coarser(A, W, lmx);
            }
            sum_fv += nfv[o];
        }
        const double ac = 1.0 / ((double)Nc + sum_fv / 8.0);
        for (int o = 0; o < 8; ++o) {
            if (lv[o] == lmin) combo_add(out, lv[o], cc[o], scale * ac);
            else combo_add(out, lv[o], cc[o], scale * ac * (double)nfv[o] / 8.0);
        }
        return 0;
    }
    if (nodd == 3) return -2;
    /* middle of a coarse edge (1 odd axis) or face (2): mean of its coarse vertices */
    const int npts = 1 << nodd;
    for (int t = 0; t < npts; ++t) {
        int64_t W[3] = {V[0], V[1], V[2]};
        int bit = 0;
        for (int a = 0; a < 3; ++a)
            if (odd[a]) {
                W[a] += ((t >> bit) & 1) ? fstep : -fstep;
                ++bit;
            }
        if (vertex_combo(A, W, scale / (double)npts, out) != 0) return -3;
    }
    return 0;
}

static int vertex_value(amr_t* A, const int64_t V[3], double out[7])
{
    combo_t cb;
    cb.n = 0;
    cb.cap = 64;
    int rc = vertex_combo(A, V, 1.0, &cb);
    if (rc != 0) return rc;
    for (int c = 0; c < 7; ++c) out[c] = 0.0;
    for (int t = 0; t < cb.n; ++t) {
        double h[7];
        if (tidal_at(A, cb.lvl[t], cb.c[t][0], cb.c[t][1], cb.c[t][2], h) != 0) return -4;
        for (int c = 0; c < 7; ++c) out[c] += cb.w[t] * h[c];
    }
    return 0;
}

/* ------------------------------------------------------------ setup API */

static int amr_init(amr_t* A, const ora_amr_desc* d)
{
    memset(A, 0, sizeof(*A));
    A->d = d;
    for (int l = 0; l <= d->lmax; ++l) {
        A->ncell[l] = l == 0 ? (int64_t)d->n * d->n * d->n : d->noct[l] * 8;
        A->H[l] = (double*)calloc((size_t)A->ncell[l] * 8, sizeof(double));
        if (!A->H[l]) return -1;
        if (l >= 1) {
            const int64_t m = side(A, l - 1);
            A->keys[l] = (int64_t*)malloc(sizeof(int64_t) * (size_t)(d->noct[l] > 0 ? d->noct[l] : 1));
            for (int64_t o = 0; o < d->noct[l]; ++o)
                A->keys[l][o] = key3(d->octs[l][3 * o], d->octs[l][3 * o + 1], d->octs[l][3 * o + 2], m);
        }
    }
    return 0;
}

static void amr_free(amr_t* A)
{
    for (int l = 0; l <= AMR_LMAX; ++l) {
        free(A->H[l]);
        free(A->keys[l]);
    }
}

/* Vertex value combination at finest-lattice point V: up to cap (leaf level,
 * i, j, k, weight) rows; returns the number of rows, or < 0 on error. */
long ora_amr_vertex_weights(const ora_amr_desc* d, const int64_t V[3], double* rows, long cap)
{
    amr_t A;
    if (amr_init(&A, d) != 0) return -10;
    combo_t cb;
    cb.n = 0;
    cb.cap = 64;
    int rc = vertex_combo(&A, V, 1.0, &cb);
    amr_free(&A);
    if (rc != 0) return rc;
    for (long t = 0; t < cb.n && t < cap; ++t) {
        rows[5 * t + 0] = cb.lvl[t];
        rows[5 * t + 1] = (double)cb.c[t][0];
        rows[5 * t + 2] = (double)cb.c[t][1];
        rows[5 * t + 3] = (double)cb.c[t][2];
        rows[5 * t + 4] = cb.w[t];
    }
    return cb.n;
}

/* d_a d_b Phi and delta (7 channels) at every cell of every level, in the
 * level order of the description (level 0 row-major, then octs x 8). */
int ora_amr_tidal(const ora_amr_desc* d, double* out)
{
    amr_t A;
    if (amr_init(&A, d) != 0) return -10;
    int64_t off = 0;
    for (int l = 0; l <= d->lmax; ++l) {
        for (int64_t idx = 0; idx < A.ncell[l]; ++idx) {
            int64_t i, j, k;
            if (l == 0) {
                i = idx / ((int64_t)d->n * d->n); j = (idx / d->n) % d->n; k = idx % d->n;
            } else {
                const int64_t o = idx / 8, ch = idx % 8;
                i = 2 * d->octs[l][3 * o] + (ch & 1);
                j = 2 * d->octs[l][3 * o + 1] + ((ch >> 1) & 1);
                k = 2 * d->octs[l][3 * o + 2] + ((ch >> 2) & 1);
            }
            if (tidal_at(&A, l, i, j, k, out + 7 * (off + idx)) != 0) {
                amr_free(&A);
                return -1;
            }
        }
        off += A.ncell[l];
    }
    amr_free(&A);
    return 0;
}

/* The 8 vertex values (7 channels each, P_1..P_8 order) of leaf (l, i, j, k). */
int ora_amr_leaf_vertices(const ora_amr_desc* d, int l, const int64_t c[3], double* out)
{
    amr_t A;
    if (amr_init(&A, d) != 0) return -10;
    const int64_t step = (int64_t)1 << (d->lmax - l);
    int rc = 0;
    for (int t = 0; t < 8 && rc == 0; ++t) {
        int64_t V[3] = {(c[0] + (t & 1)) * step, (c[1] + ((t >> 1) & 1)) * step, (c[2] + ((t >> 2) & 1)) * step};
        rc = vertex_value(&A, V, out + 7 * t);
    }
    amr_free(&A);
    return rc;
}

/* ----------------------------------------------------------------- trace */

static int cmp_desc_a(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x < y) - (x > y);
}

static double ic_ngp_a(double Qc, double chiA, double chiB, double chis)
{
    return Qc / chis * (0.5 * chis * (chiA * chiA - chiB * chiB) - (chiA * chiA * chiA - chiB * chiB * chiB) / 3.0);
}

/* Eq. (Iclensing) with the alpha of Eq. (trilinear_coef) and the d_N of App. B */
/* the d_N of Eq. (Qcompact) (Appendix B) for the trilinear field of the
 * corner values Q along the ray from A = P_1 + (a, b, c) */
static void dn_a(const double Q[8], double a, double b, double c, double h, double nx, double ny, double nz,
                 double d[4])
{
    double al1 = Q[0], al2 = Q[1] - Q[0], al3 = Q[2] - Q[0], al4 = Q[4] - Q[0];
    double al5 = Q[3] - Q[2] - Q[1] + Q[0];
    double al6 = Q[6] - Q[4] - Q[2] + Q[0];
    double al7 = Q[5] - Q[4] - Q[1] + Q[0];
    double al8 = Q[7] - Q[6] - Q[5] - Q[3] + Q[1] + Q[4] + Q[2] - Q[0];
    double h2 = h * h, h3 = h2 * h;
    d[0] = al1 + (al2 * a + al3 * b + al4 * c) / h + (al5 * a * b + al6 * b * c + al7 * a * c) / h2
           + al8 * a * b * c / h3;
    d[1] = (al2 * nx + al3 * ny + al4 * nz) / h
           + ((al6 * c + al5 * a) * ny + (al7 * c + al5 * b) * nx + (al7 * a + al6 * b) * nz) / h2
           + (al8 * b * c * nx + al8 * a * b * nz + al8 * a * c * ny) / h3;
    d[2] = (al5 * nx * ny + al7 * nx * nz + al6 * ny * nz) / h2
           + (al8 * a * ny * nz + al8 * b * nx * nz + al8 * c * nx * ny) / h3;
    d[3] = al8 / h3 * nx * ny * nz;
}

static double ic_tri_a(const double Q[8], double a, double b, double c, double h, double nx, double ny,
                       double nz, double chiA, double chiB, double chis)
{
    double d[4];
    dn_a(Q, a, b, c, h, nx, ny, nz, d);
    double R = chiB - chiA, sum = 0.0;
    for (int N = 1; N <= 4; ++N) {
        double RN = pow(R, N);
        sum += d[N - 1] * (RN / N * (chiA - chis) * chiA + RN * R / (N + 1) * (2.0 * chiA - chis)
                           + RN * R * R / (N + 2));
    }
    return sum / chis;
}

/* Method A (Eq. kappa2): Eq. (Icfinal) with K = dg/dchi = 1 - 2 chi/chi_s
 * for the cubic d_N; R = chi_B - chi_A */
static double ic_dg_tri_a(const double d[4], double chiA, double chiB, double chis)
{
    double R = chiB - chiA, sum = 0.0;
    for (int N = 1; N <= 4; ++N) {
        double RN = pow(R, N);
        sum += d[N - 1] * (-(1.0 - 2.0 * chiA / chis) * RN / N + 2.0 / chis * RN * R / (N + 1));
    }
    return sum;
}

static double pixel_angle_a(double fov, long n, long i)
{
    return n > 1 ? (double)(2 * i - (n - 1)) * (fov / (2.0 * (double)(n - 1))) : 0.0;
}

typedef struct { double sum, comp; } neu_a;

static void neu_add_a(neu_a* s, double x)
{
    double t = s->sum + x;
    if (fabs(s->sum) >= fabs(x)) s->comp += (s->sum - t) + x;
    else s->comp += (x - t) + s->sum;
    s->sum = t;
}

/*
 * One step [chi_b, chi_a] for the listed rays (or all rays when rids is NULL):
 * kappa, kborn += scale * (integrals); nseg += leaf segments. Outputs follow
 * the list order (or rayid order). shear: the two channels are the shear
 * gamma1, gamma2 (Eqs. gamma1, gamma2) instead: Q = n1n1 - n2n2 from the
 * printed Eqs. (n1n1), (n2n2), and Q = 2 n1n2 with Eq. (n1n2) in its
 * orthonormal reading (the printed form times sin theta).
 */
static int amr_trace(const ora_amr_bundle* b, const ora_amr_desc* d, double chi_a, double chi_b, double scale,
                     double a_step, double* kappa, double* kborn, int64_t* nseg, const int64_t* rids, long nrids,
                     int mode, const double* kq);

int ora_amr_trace_step(const ora_amr_bundle* b, const ora_amr_desc* d, double chi_a, double chi_b, double scale,
                       double a_step, double* kappa, double* kborn, int64_t* nseg, const int64_t* rids,
                       long nrids, int nthreads)
{
    (void)nthreads;
    return amr_trace(b, d, chi_a, chi_b, scale, a_step, kappa, kborn, nseg, rids, nrids, 0, NULL);
}

int ora_amr_trace_step_shear(const ora_amr_bundle* b, const ora_amr_desc* d, double chi_a, double chi_b,
                             double scale, double* gamma1, double* gamma2, const int64_t* rids, long nrids)
{
    return amr_trace(b, d, chi_a, chi_b, scale, 1.0, gamma1, gamma2, NULL, rids, nrids, 1, NULL);
}

/* Method A (Eq. kappa2) through the adaptive mesh: kgrad += scale * (the
 * leaf-segment integrals of (1 - 2 chi/chi_s) n.grad(Phi) - [g n.grad(Phi)]
 * at the start + [g n.grad(Phi)] at the end of the traced interval), kborn +=
 * the density term; d_a Phi per cell by central differences where the
 * same-level stencil is complete, else the coarse level's interpolated (the
 * rule of Sec. 3.3 for the tidal tensor), vertex values by the Sec. 2.7 rules. */
int ora_amr_trace_step_method_a(const ora_amr_bundle* b, const ora_amr_desc* d, double chi_a, double chi_b,
                                double scale, double a_step, double* kgrad, double* kborn, const int64_t* rids,
                                long nrids)
{
    return amr_trace(b, d, chi_a, chi_b, scale, a_step, kgrad, kborn, NULL, rids, nrids, 2, NULL);
}

/* A generic integral int K(chi) Q dchi through the adaptive mesh (Eqs. Ic,
 * Icngp, Icfinal): Q is the scalar field given in place of the potential
 * (its cell values; vertex values by the Sec. 2.7 rules), K(chi) = k[0] +
 * k[1] chi + k[2] chi^2; out += scale * (leaf-segment integrals). */
int ora_amr_trace_step_kq(const ora_amr_bundle* b, const ora_amr_desc* d, double chi_a, double chi_b, double scale,
                          const double* k, double* out, const int64_t* rids, long nrids)
{
    const long nr = rids ? nrids : (long)b->nx * b->ny;
    double* unused = (double*)calloc((size_t)(nr > 0 ? nr : 1), sizeof(double));
    int rc = amr_trace(b, d, chi_a, chi_b, scale, 1.0, out, unused, NULL, rids, nrids, 3, k);
    free(unused);
    return rc;
}

static int amr_trace(const ora_amr_bundle* b, const ora_amr_desc* d, double chi_a, double chi_b, double scale,
                     double a_step, double* kappa, double* kborn, int64_t* nseg, const int64_t* rids, long nrids,
                     int mode, const double* kq)
{
    const int shear = mode == 1, method_a = mode == 2, generic = mode == 3;
    if (!(chi_a > chi_b) || chi_b < 0.0) return -1;
    amr_t A;
    if (amr_init(&A, d) != 0) return -10;
    A.grad = method_a;
    A.scalar = generic;
    const double bpref = 1.5 * d->omega_m * ORA_H0_OVER_C_A * ORA_H0_OVER_C_A / a_step;
    const double h0 = d->box / d->n;
    const double hf = h0 / (double)((int64_t)1 << d->lmax);
    const long nr = rids ? nrids : (long)b->nx * b->ny;
    int err = 0;
    /* single thread: the memoised tidal field is shared */
    for (long slot = 0; slot < nr && !err; ++slot) {
        const long rid = rids ? (long)rids[slot] : slot;
        const long ix = rid % b->nx, iy = rid / b->nx;
        double tx = pixel_angle_a(b->fov_x, b->nx, ix), ty = pixel_angle_a(b->fov_y, b->ny, iy);
        double th = sqrt(tx * tx + ty * ty);
        double sp = th > 0 ? ty / th : 0.0, cp = th > 0 ? tx / th : 1.0;
        double st = sin(th), ct = cos(th);
        double n[3] = {st * cp, st * sp, ct};
        /* Eqs. (n1n1) + (n2n2) */
        double s2p = 2.0 * sp * cp, s2t = sin(2.0 * th);
        double w[6] = {sp * sp + cp * cp * ct * ct, cp * cp + sp * sp * ct * ct, st * st, -s2p + s2p * ct * ct,
                       -cp * s2t, -sp * s2t};
        double w2[6] = {0, 0, 0, 0, 0, 0};
        if (shear) {
            /* Eqs. (n1n1) - (n2n2) */
            w[0] = sp * sp - cp * cp * ct * ct;
            w[1] = cp * cp - sp * sp * ct * ct;
            w[2] = -st * st;
            w[3] = -s2p - s2p * ct * ct;
            w[4] = cp * s2t;
            w[5] = sp * s2t;
            /* 2 n1n2, Eq. (n1n2) times sin theta */
            w2[0] = -2.0 * ct * cp * sp;
            w2[1] = 2.0 * ct * cp * sp;
            w2[3] = 2.0 * ct * (cp * cp - sp * sp);
            w2[4] = 2.0 * st * sp;
            w2[5] = -2.0 * st * cp;
        }
        double lo = chi_b, hi = chi_a;
        if (!b->periodic) {
            for (int a = 0; a < 3; ++a) {
                double ext = (double)d->n * h0;
                if (n[a] == 0.0) {
                    if (b->obs[a] < 0 || b->obs[a] > ext) hi = lo;
                    continue;
                }
                double c0 = (0.0 - b->obs[a]) / n[a], c1 = (ext - b->obs[a]) / n[a];
                if (fmin(c0, c1) > lo) lo = fmin(c0, c1);
                if (fmax(c0, c1) < hi) hi = fmax(c0, c1);
            }
        }
        neu_a sk = {0, 0}, sb = {0, 0};
        long count = 0;
        /* Method A: n.grad(Phi) and chi at the start and the end of the interval */
        double q_start = 0.0, chi_start = 0.0, q_end = 0.0, chi_end = 0.0;
        if (hi > lo) {
            /* every finest-lattice face crossing in (lo, hi) */
            long cap = 2;
            for (int a = 0; a < 3; ++a) cap += (long)(fabs(n[a]) * (hi - lo) / hf) + 3;
            double* Lst = (double*)malloc(sizeof(double) * (size_t)cap);
            long m = 0;
            Lst[m++] = hi;
            Lst[m++] = lo;
            for (int a = 0; a < 3; ++a) {
                if (n[a] == 0.0) continue;
                double x0 = b->obs[a] + lo * n[a], x1 = b->obs[a] + hi * n[a];
                double xmin = fmin(x0, x1), xmax = fmax(x0, x1);
                for (long f = (long)floor(xmin / hf) + 1; (double)f * hf < xmax; ++f) {
                    double cc = ((double)f * hf - b->obs[a]) / n[a];
                    if (cc > lo && cc < hi && m < cap) Lst[m++] = cc;
                }
            }
            qsort(Lst, (size_t)m, sizeof(double), cmp_desc_a);
            /* group pieces by leaf */
            int cur_l = -1;
            int64_t cur_c[3] = {0, 0, 0};
            double segA = 0.0, segB = 0.0;
            long ucell[3] = {0, 0, 0};
            for (long s = 0; s < m; ++s) {
                const int at_end = (s + 1 == m);
                int have = 0;
                int lv = -1;
                int64_t c[3] = {0, 0, 0};
                double A_ = 0, B_ = 0;
                long uc[3] = {0, 0, 0};
                if (!at_end) {
                    A_ = Lst[s];
                    B_ = Lst[s + 1];
                    /* coincident crossings leave an empty piece or a rounding
                     * sliver: skip it (it joins the surrounding segments) */
                    if (!(A_ - B_ > 1e-12 * fmax(A_, hf))) continue;
                    double mid = 0.5 * (A_ + B_), p[3];
                    for (int a = 0; a < 3; ++a) p[a] = b->obs[a] + mid * n[a];
                    leaf_of_point(&A, p, &lv, c);
                    const double hl = h0 / (double)((int64_t)1 << lv);
                    for (int a = 0; a < 3; ++a) uc[a] = (long)floor(p[a] / hl);
                    have = 1;
                    if (cur_l == lv && c[0] == cur_c[0] && c[1] == cur_c[1] && c[2] == cur_c[2]) {
                        segB = B_;
                        continue;
                    }
                }
                if (cur_l >= 0) {
                    /* integrate the finished leaf segment [segB, segA] */
                    const double hl = h0 / (double)((int64_t)1 << cur_l);
                    double ik, ib;
                    if (b->interp == 0) {
                        double H[7];
                        if (tidal_at(&A, cur_l, cur_c[0], cur_c[1], cur_c[2], H) != 0) { err = 1; break; }
                        double qk = 0, q2 = 0;
                        for (int q = 0; q < 6; ++q) {
                            qk += w[q] * H[q];
                            q2 += w2[q] * H[q];
                        }
                        if (generic) {
                            ik = H[0] * (segA * (kq[0] + segA * (kq[1] / 2.0 + segA * kq[2] / 3.0))
                                         - segB * (kq[0] + segB * (kq[1] / 2.0 + segB * kq[2] / 3.0)));
                        } else if (method_a) {
                            const double qg = n[0] * H[0] + n[1] * H[1] + n[2] * H[2];
                            ik = qg * ((segA - segB) - (segA * segA - segB * segB) / b->chi_s);
                            if (count == 0) { q_start = qg; chi_start = segA; }
                            q_end = qg;
                            chi_end = segB;
                        } else {
                            ik = ic_ngp_a(qk, segA, segB, b->chi_s);
                        }
                        ib = ic_ngp_a(shear ? q2 : bpref * H[6], segA, segB, b->chi_s);
                    } else {
                        double Qk[8], Qb[8];
                        const int64_t step = (int64_t)1 << (d->lmax - cur_l);
                        for (int t = 0; t < 8; ++t) {
                            int64_t V[3] = {(cur_c[0] + (t & 1)) * step, (cur_c[1] + ((t >> 1) & 1)) * step,
                                            (cur_c[2] + ((t >> 2) & 1)) * step};
                            double val[7];
                            if (vertex_value(&A, V, val) != 0) { err = 1; break; }
                            Qk[t] = 0;
                            double q2 = 0;
                            for (int q = 0; q < 6; ++q) {
                                Qk[t] += w[q] * val[q];
                                q2 += w2[q] * val[q];
                            }
                            if (method_a) Qk[t] = n[0] * val[0] + n[1] * val[1] + n[2] * val[2];
                            if (generic) Qk[t] = val[0];
                            Qb[t] = shear ? q2 : bpref * val[6];
                        }
                        if (err) break;
                        double P1[3] = {(double)ucell[0] * hl, (double)ucell[1] * hl, (double)ucell[2] * hl};
                        double aa = b->obs[0] + segA * n[0] - P1[0];
                        double bb = b->obs[1] + segA * n[1] - P1[1];
                        double cc = b->obs[2] + segA * n[2] - P1[2];
                        if (generic) {
                            double dq[4];
                            dn_a(Qk, aa, bb, cc, hl, n[0], n[1], n[2], dq);
                            /* K about chi_A: c0 + c1 s + c2 s^2, s = chi - chi_A in [R, 0] */
                            const double c0 = kq[0] + segA * (kq[1] + segA * kq[2]), c1 = kq[1] + 2.0 * kq[2] * segA;
                            const double R = segB - segA;
                            ik = 0.0;
                            for (int N = 1; N <= 4; ++N) {
                                const double RN = pow(R, N);
                                ik -= dq[N - 1] * (c0 * RN / N + c1 * RN * R / (N + 1) + kq[2] * RN * R * R / (N + 2));
                            }
                        } else if (method_a) {
                            double dq[4];
                            dn_a(Qk, aa, bb, cc, hl, n[0], n[1], n[2], dq);
                            ik = ic_dg_tri_a(dq, segA, segB, b->chi_s);
                            if (count == 0) { q_start = dq[0]; chi_start = segA; }
                            const double R = segB - segA;
                            q_end = dq[0] + R * (dq[1] + R * (dq[2] + R * dq[3]));
                            chi_end = segB;
                        } else {
                            ik = ic_tri_a(Qk, aa, bb, cc, hl, n[0], n[1], n[2], segA, segB, b->chi_s);
                        }
                        ib = ic_tri_a(Qb, aa, bb, cc, hl, n[0], n[1], n[2], segA, segB, b->chi_s);
                    }
                    neu_add_a(&sk, ik);
                    neu_add_a(&sb, ib);
                    ++count;
                    cur_l = -1;
                }
                if (have) {
                    cur_l = lv;
                    cur_c[0] = c[0]; cur_c[1] = c[1]; cur_c[2] = c[2];
                    ucell[0] = uc[0]; ucell[1] = uc[1]; ucell[2] = uc[2];
                    segA = A_;
                    segB = B_;
                }
            }
            free(Lst);
        }
        if (method_a && count > 0) {
            /* the step's surface terms (Eq. 2nterm) */
            neu_add_a(&sk, -(b->chi_s - chi_start) * chi_start / b->chi_s * q_start);
            neu_add_a(&sk, (b->chi_s - chi_end) * chi_end / b->chi_s * q_end);
        }
        kappa[slot] += scale * (sk.sum + sk.comp);
        kborn[slot] += scale * (sb.sum + sb.comp);
        if (nseg) nseg[slot] += count;
    }
    amr_free(&A);
    return err ? -2 : 0;
}
