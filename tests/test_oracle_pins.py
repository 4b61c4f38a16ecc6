"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, an independent brute-force integration written here, an invariant, or
the paper's Gaussian-potential test (Sec. 4). A dropped term, a wrong sign or
index, or a transposed operand anywhere in the oracle fails at least one.
"""
import json
import math
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _const_H(shape, M):
    H = np.zeros(tuple(shape) + (6,))
    H[..., 0], H[..., 1], H[..., 2] = M[0, 0], M[1, 1], M[2, 2]
    H[..., 3], H[..., 4], H[..., 5] = M[0, 1], M[0, 2], M[1, 2]
    return H


# ---------------------------------------------------------------------------
# Ray geometry: Eq. (txty), Eq. (rayid), Eq. (raypos)
# ---------------------------------------------------------------------------

def test_ray_angles_and_rayid(oracle_lib):
    """Eq. (txty) puts the first and last rays at -Upsilon/2 and +Upsilon/2;
    Eq. (rayid) orders rays x fastest; Eq. (raypos) gives a unit vector whose
    transverse components point along (theta_x, theta_y)."""
    b = synth.Bundle(5, 3, 0.2, 0.1, (0, 0, 0), 10.0)
    for rid in range(b.nrays):
        ix, iy = rid % 5, rid // 5
        tx = 0.2 / 4 * ix - 0.1
        ty = 0.1 / 2 * iy - 0.05
        th = math.hypot(tx, ty)
        n, _ = oracle_lib.ray_direction(b, rid)
        assert abs(np.linalg.norm(n) - 1) < 1e-15
        assert abs(n[2] - math.cos(th)) < 1e-15
        if th > 0:
            assert np.allclose(n[:2], math.sin(th) * np.array([tx, ty]) / th, atol=1e-15)


def test_projection_is_transverse_laplacian(oracle_lib):
    """Eqs. (n1n1) + (n2n2) equal tr(H) - n^T H n for every direction (the
    Laplacian in the plane transverse to the ray)."""
    b = synth.Bundle(7, 7, 1.5, 1.2, (0, 0, 0), 10.0)
    rng = np.random.default_rng(0)
    A = rng.standard_normal((3, 3))
    M = A + A.T
    h6 = np.array([M[0, 0], M[1, 1], M[2, 2], M[0, 1], M[0, 2], M[1, 2]])
    for rid in range(b.nrays):
        n, w = oracle_lib.ray_direction(b, rid)
        assert abs(w @ h6 - (np.trace(M) - n @ M @ n)) < 1e-13


# ---------------------------------------------------------------------------
# P1, P9: constant tidal field -> closed form, NGP = trilinear
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("interp", [0, 1])
def test_constant_field_closed_form(oracle_lib, interp):
    """With H = M everywhere, Q = tr M - n^T M n is constant along the ray and
    kappa = Q [ (chi_a^2 - chi_b^2)/2 - (chi_a^3 - chi_b^3)/(3 chi_s) ] (the
    lensing kernel g of Eq. kappa integrated exactly). NGP and trilinear must
    both give it; the Born term then is 1.5 Om (H0/c)^2 delta / a times the
    same kernel integral."""
    g = synth.Grid((12, 12, 12), 48.0)
    b = synth.Bundle(9, 6, synth.deg(30), synth.deg(20), (20.0, 30.0, 1.0), 60.0, interp=interp)
    M = np.array([[1.0, 0.3, -0.2], [0.3, -0.5, 0.7], [-0.2, 0.7, 0.25]])
    H = _const_H(g.n, M)
    d = np.full(g.n, 2.5)
    steps = [synth.Step(47.0, 20.0, 1.3, 0.6), synth.Step(20.0, 0.5, 0.7, 0.8)]
    r = oracle_lib.trace(b, g, H, d, steps)
    pref = 1.5 * 0.3 * synth.H0_OVER_C ** 2
    for rid in range(b.nrays):
        n, _ = oracle_lib.ray_direction(b, rid)
        q = np.trace(M) - n @ M @ n
        ek = eb = 0.0
        for st in steps:
            G = (st.chi_a ** 2 - st.chi_b ** 2) / 2 - (st.chi_a ** 3 - st.chi_b ** 3) / (3 * b.chi_s)
            ek += st.scale * q * G
            eb += st.scale * pref * 2.5 / st.a * G
        assert abs(r.kappa[rid] - ek) <= 1e-13 * abs(ek) + 1e-15
        assert abs(r.kborn[rid] - eb) <= 1e-13 * abs(eb)


# ---------------------------------------------------------------------------
# Stencils, Eq. (tidalexample)
# ---------------------------------------------------------------------------

def test_stencils_exact_on_quadratic(oracle_lib):
    """Central differences are exact for a quadratic potential: away from the
    periodic seam, H = M at every cell."""
    n = 10
    g = synth.Grid((n, n, n), 5.0)
    h = g.h
    rng = np.random.default_rng(1)
    A = rng.standard_normal((3, 3))
    M = A + A.T
    x = (np.arange(n) + 0.5) * h
    X = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1)
    phi = 0.5 * np.einsum("...i,ij,...j->...", X, M, X) + X @ np.array([0.3, -0.1, 0.2])
    H = oracle_lib.tidal_centres(g, phi)[1:-1, 1:-1, 1:-1]
    want = np.array([M[0, 0], M[1, 1], M[2, 2], M[0, 1], M[0, 2], M[1, 2]])
    assert np.abs(H - want).max() < 1e-10 * np.abs(M).max() * 100


def test_stencils_periodic_fourier(oracle_lib):
    """On the periodic grid each stencil acting on a plane wave is exactly the
    symbol of the difference operator: (2 cos(k h) - 2)/h^2 on the diagonal and
    -sin(k_a h) sin(k_b h)/h^2 off it (each axis independently)."""
    n = 16
    g = synth.Grid((n, 12, 8), 32.0)
    h = g.h
    m = np.array([3, 2, 1])
    k = 2 * np.pi * m / (np.array(g.n) * h)
    idx = np.meshgrid(*[np.arange(s) for s in g.n], indexing="ij")
    ph = sum(k[a] * (idx[a] + 0.5) * h for a in range(3))
    phi = np.cos(ph)
    H = oracle_lib.tidal_centres(g, phi)
    diag = (2 * np.cos(k * h) - 2) / h ** 2
    for a in range(3):
        assert np.abs(H[..., a] - diag[a] * phi).max() < 1e-12
    for c, (a, bb) in zip((3, 4, 5), ((0, 1), (0, 2), (1, 2))):
        want = -np.sin(k[a] * h) * np.sin(k[bb] * h) / h ** 2 * phi
        assert np.abs(H[..., c] - want).max() < 1e-12


# ---------------------------------------------------------------------------
# P10: vertex values (Sec. 2.7)
# ---------------------------------------------------------------------------

def test_vertex_mean_conserves_mass(oracle_lib):
    """On a regular periodic mesh the vertex scheme conserves the total
    'mass' (Sec. 2.7: centre and vertex totals agree exactly), each vertex is
    the mean of its 8 cells (the weights sum to 1), and the mean over a cell's
    8 vertices summed over cells equals the centre total."""
    g = synth.Grid((6, 5, 7), 12.0)
    rng = np.random.default_rng(2)
    H = rng.standard_normal(tuple(g.n) + (6,))
    d = rng.standard_normal(g.n)
    V = oracle_lib.vertex_field(g, H, d)
    assert abs(V[..., 6].sum() - d.sum()) < 1e-12 * np.abs(d).sum()
    assert np.allclose(V[..., :6].sum(axis=(0, 1, 2)), H.sum(axis=(0, 1, 2)), atol=1e-11)
    # explicit mean for one vertex, including the periodic seam
    cells = [(i, j, k) for i in (-1, 0) for j in (-1, 0) for k in (-1, 0)]
    want = np.mean([d[i % 6, j % 5, k % 7] for (i, j, k) in cells])
    assert abs(V[0, 0, 0, 6] - want) < 1e-15
    # constant field -> constant vertices
    V1 = oracle_lib.vertex_field(g, np.ones_like(H), np.ones_like(d))
    assert np.abs(V1 - 1).max() < 1e-15


# ---------------------------------------------------------------------------
# P2: the walk tiles the interval
# ---------------------------------------------------------------------------

def test_segments_tile_the_interval(oracle_lib):
    """Sum of segment lengths = chi_a - chi_b per ray (Eq. sumIc); each segment
    lies in one cell; consecutive segments are face neighbours."""
    g = synth.Grid((8, 8, 8), 16.0)
    b = synth.Bundle(6, 5, synth.deg(50), synth.deg(40), (3.0, 14.0, 0.0), 40.0)
    r = oracle_lib.trace(b, g, np.zeros(tuple(g.n) + (6,)), np.zeros(g.n), [synth.Step(31.0, 2.0, 1, 1)])
    assert np.abs(r.sum_r - 29.0).max() < 1e-12 * 29
    for rid in (0, 7, 29):
        rows = oracle_lib.ray_segments(b, g, rid, 31.0, 2.0)
        n, _ = oracle_lib.ray_direction(b, rid)
        for chiA, chiB, cx, cy, cz in rows:
            for chi in (chiA, chiB):
                p = np.array(b.obs) + chi * n
                assert np.all(p >= np.array([cx, cy, cz]) * g.h - 1e-9)
                assert np.all(p <= (np.array([cx, cy, cz]) + 1) * g.h + 1e-9)
        # face neighbours, or edge/corner neighbours where the ray passes
        # through an edge or corner (the empty sliver between is skipped)
        steps = np.abs(np.diff(rows[:, 2:5], axis=0))
        assert np.all(steps.max(axis=1) == 1)


def test_box_clip_length(oracle_lib):
    """Without periodic wrap a ray stops at the box faces (Sec. 2.4 stop
    condition ii): the traced length is the chord inside the box."""
    g = synth.Grid((8, 8, 8), 10.0)
    b = synth.Bundle(5, 5, synth.deg(40), synth.deg(40), (5.0, 5.0, 0.0), 2000.0, periodic=False)
    r = oracle_lib.trace(b, g, np.zeros(tuple(g.n) + (6,)), np.zeros(g.n), [synth.Step(2000.0, 0.0, 1, 1)])
    for rid in range(b.nrays):
        n, _ = oracle_lib.ray_direction(b, rid)
        exits = []
        for a in range(3):
            if n[a] > 0:
                exits.append((10.0 - b.obs[a]) / n[a])
            elif n[a] < 0:
                exits.append((0.0 - b.obs[a]) / n[a])
        assert abs(r.sum_r[rid] - min(exits)) < 1e-12 * 10


# ---------------------------------------------------------------------------
# P3: closed-form integrals against brute-force quadrature of the field
# ---------------------------------------------------------------------------

def _vertex_np(Hc):
    """Independent vertex mean with np.roll: vertex (i,j,k) <- cells i-1..i."""
    out = np.zeros_like(Hc)
    for di in (0, 1):
        for dj in (0, 1):
            for dk in (0, 1):
                out += np.roll(Hc, shift=(di, dj, dk), axis=(0, 1, 2))
    return out / 8.0


def _trilerp(Vp, h, p):
    """Trilinear interpolation of the vertex array Vp (periodic) at points p."""
    n = np.array(Vp.shape[:3])
    u = p / h
    i0 = np.floor(u).astype(np.int64)
    f = u - i0
    out = 0.0
    for di in (0, 1):
        for dj in (0, 1):
            for dk in (0, 1):
                wgt = (f[:, 0] if di else 1 - f[:, 0]) * (f[:, 1] if dj else 1 - f[:, 1]) * \
                      (f[:, 2] if dk else 1 - f[:, 2])
                ii = (i0[:, 0] + di) % n[0]
                jj = (i0[:, 1] + dj) % n[1]
                kk = (i0[:, 2] + dk) % n[2]
                out = out + wgt[:, None] * Vp[ii, jj, kk]
    return out


def _gauss_legendre_line(fun, lo, hi, nsub):
    x, w = np.polynomial.legendre.leggauss(3)
    edges = np.linspace(lo, hi, nsub + 1)
    a, b = edges[:-1], edges[1:]
    pts = (0.5 * (b - a)[:, None] * x[None, :] + 0.5 * (a + b)[:, None]).ravel()
    wts = (0.5 * (b - a)[:, None] * w[None, :]).ravel()
    return float(np.sum(wts * fun(pts)))


@pytest.mark.parametrize("n,seed", [(4, 11), (8, 12)])
def test_trilinear_matches_bruteforce(oracle_lib, n, seed):
    """Eq. (Iclensing) with the d_N of Appendix B equals a brute-force
    composite Gauss-Legendre integral of g(chi) Q(x(chi)) where Q is the
    trilinear interpolant of the vertex values (Eq. trilinear_int), built here
    independently; rays wrap across the periodic seams."""
    g = synth.Grid((n, n, n), 4.0 * n)
    b = synth.Bundle(4, 3, synth.deg(60), synth.deg(50), (4.0 * n - 1.0, 1.0, 0.3), 5.0 * n, interp=1)
    phi = synth.random_field(g.n, seed)
    H, d = oracle_lib.fields(g, phi)
    steps = [synth.Step(4.7 * n, 0.2, 1.0, 0.9)]
    r = oracle_lib.trace(b, g, H, d, steps)
    Vp = _vertex_np(np.concatenate([H, d[..., None]], axis=-1))
    pref = 1.5 * 0.3 * synth.H0_OVER_C ** 2 / 0.9
    for rid in range(b.nrays):
        nh, _ = oracle_lib.ray_direction(b, rid)

        def integrand(chi, ch):
            p = np.array(b.obs)[None, :] + chi[:, None] * nh[None, :]
            V = _trilerp(Vp, g.h, p)
            M = np.zeros((len(chi), 3, 3))
            for c, (i, j) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))):
                M[:, i, j] = V[:, c]
                M[:, j, i] = V[:, c]
            q = np.trace(M, axis1=1, axis2=2) - np.einsum("i,nij,j->n", nh, M, nh)
            gk = (b.chi_s - chi) * chi / b.chi_s
            return gk * (q if ch == 0 else pref * V[:, 6])

        bk = _gauss_legendre_line(lambda c: integrand(c, 0), 0.2, 4.7 * n, 40000)
        bb = _gauss_legendre_line(lambda c: integrand(c, 1), 0.2, 4.7 * n, 40000)
        assert abs(r.kappa[rid] - bk) < 1e-7 * max(abs(bk), 1e-3)
        assert abs(r.kborn[rid] - bb) < 1e-7 * max(abs(bb), 1e-3 * pref)


def test_ngp_matches_bruteforce(oracle_lib):
    """Eq. (Iclensing_ngp): the NGP integral is the lensing kernel integrated
    against the piecewise-constant centre values; checked with a fine midpoint
    rule evaluated independently."""
    n = 6
    g = synth.Grid((n, n, n), 12.0)
    b = synth.Bundle(3, 3, synth.deg(40), synth.deg(40), (6.0, 6.0, 0.0), 15.0, interp=0)
    phi = synth.random_field(g.n, 13)
    H, d = oracle_lib.fields(g, phi)
    r = oracle_lib.trace(b, g, H, d, [synth.Step(11.5, 0.0, 1.0, 1.0)])
    npts = 2_000_000
    chi = (np.arange(npts) + 0.5) * (11.5 / npts)
    for rid in range(b.nrays):
        nh, _ = oracle_lib.ray_direction(b, rid)
        p = np.array(b.obs)[None, :] + chi[:, None] * nh[None, :]
        cell = np.floor(p / g.h).astype(np.int64) % n
        Hc = H[cell[:, 0], cell[:, 1], cell[:, 2]]
        M = np.zeros((npts, 3, 3))
        for c, (i, j) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))):
            M[:, i, j] = Hc[:, c]
            M[:, j, i] = Hc[:, c]
        q = np.trace(M, axis1=1, axis2=2) - np.einsum("i,nij,j->n", nh, M, nh)
        bk = np.sum((b.chi_s - chi) * chi / b.chi_s * q) * (11.5 / npts)
        assert abs(r.kappa[rid] - bk) < 2e-5 * np.abs(q).max() * 11.5 ** 2


# ---------------------------------------------------------------------------
# P4: the paper's Gaussian-potential test (Sec. 4)
# ---------------------------------------------------------------------------

def _gauss_q(p, centre, amp, sigma, nh):
    x = p - centre
    r2 = np.sum(x * x, axis=-1)
    e = amp * np.exp(-r2 / (2 * sigma ** 2))
    xn = x @ nh
    # tr(H) - n^T H n for H_ij = e (x_i x_j / s^4 - delta_ij / s^2)
    return e * ((r2 - xn * xn) / sigma ** 4 - 2.0 / sigma ** 2)


@pytest.mark.parametrize("n", [64])
def test_gaussian_potential_vs_quadrature(oracle_lib, n):
    """Sec. 4: a fixed Gaussian potential A exp(-r^2/2 sigma^2) in a 10 Mpc/h
    box, observer at the centre of a box face, 40x40 deg field, z_s = 0.95,
    trilinear Method B. kappa along a radial slice of the map agrees with an
    adaptive quadrature of the analytic integrand to the paper's 1% (zero
    crossings excluded), and the error shrinks with resolution."""
    from scipy.integrate import quad
    with open(os.path.join(GOLDEN, "gaussian_e1.json")) as f:
        E1 = json.load(f)
    L = E1["box"]
    amp, sig = E1["potential"]["amp"], E1["potential"]["sigma"]
    chis = synth.chi_of_z(E1["z_s"])
    nr = E1["rays"][0]
    b = synth.Bundle(nr, 1, synth.deg(E1["fov_deg"][0]), 0.0, (L / 2, L / 2, 0.0), chis, periodic=False)
    # one row of the map through its centre: theta_y = 0 (N_y = 1 reads Eq. txty as theta = 0)
    centre = np.full(3, L / 2)

    def run(ng):
        g = synth.Grid((ng, ng, ng), L)
        phi = synth.gaussian_phi(ng, L, amp, sig)
        H, d = oracle_lib.fields(g, phi)
        return oracle_lib.trace(b, g, H, d, [synth.Step(chis, 0.0, 1.0, 1.0)]).kappa

    kap = run(n)
    exact = np.zeros(nr)
    for rid in range(nr):
        nh, _ = oracle_lib.ray_direction(b, rid)
        exits = [((L if nh[a] > 0 else 0.0) - b.obs[a]) / nh[a] for a in range(3) if nh[a] != 0]
        top = min(exits)
        f = lambda c: (chis - c) * c / chis * _gauss_q(np.array(b.obs) + c * nh, centre, amp, sig, nh)
        exact[rid] = quad(f, 0.0, top, epsabs=0, epsrel=1e-11, limit=400, points=[L / 2])[0]
    keep = np.abs(exact) > 0.1 * np.abs(exact).max()
    rel = np.abs(kap - exact)[keep] / np.abs(exact[keep])
    assert rel.max() < E1["max_relative_error"][str(n)], rel.max()
    kap32 = run(32)
    rel32 = np.abs(kap32 - exact)[keep] / np.abs(exact[keep])
    assert rel32.max() < E1["max_relative_error"]["32"], rel32.max()
    assert rel.max() < rel32.max()


# ---------------------------------------------------------------------------
# P6, P7, P8: linearity, step splitting, symmetry
# ---------------------------------------------------------------------------

def test_linearity(oracle_lib):
    g = synth.Grid((8, 8, 8), 32.0)
    b = synth.Bundle(5, 4, synth.deg(20), synth.deg(15), (16.0, 16.0, 0.0), 40.0)
    p1, p2 = synth.random_field(g.n, 21), synth.random_field(g.n, 22)
    st = [synth.Step(31.0, 0.0, 1.0, 1.0)]
    r1 = oracle_lib.trace(b, g, *oracle_lib.fields(g, p1), st)
    r2 = oracle_lib.trace(b, g, *oracle_lib.fields(g, p2), st)
    r3 = oracle_lib.trace(b, g, *oracle_lib.fields(g, 2.0 * p1 - 0.5 * p2), st)
    want = 2.0 * r1.kappa - 0.5 * r2.kappa
    assert np.abs(r3.kappa - want).max() < 1e-12 * np.abs(want).max()


def test_step_splitting(oracle_lib):
    """Sec. 2.5.2: tracing in 40 steps with an unchanged field equals one step."""
    g = synth.Grid((8, 8, 8), 32.0)
    b = synth.Bundle(5, 4, synth.deg(20), synth.deg(15), (16.0, 16.0, 0.0), 31.0)
    H, d = oracle_lib.fields(g, synth.random_field(g.n, 23))
    one = oracle_lib.trace(b, g, H, d, [synth.Step(31.0, 0.0, 1.0, 1.0)])
    edges = np.linspace(31.0, 0.0, 41)
    many = oracle_lib.trace(b, g, H, d, [synth.Step(edges[i], edges[i + 1], 1.0, 1.0) for i in range(40)])
    assert np.abs(one.kappa - many.kappa).max() < 1e-12 * np.abs(one.kappa).max()
    assert np.abs(one.kborn - many.kborn).max() < 1e-12 * np.abs(one.kborn).max()


@pytest.mark.parametrize("interp", [0, 1])
def test_rotation_symmetry(oracle_lib, interp):
    """Rotating the potential by 90 degrees about the line of sight through the
    box centre rotates the map: the square bundle of Eq. (txty) maps onto itself."""
    n = 8
    g = synth.Grid((n, n, 6), 16.0)
    b = synth.Bundle(6, 6, synth.deg(30), synth.deg(30), (8.0, 8.0, 0.0), 13.0, interp=interp)
    phi = synth.random_field(g.n, 24)
    rot = np.ascontiguousarray(np.transpose(phi[:, ::-1, :], (1, 0, 2)))  # rot[i,j] = phi[j, n-1-i]
    st = [synth.Step(11.9, 0.0, 1.0, 1.0)]
    k0 = oracle_lib.trace(b, g, *oracle_lib.fields(g, phi), st).kappa.reshape(6, 6)
    k1 = oracle_lib.trace(b, g, *oracle_lib.fields(g, rot), st).kappa.reshape(6, 6)
    # kappa'[iy, ix] = kappa[N-1-ix, iy]
    want = np.array([[k0[5 - ix, iy] for ix in range(6)] for iy in range(6)])
    assert np.abs(k1 - want).max() < 1e-11 * np.abs(k0).max()


# ---------------------------------------------------------------------------
# P12: the adjoint is the transpose of the forward map
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("interp", [0, 1])
def test_adjoint_dot_product(oracle_lib, interp):
    """<J x, y> = <x, J^T y> for the whole chain Phi -> (kappa, kappa_Born)
    over two steps with different scales and scale factors."""
    g = synth.Grid((8, 8, 8), 32.0)
    b = synth.Bundle(6, 5, synth.deg(40), synth.deg(30), (16.0, 16.0, 0.0), 40.0, interp=interp)
    steps = [synth.Step(31.0, 14.0, 1.3, 0.7), synth.Step(14.0, 0.0, 0.9, 0.9)]
    x = synth.random_field(g.n, 31)
    rng = np.random.default_rng(32)
    yk, yb = rng.standard_normal(b.nrays), rng.standard_normal(b.nrays)
    r = oracle_lib.trace(b, g, *oracle_lib.fields(g, x), steps)
    lhs = r.kappa @ yk + r.kborn @ yb
    gphi, _ = oracle_lib.trace_adjoint(b, g, steps, yk, yb)
    rhs = float(np.sum(x * gphi))
    assert abs(lhs - rhs) < 1e-12 * (abs(r.kappa) @ abs(yk) + abs(r.kborn) @ abs(yb))
    # delta as an independent input: gradient splits between Phi and delta
    d = synth.random_field(g.n, 33)
    H, _ = oracle_lib.fields(g, x)
    r2 = oracle_lib.trace(b, g, H, d, steps)
    gphi2, gd2 = oracle_lib.trace_adjoint(b, g, steps, yk, yb, delta_derived=False)
    lhs2 = r2.kappa @ yk + r2.kborn @ yb
    rhs2 = float(np.sum(x * gphi2) + np.sum(d * gd2))
    assert abs(lhs2 - rhs2) < 1e-12 * (abs(r2.kappa) @ abs(yk) + abs(r2.kborn) @ abs(yb))
