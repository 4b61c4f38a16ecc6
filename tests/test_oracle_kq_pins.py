"""Pins of the oracle's generic line-of-sight integrals int K(chi) Q dchi
(Eqs. Ic, Icngp, Icfinal with a quadratic kernel; the ISW integral of Sec. 6)
and of box tiling with a relocated observer (Sec. 2.2). Each rests on a closed
form, brute-force quadrature written here, or an identity with another
oracle path."""
import math

import numpy as np
import pytest

import synth


def _vertex_np(F):
    out = np.zeros_like(F)
    for di in (0, 1):
        for dj in (0, 1):
            for dk in (0, 1):
                out += np.roll(F, shift=(di, dj, dk), axis=(0, 1, 2))
    return out / 8.0


def _trilerp(V, h, p):
    n = np.array(V.shape[:3])
    u = p / h
    i0 = np.floor(u).astype(np.int64)
    f = u - i0
    out = 0.0
    for di in (0, 1):
        for dj in (0, 1):
            for dk in (0, 1):
                wgt = (f[:, 0] if di else 1 - f[:, 0]) * (f[:, 1] if dj else 1 - f[:, 1]) * \
                      (f[:, 2] if dk else 1 - f[:, 2])
                out = out + wgt * V[(i0[:, 0] + di) % n[0], (i0[:, 1] + dj) % n[1], (i0[:, 2] + dk) % n[2]]
    return out


def _gl(fun, lo, hi, nsub):
    x, w = np.polynomial.legendre.leggauss(3)
    e = np.linspace(lo, hi, nsub + 1)
    a, b = e[:-1], e[1:]
    pts = (0.5 * (b - a)[:, None] * x[None, :] + 0.5 * (a + b)[:, None]).ravel()
    wts = (0.5 * (b - a)[:, None] * w[None, :]).ravel()
    return float(np.sum(wts * fun(pts)))


K1 = (0.7, -0.031, 0.0009)     # k0 + k1 chi + k2 chi^2
K2 = (-1.3, 0.2, -0.004)


@pytest.mark.parametrize("interp", [0, 1])
def test_constant_field_gives_the_kernel_integral(oracle_lib, interp):
    n = 8
    g = synth.Grid((n, n, n), 16.0)
    b = synth.Bundle(5, 4, synth.deg(30), synth.deg(20), (3.0, 13.0, 2.0), 40.0, interp=interp)
    Q1 = np.full(g.n, 2.5)
    Q2 = np.full(g.n, -0.75)
    steps = [synth.Step(37.0, 21.0, 1.2, 1.0), synth.Step(21.0, 0.5, 0.9, 1.0)]
    o1, o2 = oracle_lib.trace_kq(b, g, Q1, Q2, (K1, K2), steps)

    def P(k, x):
        return k[0] * x + k[1] * x ** 2 / 2 + k[2] * x ** 3 / 3
    w1 = sum(st.scale * 2.5 * (P(K1, st.chi_a) - P(K1, st.chi_b)) for st in steps)
    w2 = sum(st.scale * -0.75 * (P(K2, st.chi_a) - P(K2, st.chi_b)) for st in steps)
    assert np.abs(o1 - w1).max() < 1e-12 * abs(w1)
    assert np.abs(o2 - w2).max() < 1e-12 * abs(w2)


@pytest.mark.parametrize("n,seed", [(4, 21), (7, 22)])
def test_trilinear_matches_bruteforce(oracle_lib, n, seed):
    """Eq. (Icfinal) with the d_N of Appendix B and the quadratic kernel equals
    composite Gauss-Legendre quadrature of K(chi) Q(x(chi)), Q the trilinear
    interpolant of the vertex means built here; rays cross the periodic seams."""
    g = synth.Grid((n, n, n), 3.0 * n)
    b = synth.Bundle(4, 3, synth.deg(60), synth.deg(45), (3.0 * n - 1.0, 1.0, 0.3), 5.0 * n, interp=1)
    Q1 = synth.random_field(g.n, seed)
    Q2 = synth.random_field(g.n, seed + 100)
    lo, hi = 0.2, 4.6 * n
    o1, o2 = oracle_lib.trace_kq(b, g, Q1, Q2, (K1, K2), [synth.Step(hi, lo, 1.0, 1.0)])
    V1, V2 = _vertex_np(Q1), _vertex_np(Q2)
    for rid in range(b.nrays):
        nh, _ = oracle_lib.ray_direction(b, rid)
        for V, k, got in ((V1, K1, o1[rid]), (V2, K2, o2[rid])):
            def f(chi):
                p = np.array(b.obs)[None, :] + chi[:, None] * nh[None, :]
                return (k[0] + k[1] * chi + k[2] * chi ** 2) * _trilerp(V, g.h, p)
            want = _gl(f, lo, hi, 40000)
            l1 = _gl(lambda c: np.abs(f(c)), lo, hi, 40000)   # the integral's natural scale
            assert abs(got - want) < 1e-8 * l1, (rid, got, want)


def test_ngp_matches_midpoint_rule(oracle_lib):
    n = 6
    g = synth.Grid((n, n, n), 12.0)
    b = synth.Bundle(3, 3, synth.deg(40), synth.deg(40), (6.0, 6.0, 0.0), 15.0, interp=0)
    Q1 = synth.random_field(g.n, 23)
    o1, _ = oracle_lib.trace_kq(b, g, Q1, None, (K1, K2), [synth.Step(11.5, 0.0, 1.0, 1.0)])
    npts = 2_000_000
    chi = (np.arange(npts) + 0.5) * (11.5 / npts)
    for rid in range(b.nrays):
        nh, _ = oracle_lib.ray_direction(b, rid)
        p = np.array(b.obs)[None, :] + chi[:, None] * nh[None, :]
        c = np.floor(p / g.h).astype(np.int64) % n
        want = np.sum((K1[0] + K1[1] * chi + K1[2] * chi ** 2) * Q1[c[:, 0], c[:, 1], c[:, 2]]) * (11.5 / npts)
        assert abs(o1[rid] - want) < 2e-5 * np.abs(Q1).max() * 11.5


@pytest.mark.parametrize("interp", [0, 1])
def test_lensing_kernel_on_delta_is_the_born_term(oracle_lib, interp):
    """With K = g = chi - chi^2/chi_s and Q = 1.5 Omega_m (H0/c)^2 delta / a the
    generic integral is the density term of Eq. (kappa2), which the oracle's
    lensing path computes with Eqs. (Iclensing), (Iclensing_ngp)."""
    n = 10
    g = synth.Grid((n, n, n), 20.0)
    b = synth.Bundle(6, 5, synth.deg(25), synth.deg(20), (10.0, 9.0, 0.0), 45.0, interp=interp)
    phi = synth.random_field(g.n, 24)
    H, d = oracle_lib.fields(g, phi)
    steps = [synth.Step(44.0, 17.0, 1.1, 0.8), synth.Step(17.0, 0.0, 0.9, 0.95)]
    r = oracle_lib.trace(b, g, H, d, steps)
    got = np.zeros(b.nrays)
    for st in steps:
        pref = 1.5 * g.omega_m * synth.H0_OVER_C ** 2 / st.a
        o1, _ = oracle_lib.trace_kq(b, g, pref * d, None, ((0.0, 1.0, -1.0 / b.chi_s), (0, 0, 0)), [st])
        got += o1
    assert np.abs(got - r.kborn).max() < 1e-11 * np.abs(r.kborn).max()


def test_isw_of_a_linearly_growing_potential(oracle_lib):
    """ISW (Sec. 6): with Phi(t) = Phi_0 (1 + alpha t), the finite-difference
    Q = (Phi_curr - Phi_prev) / dt is alpha Phi_0 whatever dt, so the ISW
    integral is alpha times the integral of Phi_0 itself."""
    n = 8
    g = synth.Grid((n, n, n), 16.0)
    b = synth.Bundle(4, 4, synth.deg(20), synth.deg(20), (8.0, 8.0, 0.0), 30.0, interp=1)
    phi0 = synth.random_field(g.n, 25)
    alpha, t, dt = 0.37, 2.0, 0.013
    q = (phi0 * (1 + alpha * t) - phi0 * (1 + alpha * (t - dt))) / dt
    ker = ((2.0, 0.0, 0.0), (0.0, 0.0, 0.0))
    isw, _ = oracle_lib.trace_kq(b, g, q, None, ker, [synth.Step(29.0, 0.0, 1.0, 1.0)])
    ref, _ = oracle_lib.trace_kq(b, g, phi0, None, ker, [synth.Step(29.0, 0.0, 1.0, 1.0)])
    assert np.abs(isw - alpha * ref).max() < 1e-9 * np.abs(ref).max()


def test_tiled_boxes_with_relocated_observer(oracle_lib):
    """Sec. 2.2 tiling: three boxes stacked along the line of sight, each traced
    (without wrap) only while a ray is inside it, from an observer placed
    relative to that box's origin; NGP. The sum over the boxes equals one trace
    through the single long box that concatenates them (the same cell values,
    the same crossings)."""
    n, L = 8, 16.0
    boxes = [synth.random_field((n, n, n), 30 + i) for i in range(3)]
    Hs = [oracle_lib.tidal_centres(synth.Grid((n, n, n), L), p) for p in boxes]
    gb = synth.Grid((n, n, n), L)
    chis = 3 * L - 0.5
    total = np.zeros(20)
    for i, H in enumerate(Hs):
        b = synth.Bundle(5, 4, synth.deg(20), synth.deg(16), (L / 2, L / 2, -i * L), chis, interp=0,
                         periodic=False)
        total += oracle_lib.trace(b, gb, H, np.zeros((n, n, n)), [synth.Step(chis, 0.0, 1.0, 1.0)]).kappa
    glong = synth.Grid((n, n, 3 * n), L)
    Hl = np.concatenate(Hs, axis=2)
    bl = synth.Bundle(5, 4, synth.deg(20), synth.deg(16), (L / 2, L / 2, 0.0), chis, interp=0, periodic=False)
    want = oracle_lib.trace(bl, glong, Hl, np.zeros((n, n, 3 * n)), [synth.Step(chis, 0.0, 1.0, 1.0)]).kappa
    assert np.abs(total - want).max() < 1e-11 * np.abs(want).max()
