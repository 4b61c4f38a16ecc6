"""FP64 CPU oracle for the line-of-sight convergence integration.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this package; the library itself never does. It
shares no code with the CUDA path (see rr_oracle.c for what it computes and
which passages of Barreira et al. 2016 each function follows).

Every function here takes and returns numpy arrays; fields are promoted to
float64 before use (an FP32 input is read exactly).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rr_oracle.c")
_SRC_AMR = os.path.join(_HERE, "rr_oracle_amr.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over rays; no fused multiply-add
    contraction, so x86 and Arm give the same bits)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_AMR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", _LIB + ".tmp", _SRC, _SRC_AMR, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Bundle(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("fov_x", C.c_double), ("fov_y", C.c_double),
                ("obs", C.c_double * 3), ("chi_s", C.c_double), ("interp", C.c_int32),
                ("periodic", C.c_int32)]


class _Grid(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("box", C.c_double), ("omega_m", C.c_double)]


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        _lib.ora_tidal_centres.argtypes = [P, P, P]
        _lib.ora_delta_from_tidal.argtypes = [P, P, P]
        _lib.ora_vertex_field.argtypes = [P, P, P, P]
        _lib.ora_trace_step.argtypes = [P, P, P, P, C.c_double, C.c_double, C.c_double, C.c_double,
                                        P, P, P, P, C.c_int, P, C.c_long]
        _lib.ora_trace_step_shear.argtypes = [P, P, P, C.c_double, C.c_double, C.c_double, P, P, C.c_int, P,
                                              C.c_long]
        _lib.ora_fields_grad.argtypes = [P, P, P]
        _lib.ora_trace_step_method_a.argtypes = [P, P, P, P, C.c_double, C.c_double, C.c_double, C.c_double,
                                                 P, P, C.c_int, P, C.c_long]
        _lib.ora_trace_step_kq.argtypes = [P, P, P, P, C.c_double, C.c_double, C.c_double, P, P, P, C.c_int, P,
                                           C.c_long]
        _lib.ora_ray_segments.argtypes = [P, P, C.c_long, C.c_double, C.c_double, P, C.c_long]
        _lib.ora_ray_segments.restype = C.c_long
        _lib.ora_ray_direction.argtypes = [P, C.c_long, P, P]
        _lib.ora_trace_step_adjoint.argtypes = [P, P, C.c_double, C.c_double, C.c_double, C.c_double,
                                                P, P, P, P]
        _lib.ora_delta_from_tidal_adjoint.argtypes = [P, P, P]
        _lib.ora_tidal_centres_adjoint.argtypes = [P, P, P]
        _lib.ora_amr_vertex_weights.argtypes = [P, P, P, C.c_long]
        _lib.ora_amr_vertex_weights.restype = C.c_long
        _lib.ora_amr_tidal.argtypes = [P, P]
        _lib.ora_amr_leaf_vertices.argtypes = [P, C.c_int, P, P]
        _lib.ora_amr_trace_step_shear.argtypes = [P, P, C.c_double, C.c_double, C.c_double, P, P, P, C.c_long]
        _lib.ora_amr_trace_step_kq.argtypes = [P, P, C.c_double, C.c_double, C.c_double, P, P, P, C.c_long]
        _lib.ora_amr_trace_step_method_a.argtypes = [P, P, C.c_double, C.c_double, C.c_double, C.c_double, P, P, P,
                                                     C.c_long]
        _lib.ora_amr_trace_step.argtypes = [P, P, C.c_double, C.c_double, C.c_double, C.c_double, P, P, P, P,
                                            C.c_long, C.c_int]
    return _lib


def _ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _bundle(b) -> _Bundle:
    s = _Bundle()
    s.nx, s.ny = int(b.nx), int(b.ny)
    s.fov_x, s.fov_y = float(b.fov_x), float(b.fov_y)
    for i in range(3):
        s.obs[i] = float(b.obs[i])
    s.chi_s = float(b.chi_s)
    s.interp = int(b.interp)
    s.periodic = 1 if b.periodic else 0
    return s


def _grid(g) -> _Grid:
    s = _Grid()
    for i in range(3):
        s.n[i] = int(g.n[i])
    s.box = float(g.box)
    s.omega_m = float(g.omega_m)
    return s


# ---------------------------------------------------------------------------

def tidal_centres(grid, phi) -> np.ndarray:
    """d_a d_b Phi at cell centres, shape n^3 x 6 (xx, yy, zz, xy, xz, yz);
    Eq. (tidalexample), periodic."""
    phi = _f64(phi)
    H = np.zeros(phi.shape + (6,), np.float64)
    g = _grid(grid)
    _L().ora_tidal_centres(C.byref(g), _ptr(phi), _ptr(H))
    return H


def delta_from_tidal(grid, H) -> np.ndarray:
    """delta = tr(H) / (1.5 Omega_m (H0/c)^2) (comoving Poisson at a = 1)."""
    H = _f64(H)
    d = np.zeros(H.shape[:-1], np.float64)
    g = _grid(grid)
    _L().ora_delta_from_tidal(C.byref(g), _ptr(H), _ptr(d))
    return d


def fields(grid, phi, delta=None):
    """(H, delta) at centres; delta derived from H when not given."""
    H = tidal_centres(grid, phi)
    d = delta_from_tidal(grid, H) if delta is None else _f64(delta)
    return H, d


def vertex_field(grid, H, delta) -> np.ndarray:
    """Vertex values, shape n^3 x 7 (6 tidal components then delta); vertex
    (i,j,k) at (ih, jh, kh) is the mean of the 8 cells that share it."""
    H = _f64(H)
    delta = _f64(delta)
    V = np.zeros(H.shape[:-1] + (7,), np.float64)
    g = _grid(grid)
    _L().ora_vertex_field(C.byref(g), _ptr(H), _ptr(delta), _ptr(V))
    return V


class TraceResult:
    def __init__(self, nr):
        self.kappa = np.zeros(nr, np.float64)
        self.kborn = np.zeros(nr, np.float64)
        self.nseg = np.zeros(nr, np.int64)
        self.sum_r = np.zeros(nr, np.float64)


def trace(bundle, grid, H, delta, steps, nthreads: int = 0, result: TraceResult | None = None,
          rids=None) -> TraceResult:
    """Trace the rays of the bundle over the given steps (objects with chi_a,
    chi_b, scale, a). Returns per-ray kappa, Born kappa, segment count and the
    summed segment lengths, in rayid order (x fastest), or in the order of
    ``rids`` when only those ray ids are traced."""
    H = _f64(H)
    delta = _f64(delta)
    ids = None if rids is None else np.ascontiguousarray(rids, dtype=np.int64)
    nr = int(bundle.nx) * int(bundle.ny) if ids is None else len(ids)
    res = result if result is not None else TraceResult(nr)
    b, g = _bundle(bundle), _grid(grid)
    for st in steps:
        rc = _L().ora_trace_step(C.byref(b), C.byref(g), _ptr(H), _ptr(delta), float(st.chi_a),
                                 float(st.chi_b), float(st.scale), float(st.a), _ptr(res.kappa),
                                 _ptr(res.kborn), _ptr(res.nseg), _ptr(res.sum_r), int(nthreads),
                                 _ptr(ids), 0 if ids is None else len(ids))
        if rc != 0:
            raise ValueError("oracle: bad step interval")
    return res


def trace_shear(bundle, grid, H, steps, nthreads: int = 0, rids=None):
    """The shear (gamma1, gamma2) of the bundle over the given steps (Eqs.
    gamma1, gamma2), per ray in rayid order or in the order of ``rids``."""
    H = _f64(H)
    ids = None if rids is None else np.ascontiguousarray(rids, dtype=np.int64)
    nr = int(bundle.nx) * int(bundle.ny) if ids is None else len(ids)
    g1 = np.zeros(nr, np.float64)
    g2 = np.zeros(nr, np.float64)
    b, g = _bundle(bundle), _grid(grid)
    for st in steps:
        rc = _L().ora_trace_step_shear(C.byref(b), C.byref(g), _ptr(H), float(st.chi_a), float(st.chi_b),
                                       float(st.scale), _ptr(g1), _ptr(g2), int(nthreads), _ptr(ids),
                                       0 if ids is None else len(ids))
        if rc != 0:
            raise ValueError("oracle: bad step interval")
    return g1, g2


def fields_grad(grid, phi) -> np.ndarray:
    """d_a Phi at cell centres, [n0, n1, n2, 3], central differences."""
    g = _grid(grid)
    phi = _f64(phi)
    G = np.zeros(tuple(int(x) for x in grid.n) + (3,), np.float64)
    _L().ora_fields_grad(C.byref(g), _ptr(phi), _ptr(G))
    return G


def trace_method_a(bundle, grid, G, delta, steps, nthreads: int = 0, rids=None):
    """Method A (Eq. kappa2) over the given steps: (kgrad, kborn) per ray, in
    rayid order or in the order of ``rids``; kgrad holds the gradient integral
    and the steps' surface terms, kborn the density term, and the Method A
    convergence is their sum."""
    G = _f64(G)
    d = _f64(delta)
    ids = None if rids is None else np.ascontiguousarray(rids, dtype=np.int64)
    nr = int(bundle.nx) * int(bundle.ny) if ids is None else len(ids)
    kg = np.zeros(nr, np.float64)
    kb = np.zeros(nr, np.float64)
    b, g = _bundle(bundle), _grid(grid)
    for st in steps:
        rc = _L().ora_trace_step_method_a(C.byref(b), C.byref(g), _ptr(G), _ptr(d), float(st.chi_a),
                                          float(st.chi_b), float(st.scale), float(st.a), _ptr(kg), _ptr(kb),
                                          int(nthreads), _ptr(ids), 0 if ids is None else len(ids))
        if rc != 0:
            raise ValueError("oracle: bad step interval")
    return kg, kb


def trace_kq(bundle, grid, Q1, Q2, kernels, steps, nthreads: int = 0, rids=None):
    """Two generic integrals int K_c(chi) Q_c dchi per ray over the given steps
    (each step's field is st.scale * Q_c); kernels = (k0, k1, k2) per channel,
    K_c = k0 + k1 chi + k2 chi^2; Q2 may be None. Returns (I1, I2)."""
    Q1 = _f64(Q1)
    Q2 = None if Q2 is None else _f64(Q2)
    k = np.ascontiguousarray(np.asarray(kernels, np.float64).reshape(6))
    ids = None if rids is None else np.ascontiguousarray(rids, dtype=np.int64)
    nr = int(bundle.nx) * int(bundle.ny) if ids is None else len(ids)
    o1 = np.zeros(nr, np.float64)
    o2 = np.zeros(nr, np.float64)
    b, g = _bundle(bundle), _grid(grid)
    for st in steps:
        rc = _L().ora_trace_step_kq(C.byref(b), C.byref(g), _ptr(Q1), _ptr(Q2), float(st.chi_a), float(st.chi_b),
                                    float(st.scale), _ptr(k), _ptr(o1), _ptr(o2), int(nthreads), _ptr(ids),
                                    0 if ids is None else len(ids))
        if rc != 0:
            raise ValueError("oracle: bad step interval")
    return o1, o2


def ray_segments(bundle, grid, rid: int, chi_a: float, chi_b: float) -> np.ndarray:
    """Rows (chiA, chiB, cell_x, cell_y, cell_z) of one ray's segments."""
    b, g = _bundle(bundle), _grid(grid)
    cap = 1 << 16
    rows = np.zeros((cap, 5), np.float64)
    n = _L().ora_ray_segments(C.byref(b), C.byref(g), int(rid), float(chi_a), float(chi_b), _ptr(rows), cap)
    return rows[: min(n, cap)].copy()


def ray_direction(bundle, rid: int):
    """(n_hat, projection weights of Eqs. n1n1 + n2n2) of one ray."""
    b = _bundle(bundle)
    n = np.zeros(3, np.float64)
    w = np.zeros(6, np.float64)
    _L().ora_ray_direction(C.byref(b), int(rid), _ptr(n), _ptr(w))
    return n, w


def trace_adjoint(bundle, grid, steps, dL_dkappa, dL_dkborn=None, delta_derived: bool = True):
    """dL/dPhi at the cell centres (and dL/ddelta when delta is an independent
    input) for L with the given per-ray derivatives."""
    nr = int(bundle.nx) * int(bundle.ny)
    gk = _f64(dL_dkappa).reshape(nr)
    gb = _f64(dL_dkborn).reshape(nr) if dL_dkborn is not None else None
    shape = tuple(int(x) for x in grid.n)
    gH = np.zeros(shape + (6,), np.float64)
    gd = np.zeros(shape, np.float64)
    b, g = _bundle(bundle), _grid(grid)
    for st in steps:
        _L().ora_trace_step_adjoint(C.byref(b), C.byref(g), float(st.chi_a), float(st.chi_b),
                                    float(st.scale), float(st.a), _ptr(gk), _ptr(gb), _ptr(gH), _ptr(gd))
    if delta_derived:
        _L().ora_delta_from_tidal_adjoint(C.byref(g), _ptr(gd), _ptr(gH))
    gphi = np.zeros(shape, np.float64)
    _L().ora_tidal_centres_adjoint(C.byref(g), _ptr(gH), _ptr(gphi))
    return (gphi, None) if delta_derived else (gphi, gd)


# ---------------------------------------------------------------------------
# adaptive meshes
# ---------------------------------------------------------------------------

_AMR_LMAX = 8


class _AmrDesc(C.Structure):
    _fields_ = [("n", C.c_int32), ("lmax", C.c_int32), ("box", C.c_double), ("omega_m", C.c_double),
                ("octs", C.c_void_p * (_AMR_LMAX + 1)), ("noct", C.c_int64 * (_AMR_LMAX + 1)),
                ("phi", C.c_void_p * (_AMR_LMAX + 1))]


class _AmrBundle(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("fov_x", C.c_double), ("fov_y", C.c_double),
                ("obs", C.c_double * 3), ("chi_s", C.c_double), ("interp", C.c_int32), ("periodic", C.c_int32)]


class AmrHandle:
    """Keeps the numpy arrays of a mesh alive while the oracle reads them."""

    def __init__(self, mesh, phi=None):
        phi = mesh.phi if phi is None else phi
        self.keep = []
        d = _AmrDesc()
        d.n, d.lmax, d.box, d.omega_m = int(mesh.n), int(mesh.lmax), float(mesh.box), float(mesh.omega_m)
        for l in range(mesh.lmax + 1):
            ph = np.ascontiguousarray(phi[l], dtype=np.float64)
            self.keep.append(ph)
            d.phi[l] = ph.ctypes.data
            if l >= 1:
                oc = np.ascontiguousarray(mesh.octs[l], dtype=np.int32)
                self.keep.append(oc)
                d.octs[l] = oc.ctypes.data
                d.noct[l] = len(oc)
        self.desc = d


def amr_vertex_weights(mesh, V):
    """The value at finest-lattice point V as rows (level, i, j, k, weight) of leaf values."""
    h = AmrHandle(mesh, [np.zeros(1)] * (mesh.lmax + 1) if mesh.phi is None else None)
    v = np.ascontiguousarray(V, dtype=np.int64)
    rows = np.zeros((64, 5))
    n = _L().ora_amr_vertex_weights(C.byref(h.desc), _ptr(v), _ptr(rows), 64)
    if n < 0:
        raise ValueError(f"oracle: vertex rule failed ({n})")
    return rows[:n].copy()


def amr_tidal(mesh):
    """7 channels (H xx,yy,zz,xy,xz,yz and delta) at every cell of every level."""
    h = AmrHandle(mesh)
    total = mesh.n ** 3 + sum(8 * len(mesh.octs[l]) for l in range(1, mesh.lmax + 1))
    out = np.zeros((total, 7))
    if _L().ora_amr_tidal(C.byref(h.desc), _ptr(out)) != 0:
        raise ValueError("oracle: AMR tidal failed")
    return out


def amr_leaf_vertices(mesh, level, cell):
    h = AmrHandle(mesh)
    c = np.ascontiguousarray(cell, dtype=np.int64)
    out = np.zeros((8, 7))
    if _L().ora_amr_leaf_vertices(C.byref(h.desc), int(level), _ptr(c), _ptr(out)) != 0:
        raise ValueError("oracle: AMR vertex failed")
    return out


def _amr_bundle(bundle):
    b = _AmrBundle()
    b.nx, b.ny = int(bundle.nx), int(bundle.ny)
    b.fov_x, b.fov_y = float(bundle.fov_x), float(bundle.fov_y)
    for i in range(3):
        b.obs[i] = float(bundle.obs[i])
    b.chi_s = float(bundle.chi_s)
    b.interp = int(bundle.interp)
    b.periodic = 1 if bundle.periodic else 0
    return b


def amr_trace_shear(bundle, mesh, steps, rids=None):
    """The shear (gamma1, gamma2) of Eqs. gamma1, gamma2 through an adaptive
    mesh, per ray in rayid order or in the order of ``rids``."""
    h = AmrHandle(mesh)
    b = _amr_bundle(bundle)
    ids = None if rids is None else np.ascontiguousarray(rids, dtype=np.int64)
    nr = int(bundle.nx) * int(bundle.ny) if ids is None else len(ids)
    g1 = np.zeros(nr, np.float64)
    g2 = np.zeros(nr, np.float64)
    for st in steps:
        rc = _L().ora_amr_trace_step_shear(C.byref(b), C.byref(h.desc), float(st.chi_a), float(st.chi_b),
                                           float(st.scale), _ptr(g1), _ptr(g2), _ptr(ids),
                                           0 if ids is None else len(ids))
        if rc != 0:
            raise ValueError(f"oracle: AMR trace failed ({rc})")
    return g1, g2


def amr_trace_kq(bundle, mesh, Q1, Q2, kernels, steps, rids=None):
    """Two generic integrals int K_c(chi) Q_c dchi through an adaptive mesh;
    Q_c per level as mesh.phi is (level 0: n^3, level l: octs x 8), Q2 may be
    None; each step's field is st.scale * Q_c. Returns (I1, I2)."""
    b = _amr_bundle(bundle)
    ids = None if rids is None else np.ascontiguousarray(rids, dtype=np.int64)
    nr = int(bundle.nx) * int(bundle.ny) if ids is None else len(ids)
    ker = np.asarray(kernels, np.float64).reshape(2, 3)
    outs = []
    for Q, k in ((Q1, ker[0]), (Q2, ker[1])):
        o = np.zeros(nr, np.float64)
        if Q is not None:
            h = AmrHandle(mesh, Q)
            kk = np.ascontiguousarray(k)
            for st in steps:
                rc = _L().ora_amr_trace_step_kq(C.byref(b), C.byref(h.desc), float(st.chi_a), float(st.chi_b),
                                                float(st.scale), _ptr(kk), _ptr(o), _ptr(ids),
                                                0 if ids is None else len(ids))
                if rc != 0:
                    raise ValueError(f"oracle: AMR trace failed ({rc})")
        outs.append(o)
    return outs[0], outs[1]


def amr_trace_method_a(bundle, mesh, steps, rids=None):
    """Method A (Eq. kappa2) through an adaptive mesh: (kgrad, kborn) per ray;
    the Method A convergence is their sum."""
    h = AmrHandle(mesh)
    b = _amr_bundle(bundle)
    ids = None if rids is None else np.ascontiguousarray(rids, dtype=np.int64)
    nr = int(bundle.nx) * int(bundle.ny) if ids is None else len(ids)
    kg = np.zeros(nr, np.float64)
    kb = np.zeros(nr, np.float64)
    for st in steps:
        rc = _L().ora_amr_trace_step_method_a(C.byref(b), C.byref(h.desc), float(st.chi_a), float(st.chi_b),
                                              float(st.scale), float(st.a), _ptr(kg), _ptr(kb), _ptr(ids),
                                              0 if ids is None else len(ids))
        if rc != 0:
            raise ValueError(f"oracle: AMR trace failed ({rc})")
    return kg, kb


def amr_trace(bundle, mesh, steps, rids=None) -> TraceResult:
    """kappa, Born kappa and leaf-segment counts through an adaptive mesh."""
    h = AmrHandle(mesh)
    b = _AmrBundle()
    b.nx, b.ny = int(bundle.nx), int(bundle.ny)
    b.fov_x, b.fov_y = float(bundle.fov_x), float(bundle.fov_y)
    for i in range(3):
        b.obs[i] = float(bundle.obs[i])
    b.chi_s = float(bundle.chi_s)
    b.interp = int(bundle.interp)
    b.periodic = 1 if bundle.periodic else 0
    ids = None if rids is None else np.ascontiguousarray(rids, dtype=np.int64)
    nr = int(bundle.nx) * int(bundle.ny) if ids is None else len(ids)
    res = TraceResult(nr)
    for st in steps:
        rc = _L().ora_amr_trace_step(C.byref(b), C.byref(h.desc), float(st.chi_a), float(st.chi_b),
                                     float(st.scale), float(st.a), _ptr(res.kappa), _ptr(res.kborn),
                                     _ptr(res.nseg), _ptr(ids), 0 if ids is None else len(ids), 0)
        if rc != 0:
            raise ValueError(f"oracle: AMR trace failed ({rc})")
    return res
