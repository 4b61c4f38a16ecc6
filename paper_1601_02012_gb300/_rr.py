"""ctypes binding of librr.so: the C ABI declared in include/rr.h, same names.

Argument marshalling only -- every step of the computation runs in the CUDA
library. Device buffers may be passed as torch tensors (their data_ptr is
used) or as raw integer addresses. Streams may be a torch.cuda.Stream, a raw
cudaStream_t integer, or None for the current torch stream.

Importing this module does not touch the GPU; loading the library fails loudly
if it has not been built (there is no fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librr.so")

RR_OK = 0
RR_ERR_ARG = -1
RR_ERR_CUDA = -2
RR_ERR_OOM = -3
RR_ERR_STEP_LIMIT = -4
RR_ERR_STATE = -5
RR_ERR_NONFINITE = -6
RR_ERR_CAPACITY = -7
RR_ERR_RANGE = -8
RR_NOALLOC_MAX_RAYS = 65536

RR_NGP = 0
RR_TRILINEAR = 1
RR_PERIODIC = 1
RR_FP64_DDA = 2
RR_PLAIN_SUMS = 4
RR_SOURCE_MOMENTS = 8
RR_SHEAR = 16
RR_METHOD_A = 32
RR_GENERIC = 64
RR_AT_VERTICES = 0
RR_AT_CENTRES = 1


class rr_bundle_desc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("fov_x", C.c_double), ("fov_y", C.c_double),
                ("obs", C.c_double * 3), ("chi_s", C.c_double), ("interp", C.c_int32), ("flags", C.c_int32)]


class rr_grid_desc(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("box", C.c_double), ("omega_m", C.c_double)]


class rr_amr_desc(C.Structure):
    _fields_ = [("n", C.c_int32), ("lmax", C.c_int32), ("box", C.c_double), ("omega_m", C.c_double)]


class RRError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {rr_status_string(code)}")


_lib = None


def load() -> C.CDLL:
    """Load librr.so (built in-tree by paper_1601_02012_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"librr.so is not built ({LIB_PATH}); run paper_1601_02012_gb300.build.build()")
        lib = C.CDLL(LIB_PATH)
        P, D, I32 = C.c_void_p, C.c_double, C.c_int32
        sig = {
            "rr_status_string": ([C.c_int], C.c_char_p),
            "rr_create": ([P, C.POINTER(C.c_void_p)], C.c_int),
            "rr_create_band": ([P, I32, I32, C.POINTER(C.c_void_p)], C.c_int),
            "rr_destroy": ([P], C.c_int),
            "rr_reset": ([P, P], C.c_int),
            "rr_tidal_tensor": ([P, P, P, P, I32, P, P], C.c_int),
            "rr_footprint_bbox": ([P, P, D, D, P], C.c_int),
            "rr_upload_box": ([P, P, P, P, C.POINTER(C.c_int64), P], C.c_int),
            "rr_trace_step": ([P, P, P, D, D, D, D, P], C.c_int),
            "rr_trace_steps": ([P, P, I32, P, P, P, P, P, P, P], C.c_int),
            "rr_tidal_tensor_box": ([P, P, P, P, I32, P, P], C.c_int),
            "rr_amr_trace_steps": ([P, P, I32, P, P, P, P, P, P], C.c_int),
            "rr_finalize": ([P, P, P, P], C.c_int),
            "rr_sync_status": ([P, P], C.c_int),
            "rr_segment_count": ([P, C.POINTER(C.c_uint64), P, P], C.c_int),
            "rr_trace_step_noalloc": ([P, P, P, D, D, D, D, P, P, P], C.c_int),
            "rr_step_count": ([P, C.POINTER(C.c_int32)], C.c_int),
            "rr_trace_step_adjoint": ([P, I32, P, P, P, P], C.c_int),
            "rr_tidal_tensor_adjoint": ([P, P, I32, P, P, P], C.c_int),
            "rr_trace_backward": ([P, P, P, P, P, P, P], C.c_int),
            "rr_batch_create": ([I32, P, C.POINTER(C.c_void_p)], C.c_int),
            "rr_batch_destroy": ([P], C.c_int),
            "rr_batch_size": ([P, C.POINTER(C.c_int32)], C.c_int),
            "rr_batch_context": ([P, I32, C.POINTER(C.c_void_p)], C.c_int),
            "rr_batch_reset": ([P, P], C.c_int),
            "rr_batch_clear": ([P, P], C.c_int),
            "rr_batch_set_step": ([P, I32, P, P, D, D, D, D], C.c_int),
            "rr_batch_upload": ([P, P], C.c_int),
            "rr_batch_trace": ([P, P], C.c_int),
            "rr_batch_finalize": ([P, P, P, P], C.c_int),
            "rr_batch_sync_status": ([P, C.POINTER(C.c_uint64), P], C.c_int),
            "rr_batch_set_tuning": ([P, I32, I32, I32, I32, I32], C.c_int),
            "rr_batch_get_tuning": ([P, P], C.c_int),
            "rr_batch_autotune": ([P, I32, C.POINTER(C.c_float), P], C.c_int),
            "rr_moments": ([P, P, P], C.c_int),
            "rr_shear": ([P, P, P, P], C.c_int),
            "rr_gradient_records": ([P, P, P, P, C.c_int32, P, P], C.c_int),
            "rr_scalar_records": ([P, P, P, D, C.c_int32, P, C.c_int32, P, P], C.c_int),
            "rr_set_kernels": ([P, P], C.c_int),
            "rr_set_observer": ([P, P], C.c_int),
            "rr_source_kappa": ([P, P, C.c_int64, D, P, P, P], C.c_int),
            "rr_amr_create": ([P, P, P, C.POINTER(C.c_void_p)], C.c_int),
            "rr_amr_destroy": ([P], C.c_int),
            "rr_amr_sizes": ([P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)], C.c_int),
            "rr_amr_tidal": ([P, P, I32, P, P, P, P], C.c_int),
            "rr_amr_gradient": ([P, P, I32, P, P, P, P], C.c_int),
            "rr_amr_scalars": ([P, P, P, D, P, P, D, I32, P, P, P, P], C.c_int),
            "rr_amr_trace_step": ([P, P, P, D, D, D, D, P], C.c_int),
            "rr_fp32_peak": ([I32, I32, I32, I32, P, C.POINTER(C.c_int64), P], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def rr_status_string(code: int) -> str:
    return load().rr_status_string(int(code)).decode()


def _check(code: int, where: str) -> int:
    if code != RR_OK:
        raise RRError(code, where)
    return code


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return C.c_void_p(x)
    return C.c_void_p(x.data_ptr())


def _stream(s):
    if s is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(s, int):
        return C.c_void_p(s)
    return C.c_void_p(s.cuda_stream)


def bundle_desc(b, fp64_dda: bool = False, plain_sums: bool = False, moments: bool = False,
                shear: bool = False, method_a: bool = False, generic: bool = False) -> rr_bundle_desc:
    """rr_bundle_desc from any object with nx, ny, fov_x, fov_y, obs, chi_s,
    interp and periodic attributes."""
    d = rr_bundle_desc()
    d.nx, d.ny = int(b.nx), int(b.ny)
    d.fov_x, d.fov_y = float(b.fov_x), float(b.fov_y)
    for i in range(3):
        d.obs[i] = float(b.obs[i])
    d.chi_s = float(b.chi_s)
    d.interp = int(getattr(b, "interp", RR_TRILINEAR))
    flags = RR_PERIODIC if getattr(b, "periodic", True) else 0
    if fp64_dda:
        flags |= RR_FP64_DDA
    if plain_sums:
        flags |= RR_PLAIN_SUMS
    if moments:
        flags |= RR_SOURCE_MOMENTS
    if shear:
        flags |= RR_SHEAR
    if method_a:
        flags |= RR_METHOD_A
    if generic:
        flags |= RR_GENERIC
    d.flags = flags
    return d


def grid_desc(g) -> rr_grid_desc:
    d = rr_grid_desc()
    for i in range(3):
        d.n[i] = int(g.n[i])
    d.box = float(g.box)
    d.omega_m = float(getattr(g, "omega_m", 0.3))
    return d


# ---------------------------------------------------------------------------
# the C ABI, one Python function per entry point
# ---------------------------------------------------------------------------

def rr_create(bundle: rr_bundle_desc) -> C.c_void_p:
    h = C.c_void_p()
    _check(load().rr_create(C.byref(bundle), C.byref(h)), "rr_create")
    return h


def rr_create_band(bundle: rr_bundle_desc, y0: int, y1: int) -> C.c_void_p:
    h = C.c_void_p()
    _check(load().rr_create_band(C.byref(bundle), int(y0), int(y1), C.byref(h)), "rr_create_band")
    return h


def rr_destroy(ctx) -> None:
    _check(load().rr_destroy(ctx), "rr_destroy")


def rr_reset(ctx, stream=None) -> None:
    _check(load().rr_reset(ctx, _stream(stream)), "rr_reset")


def rr_tidal_tensor(grid: rr_grid_desc, phi, delta, rec, where: int = RR_AT_VERTICES, bbox=None,
                    stream=None) -> None:
    bb = None
    if bbox is not None:
        arr = (C.c_int32 * 6)(*[int(x) for x in bbox])
        bb = C.cast(arr, C.c_void_p)
    _check(load().rr_tidal_tensor(C.byref(grid), _ptr(phi), _ptr(delta), _ptr(rec), int(where), bb,
                                  _stream(stream)), "rr_tidal_tensor")


def rr_footprint_bbox(bundle: rr_bundle_desc, grid: rr_grid_desc, chi_a: float, chi_b: float):
    arr = (C.c_int32 * 6)()
    _check(load().rr_footprint_bbox(C.byref(bundle), C.byref(grid), float(chi_a), float(chi_b),
                                    C.cast(arr, C.c_void_p)), "rr_footprint_bbox")
    return tuple(int(x) for x in arr)


def rr_upload_box(grid: rr_grid_desc, host, dev, bbox=None, stream=None) -> int:
    """Copy the cells a boxed record call reads (the box widened by 2 cells,
    modulo n) from the host array ``host`` into the device array ``dev``;
    returns the bytes enqueued."""
    bb = None
    if bbox is not None:
        arr = (C.c_int32 * 6)(*[int(x) for x in bbox])
        bb = C.cast(arr, C.c_void_p)
    nbytes = C.c_int64(0)
    _check(load().rr_upload_box(C.byref(grid), _ptr(host), _ptr(dev), bb, C.byref(nbytes), _stream(stream)),
           "rr_upload_box")
    return int(nbytes.value)


def rr_trace_step(ctx, grid: rr_grid_desc, rec, chi_a: float, chi_b: float, scale: float = 1.0,
                  a_step: float = 1.0, stream=None) -> None:
    _check(load().rr_trace_step(ctx, C.byref(grid), _ptr(rec), float(chi_a), float(chi_b), float(scale),
                                float(a_step), _stream(stream)), "rr_trace_step")


def rr_trace_steps(ctx, grid: rr_grid_desc, recs, chi_a, chi_b, scale, a_step, boxes=None, stream=None) -> None:
    """Consecutive steps in order (equal lengths): recs[i] the record buffer
    of step i, the others per-step numbers; boxes: None (whole-grid records)
    or one 6-int box per step (box-local records of rr_tidal_tensor_box)."""
    n = len(recs)
    if not (len(chi_a) == len(chi_b) == len(scale) == len(a_step) == n):
        raise ValueError("rr_trace_steps: per-step sequences of different lengths")
    ptrs = (C.c_void_p * max(n, 1))(*[_ptr(r) for r in recs])
    arr = [(C.c_double * max(n, 1))(*[float(x) for x in v]) for v in (chi_a, chi_b, scale, a_step)]
    bx = None
    if boxes is not None:
        if len(boxes) != n:
            raise ValueError("rr_trace_steps: one box per step")
        bx = (C.c_int32 * (6 * max(n, 1)))(*[int(v) for bb in boxes for v in bb])
    _check(load().rr_trace_steps(ctx, C.byref(grid), int(n), ptrs, bx, arr[0], arr[1], arr[2], arr[3],
                                 _stream(stream)), "rr_trace_steps")


def rr_amr_trace_steps(ctx, mesh, leaf_recs, chi_a, chi_b, scale, a_step, stream=None) -> None:
    """Consecutive steps over an adaptive mesh (equal lengths): leaf_recs[i]
    the leaf records of step i."""
    n = len(leaf_recs)
    if not (len(chi_a) == len(chi_b) == len(scale) == len(a_step) == n):
        raise ValueError("rr_amr_trace_steps: per-step sequences of different lengths")
    ptrs = (C.c_void_p * max(n, 1))(*[_ptr(r) for r in leaf_recs])
    arr = [(C.c_double * max(n, 1))(*[float(x) for x in v]) for v in (chi_a, chi_b, scale, a_step)]
    _check(load().rr_amr_trace_steps(ctx, mesh, int(n), ptrs, arr[0], arr[1], arr[2], arr[3], _stream(stream)),
           "rr_amr_trace_steps")


def rr_tidal_tensor_box(grid: rr_grid_desc, phi, delta, rec, where: int, bbox, stream=None) -> None:
    bb = (C.c_int32 * 6)(*[int(v) for v in bbox])
    _check(load().rr_tidal_tensor_box(C.byref(grid), _ptr(phi), _ptr(delta), _ptr(rec), int(where), bb,
                                      _stream(stream)), "rr_tidal_tensor_box")


def rr_finalize(ctx, kappa, kappa_born=None, stream=None) -> None:
    _check(load().rr_finalize(ctx, _ptr(kappa), _ptr(kappa_born), _stream(stream)), "rr_finalize")


def rr_sync_status(ctx, stream=None) -> int:
    return int(load().rr_sync_status(ctx, _stream(stream)))


def rr_segment_count(ctx, per_ray=None, stream=None) -> int:
    tot = C.c_uint64(0)
    _check(load().rr_segment_count(ctx, C.byref(tot), _ptr(per_ray), _stream(stream)), "rr_segment_count")
    return int(tot.value)


def rr_moments(ctx, out, stream=None) -> None:
    """out: device FP64 [4, ny*nx] (A_kappa, B_kappa, A_born, B_born)."""
    _check(load().rr_moments(ctx, _ptr(out), _stream(stream)), "rr_moments")


def rr_shear(ctx, gamma1, gamma2, stream=None) -> None:
    """gamma1, gamma2: device FP64 [ny*nx] each."""
    _check(load().rr_shear(ctx, _ptr(gamma1), _ptr(gamma2), _stream(stream)), "rr_shear")


def rr_source_kappa(m_end, m_k, nrays: int, chi_k: float, kappa, kappa_born=None, stream=None) -> None:
    _check(load().rr_source_kappa(_ptr(m_end), _ptr(m_k), int(nrays), float(chi_k), _ptr(kappa), _ptr(kappa_born),
                                  _stream(stream)), "rr_source_kappa")


def rr_step_count(ctx) -> int:
    n = C.c_int32(0)
    _check(load().rr_step_count(ctx, C.byref(n)), "rr_step_count")
    return int(n.value)


def rr_trace_step_adjoint(ctx, step: int, dL_dkappa, dL_dkborn, grad_rec, stream=None) -> None:
    _check(load().rr_trace_step_adjoint(ctx, int(step), _ptr(dL_dkappa), _ptr(dL_dkborn), _ptr(grad_rec),
                                        _stream(stream)), "rr_trace_step_adjoint")


def rr_gradient_records(grid: rr_grid_desc, phi, delta, rec, where: int = RR_AT_VERTICES, bbox=None,
                        stream=None) -> None:
    """rec: 4 floats per point {d_x Phi, d_y Phi, d_z Phi, delta} (Method A)."""
    bb = None
    if bbox is not None:
        arr = (C.c_int32 * 6)(*[int(x) for x in bbox])
        bb = C.cast(arr, C.c_void_p)
    _check(load().rr_gradient_records(C.byref(grid), _ptr(phi), _ptr(delta), _ptr(rec), int(where), bb,
                                      _stream(stream)), "rr_gradient_records")


def rr_scalar_records(grid: rr_grid_desc, field, field_prev, inv_dt: float, channel: int, rec,
                      where: int = RR_AT_VERTICES, bbox=None, stream=None) -> None:
    """Channel ``channel`` of the float2 records: field, or (field - field_prev) * inv_dt."""
    bb = None
    if bbox is not None:
        arr = (C.c_int32 * 6)(*[int(x) for x in bbox])
        bb = C.cast(arr, C.c_void_p)
    _check(load().rr_scalar_records(C.byref(grid), _ptr(field), _ptr(field_prev), float(inv_dt), int(channel),
                                    _ptr(rec), int(where), bb, _stream(stream)), "rr_scalar_records")


def rr_set_kernels(ctx, kernels) -> None:
    """kernels: (k0, k1, k2) per channel, K_c(chi) = k0 + k1 chi + k2 chi^2."""
    k = (C.c_double * 6)(*[float(x) for x in np.asarray(kernels, dtype=np.float64).reshape(6)])
    _check(load().rr_set_kernels(ctx, C.cast(k, C.c_void_p)), "rr_set_kernels")


def rr_set_observer(ctx, obs) -> None:
    o = (C.c_double * 3)(*[float(x) for x in obs])
    _check(load().rr_set_observer(ctx, C.cast(o, C.c_void_p)), "rr_set_observer")


def rr_tidal_tensor_adjoint(grid: rr_grid_desc, grad_rec, where: int, dL_dphi, dL_ddelta=None, stream=None) -> None:
    _check(load().rr_tidal_tensor_adjoint(C.byref(grid), _ptr(grad_rec), int(where), _ptr(dL_dphi),
                                          _ptr(dL_ddelta), _stream(stream)), "rr_tidal_tensor_adjoint")


def rr_trace_backward(ctx, dL_dkappa, dL_dkborn, grad_rec, dL_dphi, dL_ddelta=None, stream=None) -> None:
    _check(load().rr_trace_backward(ctx, _ptr(dL_dkappa), _ptr(dL_dkborn), _ptr(grad_rec), _ptr(dL_dphi),
                                    _ptr(dL_ddelta), _stream(stream)), "rr_trace_backward")


def rr_trace_step_noalloc(bundle: rr_bundle_desc, grid: rr_grid_desc, rec, chi_a: float, chi_b: float,
                          kappa, kappa_born=None, scale: float = 1.0, a_step: float = 1.0, stream=None) -> None:
    """One step into the maps without any allocation by the library (its
    scratch is a fixed device array for at most RR_NOALLOC_MAX_RAYS rays)."""
    nr = int(bundle.nx) * int(bundle.ny)
    if nr > RR_NOALLOC_MAX_RAYS:
        raise RRError(RR_ERR_CAPACITY, f"rr_trace_step_noalloc: {nr} rays > {RR_NOALLOC_MAX_RAYS}")
    _check(load().rr_trace_step_noalloc(C.byref(bundle), C.byref(grid), _ptr(rec), float(chi_a), float(chi_b),
                                        float(scale), float(a_step), _ptr(kappa), _ptr(kappa_born),
                                        _stream(stream)), "rr_trace_step_noalloc")


# ---- batches ---------------------------------------------------------------

def rr_batch_create(bundles) -> C.c_void_p:
    arr = (rr_bundle_desc * len(bundles))(*bundles)
    h = C.c_void_p()
    _check(load().rr_batch_create(len(bundles), C.cast(arr, C.c_void_p), C.byref(h)), "rr_batch_create")
    return h


def rr_batch_destroy(b) -> None:
    _check(load().rr_batch_destroy(b), "rr_batch_destroy")


def rr_batch_context(b, i: int) -> C.c_void_p:
    h = C.c_void_p()
    _check(load().rr_batch_context(b, int(i), C.byref(h)), "rr_batch_context")
    return h


def rr_batch_reset(b, stream=None) -> None:
    _check(load().rr_batch_reset(b, _stream(stream)), "rr_batch_reset")


def rr_batch_clear(b, stream=None) -> None:
    _check(load().rr_batch_clear(b, _stream(stream)), "rr_batch_clear")


def rr_batch_set_step(b, i: int, grid: rr_grid_desc, rec, chi_a: float, chi_b: float, scale: float = 1.0,
                      a_step: float = 1.0) -> None:
    _check(load().rr_batch_set_step(b, int(i), C.byref(grid), _ptr(rec), float(chi_a), float(chi_b), float(scale),
                                    float(a_step)), "rr_batch_set_step")


def rr_batch_upload(b, stream=None) -> None:
    _check(load().rr_batch_upload(b, _stream(stream)), "rr_batch_upload")


def rr_batch_trace(b, stream=None) -> None:
    _check(load().rr_batch_trace(b, _stream(stream)), "rr_batch_trace")


def rr_batch_finalize(b, kappas, kborns=None, stream=None) -> None:
    n = len(kappas)
    ka = (C.c_void_p * n)(*[t.data_ptr() for t in kappas])
    kb = None if kborns is None else (C.c_void_p * n)(*[t.data_ptr() for t in kborns])
    _check(load().rr_batch_finalize(b, C.cast(ka, C.c_void_p), None if kb is None else C.cast(kb, C.c_void_p),
                                    _stream(stream)), "rr_batch_finalize")


def rr_batch_sync_status(b, stream=None):
    """(status code, total segments)"""
    tot = C.c_uint64(0)
    code = load().rr_batch_sync_status(b, C.byref(tot), _stream(stream))
    return int(code), int(tot.value)


def rr_batch_set_tuning(b, wx: int, bwx: int, bwy: int, chunk: int = 1, blocks_per_sm: int = 0) -> None:
    _check(load().rr_batch_set_tuning(b, int(wx), int(bwx), int(bwy), int(chunk), int(blocks_per_sm)),
           "rr_batch_set_tuning")


def rr_batch_get_tuning(b):
    arr = (C.c_int32 * 5)()
    _check(load().rr_batch_get_tuning(b, C.cast(arr, C.c_void_p)), "rr_batch_get_tuning")
    return tuple(int(x) for x in arr)


def rr_batch_autotune(b, reps: int = 3, stream=None) -> float:
    ms = C.c_float(0)
    _check(load().rr_batch_autotune(b, int(reps), C.byref(ms), _stream(stream)), "rr_batch_autotune")
    return float(ms.value)


# ---- adaptive meshes -------------------------------------------------------

def rr_amr_create(desc: rr_amr_desc, octs) -> C.c_void_p:
    """octs[l] (l = 1..lmax): int32 array-like [m_l, 3] of the refined level-(l-1)
    cells; octs[0] is ignored."""
    import numpy as np
    L = int(desc.lmax)
    keep = []
    ptrs = (C.c_void_p * (L + 1))()
    counts = (C.c_int64 * (L + 1))()
    for lv in range(1, L + 1):
        a = np.ascontiguousarray(np.asarray(octs[lv], dtype=np.int32).reshape(-1, 3))
        keep.append(a)
        ptrs[lv] = a.ctypes.data if a.size else None
        counts[lv] = a.shape[0]
    h = C.c_void_p()
    _check(load().rr_amr_create(C.byref(desc), C.cast(ptrs, C.c_void_p), C.cast(counts, C.c_void_p), C.byref(h)),
           "rr_amr_create")
    return h


def rr_amr_destroy(mesh) -> None:
    _check(load().rr_amr_destroy(mesh), "rr_amr_destroy")


def rr_amr_sizes(mesh):
    """(cells, leaves, vertices)"""
    a, b, c = C.c_int64(0), C.c_int64(0), C.c_int64(0)
    _check(load().rr_amr_sizes(mesh, C.byref(a), C.byref(b), C.byref(c)), "rr_amr_sizes")
    return int(a.value), int(b.value), int(c.value)


def rr_amr_tidal(mesh, phi, where: int, leaf_rec, cell_tidal=None, bbox=None, stream=None) -> None:
    bb = None
    if bbox is not None:
        arr = (C.c_int32 * 6)(*[int(x) for x in bbox])
        bb = C.cast(arr, C.c_void_p)
    _check(load().rr_amr_tidal(mesh, _ptr(phi), int(where), _ptr(leaf_rec), _ptr(cell_tidal), bb,
                               _stream(stream)), "rr_amr_tidal")


def rr_amr_gradient(mesh, phi, where: int, leaf_rec, cell_grad=None, bbox=None, stream=None) -> None:
    bb = None
    if bbox is not None:
        arr = (C.c_int32 * 6)(*[int(x) for x in bbox])
        bb = C.cast(arr, C.c_void_p)
    _check(load().rr_amr_gradient(mesh, _ptr(phi), int(where), _ptr(leaf_rec), _ptr(cell_grad), bb,
                                  _stream(stream)), "rr_amr_gradient")


def rr_amr_scalars(mesh, field0, prev0, inv_dt0: float, field1, prev1, inv_dt1: float, where: int, leaf_rec,
                   cell_buf=None, bbox=None, stream=None) -> None:
    bb = None
    if bbox is not None:
        arr = (C.c_int32 * 6)(*[int(x) for x in bbox])
        bb = C.cast(arr, C.c_void_p)
    _check(load().rr_amr_scalars(mesh, _ptr(field0), _ptr(prev0), float(inv_dt0), _ptr(field1), _ptr(prev1),
                                 float(inv_dt1), int(where), _ptr(leaf_rec), _ptr(cell_buf), bb, _stream(stream)),
           "rr_amr_scalars")


def rr_amr_trace_step(ctx, mesh, leaf_rec, chi_a: float, chi_b: float, scale: float = 1.0, a_step: float = 1.0,
                      stream=None) -> None:
    _check(load().rr_amr_trace_step(ctx, mesh, _ptr(leaf_rec), float(chi_a), float(chi_b), float(scale),
                                    float(a_step), _stream(stream)), "rr_amr_trace_step")


# ---- measurement -----------------------------------------------------------

def rr_fp32_peak(packed: bool, blocks: int, threads: int, iters: int, out, stream=None) -> int:
    """Launch the FP32 FMA throughput kernel; returns the FMA count of the launch."""
    n = C.c_int64()
    _check(load().rr_fp32_peak(int(bool(packed)), int(blocks), int(threads), int(iters), _ptr(out), C.byref(n),
                               _stream(stream)), "rr_fp32_peak")
    return int(n.value)
