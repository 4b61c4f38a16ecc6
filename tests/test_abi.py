"""The C ABI without a GPU: the library builds and loads, exports every entry
point that include/rr.h declares, validates arguments before touching the
device, and its host-side footprint helper covers every cell a step reads."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rr():
    from paper_1601_02012_gb300 import build
    build.build()
    from paper_1601_02012_gb300 import _rr
    _rr.load()
    return _rr


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(rr_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(rr):
    names = _declared()
    assert "rr_trace_step" in names and "rr_tidal_tensor" in names
    lib = rr.load()
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(rr):
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert rr.rr_status_string(code)
    assert "unknown" in rr.rr_status_string(42)


def test_argument_validation_is_host_side(rr):
    lib = rr.load()
    good = rr.bundle_desc(synth.Bundle(4, 4, 0.1, 0.1, (1, 1, 0), 10.0))
    h = C.c_void_p()
    assert lib.rr_create(None, C.byref(h)) == rr.RR_ERR_ARG
    for field, val in (("nx", 0), ("fov_x", -0.1), ("fov_y", 4.0), ("chi_s", 0.0), ("interp", 7), ("flags", 128)):
        bad = rr.bundle_desc(synth.Bundle(4, 4, 0.1, 0.1, (1, 1, 0), 10.0))
        setattr(bad, field, val)
        assert lib.rr_create(C.byref(bad), C.byref(h)) == rr.RR_ERR_ARG, field
    g = rr.grid_desc(synth.Grid((8, 8, 8), 16.0))
    gbad = rr.grid_desc(synth.Grid((1, 8, 8), 16.0))
    assert lib.rr_tidal_tensor(C.byref(gbad), C.c_void_p(16), None, C.c_void_p(16), 0, None, None) == rr.RR_ERR_ARG
    assert lib.rr_tidal_tensor(C.byref(g), None, None, C.c_void_p(16), 0, None, None) == rr.RR_ERR_ARG
    assert lib.rr_tidal_tensor(C.byref(g), C.c_void_p(16), None, C.c_void_p(20), 0, None, None) == rr.RR_ERR_ARG
    assert lib.rr_tidal_tensor(C.byref(g), C.c_void_p(16), None, C.c_void_p(16), 5, None, None) == rr.RR_ERR_ARG
    bb = (C.c_int32 * 6)(0, 9, 0, 8, 0, 8)
    assert lib.rr_tidal_tensor(C.byref(g), C.c_void_p(16), None, C.c_void_p(16), 0, C.cast(bb, C.c_void_p),
                               None) == rr.RR_ERR_ARG
    assert lib.rr_trace_step(None, C.byref(g), C.c_void_p(16), 1.0, 0.0, 1.0, 1.0, None) == rr.RR_ERR_ARG
    one = (C.c_double * 1)(1.0)
    recs = (C.c_void_p * 1)(16)
    assert lib.rr_trace_steps(None, C.byref(g), 1, recs, None, one, one, one, one, None) == rr.RR_ERR_ARG
    assert lib.rr_tidal_tensor_box(C.byref(g), C.c_void_p(32), None, C.c_void_p(32), 0, None, None) == rr.RR_ERR_ARG
    assert lib.rr_tidal_tensor_box(C.byref(g), C.c_void_p(32), None, C.c_void_p(16), 0, C.cast(bb, C.c_void_p),
                                   None) == rr.RR_ERR_ARG
    assert lib.rr_finalize(None, None, None, None) == rr.RR_ERR_ARG
    assert lib.rr_destroy(None) == rr.RR_ERR_ARG
    out = (C.c_int32 * 6)()
    assert lib.rr_footprint_bbox(C.byref(good), C.byref(g), 1.0, 2.0, C.cast(out, C.c_void_p)) == rr.RR_ERR_ARG


def test_upload_box_validation_is_host_side(rr):
    lib = rr.load()
    g = rr.grid_desc(synth.Grid((8, 8, 8), 16.0))
    gbad = rr.grid_desc(synth.Grid((8, 8, 5000), 16.0))
    nb = C.c_int64(-1)
    p = C.c_void_p(16)
    assert lib.rr_upload_box(None, p, p, None, C.byref(nb), None) == rr.RR_ERR_ARG
    assert lib.rr_upload_box(C.byref(gbad), p, p, None, C.byref(nb), None) == rr.RR_ERR_ARG
    assert lib.rr_upload_box(C.byref(g), None, p, None, C.byref(nb), None) == rr.RR_ERR_ARG
    assert lib.rr_upload_box(C.byref(g), p, None, None, C.byref(nb), None) == rr.RR_ERR_ARG
    for box in ((0, 9, 0, 8, 0, 8), (0, 8, 3, 3, 0, 8), (0, 8, 0, 8, 5, 4), (-(1 << 21), -(1 << 21) + 2, 0, 8, 0, 8)):
        bb = (C.c_int32 * 6)(*box)
        assert lib.rr_upload_box(C.byref(g), p, p, C.cast(bb, C.c_void_p), C.byref(nb), None) == rr.RR_ERR_ARG, box
    assert nb.value == -1   # nothing reported for a refused call


@pytest.mark.parametrize("fov,obs,chi_a,chi_b", [
    (10.0, (32.0, 32.0, 0.0), 60.0, 40.0),
    (40.0, (2.0, 60.0, 0.0), 30.0, 0.0),
    (3.0, (32.0, 32.0, 5.0), 63.0, 62.0),
])
def test_footprint_bbox_covers_oracle_walk(rr, oracle_lib, fov, obs, chi_a, chi_b):
    """Every vertex of every cell the oracle's walk visits over [chi_b, chi_a]
    lies inside the box returned by rr_footprint_bbox (indices mod n)."""
    g = synth.Grid((32, 32, 32), 64.0)
    b = synth.Bundle(9, 7, synth.deg(fov), synth.deg(fov * 0.8), obs, 64.0)
    bbox = rr.rr_footprint_bbox(rr.bundle_desc(b), rr.grid_desc(g), chi_a, chi_b)
    n = 32
    for a in range(3):
        assert 1 <= bbox[2 * a + 1] - bbox[2 * a] <= n
    inside = [np.zeros(n, bool) for _ in range(3)]
    for a in range(3):
        idx = np.arange(bbox[2 * a], bbox[2 * a + 1]) % n
        inside[a][idx] = True
    for rid in range(b.nrays):
        rows = oracle_lib.ray_segments(b, g, rid, chi_a, chi_b)
        for r in rows:
            for a in range(3):
                c = int(r[2 + a])
                assert inside[a][c % n] and inside[a][(c + 1) % n], (rid, a, c, bbox)


def test_amr_plan_validation_is_host_side(rr):
    """rr_amr_create rejects bad descriptions and meshes that are not 2:1
    balanced while building its plan on the host, before any device work."""
    lib = rr.load()
    h = C.c_void_p()

    def create(n, lmax, octs, box=8.0):
        d = rr.rr_amr_desc()
        d.n, d.lmax, d.box, d.omega_m = n, lmax, box, 0.3
        keep = [np.ascontiguousarray(np.asarray(o, np.int32).reshape(-1, 3)) for o in octs]
        ptrs = (C.c_void_p * (lmax + 1))()
        counts = (C.c_int64 * (lmax + 1))()
        for lv in range(1, lmax + 1):
            ptrs[lv] = keep[lv].ctypes.data if keep[lv].size else None
            counts[lv] = keep[lv].shape[0]
        return lib.rr_amr_create(C.byref(d), C.cast(ptrs, C.c_void_p), C.cast(counts, C.c_void_p), C.byref(h))

    empty = np.zeros((0, 3))
    assert create(1, 0, [empty]) == rr.RR_ERR_ARG                          # n < 2
    assert create(4, 9, [empty] * 10) == rr.RR_ERR_ARG                     # lmax > 8
    assert create(4, 0, [empty], box=0.0) == rr.RR_ERR_ARG                 # box
    assert create(4, 1, [empty, [[4, 0, 0]]]) == rr.RR_ERR_ARG             # parent outside the grid
    assert create(4, 1, [empty, [[1, 1, 1], [1, 1, 1]]]) == rr.RR_ERR_ARG  # refined twice
    # a level-2 oct whose level-1 parent does not exist
    assert create(4, 2, [empty, [[1, 1, 1]], [[0, 0, 0]]]) == rr.RR_ERR_ARG
    # a level-2 oct next to unrefined coarse cells: not 2:1 balanced
    assert create(4, 2, [empty, [[1, 1, 1]], [[2, 2, 2]]]) == rr.RR_ERR_ARG
    assert lib.rr_amr_create(None, None, None, C.byref(h)) == rr.RR_ERR_ARG
    assert lib.rr_amr_destroy(None) == rr.RR_ERR_ARG
    assert lib.rr_amr_sizes(None, None, None, None) == rr.RR_ERR_ARG
    assert lib.rr_amr_tidal(None, C.c_void_p(16), 0, C.c_void_p(16), None, None, None) == rr.RR_ERR_ARG
    assert lib.rr_amr_trace_step(None, None, C.c_void_p(16), 1.0, 0.0, 1.0, 1.0, None) == rr.RR_ERR_ARG


def test_source_kappa_validation_is_host_side(rr):
    lib = rr.load()
    assert lib.rr_source_kappa(None, None, 4, 1.0, C.c_void_p(16), None, None) == rr.RR_ERR_ARG
    assert lib.rr_source_kappa(C.c_void_p(16), None, 0, 1.0, C.c_void_p(16), None, None) == rr.RR_ERR_ARG
    assert lib.rr_source_kappa(C.c_void_p(16), None, 4, 0.0, C.c_void_p(16), None, None) == rr.RR_ERR_ARG
    assert lib.rr_moments(None, C.c_void_p(16), None) == rr.RR_ERR_ARG
    good = rr.bundle_desc(synth.Bundle(4, 4, 0.1, 0.1, (1, 1, 0), 10.0))
    h = C.c_void_p()
    for flags in (rr.RR_SOURCE_MOMENTS | rr.RR_FP64_DDA, rr.RR_SOURCE_MOMENTS | rr.RR_PLAIN_SUMS, 128):
        good.flags = flags
        assert lib.rr_create(C.byref(good), C.byref(h)) == rr.RR_ERR_ARG


def test_method_a_validation_is_host_side(rr):
    lib = rr.load()
    g = rr.grid_desc(synth.Grid((8, 8, 8), 16.0))
    assert lib.rr_gradient_records(C.byref(g), None, None, C.c_void_p(16), 0, None, None) == rr.RR_ERR_ARG
    assert lib.rr_gradient_records(C.byref(g), C.c_void_p(16), None, C.c_void_p(8), 0, None, None) == rr.RR_ERR_ARG
    assert lib.rr_gradient_records(C.byref(g), C.c_void_p(16), None, C.c_void_p(16), 2, None, None) == rr.RR_ERR_ARG
    good = rr.bundle_desc(synth.Bundle(4, 4, 0.1, 0.1, (1, 1, 0), 10.0))
    h = C.c_void_p()
    for other in (rr.RR_FP64_DDA, rr.RR_PLAIN_SUMS, rr.RR_SOURCE_MOMENTS, rr.RR_SHEAR):
        good.flags = rr.RR_METHOD_A | other
        assert lib.rr_create(C.byref(good), C.byref(h)) == rr.RR_ERR_ARG


def test_generic_and_relocation_validation_is_host_side(rr):
    lib = rr.load()
    g = rr.grid_desc(synth.Grid((8, 8, 8), 16.0))
    f = C.c_void_p(16)
    assert lib.rr_scalar_records(C.byref(g), None, None, 1.0, 0, f, 0, None, None) == rr.RR_ERR_ARG
    assert lib.rr_scalar_records(C.byref(g), f, None, 1.0, 2, f, 0, None, None) == rr.RR_ERR_ARG
    assert lib.rr_scalar_records(C.byref(g), f, None, float("inf"), 0, f, 0, None, None) == rr.RR_ERR_ARG
    assert lib.rr_scalar_records(C.byref(g), f, None, 1.0, 0, C.c_void_p(8), 0, None, None) == rr.RR_ERR_ARG
    assert lib.rr_set_kernels(None, f) == rr.RR_ERR_ARG
    assert lib.rr_set_observer(None, f) == rr.RR_ERR_ARG
    good = rr.bundle_desc(synth.Bundle(4, 4, 0.1, 0.1, (1, 1, 0), 10.0))
    h = C.c_void_p()
    for other in (rr.RR_FP64_DDA, rr.RR_PLAIN_SUMS, rr.RR_SOURCE_MOMENTS, rr.RR_SHEAR, rr.RR_METHOD_A):
        good.flags = rr.RR_GENERIC | other
        assert lib.rr_create(C.byref(good), C.byref(h)) == rr.RR_ERR_ARG


def test_shear_validation_is_host_side(rr):
    lib = rr.load()
    assert lib.rr_shear(None, C.c_void_p(16), C.c_void_p(16), None) == rr.RR_ERR_ARG
    good = rr.bundle_desc(synth.Bundle(4, 4, 0.1, 0.1, (1, 1, 0), 10.0))
    h = C.c_void_p()
    for other in (rr.RR_FP64_DDA, rr.RR_PLAIN_SUMS, rr.RR_SOURCE_MOMENTS):
        good.flags = rr.RR_SHEAR | other
        assert lib.rr_create(C.byref(good), C.byref(h)) == rr.RR_ERR_ARG
