"""rr_trace_step_noalloc against the regular entry points, through the C ABI.

The no-allocation entry point serves callers that cannot let the library
allocate device memory (a host framework owning the device memory pool, code
that cannot take the synchronisation cudaMalloc implies, plugin hosts that
forbid driver allocations). Its scratch is a fixed array in the library's
device memory; this file checks that two calls in a row each reproduce the
maps of rr_create + rr_trace_step + rr_finalize on the same inputs, within the
map tolerance the parity tests use, and that a bundle larger than the fixed
scratch is refused. It is collected last so that a run stopping at its first
failure has already run every other test.
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _map_err(got, want):
    got = np.asarray(got, np.float64).ravel()
    want = np.asarray(want, np.float64).ravel()
    rms = math.sqrt(float(np.mean(want * want)))
    d = got - want
    return float(np.abs(d).max() / rms), float(np.linalg.norm(d) / np.linalg.norm(want))


@pytest.fixture(scope="module")
def rrp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_02012_gb300 import build
    build.build()
    import paper_1601_02012_gb300 as pkg
    return pkg


def _regular(rrp, bundle, grid, rec, step):
    tr = rrp.Tracer(bundle)
    tr.step(grid, rec, step.chi_a, step.chi_b, step.scale, step.a)
    k, kb = tr.finalize()
    tr.close()
    return k.cpu().numpy(), kb.cpu().numpy()


@pytest.mark.parametrize("interp", [1, 0])
def test_noalloc_matches_regular_path_twice(rrp, interp):
    import torch
    from paper_1601_02012_gb300 import _rr

    g = synth.Grid((48, 48, 48), 96.0)
    phi = torch.from_numpy(synth.grf_phi(48, 96.0, 21)).cuda()
    bundle = synth.Bundle(96, 80, synth.deg(9), synth.deg(7), (48.0, 48.0, 0.0), 95.0, interp=interp)
    where = rrp.RR_AT_VERTICES if interp == 1 else rrp.RR_AT_CENTRES
    rec = rrp.record_buffer(g)
    rrp.rr_tidal_tensor(rrp.grid_desc(g), phi, None, rec, where)
    steps = [synth.Step(95.0, 40.0, 1.3, 0.8), synth.Step(40.0, 0.0, 0.9, 1.0)]
    bd, gd = _rr.bundle_desc(bundle), _rr.grid_desc(g)
    for st in steps:   # two calls in a row, different steps
        want_k, want_b = _regular(rrp, bundle, g, rec, st)
        k = torch.full((bundle.ny, bundle.nx), float("nan"), dtype=torch.float64, device="cuda")
        kb = torch.full_like(k, float("nan"))
        _rr.rr_trace_step_noalloc(bd, gd, rec, st.chi_a, st.chi_b, k, kb, st.scale, st.a)
        torch.cuda.synchronize()
        for got, want in ((k.cpu().numpy(), want_k), (kb.cpu().numpy(), want_b)):
            e_inf, e_2 = _map_err(got, want)
            assert e_inf <= TOL and e_2 <= TOL, (e_inf, e_2)


def test_noalloc_refuses_more_rays_than_its_scratch(rrp):
    import ctypes as C

    import torch
    from paper_1601_02012_gb300 import _rr

    g = synth.Grid((8, 8, 8), 16.0)
    rec = rrp.record_buffer(g)
    rec.zero_()
    big = synth.Bundle(257, 256, 0.1, 0.1, (8.0, 8.0, 0.0), 15.0)
    out = torch.zeros((256, 257), dtype=torch.float64, device="cuda")
    lib = _rr.load()
    code = lib.rr_trace_step_noalloc(C.byref(_rr.bundle_desc(big)), C.byref(_rr.grid_desc(g)),
                                     C.c_void_p(rec.data_ptr()), 15.0, 0.0, 1.0, 1.0,
                                     C.c_void_p(out.data_ptr()), None, None)
    assert code == _rr.RR_ERR_CAPACITY
    with pytest.raises(_rr.RRError):
        _rr.rr_trace_step_noalloc(_rr.bundle_desc(big), _rr.grid_desc(g), rec, 15.0, 0.0, out)
