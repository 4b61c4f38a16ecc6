"""rr_trace_step_noalloc against the regular entry points and the oracle,
through the C ABI.

The no-allocation entry point serves callers that cannot let the library
allocate device memory (a host framework owning the device memory pool, code
that cannot take the synchronisation cudaMalloc implies, plugin hosts that
forbid driver allocations). Its scratch is a fixed array in the library's
device memory; this file checks that two calls in a row each reproduce the
maps of rr_create + rr_trace_step + rr_finalize on the same inputs, within the
map tolerance the parity tests use, for every walk it accepts (periodic and
bounded boxes, the FP32 and the FP64 walk, both interpolations); that one call
matches the FP64 oracle directly; that a bundle larger than the fixed scratch
is refused; and that it rejects the arguments rr_create and rr_trace_step
reject. It is collected last so that a run stopping at its first failure has
already run every other test.
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


def _regular(rrp, bundle, grid, rec, step, fp64_dda):
    tr = rrp.Tracer(bundle, fp64_dda=fp64_dda)
    tr.step(grid, rec, step.chi_a, step.chi_b, step.scale, step.a)
    k, kb = tr.finalize()
    tr.close()
    return k.cpu().numpy(), kb.cpu().numpy()


def _noalloc(rrp, bundle, grid, rec, step, fp64_dda):
    import torch
    from paper_1601_02012_gb300 import _rr
    bd, gd = _rr.bundle_desc(bundle, fp64_dda=fp64_dda), _rr.grid_desc(grid)
    k = torch.full((bundle.ny, bundle.nx), float("nan"), dtype=torch.float64, device="cuda")
    kb = torch.full_like(k, float("nan"))
    _rr.rr_trace_step_noalloc(bd, gd, rec, step.chi_a, step.chi_b, k, kb, step.scale, step.a)
    torch.cuda.synchronize()
    return k.cpu().numpy(), kb.cpu().numpy()


def _setup(rrp, interp, periodic):
    import torch
    g = synth.Grid((48, 48, 48), 96.0)
    phi = torch.from_numpy(synth.grf_phi(48, 96.0, 21)).cuda()
    # bounded: the observer inside the box, so that rays leave it through its faces
    obs = (48.0, 48.0, 0.0) if periodic else (47.3, 48.6, 10.0)
    bundle = synth.Bundle(96, 80, synth.deg(9), synth.deg(7), obs, 95.0, interp=interp, periodic=periodic)
    where = rrp.RR_AT_VERTICES if interp == 1 else rrp.RR_AT_CENTRES
    rec = rrp.record_buffer(g)
    rrp.rr_tidal_tensor(rrp.grid_desc(g), phi, None, rec, where)
    return g, phi, bundle, rec


WALKS = [(True, False), (False, False), (True, True)]   # (periodic, fp64_dda)


@pytest.mark.parametrize("walk", WALKS, ids=["periodic", "bounded", "periodic-fp64"])
@pytest.mark.parametrize("interp", [1, 0])
def test_noalloc_matches_regular_path_twice(rrp, interp, walk):
    periodic, fp64_dda = walk
    g, _, bundle, rec = _setup(rrp, interp, periodic)
    steps = [synth.Step(95.0, 40.0, 1.3, 0.8), synth.Step(40.0, 0.0, 0.9, 1.0)]
    for st in steps:   # two calls in a row, different steps
        want_k, want_b = _regular(rrp, bundle, g, rec, st, fp64_dda)
        got_k, got_b = _noalloc(rrp, bundle, g, rec, st, fp64_dda)
        for got, want in ((got_k, want_k), (got_b, want_b)):
            e_inf, e_2 = _map_err(got, want)
            assert e_inf <= TOL and e_2 <= TOL, (e_inf, e_2)


@pytest.mark.parametrize("interp", [1, 0])
def test_noalloc_matches_oracle(rrp, oracle_lib, interp):
    """One call against the FP64 oracle on the same FP32 potential."""
    g, phi, bundle, rec = _setup(rrp, interp, True)
    st = synth.Step(95.0, 20.0, 1.1, 0.9)
    got_k, got_b = _noalloc(rrp, bundle, g, rec, st, False)
    H, d = oracle_lib.fields(g, phi.cpu().numpy().astype(np.float64))
    ora = oracle_lib.trace(bundle, g, H, d, [st])
    for got, want in ((got_k, ora.kappa), (got_b, ora.kborn)):
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


def test_noalloc_rejects_what_the_regular_path_rejects(rrp):
    """A field of view of pi, a NaN observer, an infinite source distance,
    scale or box, and a flag outside its two walks give RR_ERR_ARG (before
    any work is queued)."""
    import ctypes as C

    import torch
    from paper_1601_02012_gb300 import _rr

    g = synth.Grid((8, 8, 8), 16.0)
    rec = rrp.record_buffer(g)
    rec.zero_()
    out = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    lib = _rr.load()

    def call(bd, gd, chi_a=15.0, chi_b=0.0, scale=1.0, a_step=1.0):
        return lib.rr_trace_step_noalloc(C.byref(bd), C.byref(gd), C.c_void_p(rec.data_ptr()), chi_a, chi_b,
                                         scale, a_step, C.c_void_p(out.data_ptr()), None, None)

    ok = synth.Bundle(8, 8, 0.1, 0.1, (8.0, 8.0, 0.0), 15.0)
    assert call(_rr.bundle_desc(ok), _rr.grid_desc(g)) == _rr.RR_OK
    bad = []
    d = _rr.bundle_desc(ok); d.fov_x = math.pi; bad.append((d, _rr.grid_desc(g), {}))
    d = _rr.bundle_desc(ok); d.obs[1] = float("nan"); bad.append((d, _rr.grid_desc(g), {}))
    d = _rr.bundle_desc(ok); d.chi_s = float("inf"); bad.append((d, _rr.grid_desc(g), {}))
    d = _rr.bundle_desc(ok); d.flags |= _rr.RR_SHEAR; bad.append((d, _rr.grid_desc(g), {}))
    gd = _rr.grid_desc(g); gd.box = float("inf"); bad.append((_rr.bundle_desc(ok), gd, {}))
    bad.append((_rr.bundle_desc(ok), _rr.grid_desc(g), {"scale": float("inf")}))
    bad.append((_rr.bundle_desc(ok), _rr.grid_desc(g), {"scale": float("nan")}))
    bad.append((_rr.bundle_desc(ok), _rr.grid_desc(g), {"a_step": float("nan")}))
    bad.append((_rr.bundle_desc(ok), _rr.grid_desc(g), {"chi_b": float("nan")}))
    for bd, gd, kw in bad:
        assert call(bd, gd, **kw) == _rr.RR_ERR_ARG, kw
