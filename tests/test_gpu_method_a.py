"""Method A (RR_METHOD_A; Eq. kappa2, Sec. 3.5) against the oracle, through
the C ABI: the gradient records of rr_gradient_records, and kappa = density
term + int (1 - 2 chi/chi_s) n.grad(Phi) dchi + the steps' surface terms.

Tolerances: records per channel max|diff| <= 4e-6 max|oracle| (FP32 stencils);
maps max|x_gpu - x_ora| / rms(x_ora) <= 1e-5 and the same in the l2 norm.
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def rrp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_02012_gb300 import build
    build.build()
    import paper_1601_02012_gb300 as pkg
    return pkg


def _err(got, want):
    got = np.asarray(got, np.float64).ravel()
    want = np.asarray(want, np.float64).ravel()
    rms = math.sqrt(float(np.mean(want ** 2)))
    return float(np.abs(got - want).max() / rms), float(np.linalg.norm(got - want) / np.linalg.norm(want))


def _vertex_mean(F):
    """Mean of the 8 cells sharing each vertex (vertex i is the lower corner of
    cell i: cells i-1..i per axis), periodic."""
    out = np.zeros_like(F)
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                out += np.roll(F, (dx, dy, dz), axis=(0, 1, 2))
    return out / 8.0


@pytest.mark.parametrize("where", ["vertices", "centres"])
@pytest.mark.parametrize("with_delta", [False, True])
@pytest.mark.parametrize("shape", [(24, 20, 40), (2, 3, 5), (5, 2, 33)])
def test_gradient_records(rrp, oracle_lib, where, with_delta, shape):
    import torch
    g = synth.Grid(shape, 2.0 * shape[0])
    phi = synth.random_field(g.n, 17, np.float32)
    delta = synth.random_field(g.n, 18, np.float32) if with_delta else None
    G = oracle_lib.fields_grad(g, phi.astype(np.float64))
    _, d = oracle_lib.fields(g, phi.astype(np.float64), None if delta is None else delta.astype(np.float64))
    want = np.concatenate([G, d[..., None]], axis=-1)
    if where == "vertices":
        want = _vertex_mean(want)
    rec = rrp.gradient_buffer(g)
    dl = None if delta is None else torch.from_numpy(delta).cuda()
    rrp.rr_gradient_records(rrp.grid_desc(g), torch.from_numpy(phi).cuda(), dl, rec,
                            rrp.RR_AT_VERTICES if where == "vertices" else rrp.RR_AT_CENTRES)
    got = rec.cpu().numpy().reshape(tuple(g.n) + (4,))
    for c in range(4):
        scale = np.abs(want[..., c]).max()
        assert np.abs(got[..., c] - want[..., c]).max() <= 4e-6 * scale, c


def test_gradient_records_bbox_writes_only_the_box(rrp):
    import torch
    g = synth.Grid((16, 16, 16), 32.0)
    phi = torch.from_numpy(synth.grf_phi(16, 32.0, 19)).cuda()
    full = rrp.gradient_buffer(g)
    rrp.rr_gradient_records(rrp.grid_desc(g), phi, None, full, rrp.RR_AT_VERTICES)
    part = torch.full_like(full, float("nan"))
    bbox = (-3, 5, 10, 16, 2, 15)
    rrp.rr_gradient_records(rrp.grid_desc(g), phi, None, part, rrp.RR_AT_VERTICES, bbox)
    f = full.cpu().numpy().reshape(16, 16, 16, 4)
    p = part.cpu().numpy().reshape(16, 16, 16, 4)
    mask = np.zeros((16, 16, 16), bool)
    mask[np.ix_(np.arange(-3, 5) % 16, np.arange(10, 16), np.arange(2, 15))] = True
    assert np.array_equal(p[mask], f[mask])
    assert np.all(np.isnan(p[~mask]))


def _gpu(rrp, phi, grid, bundle, steps, delta=None):
    import torch
    ph = torch.from_numpy(np.ascontiguousarray(phi, np.float32)).cuda()
    dl = None if delta is None else torch.from_numpy(np.ascontiguousarray(delta, np.float32)).cuda()
    k, kb, nseg = rrp.trace_method_a(ph, grid, bundle, steps, delta=dl)
    torch.cuda.synchronize()
    return k.cpu().numpy().ravel(), kb.cpu().numpy().ravel(), nseg


def _oracle(oracle_lib, phi, grid, bundle, steps, delta=None, rids=None):
    p64 = np.asarray(phi, np.float32).astype(np.float64)
    d64 = None if delta is None else np.asarray(delta, np.float32).astype(np.float64)
    _, d = oracle_lib.fields(grid, p64, d64)
    kg, kb = oracle_lib.trace_method_a(bundle, grid, oracle_lib.fields_grad(grid, p64), d, steps, rids=rids)
    return kg + kb, kb


@pytest.mark.parametrize("interp", [1, 0])
@pytest.mark.parametrize("periodic", [True, False])
def test_method_a_parity_multi_step(rrp, oracle_lib, interp, periodic):
    """A ragged 37 x 29 bundle over 48^3 in five steps with different scales and
    scale factors (the surface terms then do not telescope)."""
    g = synth.Grid((48, 48, 48), 96.0)
    b = synth.Bundle(37, 29, synth.deg(14), synth.deg(11), (47.0, 49.0, 0.5), 180.0, interp=interp,
                     periodic=periodic)
    phi = synth.grf_phi(48, 96.0, 61)
    edges = [180.0, 140.0, 101.0, 66.0, 30.0, 0.0]
    steps = [synth.Step(edges[i], edges[i + 1], 1.0 - 0.04 * i, 0.55 + 0.08 * i) for i in range(5)]
    k, kb, _ = _gpu(rrp, phi, g, b, steps)
    ko, kbo = _oracle(oracle_lib, phi, g, b, steps)
    for x, y, what in ((k, ko, "kappa"), (kb, kbo, "kborn")):
        e_inf, e_2 = _err(x, y)
        assert e_inf <= TOL and e_2 <= TOL, (what, e_inf, e_2)


def test_method_a_long_steps_and_given_delta(rrp, oracle_lib):
    """One step longer than the FP32 walk's sub-step (the surface terms only at
    the interval's two ends) with an independent delta, wide field including
    the axis ray."""
    g = synth.Grid((40, 40, 40), 40.0)
    b = synth.Bundle(21, 21, synth.deg(30), synth.deg(30), (20.0, 20.0, 0.0), 140.0)
    phi = synth.grf_phi(40, 40.0, 63)
    delta = synth.random_field(g.n, 64, np.float32, scale=0.5)
    steps = [synth.Step(130.0, 1.0, 0.9, 0.8)]
    k, kb, _ = _gpu(rrp, phi, g, b, steps, delta=delta)
    ko, kbo = _oracle(oracle_lib, phi, g, b, steps, delta=delta)
    for x, y, what in ((k, ko, "kappa"), (kb, kbo, "kborn")):
        e_inf, e_2 = _err(x, y)
        assert e_inf <= TOL and e_2 <= TOL, (what, e_inf, e_2)


def test_method_a_gaussian_lens(rrp, oracle_lib):
    """Sec. 4's lens by Method A on a 129 x 129 map at 64^3 (rays stop at
    chi = 8 Mpc/h): GPU against the oracle, and within 1 % of Method B's
    oracle map away from the zero crossings (the two methods agree)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "gaussian_e1.json")) as f:
        E1 = json.load(f)
    L = E1["box"]
    nr = 129
    b = synth.Bundle(nr, nr, synth.deg(E1["fov_deg"][0]), synth.deg(E1["fov_deg"][1]), (L / 2, L / 2, 0.0),
                     synth.chi_of_z(E1["z_s"]), periodic=False)
    g = synth.Grid((64, 64, 64), L)
    phi = synth.gaussian_phi(64, L, E1["potential"]["amp"], E1["potential"]["sigma"])
    steps = [synth.Step(E1["gamma1_chi_max"], 0.0, 1.0, 1.0)]
    k, kb, _ = _gpu(rrp, phi, g, b, steps)
    ko, kbo = _oracle(oracle_lib, phi, g, b, steps)
    for x, y, what in ((k, ko, "kappa"), (kb, kbo, "kborn")):
        e_inf, e_2 = _err(x, y)
        assert e_inf <= TOL and e_2 <= TOL, (what, e_inf, e_2)
    H, d = oracle_lib.fields(g, phi.astype(np.float32).astype(np.float64))
    kB = oracle_lib.trace(b, g, H, d, steps).kappa
    keep = np.abs(kB) > 0.1 * np.abs(kB).max()
    assert (np.abs(k - kB)[keep] / np.abs(kB[keep])).max() < 0.01


def test_method_a_at_production_size_sampled(rrp, oracle_lib):
    """The 512^3, 2048 x 2048-ray, 40-step production workload by Method A;
    128 sampled rays traced by the oracle one by one."""
    w = synth.workload("prod_512")
    phi = synth.grf_phi(512, w.grid.box, w.seed)
    steps = synth.step_schedule(w.bundle.chi_s, w.nsteps, rescale=True)
    k, kb, _ = _gpu(rrp, phi, w.grid, w.bundle, steps)
    rids = np.random.default_rng(11).choice(w.bundle.nrays, 128, replace=False)
    ko, kbo = _oracle(oracle_lib, phi, w.grid, w.bundle, steps, rids=rids)
    for x, y, what in ((k, ko, "kappa"), (kb, kbo, "kborn")):
        rms = math.sqrt(float(np.mean(y ** 2)))
        assert np.abs(x[rids] - y).max() <= TOL * rms, what


def test_method_a_form_checks(rrp):
    import torch
    from paper_1601_02012_gb300 import _rr
    b = synth.Bundle(8, 8, synth.deg(5), synth.deg(5), (4.0, 4.0, 0.0), 10.0)
    for kw in ({"fp64_dda": True}, {"plain_sums": True}, {"moments": True}, {"shear": True}):
        with pytest.raises(rrp.RRError) as ei:
            rrp.Tracer(b, method_a=True, **kw)
        assert ei.value.code == _rr.RR_ERR_ARG
    g = synth.Grid((8, 8, 8), 16.0)
    tr = rrp.Tracer(b, method_a=True)
    rec = tr.record_buffer(g)
    assert tuple(rec.shape) == (512, 4)
    tr.tidal(g, torch.from_numpy(synth.random_field(8, 3, np.float32)).cuda(), rec)
    tr.step(g, rec, 10.0, 0.0)
    tr.finalize()
    with pytest.raises(rrp.RRError) as ei:   # no adjoint for Method A
        rrp.rr_trace_step_adjoint(tr.ctx, 0, torch.ones(64, dtype=torch.float64, device="cuda"), None,
                                  rrp.grad_buffer(g))
    assert ei.value.code == _rr.RR_ERR_STATE
    tr.close()
