"""Generic line-of-sight integrals (RR_GENERIC; Eqs. Ic, Icngp, Icfinal; the
ISW integral of Sec. 6) and box tiling with a relocated observer (Sec. 2.2),
against the oracle through the C ABI.

Tolerances: records max|diff| <= 4e-6 max|oracle|; maps max|x_gpu - x_ora| /
rms(x_ora) <= 1e-5 and the same in the l2 norm.
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
    out = np.zeros_like(F)
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                out += np.roll(F, (dx, dy, dz), axis=(0, 1, 2))
    return out / 8.0


@pytest.mark.parametrize("where", ["vertices", "centres"])
@pytest.mark.parametrize("shape", [(24, 20, 40), (2, 3, 5)])
def test_scalar_records(rrp, where, shape):
    """Channel 0 the field, channel 1 the finite-difference time derivative."""
    import torch
    g = synth.Grid(shape, 2.0 * shape[0])
    f = synth.random_field(g.n, 71, np.float32)
    fp = synth.random_field(g.n, 72, np.float32)
    inv_dt = 37.5
    rec = rrp.scalar_buffer(g)
    flag = rrp.RR_AT_VERTICES if where == "vertices" else rrp.RR_AT_CENTRES
    gd = rrp.grid_desc(g)
    ft, fpt = torch.from_numpy(f).cuda(), torch.from_numpy(fp).cuda()
    rrp.rr_scalar_records(gd, ft, None, 1.0, 0, rec, flag)
    rrp.rr_scalar_records(gd, ft, fpt, inv_dt, 1, rec, flag)
    got = rec.cpu().numpy().reshape(tuple(g.n) + (2,))
    want = np.stack([f.astype(np.float64), (f.astype(np.float64) - fp) * inv_dt], axis=-1)
    if where == "vertices":
        want = _vertex_mean(want)
    for c in range(2):
        scale = np.abs(want[..., c]).max()
        assert np.abs(got[..., c] - want[..., c]).max() <= 4e-6 * scale, c


def _gpu_kq(rrp, q1, q2, grid, bundle, steps, kernels):
    import torch
    tr = rrp.Tracer(bundle, generic=True)
    tr.set_kernels(kernels)
    rec = tr.record_buffer(grid)
    for st in steps:
        bbox = tr.footprint(grid, st.chi_a, st.chi_b)
        tr.scalars(grid, torch.from_numpy(np.ascontiguousarray(q1, np.float32)).cuda(), rec, 0, bbox=bbox)
        tr.scalars(grid, torch.from_numpy(np.ascontiguousarray(q2, np.float32)).cuda(), rec, 1, bbox=bbox)
        tr.step(grid, rec, st.chi_a, st.chi_b, st.scale, st.a)
    o1, o2 = tr.finalize()
    torch.cuda.synchronize()
    tr.close()
    return o1.cpu().numpy().ravel(), o2.cpu().numpy().ravel()


KERNELS = ((0.7, -0.011, 0.00004), (-1.3, 0.02, -0.0001))


@pytest.mark.parametrize("interp", [1, 0])
@pytest.mark.parametrize("periodic", [True, False])
def test_generic_integrals_parity(rrp, oracle_lib, interp, periodic):
    g = synth.Grid((48, 48, 48), 96.0)
    b = synth.Bundle(37, 29, synth.deg(14), synth.deg(11), (47.0, 49.0, 0.5), 180.0, interp=interp,
                     periodic=periodic)
    q1 = synth.grf_phi(48, 96.0, 73) * 1e4
    q2 = synth.random_field(g.n, 74, np.float32)
    edges = [180.0, 133.0, 90.0, 41.0, 0.0]
    steps = [synth.Step(edges[i], edges[i + 1], 1.0 - 0.05 * i, 1.0) for i in range(4)]
    o1, o2 = _gpu_kq(rrp, q1, q2, g, b, steps, KERNELS)
    w1, w2 = oracle_lib.trace_kq(b, g, q1.astype(np.float32).astype(np.float64),
                                 q2.astype(np.float32).astype(np.float64), KERNELS, steps)
    for x, y, what in ((o1, w1, "ch0"), (o2, w2, "ch1")):
        e_inf, e_2 = _err(x, y)
        assert e_inf <= TOL and e_2 <= TOL, (what, e_inf, e_2)


def test_isw_integral(rrp, oracle_lib):
    """The ISW integral of Sec. 6 over a growing potential: channel 0 integrates
    dPhi/dt = (Phi_curr - Phi_prev) / dt of each step (records built from two
    potentials), channel 1 the potential itself with the lensing kernel."""
    import torch
    g = synth.Grid((32, 32, 32), 64.0)
    b = synth.Bundle(40, 33, synth.deg(10), synth.deg(9), (32.0, 31.0, 0.0), 120.0)
    phi0 = synth.grf_phi(32, 64.0, 75)
    steps = synth.step_schedule(b.chi_s, 6, rescale=True)
    dt = 0.01
    ker = ((2.0, 0.0, 0.0), (0.0, 1.0, -1.0 / b.chi_s))
    tr = rrp.Tracer(b, generic=True)
    tr.set_kernels(ker)
    rec = tr.record_buffer(g)
    want1 = np.zeros(b.nrays)
    want2 = np.zeros(b.nrays)
    for i, st in enumerate(steps):
        cur = (phi0 * np.float32(st.scale)).astype(np.float32)
        prev = (phi0 * np.float32(st.scale * (1.0 - 0.03 * (i + 1)))).astype(np.float32)
        tr.scalars(g, torch.from_numpy(cur).cuda(), rec, 0, field_prev=torch.from_numpy(prev).cuda(), inv_dt=1 / dt)
        tr.scalars(g, torch.from_numpy(cur).cuda(), rec, 1)
        tr.step(g, rec, st.chi_a, st.chi_b, 1.0, st.a)
        one = synth.Step(st.chi_a, st.chi_b, 1.0, st.a)
        q = (cur.astype(np.float64) - prev.astype(np.float64)) / dt
        o1, o2 = oracle_lib.trace_kq(b, g, q, cur.astype(np.float64), ker, [one])
        want1 += o1
        want2 += o2
    o1, o2 = tr.finalize()
    tr.close()
    for x, y in ((o1.cpu().numpy(), want1), (o2.cpu().numpy(), want2)):
        e_inf, e_2 = _err(x, y)
        assert e_inf <= TOL and e_2 <= TOL, (e_inf, e_2)


def _tiles(n=32, L=64.0):
    return [(synth.grf_phi(n, L, 80 + i), synth.Grid((n, n, n), L), (L / 2, L / 2 - 3.0, -i * L)) for i in range(3)]


@pytest.mark.parametrize("interp", [1, 0])
def test_tiled_boxes_with_relocated_observer(rrp, oracle_lib, interp):
    """Sec. 2.2: a bundle through three boxes stacked along the line of sight,
    each a different realisation, traced in one context that moves the
    observer to its position relative to each box; against the oracle traced
    box by box from the same positions."""
    import torch
    L = 64.0
    b = synth.Bundle(41, 36, synth.deg(12), synth.deg(10), (0.0, 0.0, 0.0), 3 * L - 1.0, interp=interp,
                     periodic=False)
    steps = [synth.Step(3 * L - 1.0, 120.0, 0.9, 0.7), synth.Step(120.0, 50.0, 1.0, 0.8),
             synth.Step(50.0, 0.0, 1.1, 0.9)]
    tiles = _tiles()
    k, kb, _ = rrp.trace_tiles([(torch.from_numpy(p).cuda(), g, o) for p, g, o in tiles], b, steps)
    wk = np.zeros(b.nrays)
    wb = np.zeros(b.nrays)
    for p, g, o in tiles:
        bo = synth.Bundle(b.nx, b.ny, b.fov_x, b.fov_y, o, b.chi_s, interp=interp, periodic=False)
        H, d = oracle_lib.fields(g, p.astype(np.float64))
        r = oracle_lib.trace(bo, g, H, d, steps)
        wk += r.kappa
        wb += r.kborn
    for x, y, what in ((k.cpu().numpy(), wk, "kappa"), (kb.cpu().numpy(), wb, "kborn")):
        e_inf, e_2 = _err(x, y)
        assert e_inf <= TOL and e_2 <= TOL, (what, e_inf, e_2)


def test_tiled_adjoint_replays_each_observer(rrp):
    """The adjoint after a relocation replays every step from the observer it
    was traced from: with one step per box, <J x, y> = sum over boxes of
    <x_box, J_box^T y> (GPU forward against GPU adjoint)."""
    import torch
    L = 64.0
    b = synth.Bundle(33, 30, synth.deg(12), synth.deg(10), (0.0, 0.0, 0.0), 3 * L - 1.0, periodic=False)
    tiles = _tiles()
    tr = rrp.Tracer(b)
    recs = []
    for i, (p, g, o) in enumerate(tiles):
        tr.set_observer(o)
        rec = rrp.record_buffer(g)
        tr.tidal(g, torch.from_numpy(p).cuda(), rec)
        tr.step(g, rec, 3 * L - 1.0, 0.0, 1.0 + 0.1 * i, 0.8)
        recs.append(rec)
    k, kb = tr.finalize()
    rng = np.random.default_rng(81)
    yk, yb = rng.standard_normal(b.nrays), rng.standard_normal(b.nrays)
    lhs = float(k.cpu().numpy().ravel() @ yk + kb.cpu().numpy().ravel() @ yb)
    rhs = 0.0
    for i, (p, g, o) in enumerate(tiles):
        grad = rrp.grad_buffer(g)
        grad.zero_()
        rrp.rr_trace_step_adjoint(tr.ctx, i, torch.from_numpy(yk).cuda(), torch.from_numpy(yb).cuda(), grad)
        dphi = torch.zeros(g.n, dtype=torch.float32, device="cuda")
        rrp.rr_tidal_tensor_adjoint(rrp.grid_desc(g), grad, rrp.RR_AT_VERTICES, dphi, None)
        rhs += float(np.sum(p.astype(np.float64) * dphi.cpu().numpy()))
    tr.close()
    scale = float(np.abs(k.cpu().numpy().ravel()) @ np.abs(yk) + np.abs(kb.cpu().numpy().ravel()) @ np.abs(yb))
    assert abs(lhs - rhs) <= 1e-5 * scale, (lhs, rhs)


def test_generic_and_relocation_checks(rrp):
    from paper_1601_02012_gb300 import _rr
    b = synth.Bundle(8, 8, synth.deg(5), synth.deg(5), (4.0, 4.0, 0.0), 10.0)
    for kw in ({"fp64_dda": True}, {"plain_sums": True}, {"moments": True}, {"shear": True}, {"method_a": True}):
        with pytest.raises(rrp.RRError) as ei:
            rrp.Tracer(b, generic=True, **kw)
        assert ei.value.code == _rr.RR_ERR_ARG
    tr = rrp.Tracer(b)
    with pytest.raises(rrp.RRError) as ei:   # kernels only for generic contexts
        tr.set_kernels(((1, 0, 0), (1, 0, 0)))
    assert ei.value.code == _rr.RR_ERR_STATE
    g = synth.Grid((8, 8, 8), 16.0)
    rec = rrp.record_buffer(g)
    rec.zero_()
    tr.step(g, rec, 10.0, 5.0)
    with pytest.raises(rrp.RRError) as ei:   # a gap without relocation
        tr.step(g, rec, 9.0, 1.0)
    assert ei.value.code == _rr.RR_ERR_STATE
    tr.set_observer((4.0, 4.0, -16.0))
    tr.step(g, rec, 9.0, 1.0)                # allowed once after a relocation
    with pytest.raises(rrp.RRError) as ei:
        tr.step(g, rec, 0.9, 0.0)
    assert ei.value.code == _rr.RR_ERR_STATE
    with pytest.raises(rrp.RRError) as ei:
        tr.set_observer((float("nan"), 0.0, 0.0))
    assert ei.value.code == _rr.RR_ERR_ARG
    tr.close()
