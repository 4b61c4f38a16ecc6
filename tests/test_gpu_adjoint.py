"""The hand-written adjoint (rr_trace_step_adjoint, rr_tidal_tensor_adjoint,
rr_trace_backward, TraceKappa) against the FP64 oracle's gradient, against
the GPU forward map (dot-product test), and against central finite
differences on the differentiation workload.

Tolerances: ||g_gpu - g_oracle||_2 / ||g_oracle||_2 <= 1e-5 and
max|g_gpu - g_oracle| <= 1e-4 rms(g_oracle); finite differences per cell within
1e-4 of rms(g). The adjoint sums with atomics, so its order of additions (not
its value beyond rounding) varies from run to run.
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rrp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_02012_gb300 import build
    build.build()
    import paper_1601_02012_gb300 as pkg
    return pkg


def _forward(rrp, phi_t, grid, bundle, steps, delta_t=None, tracer=None):
    tr = tracer or rrp.Tracer(bundle)
    rec = rrp.record_buffer(grid)
    for st in steps:
        tr.tidal(grid, phi_t, rec, delta=delta_t)
        tr.step(grid, rec, st.chi_a, st.chi_b, st.scale, st.a)
    k, kb = tr.finalize()
    return tr, k, kb


def _rel(got, want):
    got = np.asarray(got, np.float64).ravel()
    want = np.asarray(want, np.float64).ravel()
    rms = math.sqrt(float(np.mean(want ** 2)))
    return float(np.linalg.norm(got - want) / np.linalg.norm(want)), float(np.abs(got - want).max() / rms)


@pytest.mark.parametrize("interp", [1, 0])
def test_adjoint_matches_oracle_gradient(rrp, oracle_lib, interp):
    """Multi-step, wrapping, ragged bundle; loss gradient dL/dkappa, dL/dkborn random."""
    import torch
    g = synth.Grid((16, 16, 16), 32.0)
    b = synth.Bundle(21, 18, synth.deg(30), synth.deg(25), (3.0, 29.0, 0.0), 60.0, interp=interp)
    steps = [synth.Step(60.0, 41.0, 1.2, 0.7), synth.Step(41.0, 12.5, 0.8, 0.85), synth.Step(12.5, 0.0, 1.0, 1.0)]
    phi = synth.grf_phi(16, 32.0, 41)
    rng = np.random.default_rng(42)
    yk = rng.standard_normal(b.nrays)
    yb = rng.standard_normal(b.nrays)
    tr, k, kb = _forward(rrp, torch.from_numpy(phi).cuda(), g, b, steps)
    dphi = tr.backward(g, torch.from_numpy(yk).cuda(), torch.from_numpy(yb).cuda())
    torch.cuda.synchronize()
    tr.close()
    want, _ = oracle_lib.trace_adjoint(b, g, steps, yk, yb)
    l2, mx = _rel(dphi.cpu().numpy(), want)
    assert l2 <= 1e-5 and mx <= 1e-4, (l2, mx)


def test_adjoint_with_independent_delta(rrp, oracle_lib):
    """delta given as an input: the gradient splits into dL/dPhi and dL/ddelta."""
    import torch
    g = synth.Grid((16, 12, 20), 32.0)
    b = synth.Bundle(17, 13, synth.deg(20), synth.deg(15), (16.0, 12.0, 0.0), 38.0)
    steps = [synth.Step(38.0, 15.0, 1.1, 0.9), synth.Step(15.0, 0.0, 0.9, 1.0)]
    phi = synth.random_field(g.n, 43, np.float32)
    delta = synth.random_field(g.n, 44, np.float32)
    rng = np.random.default_rng(45)
    yk = rng.standard_normal(b.nrays)
    yb = rng.standard_normal(b.nrays)
    tr, k, kb = _forward(rrp, torch.from_numpy(phi).cuda(), g, b, steps, torch.from_numpy(delta).cuda())
    ddelta = torch.zeros(tuple(g.n), dtype=torch.float32, device="cuda")
    dphi = tr.backward(g, torch.from_numpy(yk).cuda(), torch.from_numpy(yb).cuda(), ddelta=ddelta)
    torch.cuda.synchronize()
    tr.close()
    gphi, gd = oracle_lib.trace_adjoint(b, g, steps, yk, yb, delta_derived=False)
    for got, want in ((dphi.cpu().numpy(), gphi), (ddelta.cpu().numpy(), gd)):
        l2, mx = _rel(got, want)
        assert l2 <= 1e-5 and mx <= 1e-4, (l2, mx)


@pytest.mark.parametrize("interp,indep_delta", [(1, False), (0, False), (1, True)])
def test_backward_over_footprint_only(rrp, oracle_lib, interp, indep_delta):
    """rr_trace_backward zeroes and transposes only the cells within the
    stencils' reach of the logged steps' footprints: with the scratch records
    filled with NaN it gives the whole-grid result (every step's adjoint into
    zeroed records, then the whole-grid transposed stencils) and the oracle's
    gradient, on a bundle whose footprint is a small part of the grid and
    crosses the periodic seam on two axes (x below 0, z above n)."""
    import torch
    g = synth.Grid((48, 40, 56), 96.0)
    b = synth.Bundle(24, 20, synth.deg(6), synth.deg(5), (3.0, 61.0, 100.0), 40.0, interp=interp)
    steps = [synth.Step(40.0, 22.0, 1.1, 0.8), synth.Step(22.0, 0.0, 0.9, 1.0)]
    phi = synth.random_field(g.n, 71, np.float32)
    delta = synth.random_field(g.n, 72, np.float32) if indep_delta else None
    rng = np.random.default_rng(73)
    yk = rng.standard_normal(b.nrays)
    yb = rng.standard_normal(b.nrays)
    dk, db = torch.from_numpy(yk).cuda(), torch.from_numpy(yb).cuda()
    tr, k, kb = _forward(rrp, torch.from_numpy(phi).cuda(), g, b, steps,
                         torch.from_numpy(delta).cuda() if indep_delta else None)
    n = tuple(g.n)
    scratch = rrp.grad_buffer(g)
    scratch.fill_(float("nan"))
    dd_a = torch.zeros(n, dtype=torch.float32, device="cuda") if indep_delta else None
    dphi_a = tr.backward(g, dk, db, grad_rec=scratch, ddelta=dd_a)
    whole = rrp.grad_buffer(g)
    whole.zero_()
    for i in range(len(steps)):
        rrp.rr_trace_step_adjoint(tr.ctx, i, dk, db, whole)
    dphi_b = torch.zeros(n, dtype=torch.float32, device="cuda")
    dd_b = torch.zeros(n, dtype=torch.float32, device="cuda") if indep_delta else None
    where = rrp.RR_AT_VERTICES if interp == 1 else rrp.RR_AT_CENTRES
    rrp.rr_tidal_tensor_adjoint(rrp.grid_desc(g), whole, where, dphi_b, dd_b)
    torch.cuda.synchronize()
    tr.close()
    got_a, got_b = dphi_a.cpu().numpy(), dphi_b.cpu().numpy()
    assert np.isfinite(got_a).all()
    support = got_b != 0
    assert 0 < support.mean() < 0.2, support.mean()   # a small part of the grid
    assert not got_a[~support].any()
    rms = math.sqrt(float(np.mean(got_b[support].astype(np.float64) ** 2)))
    assert np.abs(got_a - got_b).max() <= 1e-6 * rms   # the atomics' order only
    want, wd = oracle_lib.trace_adjoint(b, g, steps, yk, yb, delta_derived=not indep_delta)
    l2, mx = _rel(got_a, want)
    assert l2 <= 1e-5 and mx <= 1e-4, (l2, mx)
    if indep_delta:
        ga, gb_ = dd_a.cpu().numpy(), dd_b.cpu().numpy()
        assert np.isfinite(ga).all()
        rmsd = math.sqrt(float(np.mean(gb_[gb_ != 0].astype(np.float64) ** 2)))
        assert np.abs(ga - gb_).max() <= 1e-6 * rmsd
        l2, mx = _rel(ga, wd)
        assert l2 <= 1e-5 and mx <= 1e-4, (l2, mx)


def test_dot_product_gpu(rrp):
    """<J x, y> (GPU forward) = <x, J^T y> (GPU adjoint) for the whole chain."""
    import torch
    g = synth.Grid((32, 32, 32), 64.0)
    b = synth.Bundle(48, 40, synth.deg(12), synth.deg(10), (32.0, 32.0, 0.0), 90.0)
    steps = synth.step_schedule(90.0, 4)
    x = synth.grf_phi(32, 64.0, 46)
    rng = np.random.default_rng(47)
    yk = rng.standard_normal(b.nrays)
    yb = rng.standard_normal(b.nrays)
    tr, k, kb = _forward(rrp, torch.from_numpy(x).cuda(), g, b, steps)
    lhs = float(k.cpu().numpy().ravel() @ yk + kb.cpu().numpy().ravel() @ yb)
    dphi = tr.backward(g, torch.from_numpy(yk).cuda(), torch.from_numpy(yb).cuda())
    rhs = float(np.sum(x.astype(np.float64) * dphi.cpu().numpy()))
    tr.close()
    scale = float(np.abs(k.cpu().numpy().ravel()) @ np.abs(yk) + np.abs(kb.cpu().numpy().ravel()) @ np.abs(yb))
    assert abs(lhs - rhs) <= 1e-5 * scale, (lhs, rhs)


def test_autograd_function(rrp):
    """TraceKappa.apply inside torch.autograd gives the same dL/dPhi."""
    import torch
    g = synth.Grid((16, 16, 16), 32.0)
    b = synth.Bundle(16, 16, synth.deg(10), synth.deg(10), (16.0, 16.0, 0.0), 30.0)
    steps = [synth.Step(30.0, 0.0, 1.0, 1.0)]
    phi = torch.from_numpy(synth.grf_phi(16, 32.0, 48)).cuda().requires_grad_(True)
    target = torch.zeros((16, 16), dtype=torch.float64, device="cuda")
    k, kb = rrp.TraceKappa.apply(phi, g, b, steps)
    loss = ((k - target) ** 2).sum() + 0.5 * (kb ** 2).sum()
    loss.backward()
    tr, k2, kb2 = _forward(rrp, phi.detach(), g, b, steps)
    d2 = tr.backward(g, 2 * (k2 - target), kb2)
    tr.close()
    l2, mx = _rel(phi.grad.cpu().numpy(), d2.cpu().numpy())
    assert l2 <= 1e-6 and mx <= 1e-5


def test_differentiation_workload_fd(rrp):
    """The differentiation workload: 256^3 potential, 1024^2 rays over 5x5 deg
    to chi_s = 512, one step; L = ||kappa - kappa_target||^2 with the target
    traced from a second seed's field. dL/dPhi from rr_trace_backward against
    central finite differences on 1000 random cells. kappa is linear in Phi, so
    the central difference quotient of L along a unit cell e_m is exactly
    2 <kappa - kappa_target, kappa(e_m)>: each kappa(e_m) is one GPU forward
    pass of an impulse potential, with no cancellation."""
    import torch
    w = synth.workload("adjoint_256")
    g, b = w.grid, w.bundle
    steps = [synth.Step(b.chi_s, 0.0, 1.0, 1.0)]
    phi = torch.from_numpy(synth.grf_phi_cached(256, g.box, 5)).cuda()
    phit = torch.from_numpy(synth.grf_phi_cached(256, g.box, 6)).cuda()
    tr = rrp.Tracer(b)
    rec = rrp.record_buffer(g)

    def kappa(field, footprint=None):
        tr.reset()
        tr.tidal(g, field, rec, bbox=footprint)
        tr.step(g, rec, steps[0].chi_a, steps[0].chi_b)
        k, _ = tr.finalize()
        return k

    kt = kappa(phit).clone()
    k = kappa(phi).clone()
    r = 2.0 * (k - kt)
    dphi = torch.zeros_like(phi)
    tr.backward(g, r, None, dphi=dphi)
    gmat = dphi.cpu().numpy()
    rms = math.sqrt(float(np.mean(gmat.astype(np.float64) ** 2)))
    # finite differences on 1000 random cells inside the bundle's footprint
    bbox = tr.footprint(g, steps[0].chi_a, steps[0].chi_b)
    rng = np.random.default_rng(7)
    imp = torch.zeros_like(phi)
    rec.zero_()   # records of the zero potential; each impulse writes and then clears its own box
    torch.cuda.synchronize()
    worst = 0.0
    for _ in range(1000):
        cell = tuple(int(rng.integers(bbox[2 * a] + 2, bbox[2 * a + 1] - 2)) % g.n[a] for a in range(3))
        fp = (cell[0] - 3, cell[0] + 4, cell[1] - 3, cell[1] + 4, cell[2] - 3, cell[2] + 4)
        imp[cell] = 1.0
        ke = kappa(imp, footprint=fp)
        fd = float(torch.sum(r * ke))
        imp[cell] = 0.0
        tr.tidal(g, imp, rec, bbox=fp)
        worst = max(worst, abs(fd - float(gmat[cell])) / rms)
    tr.close()
    assert worst <= 1e-4, worst


def test_differentiation_workload_vs_oracle_gradient(rrp, oracle_lib):
    """The differentiation workload at full size (256^3 potential, 1024^2 rays
    over 5x5 deg to chi_s = 512, one step) against the FP64 oracle's gradient:
    dL/dkappa and dL/dkborn non-zero on 3000 sampled rays of the bundle (the
    oracle's adjoint skips the others), dL/dPhi on the whole grid from
    rr_trace_backward and from the oracle: l2 within the tolerance above, and
    the largest difference within 1e-4 of the gradient's rms over its support
    (the cells it reaches: a gradient confined to sampled rays' footprints is
    zero on most of the grid, where an rms over every cell would shrink the
    scale the max is measured against)."""
    import torch
    w = synth.workload("adjoint_256")
    g, b = w.grid, w.bundle
    steps = [synth.Step(b.chi_s, 0.0, 1.0, 1.0)]
    phi = torch.from_numpy(synth.grf_phi_cached(256, g.box, 5)).cuda()
    rng = np.random.default_rng(11)
    rids = rng.choice(b.nrays, 3000, replace=False)
    yk = np.zeros(b.nrays)
    yb = np.zeros(b.nrays)
    yk[rids] = rng.standard_normal(len(rids))
    yb[rids] = rng.standard_normal(len(rids))
    tr, k, kb = _forward(rrp, phi, g, b, steps)
    dphi = tr.backward(g, torch.from_numpy(yk.reshape(b.ny, b.nx)).cuda(),
                       torch.from_numpy(yb.reshape(b.ny, b.nx)).cuda())
    torch.cuda.synchronize()
    got = dphi.cpu().numpy()
    tr.close()
    want, _ = oracle_lib.trace_adjoint(b, g, steps, yk, yb)
    l2, _ = _rel(got, want)
    support = want != 0.0
    rms_support = math.sqrt(float(np.mean(want[support] ** 2)))
    mx = float(np.abs(got.astype(np.float64) - want).max()) / rms_support
    assert l2 <= 1e-5 and mx <= 1e-4, (l2, mx, float(support.mean()))
