"""The trace kernel's flat (no-wrap) record addressing.

rr_trace_step addresses the records of a step with 32-bit point indices and
constant per-axis strides when the step's footprint stays at least one cell
clear of the periodic seam (and the grid has fewer than 2^31 points); other
steps use the wrap-aware addressing. Both read the same records with the same
arithmetic, so the maps must be bit-identical to the persistent batch kernel's
(which always uses wrap-aware vertex indices), and within the map tolerance of
the FP64 oracle.
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


def _map_err(got, want):
    got = np.asarray(got, np.float64).ravel()
    want = np.asarray(want, np.float64).ravel()
    rms = math.sqrt(float(np.mean(want * want)))
    d = got - want
    return float(np.abs(d).max() / rms), float(np.linalg.norm(d) / np.linalg.norm(want))


def _case():
    # observer below the box: rays enter the periodic grid at z ~ 15 and stay
    # clear of every seam over both steps
    g = synth.Grid((64, 64, 64), 128.0)
    b = synth.Bundle(40, 36, synth.deg(12), synth.deg(10), (64.3, 63.7, -30.0), 150.0)
    steps = [synth.Step(150.0, 101.3, 1.2, 0.8), synth.Step(101.3, 45.0, 0.9, 0.95)]
    return g, b, steps


def _trace_single(rrp, g, b, rec, steps):
    tr = rrp.Tracer(b)
    for st in steps:
        tr.step(g, rec, st.chi_a, st.chi_b, st.scale, st.a)
    k, kb = tr.finalize()
    segs = tr.segments()
    tr.close()
    return k.cpu().numpy(), kb.cpu().numpy(), segs


def test_flat_steps_are_chosen(rrp):
    """Every step of the case qualifies for flat addressing (footprint box
    inside [1, n - 1) on each axis)."""
    g, b, steps = _case()
    tr = rrp.Tracer(b)
    for st in steps:
        box = tr.footprint(g, st.chi_a, st.chi_b)
        for a in range(3):
            assert 1 <= box[2 * a] and box[2 * a + 1] <= g.n[a] - 1, (st.chi_a, box)
    tr.close()


def test_flat_matches_batch_bitwise_and_oracle(rrp, oracle_lib):
    import torch
    g, b, steps = _case()
    phi = synth.grf_phi(64, 128.0, 31)
    ph = torch.from_numpy(phi).cuda()
    rec = rrp.record_buffer(g)
    rrp.rr_tidal_tensor(rrp.grid_desc(g), ph, None, rec, rrp.RR_AT_VERTICES)
    k1, kb1, segs1 = _trace_single(rrp, g, b, rec, steps)

    B = rrp.Batch([b])
    for st in steps:
        B.stage(0, g, rec, st.chi_a, st.chi_b, st.scale, st.a)
        B.upload()
        B.trace()
    k2 = torch.empty((b.ny, b.nx), dtype=torch.float64, device="cuda")
    kb2 = torch.empty_like(k2)
    B.finalize([k2], [kb2])
    code, segs2 = B.sync()
    B.close()
    assert code == 0
    assert np.array_equal(k1, k2.cpu().numpy())
    assert np.array_equal(kb1, kb2.cpu().numpy())
    assert segs1 == int(np.sum(segs2))

    H, d = oracle_lib.fields(g, phi.astype(np.float64))
    ora = oracle_lib.trace(b, g, H, d, steps)
    for got, want in ((k1, ora.kappa), (kb1, ora.kborn)):
        e_inf, e_2 = _map_err(got, want)
        assert e_inf <= TOL and e_2 <= TOL, (e_inf, e_2)
    assert abs(segs1 - int(ora.nseg.sum())) <= 1e-4 * ora.nseg.sum()


def _assert_maps(pairs):
    for got, want, what in pairs:
        e_inf, e_2 = _map_err(got, want)
        assert e_inf <= TOL and e_2 <= TOL, (what, e_inf, e_2)


def test_flat_shear_form_matches_oracle(rrp, oracle_lib):
    """The shear form (kappa, Born kappa, gamma1, gamma2 in one walk) on flat steps."""
    import torch
    g, b, steps = _case()
    phi = synth.grf_phi(64, 128.0, 37)
    k, kb, g1, g2, _ = rrp.trace_shear(torch.from_numpy(phi).cuda(), g, b, steps)
    torch.cuda.synchronize()
    H, d = oracle_lib.fields(g, phi.astype(np.float64))
    ora = oracle_lib.trace(b, g, H, d, steps)
    o1, o2 = oracle_lib.trace_shear(b, g, H, steps)
    _assert_maps([(k.cpu().numpy(), ora.kappa, "kappa"), (kb.cpu().numpy(), ora.kborn, "kborn"),
                  (g1.cpu().numpy(), o1, "gamma1"), (g2.cpu().numpy(), o2, "gamma2")])


def test_flat_method_a_matches_oracle(rrp, oracle_lib):
    """Method A (gradient records, the surface terms) on flat steps."""
    import torch
    g, b, steps = _case()
    phi = synth.grf_phi(64, 128.0, 38)
    k, kb, _ = rrp.trace_method_a(torch.from_numpy(phi).cuda(), g, b, steps)
    torch.cuda.synchronize()
    p64 = phi.astype(np.float64)
    _, d = oracle_lib.fields(g, p64)
    kg, kbo = oracle_lib.trace_method_a(b, g, oracle_lib.fields_grad(g, p64), d, steps)
    _assert_maps([(k.cpu().numpy(), kg + kbo, "kappa"), (kb.cpu().numpy(), kbo, "kborn")])


def test_flat_generic_form_matches_oracle(rrp, oracle_lib):
    """Two scalar channels with their own quadratic kernels on flat steps."""
    import torch
    g, b, steps = _case()
    q1 = synth.grf_phi(64, 128.0, 39) * 1e4
    q2 = synth.random_field(g.n, 40, np.float32)
    ker = ((0.7, -0.011, 0.00004), (-1.3, 0.02, -0.0001))
    tr = rrp.Tracer(b, generic=True)
    tr.set_kernels(ker)
    rec = tr.record_buffer(g)
    for st in steps:
        tr.scalars(g, torch.from_numpy(np.ascontiguousarray(q1, np.float32)).cuda(), rec, 0)
        tr.scalars(g, torch.from_numpy(np.ascontiguousarray(q2, np.float32)).cuda(), rec, 1)
        tr.step(g, rec, st.chi_a, st.chi_b, st.scale, st.a)
    o1, o2 = tr.finalize()
    torch.cuda.synchronize()
    tr.close()
    w1, w2 = oracle_lib.trace_kq(b, g, q1.astype(np.float32).astype(np.float64),
                                 q2.astype(np.float32).astype(np.float64), ker, steps)
    _assert_maps([(o1.cpu().numpy(), w1, "ch0"), (o2.cpu().numpy(), w2, "ch1")])


def test_flat_moments_form_matches_direct_traces(rrp, oracle_lib):
    """The source-redshift moments on flat steps: kappa for the context's own
    chi_s from the moments against the oracle's direct trace."""
    import torch
    g, b, steps = _case()
    phi = synth.grf_phi(64, 128.0, 41)
    ph = torch.from_numpy(phi).cuda()
    tr = rrp.Tracer(b, moments=True)
    rec = rrp.record_buffer(g)
    for st in steps:
        tr.tidal(g, ph, rec)
        tr.step(g, rec, st.chi_a, st.chi_b, st.scale, st.a)
    k, kb = tr.finalize()
    torch.cuda.synchronize()
    tr.close()
    H, d = oracle_lib.fields(g, phi.astype(np.float64))
    ora = oracle_lib.trace(b, g, H, d, steps)
    _assert_maps([(k.cpu().numpy(), ora.kappa, "kappa"), (kb.cpu().numpy(), ora.kborn, "kborn")])
