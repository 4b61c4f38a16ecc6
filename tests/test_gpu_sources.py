"""Source-redshift moments (RR_SOURCE_MOMENTS; Eqs. Isources, Isources1)
against the oracle: one pass with moment snapshots at the step boundaries
gives kappa and Born kappa for every source distance chi_k <= chi_s, each
within the map tolerance of the oracle's direct trace of a bundle with
chi_s = chi_k (same rays)."""
import dataclasses
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
    rms = math.sqrt(float(np.mean(want ** 2)))
    return float(np.abs(got - want).max() / rms), float(np.linalg.norm(got - want) / np.linalg.norm(want))


@pytest.mark.parametrize("interp", [1, 0])
def test_kappa_for_every_step_boundary_from_one_pass(rrp, oracle_lib, interp):
    import torch
    g = synth.Grid((48, 48, 48), 96.0)
    b = synth.Bundle(33, 27, synth.deg(12), synth.deg(10), (48.0, 47.0, 0.0), 150.0, interp=interp)
    phi = synth.grf_phi(48, 96.0, 31)
    edges = [150.0, 121.0, 95.5, 70.0, 44.0, 19.0, 0.0]
    steps = [synth.Step(edges[i], edges[i + 1], 1.0 + 0.05 * i, 0.6 + 0.06 * i) for i in range(len(edges) - 1)]
    ph = torch.from_numpy(phi).cuda()
    where = rrp.RR_AT_VERTICES if interp == 1 else rrp.RR_AT_CENTRES
    rec = rrp.record_buffer(g)
    rrp.rr_tidal_tensor(rrp.grid_desc(g), ph, None, rec, where)
    tr = rrp.Tracer(b, moments=True)
    snaps = [None]   # the moments above each step boundary (none above chi_s)
    for st in steps:
        tr.step(g, rec, st.chi_a, st.chi_b, st.scale, st.a)
        snaps.append(tr.moments().clone())
    k_full, kb_full = tr.finalize()
    m_end = snaps[-1]
    H, d = oracle_lib.fields(g, phi.astype(np.float64))
    for i, chi_k in enumerate(edges[:-1]):
        k, kb = rrp.source_kappa(m_end, snaps[i], chi_k)
        bk = dataclasses.replace(b, chi_s=chi_k)
        o = oracle_lib.trace(bk, g, H, d, steps[i:])
        for got, want, what in ((k, o.kappa, "kappa"), (kb, o.kborn, "kborn")):
            e_inf, e_2 = _err(got.cpu().numpy(), want)
            assert e_inf <= TOL and e_2 <= TOL, (chi_k, what, e_inf, e_2)
    # rr_finalize of a moments context: kappa for the bundle's own chi_s
    o = oracle_lib.trace(b, g, H, d, steps)
    assert _err(k_full.cpu().numpy(), o.kappa)[0] <= TOL
    assert _err(kb_full.cpu().numpy(), o.kborn)[0] <= TOL
    tr.close()


def test_moments_form_checks(rrp):
    import torch
    from paper_1601_02012_gb300 import _rr
    b = synth.Bundle(8, 8, synth.deg(5), synth.deg(5), (4.0, 4.0, 0.0), 10.0)
    g = synth.Grid((8, 8, 8), 16.0)
    tr = rrp.Tracer(b)   # not a moments context
    with pytest.raises(rrp.RRError) as ei:
        tr.moments()
    assert ei.value.code == _rr.RR_ERR_STATE
    tr.close()
    for kw in ({"fp64_dda": True}, {"plain_sums": True}):
        with pytest.raises(rrp.RRError) as ei:
            rrp.Tracer(b, moments=True, **kw)
        assert ei.value.code == _rr.RR_ERR_ARG
    tr = rrp.Tracer(b, moments=True)
    rec = rrp.record_buffer(g)
    rrp.rr_tidal_tensor(rrp.grid_desc(g), torch.zeros(8, 8, 8, device="cuda"), None, rec, rrp.RR_AT_VERTICES)
    tr.step(g, rec, 10.0, 0.0)
    tr.finalize()
    with pytest.raises(rrp.RRError) as ei:   # the adjoint is defined for kappa only
        rrp.rr_trace_step_adjoint(tr.ctx, 0, torch.ones(64, dtype=torch.float64, device="cuda"), None,
                                  rrp.grad_buffer(g))
    assert ei.value.code == _rr.RR_ERR_STATE
    tr.close()
