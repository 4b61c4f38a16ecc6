"""pipeline_steps: a pass whose footprint records are computed on a side
stream while the previous step is traced (two record buffers) gives the maps
of the in-order pass bit for bit, on the uniform grid and on an adaptive
mesh, and both agree with the FP64 oracle."""
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


def _rel_max(got, want):
    want = np.asarray(want, np.float64)
    rms = math.sqrt(float(np.mean(want ** 2)))
    return float(np.abs(np.asarray(got, np.float64) - want).max() / rms)


def test_pipelined_uniform_pass_matches_in_order(rrp, oracle_lib):
    import torch
    g = synth.Grid((64, 64, 64), 128.0)
    b = synth.Bundle(96, 80, synth.deg(8), synth.deg(7), (64.0, 64.0, 0.0), 120.0)
    steps = synth.step_schedule(120.0, 6, rescale=True)
    phi = torch.from_numpy(synth.grf_phi(64, 128.0, 81)).cuda()
    gd = rrp.grid_desc(g)
    stream, side = torch.cuda.Stream(), torch.cuda.Stream()
    maps = []
    for nbuf in (1, 2):
        tr = rrp.Tracer(b)
        recs = [rrp.record_buffer(g) for _ in range(nbuf)]
        for r in recs:
            r.fill_(float("nan"))
        bbox = [tr.footprint(g, st.chi_a, st.chi_b) for st in steps]
        with torch.cuda.stream(stream):
            rrp.rr_reset(tr.ctx, stream)
            rrp.pipeline_steps(
                len(steps), lambda i, k, s: rrp.rr_tidal_tensor(gd, phi, None, recs[k], tr.where, bbox[i], s),
                lambda i, k, s: rrp.rr_trace_step(tr.ctx, gd, recs[k], steps[i].chi_a, steps[i].chi_b,
                                                  steps[i].scale, steps[i].a, s),
                stream, side if nbuf == 2 else None, nbuf)
            k, kb = tr.finalize(stream=stream)
        stream.synchronize()
        maps.append((k.cpu().numpy(), kb.cpu().numpy()))
        tr.close()
    assert np.array_equal(maps[0][0], maps[1][0]) and np.array_equal(maps[0][1], maps[1][1])
    H, d = oracle_lib.fields(g, phi.cpu().numpy().astype(np.float64), None)
    o = oracle_lib.trace(b, g, H, d, steps)
    assert _rel_max(maps[1][0].ravel(), o.kappa) <= 1e-5 and _rel_max(maps[1][1].ravel(), o.kborn) <= 1e-5


def test_pipelined_amr_pass_matches_in_order(rrp):
    import torch
    mesh = synth.amr_random(16, 64.0, 2, 5, threshold=1.5, child_sigma=0.8)
    pots = synth.amr_potential(mesh, synth.amr_density(mesh, 5, child_sigma=0.8))
    flat = np.concatenate([np.asarray(p, np.float64).reshape(-1) for p in pots]).astype(np.float32)
    assert sum(len(mesh.octs[l]) for l in range(1, 3)) > 0
    gm = rrp.AmrMesh(16, 2, 64.0, mesh.octs, mesh.omega_m)
    b = synth.Bundle(64, 48, synth.deg(9), synth.deg(7), (32.0, 32.0, 0.0), 60.0)
    steps = synth.step_schedule(60.0, 5, rescale=True)
    phi = torch.from_numpy(flat).cuda()
    stream, side = torch.cuda.Stream(), torch.cuda.Stream()
    maps = []
    for nbuf in (1, 2):
        tr = rrp.Tracer(b)
        recs = [gm.record_buffer(rrp.RR_AT_VERTICES) for _ in range(nbuf)]
        for r in recs:
            r.fill_(float("nan"))
        bbox = [gm.footprint(tr, st.chi_a, st.chi_b) for st in steps]
        with torch.cuda.stream(stream):
            rrp.rr_reset(tr.ctx, stream)
            rrp.pipeline_steps(
                len(steps), lambda i, k, s: gm.tidal(phi, recs[k], rrp.RR_AT_VERTICES, None, bbox[i], s),
                lambda i, k, s: tr.amr_step(gm, recs[k], steps[i].chi_a, steps[i].chi_b, steps[i].scale,
                                            steps[i].a, s),
                stream, side if nbuf == 2 else None, nbuf)
            k, kb = tr.finalize(stream=stream)
        stream.synchronize()
        maps.append((k.cpu().numpy(), kb.cpu().numpy()))
        tr.close()
    gm.close()
    assert np.isfinite(maps[1][0]).all()
    assert np.array_equal(maps[0][0], maps[1][0]) and np.array_equal(maps[0][1], maps[1][1])
