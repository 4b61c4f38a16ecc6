"""Batched lightcones: the persistent work-queue launch (rr_batch_trace), its
CUDA-graph replay and the autotuner, against per-bundle launches (the same
per-ray code, so bit-identical maps) and against the FP64 oracle."""
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


def _small_cones(n, seed, interp=1):
    cones = synth.batch_workload(n, seed=seed, sizes=(16, 24, 32), rays=(9, 70), fov_deg=(3.0, 30.0),
                                 chi_s=(20.0, 60.0))
    for c in cones:
        c.bundle.interp = interp
    return cones


def _fields(cones):
    import torch
    out = []
    for c in cones:
        out.append(torch.from_numpy(synth.grf_phi(c.grid.n[0], c.grid.box, c.field_seed)).cuda())
    return out


def _records(rrp, cones, phis, where, steps_of):
    recs = []
    for c, ph in zip(cones, phis):
        rec = rrp.record_buffer(c.grid)
        rrp.rr_tidal_tensor(rrp.grid_desc(c.grid), ph, None, rec, where)
        recs.append(rec)
    return recs


def _singles(rrp, cones, recs, steps_of, fp64=False):
    out = []
    for c, rec in zip(cones, recs):
        tr = rrp.Tracer(c.bundle, fp64_dda=fp64)
        for st in steps_of(c):
            tr.step(c.grid, rec, st.chi_a, st.chi_b, st.scale, st.a)
        k, kb = tr.finalize()
        out.append((k.cpu().numpy(), kb.cpu().numpy(), tr.segments()))
        tr.close()
    return out


def _two_steps(c):
    cs = c.bundle.chi_s
    return [synth.Step(cs, 0.45 * cs, 1.1, 0.8), synth.Step(0.45 * cs, 0.0, 0.95, 1.0)]


def _run_batch(rrp, cones, recs, steps_of, tuning=None, fp64=False):
    import torch
    B = rrp.Batch([c.bundle for c in cones], fp64_dda=fp64)
    if tuning:
        B.set_tuning(*tuning)
    nst = len(steps_of(cones[0]))
    for s in range(nst):
        for i, (c, rec) in enumerate(zip(cones, recs)):
            st = steps_of(c)[s]
            B.stage(i, c.grid, rec, st.chi_a, st.chi_b, st.scale, st.a)
        B.upload()
        B.trace()
    ks = [torch.empty((c.bundle.ny, c.bundle.nx), dtype=torch.float64, device="cuda") for c in cones]
    kbs = [torch.empty_like(k) for k in ks]
    B.finalize(ks, kbs)
    code, segs = B.sync()
    assert code == 0
    res = [(k.cpu().numpy(), kb.cpu().numpy()) for k, kb in zip(ks, kbs)]
    B.close()
    return res, segs


@pytest.mark.parametrize("interp", [1, 0])
@pytest.mark.parametrize("tuning", [None, (4, 2, 1, 1, 0), (32, 1, 4, 4, 1), (16, 4, 2, 2, 0)])
def test_batch_equals_single_launches(rrp, interp, tuning):
    cones = _small_cones(9, 11, interp)
    phis = _fields(cones)
    where = rrp.RR_AT_VERTICES if interp == 1 else rrp.RR_AT_CENTRES
    recs = _records(rrp, cones, phis, where, _two_steps)
    single = _singles(rrp, cones, recs, _two_steps)
    batch, segs = _run_batch(rrp, cones, recs, _two_steps, tuning)
    for (k1, kb1, _), (k2, kb2) in zip(single, batch):
        assert np.array_equal(k1, k2) and np.array_equal(kb1, kb2)
    assert segs == sum(s[2] for s in single)


def test_batch_plain_fp64_form(rrp):
    cones = _small_cones(5, 12)
    phis = _fields(cones)
    recs = _records(rrp, cones, phis, rrp.RR_AT_VERTICES, _two_steps)
    single = _singles(rrp, cones, recs, _two_steps, fp64=True)
    batch, _ = _run_batch(rrp, cones, recs, _two_steps, fp64=True)
    for (k1, kb1, _), (k2, kb2) in zip(single, batch):
        assert np.array_equal(k1, k2) and np.array_equal(kb1, kb2)


def test_batch_of_64_vs_oracle(rrp, oracle_lib):
    """64 small lightcones of uneven sizes in one launch, every map against the oracle."""
    cones = _small_cones(64, 13)
    phis = _fields(cones)
    recs = _records(rrp, cones, phis, rrp.RR_AT_VERTICES, _two_steps)
    batch, _ = _run_batch(rrp, cones, recs, _two_steps)
    for c, ph, (k, kb) in zip(cones, phis, batch):
        H, d = oracle_lib.fields(c.grid, ph.cpu().numpy().astype(np.float64))
        o = oracle_lib.trace(c.bundle, c.grid, H, d, _two_steps(c))
        for got, want in ((k.ravel(), o.kappa), (kb.ravel(), o.kborn)):
            rms = math.sqrt(float(np.mean(want ** 2)))
            assert np.abs(got - want).max() <= TOL * rms
            assert np.linalg.norm(got - want) <= TOL * np.linalg.norm(want)


def test_graph_replay_and_autotune(rrp):
    """[clear, tidal x n, upload, trace, finalize] captured once in a CUDA graph;
    replays reproduce the direct run, follow an in-place change of the
    potentials, and the autotuned shape gives the same maps."""
    import torch
    cones = _small_cones(12, 14)
    phis = _fields(cones)
    one = lambda c: [synth.Step(c.bundle.chi_s, 0.0, 1.0, 1.0)]
    recs = _records(rrp, cones, phis, rrp.RR_AT_VERTICES, one)
    ref, _ = _run_batch(rrp, cones, recs, one)

    B = rrp.Batch([c.bundle for c in cones])
    for i, (c, rec) in enumerate(zip(cones, recs)):
        B.stage(i, c.grid, rec, c.bundle.chi_s, 0.0)
    t, ms, cached = B.autotune(reps=2, use_cache=False)
    assert len(t) == 5 and ms > 0 and not cached
    ks = [torch.empty((c.bundle.ny, c.bundle.nx), dtype=torch.float64, device="cuda") for c in cones]
    kbs = [torch.empty_like(k) for k in ks]
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=stream):
        s = torch.cuda.current_stream()
        B.clear(s)
        for c, ph, rec in zip(cones, phis, recs):
            rrp.rr_tidal_tensor(rrp.grid_desc(c.grid), ph, None, rec, rrp.RR_AT_VERTICES, None, s)
        B.upload(s)
        B.trace(s)
        B.finalize(ks, kbs, s)
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        for (k0, kb0), k, kb in zip(ref, ks, kbs):
            assert np.array_equal(k0, k.cpu().numpy()) and np.array_equal(kb0, kb.cpu().numpy())
    for ph in phis:
        ph.mul_(-2.0)
    graph.replay()
    torch.cuda.synchronize()
    code, _ = B.sync()
    assert code == 0
    for (k0, kb0), k, kb in zip(ref, ks, kbs):
        assert np.allclose(k.cpu().numpy(), -2.0 * k0, rtol=1e-6, atol=1e-6 * np.abs(k0).max())
    B.close()
