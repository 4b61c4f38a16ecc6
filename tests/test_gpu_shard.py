"""Row bands of one bundle (rr_create_band) on one GPU: the bands' maps
concatenated in row order equal the whole bundle's maps bit for bit (same
directions, same per-ray code, same launches' tiles), and the sum of the
bands' dL/dPhi equals the whole bundle's (to the rounding of the FP32
gradient atomics), as the multi-GPU split in shard.py relies on."""
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


def _case(interp=1, obs=(24.0, 24.0, 0.0)):
    g = synth.Grid((24, 24, 24), 48.0)
    b = synth.Bundle(40, 37, synth.deg(14), synth.deg(12), obs, 47.0, interp=interp)
    steps = [synth.Step(47.0, 20.0, 1.2, 0.8), synth.Step(20.0, 0.0, 0.9, 1.0)]
    return g, b, steps


def _trace(rrp, g, b, rec, steps, rows=None):
    tr = rrp.Tracer(b, rows=rows)
    for st in steps:
        tr.step(g, rec, st.chi_a, st.chi_b, st.scale, st.a)
    k, kb = tr.finalize()
    return tr, k.cpu().numpy(), kb.cpu().numpy()


@pytest.mark.parametrize("interp", [1, 0])
@pytest.mark.parametrize("world", [2, 3, 5])
def test_bands_concatenate_to_the_whole_map_and_sum_to_its_gradient(rrp, interp, world):
    import torch
    from paper_1601_02012_gb300 import shard
    g, b, steps = _case(interp)
    ph = torch.from_numpy(synth.grf_phi(24, 48.0, 41)).cuda()
    rec = rrp.record_buffer(g)
    rrp.rr_tidal_tensor(rrp.grid_desc(g), ph, None, rec,
                        rrp.RR_AT_VERTICES if interp == 1 else rrp.RR_AT_CENTRES)
    whole, k, kb = _trace(rrp, g, b, rec, steps)
    rng = np.random.default_rng(8)
    dk = torch.from_numpy(rng.standard_normal((b.ny, b.nx))).cuda()
    gwhole = whole.backward(g, dk).cpu().numpy()
    segs = whole.segments()
    whole.close()

    parts_k, parts_kb, gsum, segsum = [], [], np.zeros_like(gwhole), 0
    for y0, y1 in shard.bands(b.ny, world):
        if y1 == y0:
            continue
        tr, kk, kkb = _trace(rrp, g, b, rec, steps, rows=(y0, y1))
        assert kk.shape == (y1 - y0, b.nx)
        parts_k.append(kk)
        parts_kb.append(kkb)
        segsum += tr.segments()
        gsum += tr.backward(g, dk[y0:y1].contiguous()).cpu().numpy()
        tr.close()
    assert np.array_equal(np.concatenate(parts_k), k)
    assert np.array_equal(np.concatenate(parts_kb), kb)
    assert segsum == segs
    assert np.linalg.norm(gsum - gwhole) <= 1e-5 * np.linalg.norm(gwhole)


def test_band_on_a_flat_step_matches_the_whole_bundle(rrp):
    """Steps clear of the periodic seam (flat record addressing): bands of the
    whole bundle still reproduce its rows."""
    import torch
    from paper_1601_02012_gb300 import shard
    g = synth.Grid((48, 48, 48), 96.0)
    b = synth.Bundle(48, 40, synth.deg(10), synth.deg(9), (48.2, 47.9, -20.0), 100.0)
    steps = [synth.Step(100.0, 60.0, 1.1, 0.9), synth.Step(60.0, 30.0, 1.0, 1.0)]
    ph = torch.from_numpy(synth.grf_phi(48, 96.0, 5)).cuda()
    rec = rrp.record_buffer(g)
    rrp.rr_tidal_tensor(rrp.grid_desc(g), ph, None, rec, rrp.RR_AT_VERTICES)
    whole, k, kb = _trace(rrp, g, b, rec, steps)
    whole.close()
    parts = []
    for y0, y1 in shard.bands(b.ny, 3):
        tr, kk, _ = _trace(rrp, g, b, rec, steps, rows=(y0, y1))
        tr.close()
        parts.append(kk)
    assert np.array_equal(np.concatenate(parts), k)


def test_sharded_autograd_on_one_rank_equals_trace_kappa(rrp):
    """ShardedTraceKappa with world = 1 is TraceKappa (no collective runs)."""
    import torch
    from paper_1601_02012_gb300 import shard
    g, b, steps = _case()
    phi = torch.from_numpy(synth.grf_phi(24, 48.0, 43)).cuda().requires_grad_(True)
    k1, kb1 = rrp.TraceKappa.apply(phi, g, b, steps)
    (k1.square().sum() + kb1.sum()).backward()
    g1 = phi.grad.clone()
    phi.grad = None
    k2, kb2 = shard.ShardedTraceKappa.apply(phi, g, b, steps, 0, 1)
    (k2.square().sum() + kb2.sum()).backward()
    assert torch.equal(k1, k2) and torch.equal(kb1, kb2)
    assert float((phi.grad - g1).norm()) <= 1e-5 * float(g1.norm())


def test_bands_with_multi_step_launches_on_box_records(rrp):
    """Bands traced by rr_trace_steps on box-local records (the footprints of
    the whole bundle, widened by a point) concatenate to the whole bundle's
    maps traced one rr_trace_step per step on whole-grid records."""
    import torch
    from paper_1601_02012_gb300 import shard
    g = synth.Grid((48, 48, 48), 96.0)
    b = synth.Bundle(48, 40, synth.deg(10), synth.deg(9), (46.0, 49.0, 3.0), 80.0)
    steps = synth.step_schedule(80.0, 7, rescale=True)
    ph = torch.from_numpy(synth.grf_phi(48, 96.0, 6)).cuda()
    rec = rrp.record_buffer(g)
    rrp.rr_tidal_tensor(rrp.grid_desc(g), ph, None, rec, rrp.RR_AT_VERTICES)
    whole, k, kb = _trace(rrp, g, b, rec, steps)
    whole.close()
    parts_k, parts_kb = [], []
    for y0, y1 in shard.bands(b.ny, 3):
        tr = rrp.Tracer(b, rows=(y0, y1))
        boxes = [tr.footprint(g, st.chi_a, st.chi_b, pad=1) for st in steps]
        recs = [tr.tidal_box(g, ph, rrp.box_record_buffer(bb), bb) for bb in boxes]
        tr.steps(g, recs, steps, boxes=boxes)
        kk, kkb = tr.finalize()
        torch.cuda.synchronize()
        parts_k.append(kk.cpu().numpy())
        parts_kb.append(kkb.cpu().numpy())
        tr.close()
    assert np.array_equal(np.concatenate(parts_k), k)
    assert np.array_equal(np.concatenate(parts_kb), kb)
