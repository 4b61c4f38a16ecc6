"""rr_trace_steps (several consecutive steps per launch, the ray's sums held
in registers between them) against one rr_trace_step per step: the same maps
and segment counts bit for bit, with steps inside and outside the flat
addressing range, more steps than one launch takes, a record buffer per step
and shared ones, NGP, a form traced step by step, and the checks; and the
FP64 oracle on one case."""
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


def _trace(rrp, bundle, grid, steps, recs, fused, **kw):
    import torch
    tr = rrp.Tracer(bundle, **kw)
    if fused:
        tr.steps(grid, recs, steps)
    else:
        for st, r in zip(steps, recs):
            tr.step(grid, r, st.chi_a, st.chi_b, st.scale, st.a)
    k, kb = tr.finalize()
    per = torch.zeros(bundle.nrays, dtype=torch.int32, device="cuda")
    n = tr.segments(per_ray=per)
    torch.cuda.synchronize()
    out = (k.cpu().numpy(), kb.cpu().numpy(), n, per.cpu().numpy(), tr.ctx)
    nlog = rrp.rr_step_count(tr.ctx)
    tr.close()
    return out[:4] + (nlog,)


def _records(rrp, bundle, grid, phis):
    import torch
    tr = rrp.Tracer(bundle)
    out = []
    for ph in phis:
        rec = rrp.record_buffer(grid)
        tr.tidal(grid, torch.from_numpy(ph).cuda(), rec)
        out.append(rec)
    tr.close()
    return out


@pytest.mark.parametrize("interp", [1, 0])
def test_steps_match_single_launches(rrp, interp):
    """20 steps (two launches' worth) from the observer on the box face: the
    steps nearest it reach the periodic seam and take their own launches;
    records alternate between two fields."""
    g = synth.Grid((64, 64, 64), 128.0)
    b = synth.Bundle(80, 72, synth.deg(9), synth.deg(8), (64.0, 64.0, 0.0), 120.0, interp=interp)
    steps = synth.step_schedule(120.0, 20, rescale=True)
    phis = [synth.grf_phi(64, 128.0, 91), synth.grf_phi(64, 128.0, 92)]
    two = _records(rrp, b, g, phis)
    recs = [two[i % 2] for i in range(len(steps))]
    one = _trace(rrp, b, g, steps, recs, False)
    fused = _trace(rrp, b, g, steps, recs, True)
    for x, y in zip(one[:2], fused[:2]):
        assert np.array_equal(x, y)
    assert one[2] == fused[2] and np.array_equal(one[3], fused[3])
    assert one[4] == fused[4] == len(steps)


def test_steps_flat_only_and_per_step_buffers(rrp, oracle_lib):
    """An observer inside the box: every step is in the flat range, so the
    steps go to one launch; each step has a buffer of its own; the maps also
    against the FP64 oracle."""
    g = synth.Grid((64, 64, 64), 128.0)
    b = synth.Bundle(96, 64, synth.deg(6), synth.deg(5), (61.0, 67.0, 20.0), 80.0)
    steps = synth.step_schedule(80.0, 9, rescale=True)
    phi = synth.grf_phi(64, 128.0, 93)
    recs = _records(rrp, b, g, [phi] * len(steps))
    one = _trace(rrp, b, g, steps, recs, False)
    fused = _trace(rrp, b, g, steps, recs, True)
    assert np.array_equal(one[0], fused[0]) and np.array_equal(one[1], fused[1])
    assert one[2] == fused[2] and np.array_equal(one[3], fused[3])
    H, d = oracle_lib.fields(g, phi.astype(np.float32).astype(np.float64), None)
    o = oracle_lib.trace(b, g, H, d, steps)
    for got, want in ((fused[0].ravel(), o.kappa), (fused[1].ravel(), o.kborn)):
        rms = math.sqrt(float(np.mean(want ** 2)))
        assert np.abs(got - want).max() <= 1e-5 * rms
    assert int(o.nseg.sum()) == fused[2]


@pytest.mark.parametrize("form", ["shear", "moments", "method_a", "generic"])
def test_steps_other_forms_match_single_launches(rrp, form):
    """The shear, moments, Method A and generic forms through rr_trace_steps
    (their extra sums in registers too) against one rr_trace_step per step:
    every output bit for bit; shear and moments also on box-local records."""
    import torch
    g = synth.Grid((32, 32, 32), 64.0)
    b = synth.Bundle(40, 36, synth.deg(8), synth.deg(7), (31.0, 33.0, 5.0), 50.0)
    steps = synth.step_schedule(50.0, 7, rescale=True)
    phi = torch.from_numpy(synth.grf_phi(32, 64.0, 94)).cuda()
    prev = torch.from_numpy(synth.grf_phi(32, 64.0, 95)).cuda()
    kw = {form: True}

    def outputs(tr):
        k, kb = tr.finalize()
        out = [k.cpu().numpy(), kb.cpu().numpy(), tr.segments()]
        if form == "shear":
            g1, g2 = tr.shear()
            out += [g1.cpu().numpy(), g2.cpu().numpy()]
        if form == "moments":
            out.append(tr.moments().cpu().numpy())
        torch.cuda.synchronize()
        return out

    def records(tr):
        rec = tr.record_buffer(g)
        if form == "generic":
            tr.scalars(g, phi, rec, channel=0, field_prev=prev, inv_dt=0.5)
            tr.scalars(g, phi, rec, channel=1)
        else:
            tr.tidal(g, phi, rec)
        return rec

    res = []
    for fused in (False, True):
        tr = rrp.Tracer(b, **kw)
        rec = records(tr)
        if fused:
            tr.steps(g, [rec] * len(steps), steps)
        else:
            for st in steps:
                tr.step(g, rec, st.chi_a, st.chi_b, st.scale, st.a)
        res.append(outputs(tr))
        tr.close()
    if form in ("shear", "moments"):
        tr = rrp.Tracer(b, **kw)
        boxes = [tr.footprint(g, st.chi_a, st.chi_b, pad=1) for st in steps]
        recs = [tr.tidal_box(g, phi, rrp.box_record_buffer(bb), bb) for bb in boxes]
        tr.steps(g, recs, steps, boxes=boxes)
        res.append(outputs(tr))
        tr.close()
    else:
        tr = rrp.Tracer(b, **kw)
        bb = tr.footprint(g, steps[0].chi_a, steps[0].chi_b, pad=1)
        with pytest.raises(rrp.RRError):   # box-local records are tidal records only
            tr.steps(g, [rrp.box_record_buffer(bb)], steps[:1], boxes=[bb])
        tr.close()
    for other in res[1:]:
        for x, y in zip(res[0], other):
            if isinstance(x, np.ndarray):
                assert np.array_equal(x, y)
            else:
                assert x == y


def test_steps_checks_leave_the_log_unchanged(rrp):
    import torch
    g = synth.Grid((32, 32, 32), 64.0)
    b = synth.Bundle(16, 16, synth.deg(5), synth.deg(5), (31.0, 33.0, 5.0), 50.0)
    steps = synth.step_schedule(50.0, 4, rescale=True)
    recs = _records(rrp, b, g, [synth.grf_phi(32, 64.0, 95)]) * len(steps)
    tr = rrp.Tracer(b)
    gap = [steps[0], steps[2]]   # the second does not continue the first
    with pytest.raises(rrp.RRError) as ei:
        tr.steps(g, recs[:2], gap)
    assert "RR_ERR_STATE" in str(ei.value)
    assert rrp.rr_step_count(tr.ctx) == 0
    bad = rrp.record_buffer(g).view(-1)[4:]   # 16-byte aligned, not 32: tidal records need 32
    with pytest.raises(rrp.RRError):
        tr.steps(g, [recs[0], bad], steps[:2])
    assert rrp.rr_step_count(tr.ctx) == 0
    tr.steps(g, [], [])
    tr.steps(g, recs, steps)
    assert rrp.rr_step_count(tr.ctx) == len(steps)
    torch.cuda.synchronize()
    tr.close()


def test_box_records_equal_whole_grid_records(rrp):
    """rr_tidal_tensor_box: the records of a box across the periodic seam,
    box-local, equal the whole-grid records of the same points bit for bit."""
    import torch
    g = synth.Grid((40, 36, 48), 80.0)
    b = synth.Bundle(8, 8, synth.deg(5), synth.deg(5), (1.0, 1.0, 1.0), 10.0)
    phi = torch.from_numpy(synth.random_field(g.n, 96, np.float32)).cuda()
    tr = rrp.Tracer(b)
    whole = tr.tidal(g, phi, rrp.record_buffer(g))
    box = (-3, 9, 30, 41, 44, 53)   # wraps in x (below 0) and z (above 48)
    rec = tr.tidal_box(g, phi, rrp.box_record_buffer(box), box)
    torch.cuda.synchronize()
    tr.close()
    W = whole.cpu().numpy().reshape(40, 36, 48, 8)
    xs = [x % 40 for x in range(box[0], box[1])]
    ys = [y % 36 for y in range(box[2], box[3])]
    zs = [z % 48 for z in range(box[4], box[5])]
    want = W[np.ix_(xs, ys, zs)].reshape(-1, 8)
    assert np.array_equal(rec.cpu().numpy()[:, :7], want[:, :7])


@pytest.mark.parametrize("obs", [(64.0, 64.0, 0.0), (2.5, 125.0, 100.0)])
def test_steps_with_box_records_match_single_launches(rrp, obs):
    """Each step reading only its footprint box's records (box-local), the
    boxes crossing the periodic seam for the second observer: the maps of one
    rr_trace_step per step on whole-grid records, bit for bit."""
    import torch
    g = synth.Grid((64, 64, 64), 128.0)
    b = synth.Bundle(72, 64, synth.deg(9), synth.deg(8), obs, 120.0)
    steps = synth.step_schedule(120.0, 18, rescale=True)
    phi = torch.from_numpy(synth.grf_phi(64, 128.0, 97)).cuda()
    tr = rrp.Tracer(b)
    whole = tr.tidal(g, phi, rrp.record_buffer(g))
    boxes = [tr.footprint(g, st.chi_a, st.chi_b, pad=1) for st in steps]
    recs = [tr.tidal_box(g, phi, rrp.box_record_buffer(bb), bb) for bb in boxes]
    tr.close()
    one = _trace(rrp, b, g, steps, [whole] * len(steps), False)
    tr = rrp.Tracer(b)
    tr.steps(g, recs, steps, boxes=boxes)
    k, kb = tr.finalize()
    n = tr.segments()
    torch.cuda.synchronize()
    tr.close()
    assert np.array_equal(one[0], k.cpu().numpy()) and np.array_equal(one[1], kb.cpu().numpy())
    assert one[2] == n


def test_box_checks(rrp):
    import torch
    g = synth.Grid((32, 32, 32), 64.0)
    b = synth.Bundle(16, 16, synth.deg(5), synth.deg(5), (31.0, 33.0, 5.0), 50.0)
    steps = synth.step_schedule(50.0, 3, rescale=True)
    phi = torch.from_numpy(synth.grf_phi(32, 64.0, 98)).cuda()
    tr = rrp.Tracer(b)
    boxes = [tr.footprint(g, st.chi_a, st.chi_b, pad=1) for st in steps]
    recs = [tr.tidal_box(g, phi, rrp.box_record_buffer(bb), bb) for bb in boxes]
    nopad = [tr.footprint(g, st.chi_a, st.chi_b) for st in steps]
    with pytest.raises(rrp.RRError):
        tr.steps(g, recs, steps, boxes=nopad)   # the footprint itself, not widened
    small = list(boxes)
    small[1] = (boxes[1][0] + 1,) + tuple(boxes[1][1:])   # misses a plane of the footprint
    with pytest.raises(rrp.RRError):
        tr.steps(g, recs, steps, boxes=small)
    assert rrp.rr_step_count(tr.ctx) == 0
    tr.close()
    for kw in ({"method_a": True}, {"fp64_dda": True}, {"plain_sums": True}):
        t2 = rrp.Tracer(b, **kw)
        with pytest.raises(rrp.RRError):
            t2.steps(g, recs, steps, boxes=boxes)
        t2.close()
    torch.cuda.synchronize()


@pytest.mark.parametrize("interp", [1, 0])
@pytest.mark.parametrize("form", ["default", "shear", "method_a", "generic"])
def test_amr_steps_match_single_launches(rrp, interp, form):
    """rr_amr_trace_steps against one rr_amr_trace_step per step on a random
    mesh, in every form of the adaptive-mesh walk: the same maps (and shear
    maps) and segment counts bit for bit, 19 steps (two launches)."""
    import torch
    mesh = synth.amr_random(16, 64.0, 2, 7, threshold=1.5, child_sigma=0.8)
    pots = synth.amr_potential(mesh, synth.amr_density(mesh, 7, child_sigma=0.8))
    flat = np.concatenate([np.asarray(p, np.float64).reshape(-1) for p in pots]).astype(np.float32)
    gm = rrp.AmrMesh(16, 2, 64.0, mesh.octs, mesh.omega_m)
    where = rrp.RR_AT_VERTICES if interp == 1 else rrp.RR_AT_CENTRES
    phi = torch.from_numpy(flat).cuda()
    b = synth.Bundle(56, 48, synth.deg(9), synth.deg(7), (31.0, 33.0, 2.0), 60.0, interp=interp)
    steps = synth.step_schedule(60.0, 19, rescale=True)
    kw = {} if form == "default" else {form: True}

    def records():
        rec = gm.record_buffer(where)
        if form == "method_a":
            return gm.gradient(phi, rec, where)
        if form == "generic":
            return gm.scalars(phi, rec, where, prev0=phi * 0.5, inv_dt0=2.0, field1=phi)
        return gm.tidal(phi, rec, where)

    recs = [records() for _ in range(2)]
    per_step = [recs[i % 2] for i in range(len(steps))]
    out = []
    for fused in (False, True):
        tr = rrp.Tracer(b, **kw)
        if fused:
            tr.amr_steps(gm, per_step, steps)
        else:
            for st, r in zip(steps, per_step):
                tr.amr_step(gm, r, st.chi_a, st.chi_b, st.scale, st.a)
        k, kb = tr.finalize()
        maps = [k.cpu().numpy(), kb.cpu().numpy()]
        if form == "shear":
            maps += [x.cpu().numpy() for x in tr.shear()]
        n = tr.segments()
        torch.cuda.synchronize()
        out.append((maps, n, rrp.rr_step_count(tr.ctx)))
        tr.close()
    gm.close()
    one, fused = out
    assert np.isfinite(one[0][0]).all()
    for x, y in zip(one[0], fused[0]):
        assert np.array_equal(x, y)
    assert one[1] == fused[1] and one[2] == fused[2] == len(steps)
