"""rr_upload_box and the streamed pass (Tracer.trace_streamed), on the device.

The copied cells must be exactly the documented ones (the box widened by 2
cells on each side, indices modulo n; nothing else written), and a boxed record
call made from those cells alone must give, bit for bit, the records it gives
from the whole field. The cells the upload leaves out hold NaN, so a read of
any of them for a point inside the box would show. A pass that streams each
step's footprint must give the maps and segment counts of the same pass on the
resident field, bit for bit (the same kernels read the same values).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

N = (32, 24, 40)
BOXES = [
    (5, 9, 3, 7, 10, 14),       # interior
    (-3, 2, 0, 5, 20, 24),      # x wraps below 0; y starts at 0 (its halo wraps)
    (28, 33, 20, 26, 1, 6),     # x and y wrap past n
    (0, 29, 2, 22, 0, 40),      # widened past n on every axis: whole axes
    (7, 8, 9, 10, 11, 12),      # one point
]


@pytest.fixture(scope="module")
def rrpkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_02012_gb300 import build
    build.build()
    import paper_1601_02012_gb300 as rrp
    return rrp


def widened_mask(n, bbox):
    axes = []
    for a in range(3):
        x0, x1 = bbox[2 * a], bbox[2 * a + 1]
        w = x1 - x0 + 4
        idx = np.arange(n[a])
        axes.append(np.ones(n[a], bool) if w >= n[a] else ((idx - (x0 - 2)) % n[a]) < w)
    return axes[0][:, None, None] & axes[1][None, :, None] & axes[2][None, None, :]


def _field(seed, n=N):
    return np.random.default_rng(seed).standard_normal(n).astype(np.float32) * np.float32(1e-5)


def _upload(rrp, grid, host_np, bbox):
    import torch
    host = torch.from_numpy(host_np).pin_memory()
    dev = torch.full(host_np.shape, float("nan"), dtype=torch.float32, device="cuda")
    nbytes = rrp.rr_upload_box(rrp.grid_desc(grid), host, dev, bbox)
    torch.cuda.synchronize()
    return dev, nbytes


@pytest.mark.parametrize("bbox", BOXES)
def test_upload_writes_exactly_the_widened_box(rrpkg, bbox):
    grid = synth.Grid(N, 64.0)
    phi = _field(1)
    dev, nbytes = _upload(rrpkg, grid, phi, bbox)
    got = dev.cpu().numpy()
    mask = widened_mask(N, bbox)
    assert nbytes == 4 * int(mask.sum())
    assert np.array_equal(got[mask], phi[mask])
    assert np.isnan(got[~mask]).all()


def test_upload_whole_field(rrpkg):
    grid = synth.Grid(N, 64.0)
    phi = _field(2)
    dev, nbytes = _upload(rrpkg, grid, phi, None)
    assert nbytes == phi.nbytes
    assert np.array_equal(dev.cpu().numpy(), phi)


@pytest.mark.parametrize("bbox", BOXES)
@pytest.mark.parametrize("kind", ["tidal_vertices", "tidal_centres", "tidal_delta", "gradient", "scalar_isw"])
def test_boxed_records_from_the_upload_alone(rrpkg, bbox, kind):
    import torch
    rrp = rrpkg
    grid = synth.Grid(N, 64.0)
    gd = rrp.grid_desc(grid)
    phi, prev, delta = _field(3), _field(4), _field(5) * np.float32(1e4)
    full = {k: torch.from_numpy(v).cuda() for k, v in (("phi", phi), ("prev", prev), ("delta", delta))}
    part = {k: _upload(rrp, grid, v, bbox)[0] for k, v in (("phi", phi), ("prev", prev), ("delta", delta))}
    npts = grid.ncells
    width = {"gradient": 4, "scalar_isw": 2}.get(kind, 8)
    recs = []
    for src in (full, part):
        rec = torch.full((npts, width), -7.0, dtype=torch.float32, device="cuda")
        where = rrp.RR_AT_CENTRES if kind == "tidal_centres" else rrp.RR_AT_VERTICES
        if kind.startswith("tidal"):
            d = src["delta"] if kind == "tidal_delta" else None
            rrp.rr_tidal_tensor(gd, src["phi"], d, rec, where, bbox)
        elif kind == "gradient":
            rrp.rr_gradient_records(gd, src["phi"], None, rec, where, bbox)
        else:
            rrp.rr_scalar_records(gd, src["phi"], src["prev"], 0.5, 0, rec, where, bbox)
            rrp.rr_scalar_records(gd, src["phi"], None, 1.0, 1, rec, where, bbox)
        torch.cuda.synchronize()
        recs.append(rec)
    assert not torch.isnan(recs[1]).any()
    assert torch.equal(recs[0], recs[1])


def _pass_case(interp):
    grid = synth.Grid((64, 64, 64), 128.0)
    bundle = synth.Bundle(48, 40, synth.deg(12.0), synth.deg(9.0), (61.3, 66.7, 0.4), 120.0, interp=interp)
    steps = synth.step_schedule(bundle.chi_s, 7)
    phi = synth.grf_phi(64, 128.0, seed=11).astype(np.float32)
    return grid, bundle, steps, phi


@pytest.mark.parametrize("interp", [1, 0])
@pytest.mark.parametrize("method_a", [False, True])
def test_streamed_pass_equals_resident_pass(rrpkg, interp, method_a):
    import torch
    rrp = rrpkg
    grid, bundle, steps, phi = _pass_case(interp)
    resident = rrp.trace_method_a if method_a else rrp.trace_kappa
    k1, kb1, s1 = resident(torch.from_numpy(phi).cuda(), grid, bundle, steps)
    torch.cuda.synchronize()

    tr = rrp.Tracer(bundle, method_a=method_a)
    try:
        stream, copy_stream = torch.cuda.Stream(), torch.cuda.Stream()
        host = torch.from_numpy(phi).pin_memory()
        bufs = [torch.full(phi.shape, float("nan"), dtype=torch.float32, device="cuda") for _ in range(2)]
        rec = tr.record_buffer(grid)
        bboxes = [tr.footprint(grid, st.chi_a, st.chi_b) for st in steps]
        tr.reset(stream)
        nbytes = tr.trace_streamed(grid, host, steps, rec, bufs, stream, copy_stream, bboxes)
        k2, kb2 = tr.finalize(stream=stream)
        s2 = tr.segments(stream=stream)
        torch.cuda.synchronize()
    finally:
        tr.close()
    assert nbytes == sum(4 * int(widened_mask(grid.n, b).sum()) for b in bboxes)
    assert nbytes < len(steps) * phi.nbytes
    assert s1 == s2
    assert torch.equal(k1, k2) and torch.equal(kb1, kb2)


def test_streamed_pass_with_delta(rrpkg):
    """A given density contrast streams beside the potential."""
    import torch
    rrp = rrpkg
    grid, bundle, steps, phi = _pass_case(1)
    delta = _field(7, grid.n) * np.float32(1e5)
    k1, kb1, _ = rrp.trace_kappa(torch.from_numpy(phi).cuda(), grid, bundle, steps,
                                 delta=torch.from_numpy(delta).cuda())
    tr = rrp.Tracer(bundle)
    try:
        stream, copy_stream = torch.cuda.Stream(), torch.cuda.Stream()
        nan = lambda: torch.full(phi.shape, float("nan"), dtype=torch.float32, device="cuda")  # noqa: E731
        rec = tr.record_buffer(grid)
        tr.reset(stream)
        tr.trace_streamed(grid, torch.from_numpy(phi).pin_memory(), steps, rec, [nan(), nan()], stream,
                          copy_stream, delta_host=torch.from_numpy(delta).pin_memory(), delta_bufs=[nan(), nan()])
        k2, kb2 = tr.finalize(stream=stream)
        torch.cuda.synchronize()
    finally:
        tr.close()
    assert torch.equal(k1, k2) and torch.equal(kb1, kb2)


def test_back_to_back_streamed_passes_share_buffers(rrpkg):
    """Two passes of two fields through the same two device buffers, queued
    without a host synchronisation between them: the second pass's first
    copies wait for the first pass's steps, so each map is its field's."""
    import torch
    rrp = rrpkg
    grid, bundle, steps, phi_a = _pass_case(1)
    phi_b = (synth.grf_phi(64, 128.0, seed=12) * 0.5).astype(np.float32)
    ref = [rrp.trace_kappa(torch.from_numpy(p).cuda(), grid, bundle, steps)[:2] for p in (phi_a, phi_b)]
    trs = [rrp.Tracer(bundle), rrp.Tracer(bundle)]
    try:
        stream, copy_stream = torch.cuda.Stream(), torch.cuda.Stream()
        bufs = [torch.full(phi_a.shape, float("nan"), dtype=torch.float32, device="cuda") for _ in range(2)]
        rec = trs[0].record_buffer(grid)
        hosts = [torch.from_numpy(p).pin_memory() for p in (phi_a, phi_b)]
        for tr, host in zip(trs, hosts):
            tr.reset(stream)
            tr.trace_streamed(grid, host, steps, rec, bufs, stream, copy_stream)
        maps = [tr.finalize(stream=stream) for tr in trs]
        torch.cuda.synchronize()
    finally:
        for tr in trs:
            tr.close()
    for (k1, kb1), (k2, kb2) in zip(ref, maps):
        assert torch.equal(k1, k2) and torch.equal(kb1, kb2)


@pytest.mark.parametrize("with_side", [False, True])
def test_streamed_grouped_pass_equals_resident_pass(rrpkg, with_side):
    """Box-local records from the streamed buffers, 4 steps per rr_trace_steps
    launch, the records on a high-priority side stream or in order; two
    passes queued back to back through the same buffers: each equals the
    resident pass bit for bit."""
    import torch
    rrp = rrpkg
    grid, bundle, steps, phi = _pass_case(1)
    k1, kb1, s1 = rrp.trace_kappa(torch.from_numpy(phi).cuda(), grid, bundle, steps, group=1)
    tr = rrp.Tracer(bundle)
    try:
        stream, copy_stream = torch.cuda.Stream(), torch.cuda.Stream()
        side = torch.cuda.Stream(priority=-1) if with_side else None
        host = torch.from_numpy(phi).pin_memory()
        bufs = [torch.full(phi.shape, float("nan"), dtype=torch.float32, device="cuda") for _ in range(2)]
        pboxes = [tr.footprint(grid, st.chi_a, st.chi_b, pad=1) for st in steps]
        brecs = [rrp.box_record_buffer(b) for b in pboxes]
        out = []
        for _ in range(2):
            tr.reset(stream)
            tr.trace_streamed(grid, host, steps, None, bufs, stream, copy_stream, pboxes, group=4, box_recs=brecs,
                              rec_stream=side)
            k2, kb2 = tr.finalize(stream=stream)
            out.append((k2.clone(), kb2.clone(), tr.segments(stream=stream)))
        torch.cuda.synchronize()
    finally:
        tr.close()
    for k2, kb2, s2 in out:
        assert s1 == s2
        assert torch.equal(k1, k2) and torch.equal(kb1, kb2)
