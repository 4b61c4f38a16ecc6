"""CUDA path against the FP64 oracle, through the C ABI, element by element.

Tolerances (map metric, on kappa and on the Born kappa):
    max|k_gpu - k_ora| / rms(k_ora) <= 1e-5  and  ||k_gpu - k_ora||_2 / ||k_ora||_2 <= 1e-5.
Records of the tidal kernel: per channel max|diff| <= 4e-6 max|oracle| (FP32 stencils).
Segment totals: within 1e-4 of the oracle's count (rounding slivers at edge
crossings may be counted on one side and not the other).
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def rrpkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_02012_gb300 import build
    build.build()
    import paper_1601_02012_gb300 as rrp
    return rrp


def map_errors(gpu, ora):
    gpu = np.asarray(gpu, np.float64).ravel()
    ora = np.asarray(ora, np.float64).ravel()
    d = gpu - ora
    rms = math.sqrt(float(np.mean(ora * ora)))
    return float(np.abs(d).max() / rms), float(np.linalg.norm(d) / np.linalg.norm(ora))


def assert_map(gpu, ora, tol=TOL, what="kappa"):
    e_inf, e_2 = map_errors(gpu, ora)
    assert e_inf <= tol and e_2 <= tol, f"{what}: max/rms {e_inf:.3e}, l2 {e_2:.3e}"


def run_gpu(rrp, phi, grid, bundle, steps, fp64_dda=False, footprint=True, delta=None):
    import torch
    ph = torch.from_numpy(np.ascontiguousarray(phi, np.float32)).cuda()
    dl = None if delta is None else torch.from_numpy(np.ascontiguousarray(delta, np.float32)).cuda()
    k, kb, nseg = rrp.trace_kappa(ph, grid, bundle, steps, delta=dl, fp64_dda=fp64_dda, footprint=footprint)
    torch.cuda.synchronize()
    return k.cpu().numpy().ravel(), kb.cpu().numpy().ravel(), nseg


def run_oracle(oracle_lib, phi, grid, bundle, steps, delta=None, rids=None):
    phi64 = np.asarray(phi, np.float32).astype(np.float64)
    d64 = None if delta is None else np.asarray(delta, np.float32).astype(np.float64)
    H, d = oracle_lib.fields(grid, phi64, d64)
    return oracle_lib.trace(bundle, grid, H, d, steps, rids=rids)


# ---------------------------------------------------------------------------
# rr_tidal_tensor
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("where", ["vertices", "centres"])
@pytest.mark.parametrize("with_delta", [False, True])
@pytest.mark.parametrize("shape", [(24, 20, 40), (2, 3, 5), (5, 2, 33), (40, 52, 96)])
def test_tidal_records(rrpkg, oracle_lib, where, with_delta, shape):
    """Every record of the grid against the oracle's stencils and vertex means;
    also grids smaller than a CTA's 8 x 32 block (indices wrap several times),
    and one whose inner blocks take their potential planes by tensor copies
    (rows a multiple of 16 bytes, tiles clear of the periodic seam)."""
    import torch
    g = synth.Grid(shape, 2.0 * shape[0])
    phi = synth.random_field(g.n, 7, np.float32)
    delta = synth.random_field(g.n, 8, np.float32) if with_delta else None
    H, d = oracle_lib.fields(g, phi.astype(np.float64), None if delta is None else delta.astype(np.float64))
    if where == "vertices":
        want = oracle_lib.vertex_field(g, H, d)
        flag = rrpkg.RR_AT_VERTICES
    else:
        want = np.concatenate([H, d[..., None]], axis=-1)
        flag = rrpkg.RR_AT_CENTRES
    rec = rrpkg.record_buffer(g)
    ph = torch.from_numpy(phi).cuda()
    dl = None if delta is None else torch.from_numpy(delta).cuda()
    rrpkg.rr_tidal_tensor(rrpkg.grid_desc(g), ph, dl, rec, flag)
    got = rec.cpu().numpy().reshape(tuple(g.n) + (8,))
    assert np.all(got[..., 7] == 0)
    for c in range(7):
        scale = np.abs(want[..., c]).max()
        err = np.abs(got[..., c] - want[..., c]).max()
        assert err <= 4e-6 * scale, (c, err / scale)


def test_tidal_bbox_on_tensor_copy_blocks(rrpkg):
    """Boxes away from the seam (all blocks take tensor copies) and across it:
    the records in the box equal the whole grid's, bit for bit."""
    import torch
    g = synth.Grid((64, 64, 128), 128.0)
    phi = torch.from_numpy(synth.random_field(g.n, 19, np.float32)).cuda()
    full = rrpkg.record_buffer(g)
    rrpkg.rr_tidal_tensor(rrpkg.grid_desc(g), phi, None, full, rrpkg.RR_AT_VERTICES)
    f = full.cpu().numpy().reshape(64, 64, 128, 8)
    for bbox in ((10, 30, 7, 45, 17, 99), (-5, 9, 50, 70, 100, 140)):
        part = torch.full_like(full, float("nan"))
        rrpkg.rr_tidal_tensor(rrpkg.grid_desc(g), phi, None, part, rrpkg.RR_AT_VERTICES, bbox)
        p = part.cpu().numpy().reshape(64, 64, 128, 8)
        mask = np.zeros((64, 64, 128), bool)
        mask[np.ix_(np.arange(bbox[0], bbox[1]) % 64, np.arange(bbox[2], bbox[3]) % 64,
                    np.arange(bbox[4], bbox[5]) % 128)] = True
        assert np.array_equal(p[mask], f[mask])
        assert np.all(np.isnan(p[~mask]))


def test_tidal_bbox_writes_only_the_box(rrpkg):
    import torch
    g = synth.Grid((16, 16, 16), 32.0)
    phi = torch.from_numpy(synth.grf_phi(16, 32.0, 9)).cuda()
    full = rrpkg.record_buffer(g)
    rrpkg.rr_tidal_tensor(rrpkg.grid_desc(g), phi, None, full, rrpkg.RR_AT_VERTICES)
    part = torch.full_like(full, float("nan"))
    bbox = (-3, 5, 10, 16, 2, 15)   # x wraps through the seam
    rrpkg.rr_tidal_tensor(rrpkg.grid_desc(g), phi, None, part, rrpkg.RR_AT_VERTICES, bbox)
    f = full.cpu().numpy().reshape(16, 16, 16, 8)
    p = part.cpu().numpy().reshape(16, 16, 16, 8)
    mask = np.zeros((16, 16, 16), bool)
    xs = np.arange(-3, 5) % 16
    mask[np.ix_(xs, np.arange(10, 16), np.arange(2, 15))] = True
    assert np.array_equal(p[mask], f[mask])
    assert np.all(np.isnan(p[~mask]))


# ---------------------------------------------------------------------------
# rr_trace_step / rr_finalize
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("interp", [1, 0])
@pytest.mark.parametrize("fp64_dda", [False, True])
def test_small_64_workload(rrpkg, oracle_lib, interp, fp64_dda):
    """64^3 GRF, box 256, 128x128 rays over 2x2 deg, chi_s = 256, one step."""
    w = synth.workload("small_64")
    w.bundle.interp = interp
    phi = synth.grf_phi(64, w.grid.box, w.seed)
    steps = [synth.Step(w.bundle.chi_s, 0.0, 1.0, 1.0)]
    k, kb, nseg = run_gpu(rrpkg, phi, w.grid, w.bundle, steps, fp64_dda=fp64_dda)
    o = run_oracle(oracle_lib, phi, w.grid, w.bundle, steps)
    assert_map(k, o.kappa)
    assert_map(kb, o.kborn, what="kborn")
    assert abs(nseg - int(o.nseg.sum())) <= 1e-4 * o.nseg.sum()
    # the map statistics: P(ell) bins and the one-point PDF
    from paper_1601_02012_gb300 import mapstats
    shape = (w.bundle.ny, w.bundle.nx)
    for got, want in ((k, o.kappa), (kb, o.kborn)):
        st = mapstats.compare(got.reshape(shape), want.reshape(shape), w.bundle.fov_x, w.bundle.fov_y)
        assert st["pl_max_rel"] <= 1e-4 and st["pdf_l1"] <= 1e-3, st


@pytest.mark.parametrize("interp", [1, 0])
def test_multistep_ragged_wrapping(rrpkg, oracle_lib, interp):
    """Ray counts that are not multiples of the 16 x 8 block tile, an observer
    near a corner so rays wrap through the periodic seams, a wide field, and
    five steps with different field scales and scale factors."""
    g = synth.Grid((32, 32, 32), 64.0)
    b = synth.Bundle(37, 13, synth.deg(40), synth.deg(25), (2.0, 61.0, 0.0), 150.0, interp=interp)
    phi = synth.grf_phi(32, 64.0, 11)
    edges = [150.0, 121.0, 90.5, 60.0, 17.25, 0.0]
    steps = [synth.Step(edges[i], edges[i + 1], 0.5 + 0.3 * i, 0.6 + 0.08 * i) for i in range(5)]
    k, kb, nseg = run_gpu(rrpkg, phi, g, b, steps)
    o = run_oracle(oracle_lib, phi, g, b, steps)
    assert_map(k, o.kappa)
    assert_map(kb, o.kborn, what="kborn")
    assert abs(nseg - int(o.nseg.sum())) <= 1e-4 * o.nseg.sum()


def test_footprint_equals_full_grid(rrpkg):
    """Restricting the records to each step's footprint changes nothing."""
    g = synth.Grid((32, 32, 32), 64.0)
    b = synth.Bundle(24, 24, synth.deg(12), synth.deg(12), (32.0, 32.0, 0.0), 120.0)
    phi = synth.grf_phi(32, 64.0, 12)
    steps = [synth.Step(120.0 - 20.0 * i, 100.0 - 20.0 * i if i < 5 else 0.0, 1.0 + 0.1 * i, 1.0) for i in range(6)]
    k1, kb1, n1 = run_gpu(rrpkg, phi, g, b, steps, footprint=True)
    k2, kb2, n2 = run_gpu(rrpkg, phi, g, b, steps, footprint=False)
    assert np.array_equal(k1, k2) and np.array_equal(kb1, kb2) and n1 == n2


def test_nonperiodic_gaussian_potential(rrpkg, oracle_lib):
    """The Sec. 4 setup: Gaussian potential in a 10 Mpc/h box, 40 x 40 deg,
    rays stop at the box faces (many enter through the sides)."""
    g = synth.Grid((64, 64, 64), 10.0)
    chis = synth.chi_of_z(0.95)
    b = synth.Bundle(48, 48, synth.deg(40), synth.deg(40), (5.0, 5.0, 0.0), chis, periodic=False)
    phi = synth.gaussian_phi(64, 10.0, 1e4, 2.0, dtype=np.float32)
    steps = [synth.Step(chis, 0.0, 1.0, 1.0)]
    k, kb, nseg = run_gpu(rrpkg, phi, g, b, steps)
    o = run_oracle(oracle_lib, phi, g, b, steps)
    assert_map(k, o.kappa)
    assert_map(kb, o.kborn, what="kborn")


@pytest.mark.parametrize("interp", [1, 0])
def test_degenerate_bundles(rrpkg, oracle_lib, interp):
    """A single ray (theta = 0 exactly: it never crosses an x or y face), a
    single row, and rays through cell edges (observer on a vertex)."""
    g = synth.Grid((16, 16, 16), 32.0)
    phi = synth.grf_phi(16, 32.0, 13)
    steps = [synth.Step(31.0, 3.0, 1.0, 1.0)]
    for b in (synth.Bundle(1, 1, 0.0, 0.0, (16.0, 16.0, 0.0), 40.0, interp=interp),
              synth.Bundle(5, 1, synth.deg(30), 0.0, (16.0, 16.0, 0.0), 40.0, interp=interp),
              synth.Bundle(3, 3, synth.deg(90), synth.deg(90), (16.0, 16.0, 0.0), 40.0, interp=interp)):
        k, kb, nseg = run_gpu(rrpkg, phi, g, b, steps)
        o = run_oracle(oracle_lib, phi, g, b, steps)
        assert_map(k, o.kappa)
        assert_map(kb, o.kborn, what="kborn")


def test_step_order_and_interval_checks(rrpkg):
    import torch
    g = synth.Grid((8, 8, 8), 16.0)
    b = synth.Bundle(4, 4, 0.1, 0.1, (8.0, 8.0, 0.0), 15.0)
    tr = rrpkg.Tracer(b)
    rec = rrpkg.record_buffer(g)
    rec.zero_()
    tr.step(g, rec, 15.0, 10.0)
    with pytest.raises(rrpkg.RRError) as e:
        tr.step(g, rec, 9.0, 5.0)       # gap after the previous step
    assert e.value.code == -5
    with pytest.raises(rrpkg.RRError):
        tr.step(g, rec, 10.0, 10.0)     # empty interval
    tr.reset()
    with pytest.raises(rrpkg.RRError):
        tr.step(g, rec, 16.0, 1.0)      # beyond the sources
    tr.step(g, rec, 12.0, 0.0)
    k, kb = tr.finalize()
    torch.cuda.synchronize()
    assert float(k.abs().max()) == 0.0
    tr.close()


# ---------------------------------------------------------------------------
# production size: 512^3, 2048^2 rays, 40 steps, sampled rays vs the oracle
# ---------------------------------------------------------------------------

def test_prod_512_sampled(rrpkg, oracle_lib):
    """The full production workload in the benchmark's launch configuration
    (footprint records per step, the FP32 walk); 512 sampled rays are traced by
    the oracle one by one. Segment counts: the sampled rays' per-ray counters
    against the oracle's counts of the same rays, within 1e-4 in total (a
    rounding sliver at an edge crossing may be counted on one side only)."""
    import torch
    w = synth.workload("prod_512")
    phi = synth.grf_phi_cached(512, w.grid.box, w.seed)
    steps = synth.step_schedule(w.bundle.chi_s, w.nsteps, rescale=True)
    ph = torch.from_numpy(phi).cuda()
    tr = rrpkg.Tracer(w.bundle)
    rec = rrpkg.record_buffer(w.grid)
    for st in steps:
        tr.tidal(w.grid, ph, rec, bbox=tr.footprint(w.grid, st.chi_a, st.chi_b))
        tr.step(w.grid, rec, st.chi_a, st.chi_b, st.scale, st.a)
    k, kb = tr.finalize()
    per_ray = torch.zeros(w.bundle.nrays, dtype=torch.int32, device="cuda")
    tr.segments(per_ray=per_ray)
    torch.cuda.synchronize()
    tr.close()
    k, kb, nseg = k.cpu().numpy().ravel(), kb.cpu().numpy().ravel(), per_ray.cpu().numpy().view(np.uint32)
    rng = np.random.default_rng(99)
    rids = rng.choice(w.bundle.nrays, 512, replace=False)
    o = run_oracle(oracle_lib, phi, w.grid, w.bundle, steps, rids=rids)
    rms = math.sqrt(float(np.mean(o.kappa ** 2)))
    assert np.abs(k[rids] - o.kappa).max() <= TOL * rms
    rmsb = math.sqrt(float(np.mean(o.kborn ** 2)))
    assert np.abs(kb[rids] - o.kborn).max() <= TOL * rmsb
    got, want = int(nseg[rids].astype(np.int64).sum()), int(o.nseg.sum())
    assert abs(got - want) <= 1e-4 * want, (got, want)
    # every sampled ray within one sliver per few hundred segments
    assert np.all(np.abs(nseg[rids].astype(np.int64) - o.nseg) <= 2)


def test_plain_sums_form(rrpkg, oracle_lib):
    """RR_PLAIN_SUMS (the FP32 walk with uncompensated sums, a comparison form)
    traces the same segments; its maps stay close to the oracle's, and the
    compensated default is at least as close on a long one-step cone."""
    import torch
    g = synth.Grid((64, 64, 64), 64.0)
    b = synth.Bundle(48, 40, synth.deg(12), synth.deg(10), (32.0, 32.0, 0.0), 600.0)
    phi = synth.grf_phi(64, 64.0, 21)
    steps = [synth.Step(600.0, 0.0, 1.0, 1.0)]
    o = run_oracle(oracle_lib, phi, g, b, steps)
    ph = torch.from_numpy(np.ascontiguousarray(phi, np.float32)).cuda()
    errs = {}
    for plain in (False, True):
        tr = rrpkg.Tracer(b, plain_sums=plain)
        rec = rrpkg.record_buffer(g)
        tr.tidal(g, ph, rec)
        tr.step(g, rec, 600.0, 0.0)
        k, kb = tr.finalize()
        errs[plain] = (map_errors(k.cpu().numpy(), o.kappa)[0], map_errors(kb.cpu().numpy(), o.kborn)[0],
                       tr.segments())
        tr.close()
    assert errs[False][2] == errs[True][2]
    assert errs[False][0] <= TOL and errs[False][1] <= TOL
    assert errs[True][0] <= 1e-3 and errs[True][1] <= 1e-3
    assert errs[False][0] <= errs[True][0] * 1.01 + 1e-7
