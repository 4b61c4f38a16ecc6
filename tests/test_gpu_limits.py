"""The largest sizes the interface accepts, against the oracle: a grid of 4096
cells along z (the per-axis maximum), an adaptive mesh refined to the deepest
level (lmax = 8), and a 4096-ray bundle through a mesh refined six levels."""
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
    rms = math.sqrt(float(np.mean(want ** 2)))
    return float(np.abs(got - want).max() / rms)


@pytest.mark.parametrize("interp", [1, 0])
def test_grid_of_4096_cells_along_z(rrp, oracle_lib, interp):
    """n = (6, 5, 4096) with h = 1 Mpc/h: the rays (along +z) cross nearly the
    whole 4096-cell axis in two steps, wrapping through x and y."""
    import torch
    g = synth.Grid((6, 5, 4096), 6.0)
    b = synth.Bundle(9, 7, synth.deg(1.0), synth.deg(1.0), (3.0, 2.5, 0.5), 4000.0, interp=interp)
    rng = np.random.default_rng(3)
    phi = (rng.standard_normal(g.n) * 1e-6).astype(np.float32)
    steps = [synth.Step(4000.0, 1500.0, 1.0, 0.8), synth.Step(1500.0, 0.0, 1.0, 1.0)]
    ph = torch.from_numpy(phi).cuda()
    k, kb, nseg = rrp.trace_kappa(ph, g, b, steps)
    H, d = oracle_lib.fields(g, phi.astype(np.float64))
    o = oracle_lib.trace(b, g, H, d, steps)
    assert _err(k.cpu().numpy().ravel(), o.kappa) <= TOL
    assert _err(kb.cpu().numpy().ravel(), o.kborn) <= TOL
    assert abs(nseg - int(o.nseg.sum())) <= max(1, 1e-4 * o.nseg.sum())


def test_amr_refined_to_level_8(rrp, oracle_lib):
    """Nested cubic refinement from a 4^3 coarse grid down to lmax = 8 (finest
    lattice 1024 per side): records, and a bundle through every level."""
    import torch
    L = 8
    box = 64.0
    widths = [box * 0.3 / (1.6 ** l) for l in range(L)]
    mesh = synth.amr_nested_cubes(4, box, L, widths)
    assert all(len(mesh.octs[l]) > 0 for l in range(1, L + 1))
    mesh.phi = synth.amr_sample(mesh, synth.gaussian_fn(1e-5, 2.0, np.full(3, box / 2)))
    mesh.phi = [np.asarray(p, np.float32).astype(np.float64) for p in mesh.phi]
    gm = rrp.AmrMesh(mesh.n, mesh.lmax, mesh.box, mesh.octs, mesh.omega_m)
    flat = np.concatenate([np.asarray(p).reshape(-1) for p in mesh.phi]).astype(np.float32)
    rec = gm.record_buffer()
    gm.tidal(torch.from_numpy(flat).cuda(), rec)
    b = synth.Bundle(15, 13, synth.deg(6), synth.deg(5), (box / 2 + 0.013, box / 2 - 0.021, 0.0), 60.0,
                     periodic=False)
    steps = [synth.Step(60.0, 31.0, 1.0, 1.0), synth.Step(31.0, 0.0, 1.0, 1.0)]
    tr = rrp.Tracer(b)
    for st in steps:
        tr.amr_step(gm, rec, st.chi_a, st.chi_b, st.scale, st.a)
    k, kb = tr.finalize()
    nseg = tr.segments()
    tr.close()
    gm.close()
    o = oracle_lib.amr_trace(b, mesh, steps)
    assert _err(k.cpu().numpy().ravel(), o.kappa) <= TOL
    assert _err(kb.cpu().numpy().ravel(), o.kborn) <= TOL
    assert abs(nseg - int(o.nseg.sum())) <= max(2, 1e-4 * o.nseg.sum())


def test_amr_deep_levels_wide_bundle(rrp, oracle_lib):
    """A lognormal-cascade mesh refined to lmax = 6 below a 16^3 coarse grid
    (3279 / 2260 / 673 / 243 / 56 / 2 octs per level, 49 687 leaves) and 4096
    rays over 40 x 40 deg through it, two steps: every ray against the oracle.
    The FP32 walk starts each sub-step from a float-float point, where the
    production AMR configuration asks for FP64 set-up at deep levels; this
    checks that reading on the deepest levels and on many rays."""
    mesh = synth.amr_random(16, 32.0, 6, 77, threshold=1.05, child_sigma=0.9)
    assert all(len(mesh.octs[l]) > 0 for l in range(1, 7))
    f = synth.fourier_fn(32.0, 40, 2 * math.pi / 32.0 * 5, 87)
    mesh.phi = [np.asarray(p, np.float32).astype(np.float64) for p in synth.amr_sample(mesh, f)]
    b = synth.Bundle(64, 64, synth.deg(40), synth.deg(40), (16.3, 15.8, 0.3), 45.0)
    steps = [synth.Step(45.0, 19.0, 1.1, 0.8), synth.Step(19.0, 0.0, 0.95, 1.0)]
    import torch
    gm = rrp.AmrMesh(mesh.n, mesh.lmax, mesh.box, mesh.octs, mesh.omega_m)
    flat = np.concatenate([np.asarray(p).reshape(-1) for p in mesh.phi]).astype(np.float32)
    rec = gm.record_buffer()
    gm.tidal(torch.from_numpy(flat).cuda(), rec)
    tr = rrp.Tracer(b)
    for st in steps:
        tr.amr_step(gm, rec, st.chi_a, st.chi_b, st.scale, st.a)
    k, kb = tr.finalize()
    nseg = tr.segments()
    tr.close()
    gm.close()
    o = oracle_lib.amr_trace(b, mesh, steps)
    assert _err(k.cpu().numpy().ravel(), o.kappa) <= TOL
    assert _err(kb.cpu().numpy().ravel(), o.kborn) <= TOL
    assert abs(nseg - int(o.nseg.sum())) <= max(2, 1e-4 * o.nseg.sum())
