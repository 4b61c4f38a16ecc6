"""Adaptive meshes on the GPU (rr_amr_*) against the FP64 oracle.

Cell tidal records (Eq. tidalexample per level, coarse interpolation at
refinement boundaries, Sec. 3.3) and leaf corner values (Sec. 2.7, Eqs.
alphac3d, alphaf3d, hanging corners) element by element; maps traced leaf by
leaf with the map metric of the uniform tests (1e-5 of the rms, max and l2);
leaf-segment counts within 1e-4 of the oracle's; the uniform limits (no
refinement; one fully refined level = the uniform grid of twice the
resolution) against the uniform kernels.
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


def _flat_phi(mesh):
    """Potential in cell order (level 0 row-major, then octs x 8 per level), FP32."""
    parts = [np.asarray(mesh.phi[0], np.float64).reshape(-1)]
    for l in range(1, mesh.lmax + 1):
        parts.append(np.asarray(mesh.phi[l], np.float64).reshape(-1))
    return np.concatenate(parts).astype(np.float32)


def _round_phi(mesh):
    """The mesh with its potential rounded to FP32 (what the GPU reads)."""
    mesh.phi = [np.asarray(p, np.float32).astype(np.float64) for p in mesh.phi]
    return mesh


def _leaves(mesh):
    """(level, i, j, k) of every leaf, in the library's leaf order (cell order)."""
    refined = [set() for _ in range(mesh.lmax + 1)]
    for l in range(1, mesh.lmax + 1):
        refined[l - 1] = {tuple(int(x) for x in r) for r in mesh.octs[l]}
    out = []
    n = mesh.n
    for i in range(n):
        for j in range(n):
            for k in range(n):
                if (i, j, k) not in refined[0]:
                    out.append((0, i, j, k))
    for l in range(1, mesh.lmax + 1):
        for p in mesh.octs[l]:
            for ch in range(8):
                c = (2 * int(p[0]) + (ch & 1), 2 * int(p[1]) + ((ch >> 1) & 1), 2 * int(p[2]) + ((ch >> 2) & 1))
                if c not in refined[l]:
                    out.append((l,) + c)
    return out


def _gpu_mesh(rrp, mesh):
    return rrp.AmrMesh(mesh.n, mesh.lmax, mesh.box, mesh.octs, mesh.omega_m)


def _random_mesh(seed=3):
    mesh = synth.amr_random(8, 16.0, 3, seed, threshold=1.2, child_sigma=0.8)   # 421, 241, 14 octs
    f = synth.fourier_fn(16.0, 40, 2 * math.pi / 16.0 * 5, seed + 10)
    mesh.phi = synth.amr_sample(mesh, f)
    return _round_phi(mesh)


def _gauss_mesh(ng=16, L=32.0):
    mesh = synth.amr_nested_cubes(ng, L, 2, [0.3 * L, 0.15 * L])
    mesh.phi = synth.amr_sample(mesh, synth.gaussian_fn(1e-5, 0.06 * L, np.full(3, L / 2)))
    return _round_phi(mesh)


def _trace_gpu(rrp, mesh, bundle, steps, where=None):
    import torch
    gm = _gpu_mesh(rrp, mesh)
    if where is None:
        where = rrp.RR_AT_VERTICES if bundle.interp == 1 else rrp.RR_AT_CENTRES
    phi = torch.from_numpy(_flat_phi(mesh)).cuda()
    rec = gm.record_buffer(where)
    gm.tidal(phi, rec, where)
    tr = rrp.Tracer(bundle)
    for st in steps:
        tr.amr_step(gm, rec, st.chi_a, st.chi_b, st.scale, st.a)
    k, kb = tr.finalize()
    nseg = tr.segments()
    out = (k.cpu().numpy().ravel(), kb.cpu().numpy().ravel(), nseg)
    tr.close()
    gm.close()
    return out


def _assert_map(got, want, tol=TOL, what="kappa"):
    d = got - want
    rms = math.sqrt(float(np.mean(want ** 2)))
    e_inf = float(np.abs(d).max() / rms)
    e_2 = float(np.linalg.norm(d) / np.linalg.norm(want))
    assert e_inf <= tol and e_2 <= tol, f"{what}: max/rms {e_inf:.3e}, l2 {e_2:.3e}"


# ---------------------------------------------------------------------------
# rr_amr_create / rr_amr_tidal
# ---------------------------------------------------------------------------

def test_plan_sizes(rrp):
    mesh = _random_mesh()
    gm = _gpu_mesh(rrp, mesh)
    assert gm.ncells == mesh.n ** 3 + sum(8 * len(mesh.octs[l]) for l in range(1, mesh.lmax + 1))
    assert gm.nleaves == mesh.nleaves() == len(_leaves(mesh))
    assert 0 < gm.nverts <= 8 * gm.nleaves
    gm.close()


def test_cell_tidal_vs_oracle(rrp, oracle_lib):
    """Every cell of every level, all 7 channels: FP32 stencils and coarse
    interpolation against the FP64 oracle on the same (FP32-rounded) potential."""
    import torch
    mesh = _random_mesh()
    assert all(len(mesh.octs[l]) > 0 for l in range(1, mesh.lmax + 1))
    gm = _gpu_mesh(rrp, mesh)
    phi = torch.from_numpy(_flat_phi(mesh)).cuda()
    cells = torch.empty((gm.ncells, 8), dtype=torch.float32, device="cuda")
    rec = gm.record_buffer(rrp.RR_AT_CENTRES)
    gm.tidal(phi, rec, rrp.RR_AT_CENTRES, cell_tidal=cells)
    got = cells.cpu().numpy()
    want = oracle_lib.amr_tidal(mesh)
    assert np.all(got[:, 7] == 0)
    for c in range(7):
        scale = np.abs(want[:, c]).max()
        err = np.abs(got[:, c] - want[:, c]).max()
        assert err <= 4e-6 * scale, (c, err / scale)
    # centre records are the leaves' own cell values
    leaves = _leaves(mesh)
    lr = rec.cpu().numpy()
    offs = np.cumsum([0, mesh.n ** 3] + [8 * len(mesh.octs[l]) for l in range(1, mesh.lmax + 1)])
    n = mesh.n
    cell_of = {}
    for l in range(1, mesh.lmax + 1):
        for o, p in enumerate(mesh.octs[l]):
            for ch in range(8):
                c = (2 * int(p[0]) + (ch & 1), 2 * int(p[1]) + ((ch >> 1) & 1), 2 * int(p[2]) + ((ch >> 2) & 1))
                cell_of[(l,) + c] = offs[l] + 8 * o + ch
    for t, lf in enumerate(leaves):
        idx = (lf[1] * n + lf[2]) * n + lf[3] if lf[0] == 0 else cell_of[lf]
        assert np.array_equal(lr[t], got[idx])
    gm.close()


@pytest.mark.parametrize("which", ["random", "gauss"])
def test_leaf_corner_values_vs_oracle(rrp, oracle_lib, which):
    """Corner values of sampled leaves (every leaf touching a coarser or finer
    leaf included) against the oracle's vertex rules."""
    import torch
    mesh = _random_mesh() if which == "random" else _gauss_mesh()
    gm = _gpu_mesh(rrp, mesh)
    phi = torch.from_numpy(_flat_phi(mesh)).cuda()
    rec = gm.record_buffer(rrp.RR_AT_VERTICES)
    gm.tidal(phi, rec, rrp.RR_AT_VERTICES)
    got = rec.cpu().numpy().reshape(-1, 8, 8)
    leaves = _leaves(mesh)
    rng = np.random.default_rng(1)
    fine = [t for t, lf in enumerate(leaves) if lf[0] > 0]
    pick = sorted(set(rng.choice(len(leaves), 120, replace=False).tolist())
                  | set(rng.choice(fine, min(160, len(fine)), replace=False).tolist()))
    want = np.stack([oracle_lib.amr_leaf_vertices(mesh, leaves[t][0], leaves[t][1:]) for t in pick])
    g = got[pick][:, :, :7]
    assert np.all(got[pick][:, :, 7] == 0)
    for c in range(7):
        scale = np.abs(want[..., c]).max()
        err = np.abs(g[..., c] - want[..., c]).max()
        assert err <= 4e-6 * scale, (c, err / scale)
    gm.close()


# ---------------------------------------------------------------------------
# rr_amr_trace_step
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("interp", [1, 0])
def test_trace_random_mesh_vs_oracle(rrp, oracle_lib, interp):
    """Three refinement levels from a lognormal cascade, rays wrapping through
    the periodic box over two steps with different scales."""
    mesh = _random_mesh()
    b = synth.Bundle(23, 17, synth.deg(30), synth.deg(22), (3.1, 12.7, 0.4), 40.0, interp=interp)
    steps = [synth.Step(40.0, 17.0, 1.1, 0.8), synth.Step(17.0, 0.0, 0.95, 1.0)]
    k, kb, nseg = _trace_gpu(rrp, mesh, b, steps)
    o = oracle_lib.amr_trace(b, mesh, steps)
    _assert_map(k, o.kappa)
    _assert_map(kb, o.kborn, what="kborn")
    assert abs(nseg - int(o.nseg.sum())) <= max(1, 1e-4 * o.nseg.sum())


@pytest.mark.parametrize("interp", [1, 0])
def test_trace_nested_gaussian_vs_oracle(rrp, oracle_lib, interp):
    """The Gaussian-potential mesh of Sec. 4 (two nested cubic refinement
    levels towards the centre), non-periodic, the observer on the z = 0 face."""
    L = 32.0
    mesh = _gauss_mesh(16, L)
    b = synth.Bundle(31, 9, synth.deg(20), synth.deg(6), (L / 2, L / 2, 0.0), 60.0, interp=interp,
                     periodic=False)
    steps = [synth.Step(60.0, 0.0, 1.0, 1.0)]
    k, kb, nseg = _trace_gpu(rrp, mesh, b, steps)
    o = oracle_lib.amr_trace(b, mesh, steps)
    _assert_map(k, o.kappa)
    _assert_map(kb, o.kborn, what="kborn")
    assert abs(nseg - int(o.nseg.sum())) <= max(1, 1e-4 * o.nseg.sum())


def test_uniform_limits(rrp):
    """No refinement: the uniform kernel on the coarse grid. One fully refined
    level: the uniform kernel on the grid of twice the resolution. Same maps to
    FP32 rounding, same segment counts."""
    import torch
    n, box = 12, 24.0
    f = synth.fourier_fn(box, 30, 2 * math.pi / box * 4, 3)
    b = synth.Bundle(19, 14, synth.deg(35), synth.deg(25), (5.0, 7.0, 1.0), 40.0)
    steps = [synth.Step(40.0, 12.0, 1.1, 0.9), synth.Step(12.0, 0.0, 1.0, 1.0)]
    full = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    for refined in (False, True):
        octs = [np.zeros((0, 3), np.int32), (full if refined else np.zeros((0, 3))).astype(np.int32)]
        mesh = synth.AmrMesh(n, box, 1, octs)
        mesh.phi = synth.amr_sample(mesh, f)
        k, kb, nseg = _trace_gpu(rrp, mesh, b, steps)
        m = 2 * n if refined else n
        g = synth.Grid((m, m, m), box)
        if refined:
            phi = np.zeros((m, m, m), np.float32)
            for o, p in enumerate(mesh.octs[1]):
                for ch in range(8):
                    phi[2 * p[0] + (ch & 1), 2 * p[1] + ((ch >> 1) & 1), 2 * p[2] + ((ch >> 2) & 1)] = \
                        mesh.phi[1][o, ch]
        else:
            phi = np.asarray(mesh.phi[0], np.float32)
        ku, kbu, nsegu = rrp.trace_kappa(torch.from_numpy(phi).cuda(), g, b, steps)
        ku = ku.cpu().numpy().ravel()
        kbu = kbu.cpu().numpy().ravel()
        _assert_map(k, ku, tol=2e-6)
        _assert_map(kb, kbu, tol=2e-6, what="kborn")
        assert abs(nseg - nsegu) <= max(1, 1e-4 * nsegu)


def test_errors_and_no_adjoint(rrp):
    import torch
    from paper_1601_02012_gb300 import _rr
    mesh = _random_mesh()
    gm = _gpu_mesh(rrp, mesh)
    rec = gm.record_buffer()
    gm.tidal(torch.from_numpy(_flat_phi(mesh)).cuda(), rec)
    b = synth.Bundle(8, 8, synth.deg(5), synth.deg(5), (1.0, 1.0, 1.0), 20.0)
    tr = rrp.Tracer(b, fp64_dda=True)
    with pytest.raises(rrp.RRError) as ei:
        tr.amr_step(gm, rec, 20.0, 0.0)
    assert ei.value.code == _rr.RR_ERR_ARG
    tr.close()
    tr = rrp.Tracer(b)
    tr.amr_step(gm, rec, 20.0, 5.0)
    with pytest.raises(rrp.RRError) as ei:   # gap between steps
        tr.amr_step(gm, rec, 4.0, 0.0)
    assert ei.value.code == _rr.RR_ERR_STATE
    k, _ = tr.finalize()
    dk = torch.ones_like(k)
    with pytest.raises(rrp.RRError) as ei:
        rrp.rr_trace_step_adjoint(tr.ctx, 0, dk, None, rrp.grad_buffer(synth.Grid((8, 8, 8), 16.0)))
    assert ei.value.code == _rr.RR_ERR_STATE
    tr.close()
    with pytest.raises(rrp.RRError):
        gm.tidal(torch.zeros(4, device="cuda"), rec, 7)
    gm.close()


def _shuffled(mesh, seed):
    """The same mesh with the octs of every level listed in a random order
    (and the potential rows with them): another cell numbering."""
    rng = np.random.default_rng(seed)
    octs, phi = [mesh.octs[0]], [mesh.phi[0]]
    for l in range(1, mesh.lmax + 1):
        perm = rng.permutation(len(mesh.octs[l]))
        octs.append(np.ascontiguousarray(mesh.octs[l][perm]))
        phi.append(np.ascontiguousarray(mesh.phi[l][perm]))
    out = synth.AmrMesh(mesh.n, mesh.box, mesh.lmax, octs, phi, mesh.omega_m)
    return out


@pytest.mark.parametrize("interp", [1, 0])
@pytest.mark.parametrize("shuffle", [False, True])
@pytest.mark.parametrize("obs", [(16.0, 15.0, 0.5), (0.7, 31.2, 30.0)])
def test_footprint_records_give_the_same_maps(rrp, interp, shuffle, obs):
    """Records of only the leaves in each step's coarse footprint box (the
    rest left as NaN) give the same maps, bit for bit, as records of the
    whole mesh: the walk reads nothing outside the box. With the octs listed
    out of order (no x-slab launches; another cell numbering) the maps are
    the same bits again. The second observer sits at a corner of the periodic
    box, so the boxes wrap through the seams (two x-slab ranges per level)."""
    import torch
    mesh = synth.amr_random(16, 32.0, 2, 6, threshold=1.5, child_sigma=0.8)
    mesh.phi = synth.amr_sample(mesh, synth.fourier_fn(32.0, 40, 2 * math.pi / 32.0 * 6, 17))
    _round_phi(mesh)
    reference = None
    if shuffle:
        b0 = synth.Bundle(21, 18, synth.deg(8), synth.deg(6), obs, 30.0, interp=interp)
        st0 = [synth.Step(30.0, 20.0, 1.2, 0.7), synth.Step(20.0, 10.0, 1.1, 0.85), synth.Step(10.0, 0.0, 1.0, 1.0)]
        reference = _trace_gpu(rrp, mesh, b0, st0)
        mesh = _shuffled(mesh, 23)
    b = synth.Bundle(21, 18, synth.deg(8), synth.deg(6), obs, 30.0, interp=interp)
    steps = [synth.Step(30.0, 20.0, 1.2, 0.7), synth.Step(20.0, 10.0, 1.1, 0.85), synth.Step(10.0, 0.0, 1.0, 1.0)]
    where = rrp.RR_AT_VERTICES if interp == 1 else rrp.RR_AT_CENTRES
    gm = _gpu_mesh(rrp, mesh)
    phi = torch.from_numpy(_flat_phi(mesh)).cuda()
    full = gm.record_buffer(where)
    gm.tidal(phi, full, where)
    maps = []
    for use_box in (False, True):
        tr = rrp.Tracer(b)
        rec = gm.record_buffer(where)
        written = 0
        for st in steps:
            if use_box:
                bb = gm.footprint(tr, st.chi_a, st.chi_b)
                assert any(bb[2 * a + 1] - bb[2 * a] < 16 for a in range(3))
                rec.fill_(float("nan"))
                gm.tidal(phi, rec, where, bbox=bb)
                ok = ~torch.isnan(rec).any(dim=1)
                written += int(ok.sum())
                assert torch.equal(rec[ok], full[ok])
            else:
                rec.copy_(full)
            tr.amr_step(gm, rec, st.chi_a, st.chi_b, st.scale, st.a)
        k, kb = tr.finalize()
        maps.append((k.cpu().numpy(), kb.cpu().numpy(), tr.segments()))
        tr.close()
        if use_box:
            assert 0 < written < len(steps) * gm.nleaves
    assert np.array_equal(maps[0][0], maps[1][0]) and np.array_equal(maps[0][1], maps[1][1])
    assert maps[0][2] == maps[1][2]
    if reference is not None:
        assert np.array_equal(reference[0], maps[0][0].ravel()) and np.array_equal(reference[1], maps[0][1].ravel())
        assert reference[2] == maps[0][2]
    gm.close()


# ---------------------------------------------------------------------------
# the shear (RR_SHEAR) through the adaptive mesh
# ---------------------------------------------------------------------------

def _trace_gpu_shear(rrp, mesh, bundle, steps):
    import torch
    gm = _gpu_mesh(rrp, mesh)
    where = rrp.RR_AT_VERTICES if bundle.interp == 1 else rrp.RR_AT_CENTRES
    rec = gm.record_buffer(where)
    gm.tidal(torch.from_numpy(_flat_phi(mesh)).cuda(), rec, where)
    tr = rrp.Tracer(bundle, shear=True)
    for st in steps:
        tr.amr_step(gm, rec, st.chi_a, st.chi_b, st.scale, st.a)
    k, kb = tr.finalize()
    g1, g2 = tr.shear()
    out = [x.cpu().numpy().ravel() for x in (k, kb, g1, g2)]
    tr.close()
    gm.close()
    return out


@pytest.mark.parametrize("interp", [1, 0])
def test_shear_random_mesh_vs_oracle(rrp, oracle_lib, interp):
    """gamma1, gamma2 (Eqs. gamma1, gamma2) over three refinement levels and
    two steps, with kappa and Born kappa of the same walk unchanged."""
    mesh = _random_mesh()
    b = synth.Bundle(23, 17, synth.deg(30), synth.deg(22), (3.1, 12.7, 0.4), 40.0, interp=interp)
    steps = [synth.Step(40.0, 17.0, 1.1, 0.8), synth.Step(17.0, 0.0, 0.95, 1.0)]
    k, kb, g1, g2 = _trace_gpu_shear(rrp, mesh, b, steps)
    o = oracle_lib.amr_trace(b, mesh, steps)
    w1, w2 = oracle_lib.amr_trace_shear(b, mesh, steps)
    _assert_map(k, o.kappa)
    _assert_map(kb, o.kborn, what="kborn")
    _assert_map(g1, w1, what="gamma1")
    _assert_map(g2, w2, what="gamma2")


def test_shear_nested_gaussian_vs_oracle(rrp, oracle_lib):
    """Sec. 4's mesh (two refined cubes towards the lens): the shear of the
    axisymmetric lens is tangential, so gamma2 is only the mesh's anisotropy;
    its errors are measured in units of rms(gamma1)."""
    L = 32.0
    mesh = _gauss_mesh(16, L)
    b = synth.Bundle(31, 31, synth.deg(20), synth.deg(20), (L / 2, L / 2, 0.0), 60.0, periodic=False)
    steps = [synth.Step(60.0, 0.0, 1.0, 1.0)]
    _, _, g1, g2 = _trace_gpu_shear(rrp, mesh, b, steps)
    w1, w2 = oracle_lib.amr_trace_shear(b, mesh, steps)
    _assert_map(g1, w1, what="gamma1")
    rms1 = math.sqrt(float(np.mean(w1 ** 2)))
    assert np.abs(g2 - w2).max() <= TOL * rms1


def _trace_gpu_method_a(rrp, mesh, bundle, steps):
    import torch
    gm = _gpu_mesh(rrp, mesh)
    where = rrp.RR_AT_VERTICES if bundle.interp == 1 else rrp.RR_AT_CENTRES
    rec = gm.record_buffer(where)
    gm.gradient(torch.from_numpy(_flat_phi(mesh)).cuda(), rec, where)
    tr = rrp.Tracer(bundle, method_a=True)
    for st in steps:
        tr.amr_step(gm, rec, st.chi_a, st.chi_b, st.scale, st.a)
    k, kb = tr.finalize()
    out = [x.cpu().numpy().ravel() for x in (k, kb)]
    tr.close()
    gm.close()
    return out


@pytest.mark.parametrize("interp", [1, 0])
def test_method_a_random_mesh_vs_oracle(rrp, oracle_lib, interp):
    """Method A (Eq. kappa2) over three refinement levels and two steps with
    different scales (the surface terms do not telescope): kappa (all three
    terms) and the density term."""
    mesh = _random_mesh()
    b = synth.Bundle(23, 17, synth.deg(30), synth.deg(22), (3.1, 12.7, 0.4), 40.0, interp=interp)
    steps = [synth.Step(40.0, 17.0, 1.1, 0.8), synth.Step(17.0, 0.0, 0.95, 1.0)]
    k, kb = _trace_gpu_method_a(rrp, mesh, b, steps)
    kg, kbo = oracle_lib.amr_trace_method_a(b, mesh, steps)
    _assert_map(k, kg + kbo)
    _assert_map(kb, kbo, what="kborn")


@pytest.mark.parametrize("interp", [1, 0])
def test_method_a_nested_gaussian_vs_oracle(rrp, oracle_lib, interp):
    """Sec. 4's mesh, bounded box, the observer on its face: the rays enter
    and leave the box, so the surface terms sit on the box faces."""
    L = 32.0
    mesh = _gauss_mesh(16, L)
    b = synth.Bundle(31, 9, synth.deg(20), synth.deg(6), (L / 2, L / 2, 0.0), 60.0, interp=interp,
                     periodic=False)
    steps = [synth.Step(60.0, 20.0, 0.9, 1.0), synth.Step(20.0, 0.0, 1.0, 1.0)]
    k, kb = _trace_gpu_method_a(rrp, mesh, b, steps)
    kg, kbo = oracle_lib.amr_trace_method_a(b, mesh, steps)
    _assert_map(k, kg + kbo)
    _assert_map(kb, kbo, what="kborn")


def _flat(levels):
    return np.concatenate([np.asarray(q, np.float64).reshape(-1) for q in levels]).astype(np.float32)


@pytest.mark.parametrize("interp", [1, 0])
def test_generic_integrals_random_mesh_vs_oracle(rrp, oracle_lib, interp):
    """Generic integrals (RR_GENERIC) over three refinement levels: channel 0
    a finite-difference time derivative (the ISW integrand of Sec. 6) of two
    fields, channel 1 a field with the lensing kernel, two steps."""
    import torch
    mesh = _random_mesh()
    cur = [np.asarray(p, np.float32).astype(np.float64) for p in mesh.phi]
    prev = [np.asarray(0.9 * p + 0.01, np.float32).astype(np.float64) for p in mesh.phi]
    inv_dt = 20.0
    b = synth.Bundle(23, 17, synth.deg(30), synth.deg(22), (3.1, 12.7, 0.4), 40.0, interp=interp)
    steps = [synth.Step(40.0, 17.0, 1.1, 1.0), synth.Step(17.0, 0.0, 0.95, 1.0)]
    ker = ((2.0, 0.01, 0.0), (0.0, 1.0, -1.0 / 40.0))
    gm = _gpu_mesh(rrp, mesh)
    where = rrp.RR_AT_VERTICES if interp == 1 else rrp.RR_AT_CENTRES
    rec = gm.record_buffer(where)
    fc, fp = torch.from_numpy(_flat(cur)).cuda(), torch.from_numpy(_flat(prev)).cuda()
    gm.scalars(fc, rec, where, prev0=fp, inv_dt0=inv_dt, field1=fc)
    tr = rrp.Tracer(b, generic=True)
    tr.set_kernels(ker)
    for st in steps:
        tr.amr_step(gm, rec, st.chi_a, st.chi_b, st.scale, st.a)
    o1, o2 = tr.finalize()
    got = [x.cpu().numpy().ravel() for x in (o1, o2)]
    tr.close()
    gm.close()
    q = [(np.asarray(c, np.float32).astype(np.float64) - np.asarray(p_, np.float32).astype(np.float64)) * inv_dt
         for c, p_ in zip(cur, prev)]
    want = oracle_lib.amr_trace_kq(b, mesh, q, cur, ker, steps)
    _assert_map(got[0], want[0], what="isw")
    _assert_map(got[1], want[1], what="channel 1")


@pytest.mark.parametrize("seed", range(6))
def test_random_meshes_and_bundles(rrp, oracle_lib, seed):
    """Seeded sweep: random refinement (1-3 levels), random bundles (ragged,
    up to 50 deg, observers inside or outside the box, periodic or bounded),
    uneven steps; kappa, Born kappa, the shear and Method A against the oracle."""
    rng = np.random.default_rng(500 + seed)
    n = int(rng.choice([6, 8]))
    box = float(rng.uniform(8.0, 20.0))
    mesh = synth.amr_random(n, box, int(rng.integers(1, 4)), 40 + seed, threshold=float(rng.uniform(1.0, 1.6)),
                            child_sigma=0.8)
    f = synth.fourier_fn(box, 30, 2 * math.pi / box * 4, 60 + seed)
    mesh.phi = synth.amr_sample(mesh, f)
    _round_phi(mesh)
    periodic = bool(rng.integers(0, 2))
    obs = tuple(float(x) for x in rng.uniform(-0.2, 1.2, size=3) * box)
    if not periodic:
        obs = (obs[0], obs[1], float(rng.uniform(-0.4, 0.1) * box))
    chis = float(rng.uniform(0.8, 2.5) * box)
    b = synth.Bundle(int(rng.integers(1, 24)), int(rng.integers(1, 24)), synth.deg(float(rng.uniform(2, 50))),
                     synth.deg(float(rng.uniform(2, 50))), obs, chis, interp=int(rng.integers(0, 2)),
                     periodic=periodic)
    mid = float(rng.uniform(0.3, 0.7) * chis)
    steps = [synth.Step(chis, mid, float(rng.uniform(0.6, 1.4)), 0.9),
             synth.Step(mid, float(rng.uniform(0.0, 0.1) * chis), float(rng.uniform(0.6, 1.4)), 1.0)]
    k, kb, g1, g2 = _trace_gpu_shear(rrp, mesh, b, steps)
    o = oracle_lib.amr_trace(b, mesh, steps)
    w1, w2 = oracle_lib.amr_trace_shear(b, mesh, steps)
    ka, kba = _trace_gpu_method_a(rrp, mesh, b, steps)
    wg, wb = oracle_lib.amr_trace_method_a(b, mesh, steps)
    for got, want, what in ((k, o.kappa, "kappa"), (kb, o.kborn, "kborn"), (g1, w1, "gamma1"), (g2, w2, "gamma2"),
                            (ka, wg + wb, "kappa A"), (kba, wb, "kborn A")):
        if not np.any(want):
            assert np.abs(got).max() == 0.0, what
            continue
        _assert_map(got, want, what=what)
