"""Shear (RR_SHEAR; Eqs. gamma1, gamma2) against the oracle, through the C ABI.

The shear form accumulates (gamma1, gamma2) in the same walk as kappa and
Born kappa. Tolerance: the map metric of kappa on each of the four maps,
max|x_gpu - x_ora| / rms(x_ora) <= 1e-5 and ||x_gpu - x_ora|| / ||x_ora|| <= 1e-5.
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


def _err(got, want):
    got = np.asarray(got, np.float64).ravel()
    want = np.asarray(want, np.float64).ravel()
    rms = math.sqrt(float(np.mean(want ** 2)))
    return float(np.abs(got - want).max() / rms), float(np.linalg.norm(got - want) / np.linalg.norm(want))


def _gpu(rrp, phi, grid, bundle, steps, footprint=True):
    import torch
    ph = torch.from_numpy(np.ascontiguousarray(phi, np.float32)).cuda()
    out = rrp.trace_shear(ph, grid, bundle, steps, footprint=footprint)
    torch.cuda.synchronize()
    return [x.cpu().numpy().ravel() for x in out[:4]] + [out[4]]


def _oracle(oracle_lib, phi, grid, bundle, steps, rids=None):
    H, d = oracle_lib.fields(grid, np.asarray(phi, np.float32).astype(np.float64))
    o = oracle_lib.trace(bundle, grid, H, d, steps, rids=rids)
    g1, g2 = oracle_lib.trace_shear(bundle, grid, H, steps, rids=rids)
    return o.kappa, o.kborn, g1, g2


@pytest.mark.parametrize("interp", [1, 0])
@pytest.mark.parametrize("periodic", [True, False])
def test_shear_parity_multi_step(rrp, oracle_lib, interp, periodic):
    """A ragged 37 x 29 bundle (several ray tiles and partial ones) over 48^3
    in five steps with different scales: all four maps."""
    g = synth.Grid((48, 48, 48), 96.0)
    b = synth.Bundle(37, 29, synth.deg(14), synth.deg(11), (47.0, 49.0, 0.5), 180.0, interp=interp,
                     periodic=periodic)
    phi = synth.grf_phi(48, 96.0, 41)
    edges = [180.0, 140.0, 101.0, 66.0, 30.0, 0.0]
    steps = [synth.Step(edges[i], edges[i + 1], 1.0 - 0.04 * i, 0.55 + 0.08 * i) for i in range(5)]
    got = _gpu(rrp, phi, g, b, steps)
    want = _oracle(oracle_lib, phi, g, b, steps)
    for x, y, what in zip(got[:4], want, ("kappa", "kborn", "gamma1", "gamma2")):
        e_inf, e_2 = _err(x, y)
        assert e_inf <= TOL and e_2 <= TOL, (what, e_inf, e_2)


def test_shear_wide_field_with_central_ray(rrp, oracle_lib):
    """An odd bundle whose central ray is exactly on the z axis (theta = 0,
    phi = 0 by convention) over a 40 x 40 deg field: rays far from the axis
    and the axis ray itself."""
    g = synth.Grid((40, 40, 40), 40.0)
    b = synth.Bundle(21, 21, synth.deg(40), synth.deg(40), (20.0, 20.0, 0.0), 60.0, periodic=True)
    phi = synth.grf_phi(40, 40.0, 43)
    steps = [synth.Step(60.0, 25.0, 1.0, 0.7), synth.Step(25.0, 0.0, 1.1, 0.9)]
    got = _gpu(rrp, phi, g, b, steps)
    want = _oracle(oracle_lib, phi, g, b, steps)
    for x, y, what in zip(got[:4], want, ("kappa", "kborn", "gamma1", "gamma2")):
        e_inf, e_2 = _err(x, y)
        assert e_inf <= TOL and e_2 <= TOL, (what, e_inf, e_2)
    c = 10 * 21 + 10   # the axis ray
    for x, y in zip(got[2:4], want[2:4]):
        assert abs(x[c] - y[c]) <= TOL * math.sqrt(float(np.mean(y ** 2)))


def test_shear_form_keeps_kappa(rrp):
    """The shear form traces the same segments and leaves kappa and Born kappa
    as the default form computes them."""
    import torch
    g = synth.Grid((32, 32, 32), 64.0)
    b = synth.Bundle(45, 38, synth.deg(9), synth.deg(8), (31.0, 33.0, 0.0), 120.0)
    ph = torch.from_numpy(synth.grf_phi(32, 64.0, 47)).cuda()
    steps = synth.step_schedule(b.chi_s, 4)
    k0, kb0, n0 = rrp.trace_kappa(ph, g, b, steps)
    k1, kb1, _, _, n1 = rrp.trace_shear(ph, g, b, steps)
    torch.cuda.synchronize()
    assert n0 == n1
    for x, y in ((k1, k0), (kb1, kb0)):
        x, y = x.cpu().numpy(), y.cpu().numpy()
        assert np.abs(x - y).max() <= 1e-6 * math.sqrt(float(np.mean(y ** 2)))


def test_gaussian_lens_shear(rrp, oracle_lib):
    """Sec. 4 (the Gaussian lens, trilinear, 40 x 40 deg, z_s = 0.95) on a
    129 x 129 map at 64^3. The shear of a lens axisymmetric about the central
    ray is tangential, i.e. pure gamma1 in the polar frame: gamma2 is only the
    cubic mesh's anisotropy (~1e-3 of gamma1), so its errors are measured in
    units of the shear's own scale, rms(gamma1). gamma2 vanishes to FP32
    rounding on the map's four mirror lines (central row and column, both
    diagonals), which are symmetry planes of the lens and of the mesh."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "gaussian_e1.json")) as f:
        E1 = json.load(f)
    L = E1["box"]
    nr = 129   # odd: the mirror lines are rows and columns of rays
    b = synth.Bundle(nr, nr, synth.deg(E1["fov_deg"][0]), synth.deg(E1["fov_deg"][1]), (L / 2, L / 2, 0.0),
                     synth.chi_of_z(E1["z_s"]), periodic=False)
    g = synth.Grid((64, 64, 64), L)
    phi = synth.gaussian_phi(64, L, E1["potential"]["amp"], E1["potential"]["sigma"])
    steps = [synth.Step(E1["gamma1_chi_max"], 0.0, 1.0, 1.0)]
    got = _gpu(rrp, phi, g, b, steps)
    want = _oracle(oracle_lib, phi, g, b, steps)
    for x, y, what in zip(got[:3], want[:3], ("kappa", "kborn", "gamma1")):
        if what == "kborn":
            continue   # no density here
        e_inf, e_2 = _err(x, y)
        assert e_inf <= TOL and e_2 <= TOL, (what, e_inf, e_2)
    rms1 = math.sqrt(float(np.mean(want[2] ** 2)))
    assert np.abs(got[3] - want[3]).max() <= TOL * rms1
    assert np.abs(want[3]).max() <= 2e-3 * np.abs(want[2]).max()
    g1 = got[2].reshape(nr, nr)
    g2 = got[3].reshape(nr, nr)
    peak = np.abs(g1).max()
    i = np.arange(nr)
    for line in (g2[nr // 2, :], g2[:, nr // 2], g2[i, i], g2[i, nr - 1 - i]):
        assert np.abs(line).max() <= 1e-5 * peak


def test_rotated_elliptical_lens_shear(rrp, oracle_lib):
    """A lens without axial symmetry: an elliptical Gaussian potential
    (sigma 2, 1 and 1.5 Mpc/h) rotated by 30 deg about the line of sight, so
    that gamma2 is of the size of gamma1. All four maps, each at its own rms,
    within the map tolerance of the oracle."""
    L, n = 10.0, 64
    h = L / n
    x = (np.arange(n) + 0.5) * h - L / 2
    dx, dy, dz = x[:, None, None], x[None, :, None], x[None, None, :] - 0.1 * L
    ca, sa = math.cos(math.radians(30.0)), math.sin(math.radians(30.0))
    xr, yr = ca * dx + sa * dy, -sa * dx + ca * dy
    phi = 1e-4 * np.exp(-(xr ** 2 / (2 * 2.0 ** 2) + yr ** 2 / (2 * 1.0 ** 2) + dz ** 2 / (2 * 1.5 ** 2)))
    g = synth.Grid((n, n, n), L)
    b = synth.Bundle(97, 89, synth.deg(40), synth.deg(36), (L / 2, L / 2, 0.0), 9.5, periodic=False)
    steps = [synth.Step(8.0, 3.1, 1.0, 1.0), synth.Step(3.1, 0.0, 1.0, 1.0)]
    got = _gpu(rrp, phi, g, b, steps)
    want = _oracle(oracle_lib, phi, g, b, steps)
    for x_, y_, what in zip(got[:4], want, ("kappa", "kborn", "gamma1", "gamma2")):
        e_inf, e_2 = _err(x_, y_)
        assert e_inf <= TOL and e_2 <= TOL, (what, e_inf, e_2)
    rms1 = math.sqrt(float(np.mean(want[2] ** 2)))
    rms2 = math.sqrt(float(np.mean(want[3] ** 2)))
    assert rms2 >= 0.3 * rms1, (rms1, rms2)


def test_shear_at_production_size_sampled(rrp, oracle_lib):
    """The 512^3, 2048 x 2048-ray, 40-step production workload in the shear
    form; 128 sampled rays are traced by the oracle one by one."""
    w = synth.workload("prod_512")
    phi = synth.grf_phi(512, w.grid.box, w.seed)
    steps = synth.step_schedule(w.bundle.chi_s, w.nsteps, rescale=True)
    got = _gpu(rrp, phi, w.grid, w.bundle, steps)
    rids = np.random.default_rng(7).choice(w.bundle.nrays, 128, replace=False)
    want = _oracle(oracle_lib, phi, w.grid, w.bundle, steps, rids=rids)
    for x, y, what in zip(got[:4], want, ("kappa", "kborn", "gamma1", "gamma2")):
        rms = math.sqrt(float(np.mean(y ** 2)))
        assert np.abs(x[rids] - y).max() <= TOL * rms, what


def test_shear_form_checks(rrp):
    import torch
    from paper_1601_02012_gb300 import _rr
    b = synth.Bundle(8, 8, synth.deg(5), synth.deg(5), (4.0, 4.0, 0.0), 10.0)
    tr = rrp.Tracer(b)   # not a shear context
    with pytest.raises(rrp.RRError) as ei:
        tr.shear()
    assert ei.value.code == _rr.RR_ERR_STATE
    tr.close()
    for kw in ({"fp64_dda": True}, {"plain_sums": True}, {"moments": True}):
        with pytest.raises(rrp.RRError) as ei:
            rrp.Tracer(b, shear=True, **kw)
        assert ei.value.code == _rr.RR_ERR_ARG
    # reset clears the shear too
    g = synth.Grid((8, 8, 8), 16.0)
    tr = rrp.Tracer(b, shear=True)
    rec = rrp.record_buffer(g)
    rrp.rr_tidal_tensor(rrp.grid_desc(g), torch.from_numpy(synth.random_field(8, 3, np.float32)).cuda(), None,
                        rec, rrp.RR_AT_VERTICES)
    tr.step(g, rec, 10.0, 0.0)
    g1, _ = tr.shear()
    assert float(g1.abs().max()) > 0
    tr.reset()
    g1, g2 = tr.shear()
    torch.cuda.synchronize()
    assert float(g1.abs().max()) == 0 and float(g2.abs().max()) == 0
    tr.close()
