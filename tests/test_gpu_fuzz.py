"""Randomised parity sweep: every trace form against the oracle on small,
irregular cases -- non-cubic grids, ragged bundles, wide fields, observers
inside or outside the box, periodic or bounded boxes, both interpolations,
steps of uneven lengths and scales. Each case is seeded and reproducible;
tolerance: the map metric of the other parity tests (1e-5 of the rms, max and
l2), on every map the form writes."""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5
FORMS = ["default", "shear", "method_a", "generic", "moments"]


@pytest.fixture(scope="module")
def rrp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_02012_gb300 import build
    build.build()
    import paper_1601_02012_gb300 as pkg
    return pkg


def _case(seed):
    rng = np.random.default_rng(1000 + seed)
    n = tuple(int(x) for x in rng.integers(6, 28, size=3))
    h = float(rng.uniform(0.5, 3.0))
    g = synth.Grid(n, n[0] * h)
    ext = np.array(n) * h
    periodic = bool(rng.integers(0, 2))
    interp = int(rng.integers(0, 2))
    obs = tuple(float(x) for x in rng.uniform(-0.3, 1.3, size=3) * ext)
    if not periodic:   # an observer below the box, looking into it along +z
        obs = (obs[0], obs[1], float(rng.uniform(-0.5, 0.2) * ext[2]))
    nx, ny = int(rng.integers(1, 40)), int(rng.integers(1, 40))
    fov = (synth.deg(float(rng.uniform(1, 60))), synth.deg(float(rng.uniform(1, 60))))
    chis = float(rng.uniform(0.5, 3.0) * ext.max())
    b = synth.Bundle(nx, ny, fov[0], fov[1], obs, chis, interp=interp, periodic=periodic)
    nst = int(rng.integers(1, 5))
    edges = np.sort(rng.uniform(0.0, chis, size=nst - 1))[::-1]
    edges = [chis] + list(edges)
    edges.append(float(rng.uniform(0, 0.2) * edges[-1]))   # the last step ends short of the observer
    steps = [synth.Step(float(edges[i]), float(edges[i + 1]), float(rng.uniform(0.5, 1.5)),
                        float(rng.uniform(0.5, 1.0))) for i in range(nst)]
    phi = synth.random_field(n, 2000 + seed, np.float32)
    return g, b, steps, phi


def _err(got, want):
    got = np.asarray(got, np.float64).ravel()
    want = np.asarray(want, np.float64).ravel()
    rms = math.sqrt(float(np.mean(want ** 2)))
    if rms == 0.0:
        return float(np.abs(got).max()), 0.0
    return float(np.abs(got - want).max() / rms), float(np.linalg.norm(got - want) / np.linalg.norm(want))


def _gpu(rrp, form, g, b, steps, phi):
    import torch
    ph = torch.from_numpy(phi).cuda()
    kw = {"shear": form == "shear", "method_a": form == "method_a", "generic": form == "generic",
          "moments": form == "moments"}
    tr = rrp.Tracer(b, **kw)
    rec = tr.record_buffer(g)
    kern = ((0.3, 0.02, -0.001), (0.0, 1.0, -1.0 / b.chi_s))
    if form == "generic":
        tr.set_kernels(kern)
    for st in steps:
        bbox = tr.footprint(g, st.chi_a, st.chi_b)
        if form == "generic":
            tr.scalars(g, ph, rec, 0, bbox=bbox)
            tr.scalars(g, ph, rec, 1, bbox=bbox)
        else:
            tr.tidal(g, ph, rec, bbox=bbox)
        tr.step(g, rec, st.chi_a, st.chi_b, st.scale, st.a)
    k, kb = tr.finalize()
    out = [k.cpu().numpy().ravel(), kb.cpu().numpy().ravel()]
    if form == "shear":
        out += [x.cpu().numpy().ravel() for x in tr.shear()]
    tr.close()
    return out, kern


def _oracle(oracle_lib, form, g, b, steps, phi, kern):
    p64 = phi.astype(np.float64)
    H, d = oracle_lib.fields(g, p64)
    if form == "method_a":
        kg, kb = oracle_lib.trace_method_a(b, g, oracle_lib.fields_grad(g, p64), d, steps)
        return [kg + kb, kb]
    if form == "generic":
        return list(oracle_lib.trace_kq(b, g, p64, p64, kern, steps))
    r = oracle_lib.trace(b, g, H, d, steps)
    out = [r.kappa, r.kborn]
    if form == "shear":
        out += list(oracle_lib.trace_shear(b, g, H, steps))
    return out


@pytest.mark.parametrize("seed", range(40))
def test_random_cases_all_forms(rrp, oracle_lib, seed):
    g, b, steps, phi = _case(seed)
    for form in FORMS:
        got, kern = _gpu(rrp, form, g, b, steps, phi)
        want = _oracle(oracle_lib, form, g, b, steps, phi, kern)
        for i, (x, y) in enumerate(zip(got, want)):
            if not np.any(y):   # rays that never enter a bounded box
                assert np.abs(x).max() == 0.0, (seed, form, i)
                continue
            e_inf, e_2 = _err(x, y)
            assert e_inf <= TOL and e_2 <= TOL, (seed, form, i, e_inf, e_2, g.n, b, steps)
