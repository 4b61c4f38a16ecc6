"""Map statistics (flat-sky P(ell) and one-point PDF) against closed forms."""
import math

import numpy as np

from paper_1601_02012_gb300 import mapstats as ms


def test_white_noise_spectrum_is_flat_at_sigma2_times_pixel_area():
    rng = np.random.default_rng(0)
    m = rng.standard_normal((512, 512)) * 3.0
    fov = 0.2
    ell, p, counts = ms.power_spectrum(m, fov, fov)
    area = (fov / 511) ** 2
    good = counts > 200
    assert np.all(np.abs(p[good] / (9.0 * area) - 1.0) < 0.15)


def test_single_mode_lands_in_its_ell_bin():
    ny, nx, fov = 128, 128, 0.1
    x = np.arange(nx)
    mode = 7
    m = np.cos(2 * math.pi * mode * x / nx)[None, :].repeat(ny, 0)
    ell, p, counts = ms.power_spectrum(m, fov, fov)
    want = 2 * math.pi * mode / fov
    top = int(np.nanargmax(p))
    edges = np.geomspace(2 * math.pi / fov, math.pi * nx / fov, len(ell) + 1)
    assert edges[top] <= want < edges[top + 1]


def test_pdf_of_a_gaussian_sample():
    rng = np.random.default_rng(1)
    v = rng.standard_normal(2_000_000)
    edges, d = ms.pdf(v, nbins=50, nsigma=4.0)
    c = 0.5 * (edges[1:] + edges[:-1])
    assert np.max(np.abs(d - np.exp(-c * c / 2) / math.sqrt(2 * math.pi))) < 5e-3


def test_compare_of_identical_and_scaled_maps():
    rng = np.random.default_rng(2)
    m = rng.standard_normal((64, 64))
    r = ms.compare(m, m, 0.1, 0.1)
    assert r["max_over_rms"] == 0 and r["pl_max_rel"] == 0 and r["pdf_l1"] == 0
    r = ms.compare(1.001 * m, m, 0.1, 0.1)
    assert abs(r["pl_max_rel"] - (1.001 ** 2 - 1)) < 1e-9
