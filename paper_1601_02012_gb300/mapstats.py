"""Statistics of convergence maps: the flat-sky angular power spectrum and the
one-point PDF (the map statistics of Sec. 5, used here to state how far two
maps of the same bundle -- e.g. the GPU's and the FP64 oracle's -- differ
beyond the pixel-wise metric). Plain numpy, host side.

A map is the [ny, nx] array of a bundle in rayid order (x fastest); its rays
sit on the Eq. (txty) grid, spanning fov_x x fov_y radians.
"""
from __future__ import annotations

import math

import numpy as np


def power_spectrum(kmap, fov_x: float, fov_y: float, nbins: int = 20):
    """Azimuthally averaged |FFT|^2 of the mean-subtracted map in `nbins`
    logarithmic bins of the flat-sky multipole ell = 2 pi m / Upsilon (m the
    Fourier index along each axis), between the fundamental and the Nyquist
    multipole. Returns (bin centres, power per bin, modes per bin); empty bins
    have power NaN. Normalisation: P = |FFT|^2 * (pixel area) / (number of
    pixels), so that the result does not depend on the resolution."""
    m = np.asarray(kmap, np.float64)
    ny, nx = m.shape
    m = m - m.mean()
    f = np.fft.fft2(m)
    ex = 2.0 * math.pi * np.fft.fftfreq(nx, d=1.0 / nx) / fov_x
    ey = 2.0 * math.pi * np.fft.fftfreq(ny, d=1.0 / ny) / fov_y
    ell = np.sqrt(ey[:, None] ** 2 + ex[None, :] ** 2)
    area = (fov_x / max(nx - 1, 1)) * (fov_y / max(ny - 1, 1))
    p2 = (np.abs(f) ** 2) * area / (nx * ny)
    lo = 2.0 * math.pi / max(fov_x, fov_y)
    hi = math.pi * min(nx / fov_x, ny / fov_y)
    edges = np.geomspace(lo, hi, nbins + 1)
    idx = np.digitize(ell.ravel(), edges) - 1
    ok = (idx >= 0) & (idx < nbins)
    counts = np.bincount(idx[ok], minlength=nbins)
    sums = np.bincount(idx[ok], weights=p2.ravel()[ok], minlength=nbins)
    with np.errstate(invalid="ignore", divide="ignore"):
        power = np.where(counts > 0, sums / np.maximum(counts, 1), np.nan)
    return np.sqrt(edges[:-1] * edges[1:]), power, counts


def pdf(kmap, nbins: int = 100, nsigma: float = 5.0, centre=None, sigma=None):
    """Histogram density of the map values in `nbins` bins over centre +-
    nsigma * sigma (default: the map's own mean and standard deviation).
    Returns (bin edges, density)."""
    v = np.asarray(kmap, np.float64).ravel()
    c = float(v.mean()) if centre is None else float(centre)
    s = float(v.std()) if sigma is None else float(sigma)
    edges = np.linspace(c - nsigma * s, c + nsigma * s, nbins + 1)
    dens, _ = np.histogram(v, bins=edges, density=False)
    return edges, dens / (v.size * (edges[1] - edges[0]))


def compare(test, ref, fov_x: float, fov_y: float):
    """How map `test` differs from map `ref` (same bundle):
    max_over_rms  max |test - ref| / rms(ref);
    l2            ||test - ref|| / ||ref||;
    pl_max_rel    largest relative difference of the P(ell) bins;
    pdf_l1        L1 distance of the two PDFs on the reference's bins
                  (100 bins over +-5 sigma of the reference), in units of
                  the PDF's own L1 norm (0: identical histograms, 2: disjoint)."""
    t = np.asarray(test, np.float64)
    r = np.asarray(ref, np.float64)
    d = t - r
    rms = math.sqrt(float(np.mean(r * r)))
    _, pt, _ = power_spectrum(t, fov_x, fov_y)
    _, pr, _ = power_spectrum(r, fov_x, fov_y)
    ok = np.isfinite(pr) & (pr > 0)
    edges, hr = pdf(r)
    _, ht = pdf(t, centre=float(r.mean()), sigma=float(r.std()))
    width = edges[1] - edges[0]
    return {
        "max_over_rms": float(np.abs(d).max() / rms),
        "l2": float(np.linalg.norm(d) / np.linalg.norm(r)),
        "pl_max_rel": float(np.max(np.abs(pt[ok] - pr[ok]) / pr[ok])),
        "pdf_l1": float(np.sum(np.abs(ht - hr)) * width),
    }
