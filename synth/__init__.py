"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module holds none of the ray-tracing arithmetic: it only draws fields,
describes ray bundles and lays out the per-step schedule that a caller would
hand to the library. Everything is deterministic in the seed.

Units: comoving Mpc/h for lengths; the potential is Phi/c^2 (dimensionless),
so that the convergence is kappa = int g(chi_s, chi) Q dchi with no 1/c^2
prefactor (Eq. kappa of Barreira et al. 2016, with Phi measured in c^2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

#: Hubble distance c/H0 in Mpc/h (H0 = 100 h km/s/Mpc).
HUBBLE_DISTANCE = 2997.92458
#: H0/c in h/Mpc.
H0_OVER_C = 1.0 / HUBBLE_DISTANCE


# ---------------------------------------------------------------------------
# Bundles and grids
# ---------------------------------------------------------------------------

@dataclass
class Bundle:
    """A light bundle: N_x x N_y rays over an opening angle Upsilon_x x Upsilon_y
    (Sec. 2.4, Eq. txty), observer at ``obs`` in box coordinates (Sec. 2.2),
    source at comoving distance ``chi_s``."""
    nx: int
    ny: int
    fov_x: float          # radians
    fov_y: float          # radians
    obs: tuple            # (x, y, z) in Mpc/h
    chi_s: float          # Mpc/h
    interp: int = 1       # 0 = NGP (Eq. Icngp), 1 = trilinear (Eq. Icfinal)
    periodic: bool = True

    @property
    def nrays(self) -> int:
        return self.nx * self.ny


@dataclass
class Grid:
    """Uniform cubic-cell grid of n[0] x n[1] x n[2] cells, cell size h = box/n[0]."""
    n: tuple
    box: float
    omega_m: float = 0.3

    @property
    def h(self) -> float:
        return self.box / self.n[0]

    @property
    def ncells(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])


def deg(x: float) -> float:
    return x * math.pi / 180.0


# ---------------------------------------------------------------------------
# Fields
# ---------------------------------------------------------------------------

def _kgrid(n: int, box: float):
    k1 = 2.0 * np.pi * np.fft.fftfreq(n, d=box / n)
    kz = 2.0 * np.pi * np.fft.rfftfreq(n, d=box / n)
    return k1, kz


def grf_phi(n: int, box: float, seed: int, omega_m: float = 0.3,
            spectral_index: float = -3.0, rms_delta: float = 1.0,
            dtype=np.float32) -> np.ndarray:
    """Gaussian random potential Phi/c^2 on the n^3 cell centres, [ix][iy][iz]
    with z fastest, periodic.

    P_Phi(k) = A k^spectral_index for 0 < |k| <= k_Nyq = pi n / box (spherical
    cut; the Nyquist planes are zeroed). White noise is drawn in real space with
    numpy's PCG64(seed), transformed, shaped by sqrt(P) and transformed back, all
    in FP64. The amplitude A makes the continuum density contrast
    delta = -k^2 Phi / (1.5 Omega_m (H0/c)^2) (comoving Poisson equation at
    a = 1) have the requested rms. The result is cast to ``dtype`` last.
    """
    import scipy.fft as sfft

    rng = np.random.Generator(np.random.PCG64(seed))
    white = rng.standard_normal((n, n, n))
    wk = sfft.rfftn(white, workers=-1)
    del white
    k1, kz = _kgrid(n, box)
    kx = k1[:, None, None]
    ky = k1[None, :, None]
    kzz = kz[None, None, :]
    k2 = kx * kx + ky * ky + kzz * kzz
    knyq = math.pi * n / box
    shape = np.zeros_like(k2)
    live = (k2 > 0) & (k2 <= knyq * knyq)
    shape[live] = np.sqrt(k2[live]) ** (0.5 * spectral_index)
    # zero the Nyquist planes so the field is exactly real-symmetric
    if n % 2 == 0:
        shape[n // 2, :, :] = 0.0
        shape[:, n // 2, :] = 0.0
        shape[:, :, -1] = 0.0
    wk *= shape
    phi = sfft.irfftn(wk, s=(n, n, n), workers=-1)
    dk = sfft.irfftn(-k2 * wk, s=(n, n, n), workers=-1)
    del wk
    pref = 1.5 * omega_m * H0_OVER_C ** 2
    rms = float(np.sqrt(np.mean((dk / pref) ** 2)))
    phi *= rms_delta / rms
    return np.ascontiguousarray(phi.astype(dtype, copy=False))


def gaussian_phi(n: int, box: float, amp: float, sigma: float,
                 centre=None, dtype=np.float64) -> np.ndarray:
    """Gaussian potential A exp(-r^2 / 2 sigma^2) sampled at cell centres
    (Eq. gaussian, Sec. 4)."""
    h = box / n
    c = np.full(3, box / 2.0) if centre is None else np.asarray(centre, float)
    x = (np.arange(n) + 0.5) * h
    dx = (x - c[0])[:, None, None]
    dy = (x - c[1])[None, :, None]
    dz = (x - c[2])[None, None, :]
    r2 = dx * dx + dy * dy + dz * dz
    return np.ascontiguousarray((amp * np.exp(-r2 / (2.0 * sigma * sigma))).astype(dtype))


def random_field(n, seed, dtype=np.float64, scale=1.0) -> np.ndarray:
    """White-noise field (tiny parity cases and adjoint probes)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if isinstance(n, int):
        n = (n, n, n)
    return np.ascontiguousarray((scale * rng.standard_normal(tuple(n))).astype(dtype))


# ---------------------------------------------------------------------------
# Background cosmology for the per-step schedule (flat LCDM)
# ---------------------------------------------------------------------------

def _E(z, omega_m):
    return math.sqrt(omega_m * (1.0 + z) ** 3 + (1.0 - omega_m))


def chi_of_z(z: float, omega_m: float = 0.3) -> float:
    """Comoving distance c int_0^z dz/H(z) in Mpc/h (Sec. 2.2)."""
    from scipy.integrate import quad
    val, _ = quad(lambda zz: 1.0 / _E(zz, omega_m), 0.0, z, epsabs=0, epsrel=1e-13, limit=200)
    return HUBBLE_DISTANCE * val


def z_of_chi(chi: float, omega_m: float = 0.3) -> float:
    from scipy.optimize import brentq
    if chi <= 0:
        return 0.0
    return brentq(lambda z: chi_of_z(z, omega_m) - chi, 0.0, 20.0, xtol=1e-15, rtol=1e-15)


def growth(a: float, omega_m: float = 0.3) -> float:
    """Linear growth factor D(a) of flat LCDM, normalised to D(1) = 1:
    D(a) propto H(a) int_0^a da' / (a' H(a'))^3."""
    from scipy.integrate import quad

    def unnorm(aa):
        if aa <= 0:
            return 0.0
        e = math.sqrt(omega_m / aa ** 3 + (1.0 - omega_m))
        val, _ = quad(lambda x: 1.0 / (x * math.sqrt(omega_m / x ** 3 + (1.0 - omega_m))) ** 3,
                      0.0, aa, epsabs=0, epsrel=1e-12, limit=200)
        return e * val

    return unnorm(a) / unnorm(1.0)


@dataclass
class Step:
    chi_a: float     # far end (the step starts here; chi decreases)
    chi_b: float     # near end
    scale: float     # multiplies every channel of the field for this step
    a: float         # scale factor held constant over the step


def step_schedule(chi_s: float, nsteps: int, omega_m: float = 0.3,
                  rescale: bool = True) -> list:
    """Equal-Delta-a steps between a(chi_s) and 1. Each step covers the distance
    light travels during it, [chi_a, chi_b) with chi_a > chi_b (Sec. 2.5.2).
    The field of a step is Phi_k = s_k Phi with s_k = D(a_k)/a_k (comoving
    Poisson: Phi propto delta/a), a_k taken at the step's far end, when the
    N-body code computed the field. With rescale=False every s_k = 1 and a_k = 1.
    """
    a_src = 1.0 / (1.0 + z_of_chi(chi_s, omega_m))
    a_edges = np.linspace(a_src, 1.0, nsteps + 1)
    chis = [chi_s] + [chi_of_z(1.0 / a - 1.0, omega_m) for a in a_edges[1:-1]] + [0.0]
    steps = []
    for k in range(nsteps):
        ak = float(a_edges[k])
        if rescale:
            s = growth(ak, omega_m) / ak
            steps.append(Step(chis[k], chis[k + 1], s, ak))
        else:
            steps.append(Step(chis[k], chis[k + 1], 1.0, 1.0))
    return steps


# ---------------------------------------------------------------------------
# The workloads (sizes as the paper's experiments and the production setup)
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    grid: Grid
    bundle: Bundle
    nsteps: int
    seed: int
    rescale: bool = False
    notes: str = ""


def workload(name: str) -> Workload:
    """Named synthetic workloads.

    small_64: 64^3 GRF, box 256 Mpc/h, 128x128 rays over 2x2 deg, chi_s = 256,
        one step, observer at the centre of the z = 0 face.
    prod_512: 512^3 FP32 GRF, box 1024 Mpc/h, 2048x2048 rays over 10x10 deg,
        chi_s = 1000, 40 steps of equal Delta a with Phi rescaled by D(a)/a
        (flat LCDM, Omega_m = 0.3).
    mid_256: 256^3 GRF, box 512 (same cell size as prod_512), 1024x1024 rays
        over 10x10 deg, chi_s = 500, 20 rescaled steps (profiling case: inputs
        larger than L2, a few GB on the device).
    adjoint_256: 256^3 GRF, box 512, 1024x1024 rays over 5x5 deg, chi_s = 512,
        one step.
    """
    if name == "small_64":
        g = Grid((64, 64, 64), 256.0)
        b = Bundle(128, 128, deg(2.0), deg(2.0), (128.0, 128.0, 0.0), 256.0)
        return Workload(name, g, b, 1, 1)
    if name == "prod_512":
        g = Grid((512, 512, 512), 1024.0)
        b = Bundle(2048, 2048, deg(10.0), deg(10.0), (512.0, 512.0, 0.0), 1000.0)
        return Workload(name, g, b, 40, 2, rescale=True)
    if name == "mid_256":
        g = Grid((256, 256, 256), 512.0)
        b = Bundle(1024, 1024, deg(10.0), deg(10.0), (256.0, 256.0, 0.0), 500.0)
        return Workload(name, g, b, 20, 6, rescale=True)
    if name == "adjoint_256":
        g = Grid((256, 256, 256), 512.0)
        b = Bundle(1024, 1024, deg(5.0), deg(5.0), (256.0, 256.0, 0.0), 512.0)
        return Workload(name, g, b, 1, 5)
    raise KeyError(name)


def grf_phi_cached(n: int, box: float, seed: int, omega_m: float = 0.3) -> np.ndarray:
    """grf_phi (FP32) memoised on disk under $RR_CACHE (default: the system
    temporary directory), so that repeated runs on one machine draw it once."""
    import os
    import tempfile
    root = os.environ.get("RR_CACHE", os.path.join(tempfile.gettempdir(), "rr_cache"))
    os.makedirs(root, exist_ok=True)
    path = os.path.join(root, f"grf_n{n}_L{box:g}_s{seed}_om{omega_m:g}.npy")
    if os.path.exists(path):
        return np.load(path)
    phi = grf_phi(n, box, seed, omega_m)
    tmp = path + f".{os.getpid()}.tmp.npy"
    np.save(tmp, phi)
    os.replace(tmp, path)
    return phi


def grf_phi_torch(n: int, box: float, seed: int, device="cuda", omega_m: float = 0.3,
                  spectral_index: float = -3.0, rms_delta: float = 1.0):
    """The grf_phi recipe (same spectrum, cut and normalisation) drawn and
    transformed on a torch device: white noise from torch.Generator(seed)
    (Philox on CUDA), FP64 FFTs, FP32 result. Deterministic for a seed on a
    given device type; its values differ from grf_phi's (another generator)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    white = torch.randn((n, n, n), generator=gen, device=device, dtype=torch.float64)
    wk = torch.fft.rfftn(white)
    del white
    k1 = 2.0 * math.pi * torch.fft.fftfreq(n, d=box / n, device=device, dtype=torch.float64)
    kz = 2.0 * math.pi * torch.fft.rfftfreq(n, d=box / n, device=device, dtype=torch.float64)
    k2 = k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + kz[None, None, :] ** 2
    knyq = math.pi * n / box
    live = (k2 > 0) & (k2 <= knyq * knyq)
    shape = torch.where(live, k2.clamp_min(1e-300) ** (0.25 * spectral_index), torch.zeros_like(k2))
    if n % 2 == 0:
        shape[n // 2, :, :] = 0.0
        shape[:, n // 2, :] = 0.0
        shape[:, :, -1] = 0.0
    wk *= shape
    del shape, live
    dk = torch.fft.irfftn(-k2 * wk, s=(n, n, n))
    pref = 1.5 * omega_m * H0_OVER_C ** 2
    rms = float(torch.sqrt(torch.mean((dk / pref) ** 2)))
    del dk
    phi = torch.fft.irfftn(wk, s=(n, n, n))
    del wk, k2
    phi *= rms_delta / rms
    return phi.to(torch.float32).contiguous()


@dataclass
class Cone:
    """One lightcone of a batch: its grid, bundle and field seed."""
    grid: Grid
    bundle: Bundle
    field_seed: int


def batch_workload(n: int = 64, seed: int = 4, sizes=(128, 256, 512), rays=(256, 2048),
                   fov_deg=(1.0, 10.0), chi_s=(200.0, 1000.0)) -> list:
    """Independent lightcones of uneven sizes: grid side drawn uniformly from
    `sizes`, box side = chi_s (observer at the centre of the z = 0 face, one
    step from chi_s to 0), ray-grid side log-uniform in `rays` rounded to a
    multiple of 32, field of view uniform in `fov_deg`, chi_s uniform in
    `chi_s`; all from numpy's PCG64(seed); cone i's field seed is 1000 + i."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cones = []
    for i in range(n):
        ng = int(rng.choice(np.asarray(sizes)))
        side = int(round(math.exp(rng.uniform(math.log(rays[0]), math.log(rays[1]))) / 32.0)) * 32
        side = max(32, side)
        fov = deg(float(rng.uniform(*fov_deg)))
        cs = float(rng.uniform(*chi_s))
        g = Grid((ng, ng, ng), cs)
        b = Bundle(side, side, fov, fov, (cs / 2.0, cs / 2.0, 0.0), cs)
        cones.append(Cone(g, b, 1000 + i))
    return cones


# ---------------------------------------------------------------------------
# Adaptive meshes (an octree over a periodic coarse grid)
# ---------------------------------------------------------------------------

@dataclass
class AmrMesh:
    """An octree mesh: an n^3 periodic coarse grid (level 0, cell size
    h0 = box/n) whose cells may be refined into octs of 8 children, down to
    level lmax (cell size h0 / 2^l).

    octs[l] (l = 1..lmax): int32 array (m_l, 3) of the level-(l-1) cells that
    are refined, in level-(l-1) integer coordinates, sorted lexicographically;
    each is the parent of the 8 level-l cells 2 (i,j,k) + (dx, dy, dz),
    child index dx + 2 dy + 4 dz. Neighbouring leaves differ by at most one
    level across faces, edges and corners (2:1 balance).
    phi[l]: level 0 an (n, n, n) array, level l >= 1 an (m_l, 8) array: the
    potential at every cell centre of that level (leaves and parents)."""
    n: int
    box: float
    lmax: int
    octs: list
    phi: list = None
    omega_m: float = 0.3

    def h(self, level: int) -> float:
        return self.box / self.n / (1 << level)

    def nleaves(self) -> int:
        total = self.n ** 3
        for l in range(1, self.lmax + 1):
            total += 7 * len(self.octs[l])
        return total


def _neighbours26(cells: np.ndarray, m: int) -> np.ndarray:
    offs = np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)], np.int64)
    return ((cells[:, None, :] + offs[None, :, :]) % m).reshape(-1, 3)


def _unique_rows(a: np.ndarray) -> np.ndarray:
    if len(a) == 0:
        return a.reshape(0, 3).astype(np.int32)
    return np.unique(a.astype(np.int64), axis=0).astype(np.int32)


def amr_balance(n: int, lmax: int, flags: list) -> list:
    """From refinement flags flags[l] (level-l cells to refine, l = 0..lmax-1)
    build a 2:1-balanced octree: a refined level-l cell needs its parent's 26
    neighbours refined (so its own neighbours exist), applied bottom-up; cells
    whose parent is not refined are dropped, top-down. Returns octs[0..lmax]
    (octs[0] unused)."""
    fl = [_unique_rows(np.asarray(f).reshape(-1, 3)) for f in flags] + [np.zeros((0, 3), np.int32)]
    for l in range(lmax - 1, 0, -1):
        if len(fl[l]) == 0:
            continue
        parents = fl[l] // 2
        fl[l - 1] = _unique_rows(np.concatenate([fl[l - 1], _neighbours26(parents, n << (l - 1)),
                                                 parents]))
    octs = [np.zeros((0, 3), np.int32)]
    for l in range(1, lmax + 1):
        cand = fl[l - 1]
        if l >= 2 and len(cand):
            # keep only cells that exist: their parent is refined
            m = np.int64(n << (l - 2))
            have = octs[l - 1].astype(np.int64)
            par = (cand // 2).astype(np.int64)
            keep = np.isin((par[:, 0] * m + par[:, 1]) * m + par[:, 2], (have[:, 0] * m + have[:, 1]) * m + have[:, 2])
            cand = cand[keep]
        octs.append(cand.astype(np.int32))
    return octs


def amr_nested_cubes(n: int, box: float, lmax: int, half_widths) -> AmrMesh:
    """Hierarchically nested cubic refinements around the box centre (the
    paper's Gaussian test, Sec. 4): a level-l cell is refined when its centre
    lies within half_widths[l] (Mpc/h) of the centre along every axis."""
    flags = []
    c = box / 2.0
    for l in range(lmax):
        m = n << l
        h = box / m
        x = (np.arange(m) + 0.5) * h
        inside = np.nonzero(np.abs(x - c) < half_widths[l])[0]
        if len(inside) == 0:
            flags.append(np.zeros((0, 3), np.int32))
            continue
        g = np.stack(np.meshgrid(inside, inside, inside, indexing="ij"), -1).reshape(-1, 3)
        flags.append(g.astype(np.int32))
    return AmrMesh(n, box, lmax, amr_balance(n, lmax, flags))


_KIDS = np.array([(i & 1, (i >> 1) & 1, (i >> 2) & 1) for i in range(8)], np.int64)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea & Flood 2014) on uint64 arrays."""
    x = x + np.uint64(0x9E3779B97F4A7C15)
    x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return x ^ (x >> np.uint64(31))


def _hash_normal(level: int, cells: np.ndarray, seed: int) -> np.ndarray:
    """One standard normal per level-l cell (rows of integer coordinates), a
    pure function of (seed, level, coordinates): SplitMix64 over the key, two
    53-bit uniforms, Box-Muller. Independent of the order cells are visited."""
    with np.errstate(over="ignore"):
        h = _splitmix64(np.full(len(cells), (np.uint64(seed) << np.uint64(8)) ^ np.uint64(level), np.uint64))
        for a in range(3):
            h = _splitmix64(h ^ cells[:, a].astype(np.uint64))
        h2 = _splitmix64(h ^ np.uint64(0xD1B54A32D192ED03))
    u1 = ((h >> np.uint64(11)).astype(np.float64) + 0.5) / 9007199254740992.0
    u2 = (h2 >> np.uint64(11)).astype(np.float64) / 9007199254740992.0
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def _cascade(level: int, parents: np.ndarray, rho_parent: np.ndarray, seed: int, child_sigma: float):
    """Children (m, 8, 3) of level-(l-1) cells and their densities (m, 8):
    rho_parent times lognormal factors of rms child_sigma normalised to mean 1
    over the 8 siblings (mass conserving)."""
    child = 2 * parents.astype(np.int64)[:, None, :] + _KIDS[None]
    f = np.exp(child_sigma * _hash_normal(level, child.reshape(-1, 3), seed)).reshape(-1, 8)
    f /= f.mean(axis=1, keepdims=True)
    return child, rho_parent[:, None] * f


def _lognormal_coarse(n: int, box: float, seed: int, sigma_ln: float) -> np.ndarray:
    """rho = exp(g - sigma^2/2) on the n^3 grid, g Gaussian with P_g propto
    k^-2 and rms sigma_ln (numpy PCG64(seed) white noise, FP64 FFTs)."""
    import scipy.fft as sfft
    rng = np.random.Generator(np.random.PCG64(seed))
    wk = sfft.rfftn(rng.standard_normal((n, n, n)), workers=-1)
    k1, kz = _kgrid(n, box)
    k2 = k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + kz[None, None, :] ** 2
    shape = np.where(k2 > 0, 1.0 / np.sqrt(np.maximum(k2, 1e-300)), 0.0)
    g = sfft.irfftn(wk * shape, s=(n, n, n), workers=-1)
    g *= sigma_ln / g.std()
    return np.exp(g - 0.5 * sigma_ln ** 2)


def amr_random(n: int, box: float, lmax: int, seed: int, sigma_ln: float = 1.5, child_sigma: float = 0.5,
               threshold: float = 8.0) -> AmrMesh:
    """Refinement driven by a lognormal density: rho = exp(g - sigma^2/2) on
    the coarse grid (g Gaussian, P_g propto k^-2, rms sigma_ln), passed to the
    children by a multiplicative cascade (lognormal factors of rms child_sigma,
    a hash of the seed, level and cell, normalised to mean 1 over the 8
    siblings); a level-l cell is refined when its mass rho (h_l/h_0)^3 exceeds
    `threshold` times the mean cell mass of level 0; then 2:1 balanced."""
    rho = _lognormal_coarse(n, box, seed, sigma_ln)
    cells = np.stack(np.nonzero(rho > threshold), -1).astype(np.int64)
    rho_cells = rho[tuple(cells.T)]
    flags = [cells.astype(np.int32)]
    for l in range(1, lmax):
        if len(cells) == 0:
            flags.append(np.zeros((0, 3), np.int32))
            continue
        child, rho_child = _cascade(l, cells, rho_cells, seed, child_sigma)
        child, rho_child = child.reshape(-1, 3), rho_child.reshape(-1)
        sel = rho_child / 8.0 ** l > threshold
        cells, rho_cells = child[sel], rho_child[sel]
        flags.append(cells.astype(np.int32))
    return AmrMesh(n, box, lmax, amr_balance(n, lmax, flags))


def _level_keys(mesh: AmrMesh, l: int):
    """Integer coordinates (m_l * 8, 3) of every level-l cell in cell order,
    and their periodic keys."""
    m = np.int64(mesh.n << l)
    if l == 0:
        ii = np.arange(mesh.n, dtype=np.int64)
        c = np.stack(np.meshgrid(ii, ii, ii, indexing="ij"), -1).reshape(-1, 3)
    else:
        c = (2 * mesh.octs[l].astype(np.int64)[:, None, :] + _KIDS[None]).reshape(-1, 3)
    return c, (c[:, 0] * m + c[:, 1]) * m + c[:, 2]


def _lookup(keys_sorted, order, m, c):
    """Cell-order index of the level cells at coordinates c (periodic), -1 where absent."""
    c = np.mod(c, m)
    k = (c[..., 0] * m + c[..., 1]) * m + c[..., 2]
    pos = np.clip(np.searchsorted(keys_sorted, k), 0, len(keys_sorted) - 1)
    hit = keys_sorted[pos] == k
    return np.where(hit, order[pos], -1)


def amr_density(mesh: AmrMesh, seed: int, sigma_ln: float = 1.5, child_sigma: float = 0.5) -> list:
    """The density of amr_random(seed, sigma_ln, child_sigma) at every cell of
    every level of the mesh: level 0 (n, n, n), level l (m_l, 8)."""
    rho0 = _lognormal_coarse(mesh.n, mesh.box, seed, sigma_ln)
    out = [rho0]
    flat_prev = rho0.reshape(-1)
    keys_prev = None
    for l in range(1, mesh.lmax + 1):
        par = mesh.octs[l].astype(np.int64)
        if l == 1:
            rp = rho0[tuple(par.T)]
        else:
            ks, order = keys_prev
            idx = _lookup(ks, order, np.int64(mesh.n << (l - 1)), par)
            rp = flat_prev[idx]
        _, rho_l = _cascade(l, par, rp, seed, child_sigma)
        out.append(rho_l)
        flat_prev = rho_l.reshape(-1)
        _, k = _level_keys(mesh, l)
        order = np.argsort(k, kind="stable")
        keys_prev = (k[order], order)
    return out


def amr_potential(mesh: AmrMesh, rho: list, omega_m: float = 0.3, sweeps: int = 8) -> list:
    """Phi/c^2 at every cell of every level from the density (comoving Poisson
    equation at a = 1, lap Phi = 1.5 Omega_m (H0/c)^2 delta, delta = rho /
    mean(rho_0) - 1). Level 0: FFT solve with the eigenvalues of the 7-point
    Laplacian. Level l >= 1: the coarser level's Phi interpolated trilinearly
    from the 8 nearest coarser centres, then `sweeps` red-black Gauss-Seidel
    sweeps of the 7-point equation on the cells whose 6 face neighbours exist
    at that level (the others keep the interpolated value: Dirichlet)."""
    import scipy.fft as sfft
    n, box = mesh.n, mesh.box
    pref = 1.5 * omega_m * H0_OVER_C ** 2
    mean0 = float(rho[0].mean())
    d0 = rho[0] / mean0 - 1.0
    h0 = box / n
    k1, kz = _kgrid(n, box)
    lam = ((2.0 - 2.0 * np.cos(k1 * h0))[:, None, None] + (2.0 - 2.0 * np.cos(k1 * h0))[None, :, None]
           + (2.0 - 2.0 * np.cos(kz * h0))[None, None, :]) / (h0 * h0)
    dk = sfft.rfftn(d0, workers=-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        pk = np.where(lam > 0, -pref * dk / lam, 0.0)
    phi = [sfft.irfftn(pk, s=(n, n, n), workers=-1)]
    prev_flat = phi[0].reshape(-1)
    _, k0 = _level_keys(mesh, 0)
    prev = (k0, np.arange(len(k0)))   # level 0 keys are already sorted
    faces = np.array([(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)], np.int64)
    for l in range(1, mesh.lmax + 1):
        c, k = _level_keys(mesh, l)
        if len(c) == 0:
            phi.append(np.zeros((0, 8)))
            continue
        m_prev = np.int64(n << (l - 1))
        # trilinear from the coarser level: centre x/2 - 1/4 in coarse-centre units
        lo = np.where(c % 2 == 0, c // 2 - 1, (c - 1) // 2)
        fr = np.where(c % 2 == 0, 0.75, 0.25)
        val = np.zeros(len(c))
        for t in range(8):
            d = _KIDS[t]
            idx = _lookup(prev[0], prev[1], m_prev, lo + d[None])
            if np.any(idx < 0):
                raise ValueError("amr_potential: mesh is not 2:1 balanced")
            w = np.prod(np.where(d[None] == 1, fr, 1.0 - fr), axis=1)
            val += w * prev_flat[idx]
        order = np.argsort(k, kind="stable")
        ks = k[order]
        m = np.int64(n << l)
        nb = np.stack([_lookup(ks, order, m, c + f[None]) for f in faces], 1)
        inner = np.all(nb >= 0, axis=1)
        hl = box / float(m)
        src = (hl * hl * pref) * (rho[l].reshape(-1) / mean0 - 1.0)
        colour = (c.sum(axis=1) % 2)
        for _ in range(sweeps):
            for col in (0, 1):
                sel = np.nonzero(inner & (colour == col))[0]
                val[sel] = (val[nb[sel]].sum(axis=1) - src[sel]) / 6.0
        phi.append(val.reshape(-1, 8))
        prev_flat = val
        prev = (ks, order)
    return phi


def amr_cell_centres(mesh: AmrMesh, level: int) -> np.ndarray:
    """Cell centres of a level: (n,n,n,3) for level 0, (m,8,3) for octs."""
    h = mesh.h(level)
    if level == 0:
        x = (np.arange(mesh.n) + 0.5) * h
        return np.stack(np.meshgrid(x, x, x, indexing="ij"), -1)
    kids = np.array([(i & 1, (i >> 1) & 1, (i >> 2) & 1) for i in range(8)], np.float64)
    base = 2.0 * mesh.octs[level].astype(np.float64)
    return (base[:, None, :] + kids[None] + 0.5) * h


def amr_sample(mesh: AmrMesh, fn) -> list:
    """phi[l] = fn(centres) for every level (fn maps (..., 3) positions to values)."""
    return [np.ascontiguousarray(fn(amr_cell_centres(mesh, l))) for l in range(mesh.lmax + 1)]


def gaussian_fn(amp: float, sigma: float, centre):
    c = np.asarray(centre, np.float64)

    def f(p):
        d = p - c
        return amp * np.exp(-np.sum(d * d, axis=-1) / (2.0 * sigma * sigma))
    return f


def fourier_fn(box: float, nmodes: int, kmax: float, seed: int, spectral_index: float = -3.0,
               omega_m: float = 0.3, rms_delta: float = 1.0):
    """A smooth periodic random potential: sum of nmodes plane waves
    a_k cos(k.x + p_k) with integer wave vectors (periodic in the box),
    |k| <= kmax, a_k^2 propto |k|^spectral_index, scaled so that the
    continuum delta = -lap(Phi)/(1.5 Om (H0/c)^2) has the requested rms."""
    rng = np.random.Generator(np.random.PCG64(seed))
    kf = 2.0 * math.pi / box
    mmax = int(kmax / kf)
    ks, amps = [], []
    while len(ks) < nmodes:
        m = rng.integers(-mmax, mmax + 1, size=3)
        kk = kf * m.astype(np.float64)
        kn = float(np.sqrt(kk @ kk))
        if kn == 0.0 or kn > kmax:
            continue
        ks.append(kk)
        amps.append(kn ** (0.5 * spectral_index) * rng.standard_normal())
    ks = np.array(ks)
    amps = np.array(amps)
    ph = rng.uniform(0, 2 * math.pi, nmodes)
    pref = 1.5 * omega_m * H0_OVER_C ** 2
    var = 0.5 * np.sum((amps * np.sum(ks * ks, axis=1) / pref) ** 2)
    amps *= rms_delta / math.sqrt(var)

    def f(p):
        out = np.zeros(p.shape[:-1])
        for i in range(nmodes):
            out += amps[i] * np.cos(p @ ks[i] + ph[i])
        return out
    return f


# ---------------------------------------------------------------------------
# Adaptive-mesh workloads
# ---------------------------------------------------------------------------

@dataclass
class AmrWorkload:
    name: str
    n: int
    box: float
    lmax: int
    seed: int
    sigma_ln: float
    child_sigma: float
    threshold: float
    bundle: Bundle
    nsteps: int
    rescale: bool = True


def amr_workload(name: str) -> AmrWorkload:
    """Named adaptive-mesh workloads (lognormal density, sigma_ln = 1.5, cascade
    child_sigma = 0.5, refinement where the cell mass exceeds 8x the mean,
    Phi by amr_potential; equal-Delta-a steps with Phi rescaled by D(a)/a).

    amr_256: 256^3 coarse grid, box 512 Mpc/h, up to 4 extra levels (about
        21.7M leaves), 4096 x 4096 rays over 5 x 5 deg to chi_s = 500, 32 steps.
    amr_128: 128^3 coarse grid, box 256, up to 4 levels, 1024 x 1024 rays over
        5 x 5 deg to chi_s = 250, 8 steps (profiling case: leaf records larger
        than L2, about 1 GB on the device).
    """
    if name == "amr_256":
        b = Bundle(4096, 4096, deg(5.0), deg(5.0), (256.0, 256.0, 0.0), 500.0)
        return AmrWorkload(name, 256, 512.0, 4, 8, 1.5, 0.5, 8.0, b, 32)
    if name == "amr_128":
        b = Bundle(1024, 1024, deg(5.0), deg(5.0), (128.0, 128.0, 0.0), 250.0)
        return AmrWorkload(name, 128, 256.0, 4, 9, 1.5, 0.5, 8.0, b, 8)
    raise KeyError(name)


def amr_workload_mesh(w: AmrWorkload, omega_m: float = 0.3):
    """(mesh with FP64 phi per level, flat FP32 phi in cell order) of an
    adaptive-mesh workload, memoised on disk under $RR_CACHE like
    grf_phi_cached."""
    import os
    import tempfile
    root = os.environ.get("RR_CACHE", os.path.join(tempfile.gettempdir(), "rr_cache"))
    os.makedirs(root, exist_ok=True)
    path = os.path.join(root, f"amr_{w.n}_L{w.box:g}_l{w.lmax}_s{w.seed}_t{w.threshold:g}_v2.npz")
    if os.path.exists(path):
        z = np.load(path)
        octs = [np.zeros((0, 3), np.int32)] + [z[f"octs{l}"] for l in range(1, w.lmax + 1)]
        mesh = AmrMesh(w.n, w.box, w.lmax, octs, omega_m=omega_m)
        flat = z["phi"]
    else:
        mesh = amr_random(w.n, w.box, w.lmax, w.seed, w.sigma_ln, w.child_sigma, w.threshold)
        mesh.omega_m = omega_m
        rho = amr_density(mesh, w.seed, w.sigma_ln, w.child_sigma)
        phi = amr_potential(mesh, rho, omega_m)
        flat = np.concatenate([np.asarray(p, np.float64).reshape(-1) for p in phi]).astype(np.float32)
        tmp = path + f".{os.getpid()}.tmp.npz"
        np.savez(tmp, phi=flat, **{f"octs{l}": mesh.octs[l] for l in range(1, w.lmax + 1)})
        os.replace(tmp, path)
    # per-level FP64 copies of the FP32 values (what both sides read)
    parts, off = [], 0
    sizes = [w.n ** 3] + [8 * len(mesh.octs[l]) for l in range(1, w.lmax + 1)]
    for l, sz in enumerate(sizes):
        p = flat[off:off + sz].astype(np.float64)
        parts.append(p.reshape(w.n, w.n, w.n) if l == 0 else p.reshape(-1, 8))
        off += sz
    mesh.phi = parts
    return mesh, flat
