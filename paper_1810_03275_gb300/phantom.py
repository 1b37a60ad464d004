"""Seeded synthetic inputs: ellipse phantoms with metal disks, their exact
parallel-beam line integrals, noise, and the metal-trace mask.

This module is the one piece shared by the CUDA path's tests/benchmarks and the
CPU oracle.  It holds none of the reconstruction method's arithmetic: the
sinogram is the *continuous* line integral of the piecewise-constant phantom
(what a scanner measures, computed exactly from the ellipse/ray intersections),
not the discrete operator R_h, so the data carry a realistic model mismatch.

Stand-ins for the thesis's data (its Shepp-Logan, walnut and scanner sets are not
used): 0-1 ellipse phantoms, metal disks of value 10, 1 % Gaussian or 1e5-photon
Poisson noise.  All randomness comes from numpy's PCG64 with an explicit seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class Ellipse:
    cx: float
    cy: float
    a: float      # semi-axis along the rotated x axis
    b: float      # semi-axis along the rotated y axis
    phi: float    # rotation (radians)
    value: float


@dataclass
class Phantom:
    n: int
    h: float
    tissue: List[Ellipse] = field(default_factory=list)
    metal: List[Ellipse] = field(default_factory=list)

    @property
    def all(self) -> List[Ellipse]:
        return list(self.tissue) + list(self.metal)


def pixel_centres(n: int, h: float = 1.0) -> np.ndarray:
    """Centred pixel grid: x_i = h (i - (n-1)/2), i = 0..n-1."""
    return h * (np.arange(n, dtype=np.float64) - 0.5 * (n - 1))


def random_phantom(n: int, n_ellipses: int, seed: int, h: float = 1.0,
                   n_metal: int = 0, metal_radius=(4.0, 10.0), metal_value: float = 10.0) -> Phantom:
    """K ellipses: centres uniform in the disk of radius 0.6 n h/2, semi-axes
    U[0.05, 0.4] n h/2, rotation U[0, pi), value U[0, 1]; painted in order (a
    later ellipse overwrites).  Then ``n_metal`` disks of radius U[metal_radius]
    (pixels) and value ``metal_value`` with centres in the disk of radius
    0.35 n h/2, painted last."""
    rng = np.random.Generator(np.random.PCG64(seed))
    R = 0.5 * n * h
    tissue = []
    for _ in range(n_ellipses):
        r = 0.6 * R * np.sqrt(rng.uniform())
        t = rng.uniform(0.0, 2.0 * np.pi)
        a = rng.uniform(0.05, 0.4) * R
        b = rng.uniform(0.05, 0.4) * R
        tissue.append(Ellipse(r * np.cos(t), r * np.sin(t), a, b, rng.uniform(0.0, np.pi), rng.uniform(0.0, 1.0)))
    metal = []
    for _ in range(n_metal):
        r = 0.35 * R * np.sqrt(rng.uniform())
        t = rng.uniform(0.0, 2.0 * np.pi)
        rad = rng.uniform(*metal_radius) * h
        metal.append(Ellipse(r * np.cos(t), r * np.sin(t), rad, rad, 0.0, metal_value))
    return Phantom(n, h, tissue, metal)


def _inside(e: Ellipse, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    c, s = np.cos(e.phi), np.sin(e.phi)
    dx, dy = x - e.cx, y - e.cy
    qx = c * dx + s * dy
    qy = -s * dx + c * dy
    return (qx / e.a) ** 2 + (qy / e.b) ** 2 <= 1.0


def rasterize(ph: Phantom, which: str = "all") -> np.ndarray:
    """Pixel-centre inclusion image u[i, j] (i <-> x, j <-> y), later shapes overwrite."""
    xs = pixel_centres(ph.n, ph.h)
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    u = np.zeros((ph.n, ph.n))
    shapes = {"all": ph.all, "tissue": ph.tissue, "metal": ph.metal}[which]
    for e in shapes:
        u[_inside(e, X, Y)] = e.value
    return u


def bin_centres(n_bins: int, ds: float = 1.0) -> np.ndarray:
    """Detector bin centres s_k = (k - (M-1)/2) ds."""
    return ds * (np.arange(n_bins, dtype=np.float64) - 0.5 * (n_bins - 1))


def _chords(e: Ellipse, s: np.ndarray, ct: np.ndarray, st: np.ndarray):
    """Entry/exit parameters t1 <= t2 of the rays {s (cos, sin) + t (-sin, cos)}
    through the ellipse (NaN where the ray misses)."""
    c, sn = np.cos(e.phi), np.sin(e.phi)
    px, py = s * ct - e.cx, s * st - e.cy        # ray point at t = 0, relative to the centre
    dx, dy = -st, ct                             # ray direction
    qx0, qy0 = c * px + sn * py, -sn * px + c * py
    qdx, qdy = c * dx + sn * dy, -sn * dx + c * dy
    A = (qdx / e.a) ** 2 + (qdy / e.b) ** 2
    B = 2.0 * (qx0 * qdx / e.a ** 2 + qy0 * qdy / e.b ** 2)
    C = (qx0 / e.a) ** 2 + (qy0 / e.b) ** 2 - 1.0
    disc = B * B - 4.0 * A * C
    ok = disc > 0.0
    sq = np.sqrt(np.where(ok, disc, 0.0))
    t1 = np.where(ok, (-B - sq) / (2.0 * A), np.nan)
    t2 = np.where(ok, (-B + sq) / (2.0 * A), np.nan)
    return t1, t2


def line_integrals(ph: Phantom, theta: np.ndarray, n_bins: int, ds: float = 1.0,
                   which: str = "all") -> np.ndarray:
    """Exact line integrals f[l, k] of the painted (overwrite) phantom along the
    ray at angle theta_l and detector offset s_k: along each ray the phantom is
    piecewise constant between ellipse boundary crossings, and each segment takes
    the value of the last-painted shape containing it."""
    theta = np.asarray(theta, dtype=np.float64)
    chunk = max(1, 2_000_000 // max(n_bins * max(len(ph.all), 1), 1))
    if theta.shape[0] > chunk:
        return np.concatenate([line_integrals(ph, theta[a:a + chunk], n_bins, ds, which)
                               for a in range(0, theta.shape[0], chunk)], axis=0)
    shapes = {"all": ph.all, "tissue": ph.tissue, "metal": ph.metal}[which]
    s = bin_centres(n_bins, ds)[None, :]
    ct = np.cos(theta)[:, None]
    st = np.sin(theta)[:, None]
    shape = (theta.shape[0], n_bins)
    if not shapes:
        return np.zeros(shape)
    t1s, t2s = [], []
    for e in shapes:
        t1, t2 = _chords(e, s, ct, st)
        t1s.append(np.broadcast_to(t1, shape))
        t2s.append(np.broadcast_to(t2, shape))
    T1 = np.stack(t1s, -1)
    T2 = np.stack(t2s, -1)
    pts = np.sort(np.concatenate([T1, T2], -1), axis=-1)     # NaNs sort last
    vals = np.array([e.value for e in shapes])
    total = np.zeros(shape)
    for q in range(pts.shape[-1] - 1):
        lo, hi = pts[..., q], pts[..., q + 1]
        seg = hi - lo
        good = np.isfinite(seg) & (seg > 0)
        mid = 0.5 * (lo + hi)
        top = np.zeros(shape)
        for kk in range(len(shapes)):
            inside = (mid >= T1[..., kk]) & (mid <= T2[..., kk])
            top = np.where(inside, vals[kk], top)
        total += np.where(good, seg * top, 0.0)
    return total


def metal_trace(ph: Phantom, theta: np.ndarray, n_bins: int, ds: float = 1.0,
                margin_bins: float = 1.0) -> np.ndarray:
    """Rays meeting a metal disk, widened by ``margin_bins`` detector bins (the
    half-width of the linear-interpolation footprint): mask[l, k] = 1 where
    |s_k - (c_x cos + c_y sin)| < r + margin."""
    s = bin_centres(n_bins, ds)[None, :]
    ct = np.cos(np.asarray(theta))[:, None]
    st = np.sin(np.asarray(theta))[:, None]
    mask = np.zeros((len(theta), n_bins), dtype=bool)
    for e in ph.metal:
        sc = e.cx * ct + e.cy * st
        mask |= np.abs(s - sc) < (e.a + margin_bins * ds)
    return mask.astype(np.uint8)


def gaussian_noise(f: np.ndarray, rel: float, seed: int):
    """f + N(0, sigma_n^2) with sigma_n = rel * max|f|.  Returns (noisy, sigma_n)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sigma_n = rel * float(np.max(np.abs(f))) if f.size else 0.0
    return f + sigma_n * rng.standard_normal(f.shape), sigma_n


def poisson_noise(f: np.ndarray, f_tissue_max: float, seed: int, photons: float = 1e5,
                  kappa_target: float = 4.0):
    """Photon-count noise: kappa is set so the thickest tissue-only ray has
    kappa * f = kappa_target; counts ~ Poisson(I0 exp(-kappa f)),
    f_noisy = -log(max(counts, 1)/I0)/kappa.  Returns (noisy, kappa)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    kappa = kappa_target / max(f_tissue_max, 1e-12)
    counts = rng.poisson(photons * np.exp(-kappa * f))
    return -np.log(np.maximum(counts, 1) / photons) / kappa, kappa


@dataclass
class Problem:
    """One synthetic reconstruction problem (inputs of tv_pd_solve)."""
    name: str
    n: int
    n_angles: int
    n_bins: int
    h: float
    ds: float
    theta: np.ndarray
    truth: np.ndarray          # rasterised phantom
    f_clean: np.ndarray        # exact line integrals
    f: np.ndarray              # noisy data
    mask: np.ndarray           # metal trace (uint8, 1 = on trace)
    alpha: float
    delta: float
    iters: int
    dtype: str


def uniform_angles(n_angles: int) -> np.ndarray:
    return np.arange(n_angles, dtype=np.float64) * (np.pi / n_angles)


def make_problem(name: str, n: int, n_angles: int, n_bins: int, *, seed: int, n_ellipses: int = 6,
                 n_metal: int = 0, noise: str = "gaussian", alpha: float = 0.01,
                 delta_sigmas: float = 3.0, iters: int = 200, dtype: str = "f32",
                 h: float = 1.0, ds: float = 1.0) -> Problem:
    theta = uniform_angles(n_angles)
    ph = random_phantom(n, n_ellipses, seed, h=h, n_metal=n_metal)
    truth = rasterize(ph)
    f_clean = line_integrals(ph, theta, n_bins, ds)
    if noise == "gaussian":
        f, sigma_n = gaussian_noise(f_clean, 0.01, seed + 1)
        delta = delta_sigmas * sigma_n
    elif noise == "poisson":
        f_tissue = line_integrals(ph, theta, n_bins, ds, which="tissue")
        f, _ = poisson_noise(f_clean, float(f_tissue.max()), seed + 1)
        mask0 = metal_trace(ph, theta, n_bins, ds).astype(bool)
        resid = (f - f_clean)[~mask0]
        delta = delta_sigmas * float(np.sqrt(np.mean(resid ** 2))) if resid.size else 0.0
    else:
        f, delta = f_clean.copy(), 0.0
    mask = metal_trace(ph, theta, n_bins, ds) if n_metal else np.zeros(f.shape, np.uint8)
    return Problem(name, n, n_angles, n_bins, h, ds, theta, truth, f_clean, f, mask,
                   alpha, delta, iters, dtype)


def config_plain_fp64(seed: int = 1) -> Problem:
    """64x64, 6 ellipses, 90 angles on [0, pi), 95 bins, 1 % Gaussian noise,
    alpha = 0.01, delta = 3 sigma_n, 200 iterations, FP64."""
    return make_problem("plain_fp64_64", 64, 90, 95, seed=seed, n_ellipses=6, noise="gaussian",
                        alpha=0.01, iters=200, dtype="f64")


def config_bf16_2048(seed: int = 5) -> Problem:
    """2048x2048 ellipse phantom with 6 metal disks, 2048 angles, 2897 bins
    (ceil(sqrt(2) 2048)), 1e5-photon Poisson noise, 300 iterations; the projector
    operands are stored in bfloat16."""
    return make_problem("bf16_2048", 2048, 2048, 2897, seed=seed, n_ellipses=10, n_metal=6,
                        noise="poisson", alpha=0.3, iters=300, dtype="bf16")


def config_batched(count: int = 64, seed: int = 11, iters: int = 300, sizes=(256, 384, 512, 768, 1024),
                   views=(180, 1440), n_ellipses: int = 4, n_metal: int = 2):
    """`count` slices of uneven size: n uniform in `sizes`, view count uniform in
    [views[0], views[1]], bins ceil(sqrt(2) n); `n_ellipses` ellipses and `n_metal`
    metal disks each, 1e5-photon Poisson noise; FP32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for s in range(count):
        n = int(sizes[int(rng.integers(0, len(sizes)))])
        N = int(rng.integers(views[0], views[1] + 1))
        M = int(np.ceil(np.sqrt(2.0) * n))
        out.append(make_problem(f"batch_{s}", n, N, M, seed=seed * 1000 + s, n_ellipses=n_ellipses, n_metal=n_metal,
                                noise="poisson", alpha=0.3, iters=iters, dtype="f32"))
    return out


def config_mar_fp32(seed: int = 2, n_metal: Optional[int] = None) -> Problem:
    """512x512 ellipse phantom plus 2-4 metal disks (radius 4-10 px, value 10),
    720 angles, 729 bins, 1e5-photon Poisson noise, metal-trace inequality
    constraint and delta-ball elsewhere, 500 iterations, FP32."""
    if n_metal is None:
        n_metal = int(np.random.Generator(np.random.PCG64(seed + 100)).integers(2, 5))
    return make_problem("mar_fp32_512", 512, 720, 729, seed=seed, n_ellipses=10, n_metal=n_metal,
                        noise="poisson", alpha=0.3, iters=500, dtype="f32")
