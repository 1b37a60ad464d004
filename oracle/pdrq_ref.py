"""FP64 numpy oracle for everything around R_h: the discrete gradient and
divergence, the pointwise resolvents, the inverse-norm Fourier preconditioner,
the impulse-response, circulant and Richardson preconditioners, the power
iterations, Alg. 4 (PDRQS1), Alg. 3 (PDRQS2, unconstrained), Alg. 5 (PDRQS1 with
u >= 0), Alg. 1 (Chambolle-Pock), ADMM with PCG, and the metal-trace estimation.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every function follows
the thesis step by step, with library primitives (numpy FFT) as single steps;
no fusion, no reordering.  Readings of passages where the thesis is silent,
ambiguous or garbled are stated where they are used.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np

from .radon import Geometry, rh_adjoint, rh_forward


# ----------------------------------------------------------------------------
# Sec. 3.1: discrete gradient (forward differences, Neumann) and divergence
# (backward differences, Dirichlet), div_h = -grad_h^*.
# ----------------------------------------------------------------------------
def grad(u: np.ndarray, h: float = 1.0):
    """grad_h u = (d_x u, d_y u): (u[i+1,j]-u[i,j])/h for i < n-1, else 0; the
    same along j.  Sec. 3.1."""
    u = np.asarray(u, dtype=np.float64)
    px = np.zeros_like(u)
    py = np.zeros_like(u)
    px[:-1, :] = (u[1:, :] - u[:-1, :]) / h
    py[:, :-1] = (u[:, 1:] - u[:, :-1]) / h
    return px, py


def div(px: np.ndarray, py: np.ndarray, h: float = 1.0) -> np.ndarray:
    """div_h p = (d_1(p) + d_2(p))/h with d_1 = p_1 at the first row, p_i - p_{i-1}
    inside, -p_{n-1} at the last row (0-based: px[0], px[i]-px[i-1], -px[n-2]);
    d_2 the same along j.  Sec. 3.1.  For n = 1 the gradient is the zero map and
    so is its adjoint."""
    px = np.asarray(px, dtype=np.float64)
    py = np.asarray(py, dtype=np.float64)
    n = px.shape[0]
    d1 = np.zeros_like(px)
    d2 = np.zeros_like(py)
    if n >= 2:
        d1[0, :] = px[0, :]
        d1[1:n - 1, :] = px[1:n - 1, :] - px[0:n - 2, :]
        d1[n - 1, :] = -px[n - 2, :]
        d2[:, 0] = py[:, 0]
        d2[:, 1:n - 1] = py[:, 1:n - 1] - py[:, 0:n - 2]
        d2[:, n - 1] = -py[:, n - 2]
    return (d1 + d2) / h


def tv_norm(u: np.ndarray, h: float = 1.0) -> float:
    """Isotropic ||grad_h u||_1 = sum sqrt(q1^2 + q2^2), Sec. 3.1."""
    px, py = grad(u, h)
    return float(np.sum(np.sqrt(px * px + py * py)))


# ----------------------------------------------------------------------------
# Sec. 4.3 / 4.3.1 / 4.4: inverse-norm preconditioner
#   M^{-1} y = F^{-1}( F(y) * ||xi||_eps / (sigma^2 c + (sigma tau)^2 F(kappa_Delta) ||xi||_eps) )
# Readings: F(kappa_Delta)_{ij} = 4 sin^2(pi i/n) + 4 sin^2(pi j/n) (the printed
# formula repeats i; the closed form of the periodic 5-point stencil has j);
# ||xi|| is the norm of the wrapped signed angular frequency 2 pi (i~, j~)/n,
# i~ in (-n/2, n/2]; eps > 0 is kept in the algorithm (Alg. 4 prints it without
# eps, which would zero the mean mode).
# ----------------------------------------------------------------------------
def lap_symbol(n: int) -> np.ndarray:
    """DFT of the periodic Laplacian stencil kappa_Delta, Sec. 4.3."""
    s = np.sin(np.pi * np.arange(n) / n) ** 2
    return 4.0 * s[:, None] + 4.0 * s[None, :]


def freq_norm(n: int, eps: float) -> np.ndarray:
    """||xi||_eps = sqrt(|xi|^2 + eps^2) on the DFT grid, Sec. 4.3.1."""
    xi = 2.0 * np.pi * np.fft.fftfreq(n)
    return np.sqrt(xi[:, None] ** 2 + xi[None, :] ** 2 + eps * eps)


def precond_symbol(n: int, sigma: float, tau: float, c: float, eps: float) -> np.ndarray:
    """Fourier multiplier of M^{-1} in Alg. 4."""
    nrm = freq_norm(n, eps)
    L = lap_symbol(n)
    return nrm / (sigma * sigma * c + (sigma * tau) ** 2 * L * nrm)


def precond_symbol_nonneg(n: int, sigma: float, tau: float, c: float, eps: float) -> np.ndarray:
    """Fourier multiplier of M^{-1} in Alg. 5 (non-negativity, Sec. "Non-negativity
    constraints"): there T = id + sigma^2 K^*K, so M = id + c sigma^2 F^{-1}(1/||xi||) F
    - (sigma tau)^2 Delta_p and M^{-1} multiplies by
    ||xi|| / (||xi|| + sigma^2 c + (sigma tau)^2 F(kappa_Delta) ||xi||)."""
    nrm = freq_norm(n, eps)
    L = lap_symbol(n)
    return nrm / (nrm + sigma * sigma * c + (sigma * tau) ** 2 * L * nrm)


def impulse_response_kernel_dft(geo: Geometry, floor: float = 1e-3) -> np.ndarray:
    """Sec. "Impulse response preconditioners": the DFT of the point-symmetrised impulse
    response of R_h^* R_h, the approximation s of R_h^* R_h used in place of 1/||xi||.
    Readings: the impulse sits at (n//2, n//2) (for even n the lower right of the middle
    four pixels, as printed; the middle pixel for odd n); "symmetric" is taken as point
    symmetry about it, k(x) = (k~(x) + k~(-x))/2 after moving the impulse to the origin,
    which makes the convolution self-adjoint and the DFT real; the DFT is bounded below by
    floor * its maximum (the thesis is silent on signs; R_h^* R_h is positive
    semidefinite, and its discrete impulse response has small negative DFT values at the
    highest frequencies)."""
    n = geo.n
    c = n // 2
    d = np.zeros((n, n))
    d[c, c] = 1.0
    kt = np.roll(rh_adjoint(rh_forward(d, geo), geo), (-c, -c), axis=(0, 1))
    k = 0.5 * (kt + np.roll(kt[::-1, ::-1], (1, 1), axis=(0, 1)))      # k(x) and k(-x mod n)
    F = np.real(np.fft.fft2(k))
    return np.maximum(F, floor * F.max())


def precond_symbol_from(n: int, sigma: float, tau: float, c: float, s: np.ndarray, nonneg: bool = False) -> np.ndarray:
    """Fourier multiplier of M^{-1} for M = sigma^2 c S - (sigma tau)^2 Delta_p (+ id for Alg.
    5), S the convolution whose DFT is s: s = 1/||xi||_eps gives precond_symbol /
    precond_symbol_nonneg, s = impulse_response_kernel_dft the impulse-response preconditioner."""
    L = lap_symbol(n)
    return 1.0 / ((1.0 if nonneg else 0.0) + sigma * sigma * c * s + (sigma * tau) ** 2 * L)


def precond_apply(y: np.ndarray, symbol: np.ndarray) -> np.ndarray:
    """x = F^{-1}(F(y) * symbol) with the 2-D DFT (numpy FFT as one step)."""
    return np.real(np.fft.ifft2(np.fft.fft2(np.asarray(y, dtype=np.float64)) * symbol))


# ----------------------------------------------------------------------------
# Sec. "Circulant matrix preconditioner": R_h^* R_h and -Delta_h approximated by
# circulant matrices acting on the image flattened to a vector of n^2 entries, and
# inverted with the 1-D DFT F_{h,1} of length n^2.
# Readings: the image u[i, j] is flattened with the first index running fastest,
# t = i + n j (column-major, the order of the thesis's MATLAB arrays); the impulse is
# the same point function as in the impulse-response section, at (n//2, n//2), flat
# index p = n//2 + n (n//2); its response is moved to index 0 (the first column of the
# circulant is the response to the first unit vector) and then symmetrised as
# printed, k_t = (k~_t + k~_{(n^2 - t) mod n^2}) / 2; the Laplace kernel comes from
# -Delta_h delta = -div_h grad_h delta by the same steps; the DFT of k is bounded
# below by 1e-3 of its maximum, as for the impulse-response preconditioner.
# ----------------------------------------------------------------------------
def flatten(u: np.ndarray) -> np.ndarray:
    """Image -> vector, t = i + n j."""
    return np.asarray(u).reshape(-1, order="F")


def unflatten(x: np.ndarray, n: int) -> np.ndarray:
    return np.asarray(x).reshape((n, n), order="F")


def circulant_first_column(response: np.ndarray) -> np.ndarray:
    """The symmetrised first column k of the circulant from the response (n x n) to the
    impulse at (n//2, n//2)."""
    n = response.shape[0]
    p = n // 2 + n * (n // 2)
    kt = np.roll(flatten(response), -p)                    # impulse moved to index 0
    return 0.5 * (kt + kt[(-np.arange(n * n)) % (n * n)])


def circulant_kernel_dft(geo: Geometry, floor: float = 1e-3) -> np.ndarray:
    """F_{h,1}(k), k the symmetrised circulant column of R_h^* R_h (length n^2, real by
    the symmetry), bounded below by floor * its maximum."""
    n = geo.n
    d = np.zeros((n, n))
    d[n // 2, n // 2] = 1.0
    k = circulant_first_column(rh_adjoint(rh_forward(d, geo), geo))
    F = np.real(np.fft.fft(k))
    return np.maximum(F, floor * F.max())


def circulant_laplace_dft(n: int, h: float = 1.0) -> np.ndarray:
    """F_{h,1}(kappa_Delta), kappa_Delta the symmetrised circulant column of -Delta_h."""
    d = np.zeros((n, n))
    d[n // 2, n // 2] = 1.0
    return np.real(np.fft.fft(circulant_first_column(-div(*grad(d, h), h))))


def precond_symbol_circulant(n: int, sigma: float, tau: float, c: float, s1: np.ndarray, lap1: np.ndarray,
                             nonneg: bool = False) -> np.ndarray:
    """1-D multiplier of M^{-1}, M = sigma^2 c C_k + (sigma tau)^2 C_Delta (+ id for Alg. 5)."""
    return 1.0 / ((1.0 if nonneg else 0.0) + sigma * sigma * c * s1 + (sigma * tau) ** 2 * lap1)


def precond_apply_circulant(y: np.ndarray, symbol1: np.ndarray) -> np.ndarray:
    """x = F_{h,1}^{-1}(F_{h,1}(y) * symbol1) on the flattened image."""
    y = np.asarray(y, dtype=np.float64)
    return unflatten(np.real(np.fft.ifft(np.fft.fft(flatten(y)) * symbol1)), y.shape[0])


# ----------------------------------------------------------------------------
# Sec. "Suitable Preconditioners": Richardson, M = m id with m >= ||T||.
# Reading: with T = sigma^2 Rt^* Rt + (sigma tau)^2 (-Delta_h) the constant is taken
# as m = sigma^2 c + (sigma tau)^2 8 / h^2, c >= ||Rt^* Rt|| from the power iteration
# (with S = id) and 8 / h^2 >= ||-Delta_h||, so M - T >= 0 holds term by term.
# ----------------------------------------------------------------------------
def richardson_m(sigma: float, tau: float, c: float, h: float = 1.0, nonneg: bool = False) -> float:
    return (1.0 if nonneg else 0.0) + sigma * sigma * c + (sigma * tau) ** 2 * 8.0 / (h * h)


# ----------------------------------------------------------------------------
# Sec. 3.3 / 3.5: pointwise resolvents.
# Per-bin data term g_r(z) = (w_r/2)(z - a_r)^2 + I_[lo_r, hi_r](z).  By
# Lemma lem_loc the resolvent of sigma*G1^* acts per bin, and by the Moreau
# identity (Sec. 1.3) it is v - sigma * prox_{g_r/sigma}(v/sigma), where the
# prox of a 1-D quadratic plus a box is the clipped unconstrained minimiser:
#     (id + sigma d g_r^*)^{-1}(v) = v - sigma * clip((v + w a)/(sigma + w), lo, hi).
# Special cases reproduce every resolvent printed in Sec. 3.3-3.5 (tested).
# ----------------------------------------------------------------------------
def prox_dual(v, sigma, w, a, lo, hi):
    """Resolvent of sigma * g^* for the box-quadratic data term above."""
    v = np.asarray(v, dtype=np.float64)
    z = (v + w * a) / (sigma + w)
    return v - sigma * np.clip(z, lo, hi)


def tv_project(zx, zy, lam: float, tau: float):
    """Projection onto the pointwise isotropic ball of radius lam/tau:
    z / max(1, tau |z| / lam)  (Alg. 4; Sec. 3.3 for the unscaled ball)."""
    zx = np.asarray(zx, dtype=np.float64)
    zy = np.asarray(zy, dtype=np.float64)
    if lam <= 0.0:
        return np.zeros_like(zx), np.zeros_like(zy)
    den = np.maximum(1.0, tau * np.sqrt(zx * zx + zy * zy) / lam)
    return zx / den, zy / den


def conj_data_term(t, w, a, lo, hi):
    """g_r^*(t) = sup_{lo <= z <= hi} t z - (w/2)(z - a)^2 per bin (Lemma
    lem_f_ast1 and its variants).  +inf where the supremum is unbounded."""
    t = np.asarray(t, dtype=np.float64)
    w = np.broadcast_to(np.asarray(w, dtype=np.float64), t.shape)
    a = np.broadcast_to(np.asarray(a, dtype=np.float64), t.shape)
    lo = np.broadcast_to(np.asarray(lo, dtype=np.float64), t.shape)
    hi = np.broadcast_to(np.asarray(hi, dtype=np.float64), t.shape)
    out = np.empty_like(t)
    pos = w > 0
    with np.errstate(invalid="ignore", divide="ignore"):
        zq = np.clip(a + t / np.where(pos, w, 1.0), lo, hi)
        vq = t * zq - 0.5 * w * (zq - a) ** 2
        zl = np.where(t > 0, hi, np.where(t < 0, lo, 0.0))
        vl = np.where(t == 0, 0.0, t * zl)
    out[pos] = vq[pos]
    out[~pos] = vl[~pos]
    return out


def make_descriptors(f, metal_mask, delta: float, trace_ratio: float = 0.8):
    """Per-bin data term (w, a, lo, hi) of problem (C_h) with the data tolerance:
    off the metal trace  w = 1, a = f, [lo, hi] = [f - delta, f + delta]
    (delta < 0: no box, the thesis's plain quadratic fit);
    on the metal trace   w = 0, lo = C = trace_ratio * f, hi = +inf
    (the inequality constraint R_h u >= C of Sec. 2.2 / 3.2 with the pointwise
    threshold C = 0.8 f of Sec. 5.2)."""
    f = np.asarray(f, dtype=np.float64)
    m = np.asarray(metal_mask).astype(bool) if metal_mask is not None else np.zeros(f.shape, bool)
    w = np.where(m, 0.0, 1.0)
    a = np.where(m, 0.0, f)
    if delta >= 0:
        lo = np.where(m, trace_ratio * f, f - delta)
        hi = np.where(m, np.inf, f + delta)
    else:
        lo = np.where(m, trace_ratio * f, -np.inf)
        hi = np.full(f.shape, np.inf)
    return w, a, lo, hi


# ----------------------------------------------------------------------------
# Sec. 2 (filtered backprojection): the detector-axis ramp filter F_1^{-1} |omega| F_1
# (the Ram-Lak filter) and the filtered backprojection that inverts the Radon transform.
# Readings: the filter is the band-limited ramp sampled in space (the classical Ram-Lak
# kernel k(0) = 1/(4 ds^2), k(m) = -1/(pi^2 m^2 ds^2) for odd m, 0 for even m != 0),
# applied per view as the linear (not circular) convolution ds sum_m k(m) g(k - m) over
# the detector; the backprojection integral over [0, pi) becomes (pi / N) R_h^* (angles
# taken as uniform; the data are line integrals, the thesis's R_h with h = ds = 1).
# ----------------------------------------------------------------------------
def ramlak_kernel(M: int, ds: float = 1.0) -> np.ndarray:
    """k(m) for m = -(M-1) .. M-1 (index m + M - 1)."""
    m = np.arange(-(M - 1), M)
    k = np.zeros(2 * M - 1)
    k[M - 1] = 1.0 / (4.0 * ds * ds)
    odd = (m % 2) != 0
    k[odd] = -1.0 / (np.pi ** 2 * m[odd].astype(np.float64) ** 2 * ds * ds)
    return k


def ramp_filter(g: np.ndarray, ds: float = 1.0) -> np.ndarray:
    """Per view: y(k) = ds sum_{k'} k_RL(k - k') g(k'), k = 0..M-1 (linear convolution)."""
    g = np.asarray(g, dtype=np.float64)
    M = g.shape[1]
    ker = ramlak_kernel(M, ds)
    return np.stack([ds * np.convolve(row, ker)[M - 1:2 * M - 1] for row in g])


def fbp(g: np.ndarray, geo: Geometry) -> np.ndarray:
    """Filtered backprojection (pi / N) R_h^*(ramp_filter(g))."""
    return (np.pi / geo.n_angles) * rh_adjoint(ramp_filter(g, geo.ds), geo)


# ----------------------------------------------------------------------------
# Sec. "Real metal artifacts": estimating the metal trace D_0 from a reconstruction.
# The pixels whose reconstructed value exceeds a threshold are marked, the marks are
# dilated (by 5 px in the thesis's experiment), and the sinogram bins that the marked
# pixels project onto form the trace.  Readings: the thesis says "back projection" for
# the image-to-sinogram step, which is R_h (the forward projection); the dilation uses
# the disk {di^2 + dj^2 <= r^2}; a bin belongs to the trace when R_h of the 0/1 image of
# marked pixels exceeds proj_tol (a bin that no marked pixel touches gets exactly 0).
# ----------------------------------------------------------------------------
def dilate_disk(marked: np.ndarray, radius: int) -> np.ndarray:
    """Binary dilation of a 0/1 image by the disk of the given radius (in pixels)."""
    marked = np.asarray(marked).astype(bool)
    n0, n1 = marked.shape
    out = np.zeros_like(marked)
    r = int(radius)
    for di in range(-r, r + 1):
        for dj in range(-r, r + 1):
            if di * di + dj * dj > r * r:
                continue
            # out[i, j] |= marked[i + di, j + dj] where that pixel exists
            src = marked[max(di, 0):n0 + min(di, 0), max(dj, 0):n1 + min(dj, 0)]
            out[max(-di, 0):n0 + min(-di, 0), max(-dj, 0):n1 + min(-dj, 0)] |= src
    return out


def metal_trace_estimate(u: np.ndarray, geo: Geometry, threshold: float, radius: int = 5,
                         proj_tol: float = 1e-6):
    """(marked image, sinogram trace mask) from a reconstruction u."""
    marked = dilate_disk(np.asarray(u) > threshold, radius)
    trace = rh_forward(marked.astype(np.float64), geo) > proj_tol
    return marked.astype(np.uint8), trace.astype(np.uint8)


# ----------------------------------------------------------------------------
# Sec. 4.3 / 5.1: power iterations.
# beta ~ ||R_h|| (the problem is solved with R_h/beta, f/beta, lambda/beta^2,
# Sec. 5.1); c ~ 1.05 lambda_max(Mt^{-1} Rt^* Rt) with Mt = F^{-1}(1/||xi||_eps) F
# (Sec. 4.3.1), iterated in the symmetric form Mt^{-1/2} Rt^* Rt Mt^{-1/2}.
# Both run a fixed count from the same deterministic start: the R2
# low-discrepancy pattern x_ij = frac(1/2 + i/g + j/g^2) - 1/2 (g the plastic
# number), normalised.  (The all-ones image is orthogonal to the symmetric-broken
# top eigenvectors of these operators and stalls below lambda_max.)
# ----------------------------------------------------------------------------
PLASTIC = 1.32471795724474602596


def power_start(n: int) -> np.ndarray:
    i = np.arange(n, dtype=np.float64)
    x = np.mod(0.5 + i[:, None] / PLASTIC + i[None, :] / (PLASTIC * PLASTIC), 1.0) - 0.5
    nx = np.linalg.norm(x)
    return x / nx if nx > 0 else x


def power_beta(geo: Geometry, iters: int = 50) -> float:
    n = geo.n
    x = power_start(n)
    lam = 0.0
    for _ in range(iters):
        y = rh_adjoint(rh_forward(x, geo), geo)
        lam = float(np.sum(x * y))
        ny = float(np.linalg.norm(y))
        if ny == 0.0:
            return 0.0
        x = y / ny
    return float(np.sqrt(max(lam, 0.0)))


def power_c(geo: Geometry, beta: float, eps: float, iters: int = 50, margin: float = 1.05,
            s: Optional[np.ndarray] = None, circulant: bool = False) -> float:
    """c = margin x the largest eigenvalue of S^{-1/2} Rt^* Rt S^{-1/2} (S the convolution
    with 2-D DFT s; default s = 1/||xi||_eps, Sec. 4.3.1; with circulant=True, S the
    circulant with 1-D DFT s on the flattened image), by power iteration from the R2 start."""
    n = geo.n
    half = np.sqrt(freq_norm(n, eps)) if s is None else 1.0 / np.sqrt(s)

    def mhalf(x):
        if circulant:
            return precond_apply_circulant(x, half)
        return np.real(np.fft.ifft2(np.fft.fft2(x) * half))

    z = power_start(n)
    lam = 0.0
    for _ in range(iters):
        x = mhalf(z)
        y = mhalf(rh_adjoint(rh_forward(x, geo), geo) / (beta * beta))
        lam = float(np.sum(z * y))
        ny = float(np.linalg.norm(y))
        if ny == 0.0:
            return 0.0
        z = y / ny
    return margin * lam


# ----------------------------------------------------------------------------
# Alg. 4 (PDRQS1) for problem (C_h), with K = [R; tau grad] on the scaled problem.
# ----------------------------------------------------------------------------
@dataclass
class PDRQState:
    u: np.ndarray       # primal iterate (original scale of u; u is not rescaled)
    Ru: np.ndarray      # cached Rt u = R_h u / beta (Sec. 4.4: R_h u is saved)
    v1b: np.ndarray     # bar v_1 (sinogram)
    v2bx: np.ndarray    # bar v_2 (two image planes)
    v2by: np.ndarray
    t1: Optional[np.ndarray] = None   # last resolvent outputs (dual certificates)
    t2x: Optional[np.ndarray] = None
    t2y: Optional[np.ndarray] = None
    k: int = 0
    ub: Optional[np.ndarray] = None   # bar u of Alg. 5 (non-negativity); None for Alg. 4

    @staticmethod
    def zeros(geo: Geometry) -> "PDRQState":
        n = geo.n
        return PDRQState(np.zeros((n, n)), np.zeros(geo.sino_shape), np.zeros(geo.sino_shape),
                         np.zeros((n, n)), np.zeros((n, n)))

    def copy(self) -> "PDRQState":
        c = lambda a: None if a is None else a.copy()
        return PDRQState(self.u.copy(), self.Ru.copy(), self.v1b.copy(), self.v2bx.copy(),
                         self.v2by.copy(), c(self.t1), c(self.t2x), c(self.t2y), self.k, c(self.ub))


def pdrq_solve(geo: Geometry, desc, alpha: float, iters: int, *, sigma: float, tau: float,
               eps: float, beta: float, c: float, state: Optional[PDRQState] = None,
               callback=None, symbol: Optional[np.ndarray] = None, circulant: bool = False) -> PDRQState:
    """Run ``iters`` iterations of Alg. 4 on the problem scaled by beta (Sec. 5.1).
    symbol: the multiplier of M^{-1} (default: the inverse-norm one); circulant=True
    applies it with the 1-D DFT of the flattened image (circulant preconditioner).

    desc = (w, a, lo, hi) per bin in the original scale (see make_descriptors).
    One iteration, in the order of Alg. 4:
        u_tmp = -sigma ( Rt^*(v1b + sigma Rt u) - tau div(v2b + sigma tau grad u) )
        u_new = u + F^{-1}( F(u_tmp) * m )
        v1 = v1b + sigma Rt u_new ;  v2 = v2b + sigma tau grad u_new
        t1 = (id + sigma d G1^*)^{-1}(2 v1 - v1b) ;  v1b += t1 - v1
        t2 = P_{lambda/tau}(2 v2 - v2b)           ;  v2b += t2 - v2
        u  = u_new
    with Rt = R_h/beta, lambda = alpha/beta^2 and the bounds of G1 divided by beta.
    """
    h = geo.h
    w, a, lo, hi = (np.asarray(x, dtype=np.float64) for x in desc)
    at, lot, hit = a / beta, lo / beta, hi / beta
    lam = alpha / (beta * beta)
    m = precond_symbol(geo.n, sigma, tau, c, eps) if symbol is None else symbol
    st = PDRQState.zeros(geo) if state is None else state.copy()
    for _ in range(iters):
        y1 = st.v1b + sigma * st.Ru
        gx, gy = grad(st.u, h)
        y2x = st.v2bx + sigma * tau * gx
        y2y = st.v2by + sigma * tau * gy
        u_tmp = -sigma * (rh_adjoint(y1, geo) / beta - tau * div(y2x, y2y, h))
        u_new = st.u + (precond_apply_circulant(u_tmp, m) if circulant else precond_apply(u_tmp, m))
        Ru_new = rh_forward(u_new, geo) / beta
        v1 = st.v1b + sigma * Ru_new
        gx, gy = grad(u_new, h)
        v2x = st.v2bx + sigma * tau * gx
        v2y = st.v2by + sigma * tau * gy
        t1 = prox_dual(2.0 * v1 - st.v1b, sigma, w, at, lot, hit)
        st.v1b = st.v1b + t1 - v1
        t2x, t2y = tv_project(2.0 * v2x - st.v2bx, 2.0 * v2y - st.v2by, lam, tau)
        st.v2bx = st.v2bx + t2x - v2x
        st.v2by = st.v2by + t2y - v2y
        st.u, st.Ru = u_new, Ru_new
        st.t1, st.t2x, st.t2y = t1, t2x, t2y
        st.k += 1
        if callback is not None:
            callback(st)
    return st


def pdrq2_solve(geo: Geometry, f, alpha: float, iters: int, *, sigma: float, tau: float, eps: float,
                beta: float, c: float, state: Optional[PDRQState] = None, symbol: Optional[np.ndarray] = None,
                circulant: bool = False) -> PDRQState:
    """Run ``iters`` iterations of Alg. 3 (PDRQS2) for the unconstrained problem (U_h),
    min 1/2 ||R_h u - f||^2 + alpha ||grad_h u||_1, on the problem scaled by beta.  Only
    the TV term is dualised; the data term stays in the quadratic part, so
    T = sigma Rt^* Rt + (sigma tau)^2 (-Delta_h) and the multiplier of M^{-1} is
    ||xi|| / (sigma c + (sigma tau)^2 L ||xi||).  One iteration, in the order of Alg. 3:
        u_tmp = sigma tau div v2b + sigma Rt^*(ft - Rt u) + (sigma tau)^2 div grad u
        u_new = u + F^{-1}( F(u_tmp) * m )
        v2 = v2b + sigma tau grad u_new
        t2 = P_{lambda/tau}(2 v2 - v2b) ;  v2b += t2 - v2 ;  u = u_new
    Reading: the printed quadratic part carries -(sigma tau)^2 Delta_h u with the
    Laplacian taken as the positive semidefinite -div_h grad_h (so that T >= 0), i.e.
    +(sigma tau)^2 div_h grad_h u here.  symbol / circulant as in pdrq_solve, where the
    symbol passed must already hold sigma c in place of sigma^2 c.  The state's Ru is
    Rt u and t1 = Rt u - ft (the data term's gradient, its optimal dual), so that
    diagnostics() applies with the unconstrained descriptors."""
    h = geo.h
    ft = np.asarray(f, dtype=np.float64) / beta
    lam = alpha / (beta * beta)
    m = precond_symbol(geo.n, sigma, tau, c / sigma, eps) if symbol is None else symbol
    st = PDRQState.zeros(geo) if state is None else state.copy()
    for _ in range(iters):
        gx, gy = grad(st.u, h)
        u_tmp = (sigma * tau * div(st.v2bx, st.v2by, h) + sigma * rh_adjoint(ft - st.Ru, geo) / beta
                 + (sigma * tau) ** 2 * div(gx, gy, h))
        u_new = st.u + (precond_apply_circulant(u_tmp, m) if circulant else precond_apply(u_tmp, m))
        gx, gy = grad(u_new, h)
        v2x = st.v2bx + sigma * tau * gx
        v2y = st.v2by + sigma * tau * gy
        t2x, t2y = tv_project(2.0 * v2x - st.v2bx, 2.0 * v2y - st.v2by, lam, tau)
        st.v2bx = st.v2bx + t2x - v2x
        st.v2by = st.v2by + t2y - v2y
        st.u = u_new
        st.Ru = rh_forward(u_new, geo) / beta
        st.t1, st.t2x, st.t2y = st.Ru - ft, t2x, t2y
        st.k += 1
    return st


def pdrq5_solve(geo: Geometry, desc, alpha: float, iters: int, *, sigma: float, tau: float,
                eps: float, beta: float, c: float, state: Optional[PDRQState] = None,
                callback=None) -> PDRQState:
    """Run ``iters`` iterations of Alg. 5 (PDRQS1 with u >= 0, Sec. "Non-negativity
    constraints") on the problem scaled by beta.  The added term I_{u >= 0} is the
    primal function F of the splitting, with resolvent max(., 0) (Lemma
    lem_resolv_non_neg, d = 0); its effect enters through bar u.  One iteration, in the
    order of Alg. 5:
        u_tmp = bar u - u - sigma ( Rt^*(v1b + sigma Rt u) - tau div(v2b + sigma tau grad u) )
        u_new = u + F^{-1}( F(u_tmp) * m5 ),  m5 = ||xi|| / (||xi|| + sigma^2 c + (sigma tau)^2 L ||xi||)
        v1, v2, t1, t2, v1b, v2b as in Alg. 4
        bar u += max(2 u_new - bar u, 0) - u_new ;  u = u_new
    The data term is the per-bin (w, a, lo, hi) of make_descriptors, as in pdrq_solve."""
    h = geo.h
    w, a, lo, hi = (np.asarray(x, dtype=np.float64) for x in desc)
    at, lot, hit = a / beta, lo / beta, hi / beta
    lam = alpha / (beta * beta)
    m = precond_symbol_nonneg(geo.n, sigma, tau, c, eps)
    st = PDRQState.zeros(geo) if state is None else state.copy()
    if st.ub is None:
        st.ub = np.zeros_like(st.u)
    for _ in range(iters):
        y1 = st.v1b + sigma * st.Ru
        gx, gy = grad(st.u, h)
        y2x = st.v2bx + sigma * tau * gx
        y2y = st.v2by + sigma * tau * gy
        u_tmp = st.ub - st.u - sigma * (rh_adjoint(y1, geo) / beta - tau * div(y2x, y2y, h))
        u_new = st.u + precond_apply(u_tmp, m)
        Ru_new = rh_forward(u_new, geo) / beta
        v1 = st.v1b + sigma * Ru_new
        gx, gy = grad(u_new, h)
        v2x = st.v2bx + sigma * tau * gx
        v2y = st.v2by + sigma * tau * gy
        t1 = prox_dual(2.0 * v1 - st.v1b, sigma, w, at, lot, hit)
        st.v1b = st.v1b + t1 - v1
        t2x, t2y = tv_project(2.0 * v2x - st.v2bx, 2.0 * v2y - st.v2by, lam, tau)
        st.v2bx = st.v2bx + t2x - v2x
        st.v2by = st.v2by + t2y - v2y
        st.ub = st.ub + np.maximum(2.0 * u_new - st.ub, 0.0) - u_new
        st.u, st.Ru = u_new, Ru_new
        st.t1, st.t2x, st.t2y = t1, t2x, t2y
        st.k += 1
        if callback is not None:
            callback(st)
    return st


# ----------------------------------------------------------------------------
# Sec. "Alternating Direction Method of Multipliers" (ADMM with PCG inner solves) for
# the unconstrained problem, on the beta-scaled problem: z = (w, v) = K u with
# K = [Rt; grad_h], f(z) = 1/2 ||w - ft||^2 + lambda ||v||_1, weighting
# Lambda = diag(I, tau I), scaled multiplier eta = (eta_w, eta_v).
# ----------------------------------------------------------------------------
@dataclass
class ADMMState:
    u: np.ndarray
    Ru: np.ndarray      # Rt u
    w: np.ndarray       # z_w (sinogram)
    vx: np.ndarray      # z_v (two image planes)
    vy: np.ndarray
    ew: np.ndarray      # eta_w
    evx: np.ndarray     # eta_v
    evy: np.ndarray
    k: int = 0

    @staticmethod
    def zeros(geo: Geometry) -> "ADMMState":
        n = geo.n
        z = lambda: np.zeros((n, n))
        return ADMMState(z(), np.zeros(geo.sino_shape), np.zeros(geo.sino_shape), z(), z(),
                         np.zeros(geo.sino_shape), z(), z())

    def copy(self) -> "ADMMState":
        return ADMMState(*(getattr(self, f).copy() for f in ("u", "Ru", "w", "vx", "vy", "ew", "evx", "evy")),
                         k=self.k)


def pcg(apply_A, b: np.ndarray, x0: np.ndarray, iters: int, apply_Minv) -> np.ndarray:
    """`iters` steps of the preconditioned conjugate gradient method for A x = b from x0
    (A symmetric positive definite, M^{-1} symmetric positive definite), textbook form;
    stops early only when the preconditioned residual vanishes exactly."""
    x = np.array(x0, dtype=np.float64)
    r = b - apply_A(x)
    z = apply_Minv(r)
    p = z.copy()
    rz = float(np.sum(r * z))
    for _ in range(iters):
        if rz == 0.0:
            break
        Ap = apply_A(p)
        alpha = rz / float(np.sum(p * Ap))
        x = x + alpha * p
        r = r - alpha * Ap
        z = apply_Minv(r)
        rz_new = float(np.sum(r * z))
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x


def soft_threshold2(ux, uy, t: float):
    """argmin_x 1/2 ||x - u||^2 + t ||x|| per pixel (Lemma lem_soft_thres2d): 0 if
    ||u|| <= t, else (1 - t/||u||) u."""
    nrm = np.sqrt(ux * ux + uy * uy)
    fac = np.where(nrm > t, 1.0 - t / np.where(nrm > 0, nrm, 1.0), 0.0)
    return fac * ux, fac * uy


def admm_solve(geo: Geometry, f, alpha: float, iters: int, *, mu: float, tau: float, cg_iters: int,
               beta: float, minv_symbol: np.ndarray, circulant: bool = False,
               state: Optional[ADMMState] = None) -> ADMMState:
    """``iters`` ADMM iterations for min 1/2 ||R_h u - f||^2 + alpha ||grad_h u||_1 (scaled by
    beta).  One iteration, in the thesis's order:
        u   = PCG_{cg_iters}( Rt^* Rt + tau^2 (-Delta_h),  Rt^*(w - eta_w) - tau^2 div_h(v - eta_v) ),
              warm-started at the current u, preconditioned by the multiplier minv_symbol
              (2-D DFT, or the 1-D DFT of the flattened image with circulant=True)
        w   = (ft + mu (Rt u + eta_w)) / (1 + mu)
        v   = soft_threshold(grad_h u + eta_v, lambda / (mu tau^2))
        eta_w -= w - Rt u ;  eta_v -= v - grad_h u
    Readings: the multiplier is the scaled one with step 1 (the printed factor mu belongs
    to the unscaled multiplier); the v-step's weight "mu nu" is mu tau^2, from
    Lambda = diag(I, tau I)."""
    h = geo.h
    ft = np.asarray(f, dtype=np.float64) / beta
    lam = alpha / (beta * beta)
    st = ADMMState.zeros(geo) if state is None else state.copy()
    t2 = tau * tau

    def apply_A(x):
        return rh_adjoint(rh_forward(x, geo) / beta, geo) / beta - t2 * div(*grad(x, h), h)

    def apply_Minv(y):
        return precond_apply_circulant(y, minv_symbol) if circulant else precond_apply(y, minv_symbol)

    for _ in range(iters):
        b = rh_adjoint(st.w - st.ew, geo) / beta - t2 * div(st.vx - st.evx, st.vy - st.evy, h)
        st.u = pcg(apply_A, b, st.u, cg_iters, apply_Minv)
        st.Ru = rh_forward(st.u, geo) / beta
        gx, gy = grad(st.u, h)
        st.w = (ft + mu * (st.Ru + st.ew)) / (1.0 + mu)
        st.vx, st.vy = soft_threshold2(gx + st.evx, gy + st.evy, lam / (mu * t2))
        st.ew = st.ew - (st.w - st.Ru)
        st.evx = st.evx - (st.vx - gx)
        st.evy = st.evy - (st.vy - gy)
        st.k += 1
    return st


def cp_solve(geo: Geometry, desc, alpha: float, iters: int, *, beta: float,
             sigma: Optional[float] = None, tau: Optional[float] = None,
             u0: Optional[np.ndarray] = None, nonneg: bool = False) -> np.ndarray:
    """Alg. 1 (Chambolle-Pock) for problem (C_h) on the same beta-scaled problem,
    used only as an independent minimiser: (C_h) has a unique solution when R_h
    is injective (Sec. 3.2), so Alg. 1 and Alg. 4 must agree there.  Notation of
    Alg. 1: tau is the dual and sigma the primal step, sigma tau (||Rt||^2 + 8/h^2) < 1.
    nonneg: the primal step ends with the projection onto u >= 0 (the resolvent of
    I_{u >= 0}), giving the minimiser of the problem Alg. 5 solves."""
    h = geo.h
    w, a, lo, hi = (np.asarray(x, dtype=np.float64) for x in desc)
    at, lot, hit = a / beta, lo / beta, hi / beta
    lam = alpha / (beta * beta)
    L2 = 1.0 + 8.0 / (h * h)   # ||Rt|| = 1 up to the power-iteration estimate
    if sigma is None or tau is None:
        sigma = tau = 0.99 / np.sqrt(L2 * 1.02)
    n = geo.n
    u = np.zeros((n, n)) if u0 is None else np.array(u0, dtype=np.float64)
    ub = u.copy()
    v = np.zeros(geo.sino_shape)
    wx = np.zeros((n, n))
    wy = np.zeros((n, n))
    for _ in range(iters):
        gx, gy = grad(ub, h)
        wbx, wby = wx + tau * gx, wy + tau * gy
        vb = v + tau * rh_forward(ub, geo) / beta
        wx, wy = tv_project(wbx, wby, lam, 1.0)
        v = prox_dual(vb, tau, w, at, lot, hit)
        u_new = u + sigma * div(wx, wy, h) - sigma * rh_adjoint(v, geo) / beta
        if nonneg:
            u_new = np.maximum(u_new, 0.0)
        ub = 2.0 * u_new - u
        u = u_new
    return u


def diagnostics(geo: Geometry, desc, alpha: float, u: np.ndarray, *, beta: float = 1.0,
                tau: float = 1.0, t1=None, t2x=None, t2y=None) -> dict:
    """Objective of (C_h) in the original scale, its parts, the constraint
    violation, and -- given dual certificates t = (t1, t2) of the beta-scaled
    saddle problem -- the Fenchel-Young gap G(Ku) + G^*(t) - <Ku, t> (box
    indicators left out; they are reported as the violation) and ||K^* t||."""
    w, a, lo, hi = (np.asarray(x, dtype=np.float64) for x in desc)
    Ru = rh_forward(u, geo)
    data = 0.5 * float(np.sum(w * (Ru - a) ** 2))
    tv = tv_norm(u, geo.h)
    viol = float(max(0.0, np.max(lo - Ru, initial=0.0), np.max(Ru - hi, initial=0.0)))
    out = {"objective": data + alpha * tv, "data_fit": data, "tv": tv, "violation": viol}
    if t1 is not None:
        lam = alpha / (beta * beta)
        z = Ru / beta
        at, lot, hit = a / beta, lo / beta, hi / beta
        gz = 0.5 * w * (z - at) ** 2
        g1 = float(np.sum(gz + conj_data_term(t1, w, at, lot, hit) - z * t1))
        gx, gy = grad(u, geo.h)
        g2 = float(np.sum(lam * np.sqrt(gx * gx + gy * gy) - tau * (gx * t2x + gy * t2y)))
        kt = rh_adjoint(t1, geo) / beta - tau * div(t2x, t2y, geo.h)
        out["gap"] = g1 + g2
        out["dual_residual"] = float(np.linalg.norm(kt))
    return out


def pdrq_grad(geo: Geometry, f, mask, delta: float, alpha: float, iters: int, cot_u, *, sigma: float, tau: float,
              eps: float, beta: float, c: float, trace_ratio: float = 0.8):
    """Reverse mode of `iters` iterations of Alg. 4 from zero: the derivatives of
    <cot_u, u_iters> with respect to the data f (through the data term of
    make_descriptors) and to alpha, by the chain rule through each step of the
    iteration in reverse order (beta and c held fixed).  Where clip or the TV
    projection has a kink the inside branch is taken.  Returns (df, dalpha).
    Pinned by central finite differences of pdrq_solve (tests/test_oracle_grad.py)."""
    h = geo.h
    f = np.asarray(f, dtype=np.float64)
    m = np.zeros(f.shape, bool) if mask is None else np.asarray(mask).astype(bool)
    desc = make_descriptors(f, m, delta, trace_ratio)
    w, a, lo, hi = desc
    at, lot, hit = a / beta, lo / beta, hi / beta
    lam = alpha / (beta * beta)
    sym = precond_symbol(geo.n, sigma, tau, c, eps)
    kw = dict(sigma=sigma, tau=tau, eps=eps, beta=beta, c=c)
    states = [PDRQState.zeros(geo)]
    for _ in range(iters):
        states.append(pdrq_solve(geo, desc, alpha, 1, state=states[-1], **kw))
    bu = np.array(cot_u, dtype=np.float64)
    b1 = np.zeros(geo.sino_shape)
    b2x = np.zeros(geo.image_shape)
    b2y = np.zeros(geo.image_shape)
    df = np.zeros(geo.sino_shape)
    dlam = 0.0
    st_ = sigma * tau
    for k in reversed(range(iters)):
        s0, s1 = states[k], states[k + 1]
        # t1 = z1 - sigma clip(q, lo, hi), q = (z1 + w a)/(sigma + w), z1 = v1b + 2 sigma Rt u'
        z1 = s0.v1b + 2.0 * sigma * s1.Ru
        q = (z1 + w * at) / (sigma + w)
        below, above = q < lot, q > hit
        inside = ~(below | above)
        A1 = b1
        dz1 = np.where(inside, A1 * (1.0 - sigma / (sigma + w)), A1)
        da = np.where(inside, -sigma * w / (sigma + w) * A1, 0.0)
        dlo = np.where(below, -sigma * A1, 0.0)
        dhi = np.where(above, -sigma * A1, 0.0)
        df += np.where(m, trace_ratio * dlo, da + dlo + dhi) / beta
        dRu = -sigma * A1 + 2.0 * sigma * dz1
        # t2 = P(z2), z2 = v2b + 2 sigma tau grad u'
        gx, gy = grad(s1.u, h)
        zx, zy = s0.v2bx + 2.0 * st_ * gx, s0.v2by + 2.0 * st_ * gy
        nz = np.sqrt(zx * zx + zy * zy)
        proj = tau * nz > lam
        with np.errstate(invalid="ignore", divide="ignore"):
            nx, ny = np.where(proj, zx / nz, 0.0), np.where(proj, zy / nz, 0.0)
            dot = nx * b2x + ny * b2y
            sc = np.where(proj, lam / (tau * nz), 1.0)
        dx = np.where(proj, sc * (b2x - nx * dot), b2x)
        dy = np.where(proj, sc * (b2y - ny * dot), b2y)
        dlam += float(np.sum(np.where(proj, dot / tau, 0.0)))
        dgx, dgy = -st_ * b2x + 2.0 * st_ * dx, -st_ * b2y + 2.0 * st_ * dy
        # u' = u - sigma P(Rt^* y1 - tau div y2)
        du1 = bu + rh_adjoint(dRu, geo) / beta - div(dgx, dgy, h)
        dr = -sigma * precond_apply(du1, sym)
        dy1 = rh_forward(dr, geo) / beta
        ex, ey = grad(dr, h)
        dy2x, dy2y = tau * ex, tau * ey
        bu = du1 + sigma * rh_adjoint(dy1, geo) / beta - st_ * div(dy2x, dy2y, h)
        b1 = dz1 + dy1
        b2x, b2y = dx + dy2x, dy + dy2y
    return df, dlam / (beta * beta)
