"""Pins of the oracle's grad_h/div_h (Sec. 3.1), the Fourier preconditioner
(Sec. 4.3.1, Alg. 4) and the power iterations, against closed forms and library
routines that do not come from the oracle."""
import numpy as np
import pytest
import scipy.fft
import scipy.linalg

import oracle
from oracle import Geometry


@pytest.mark.parametrize("n,h", [(1, 1.0), (2, 1.0), (7, 1.0), (16, 0.5)])
def test_grad_div_adjoint(n, h):
    """<grad u, p> = -<u, div p> (Sec. 3.1): the two are written from their own
    formulas, so agreement pins both."""
    rng = np.random.default_rng(n)
    u = rng.standard_normal((n, n))
    px, py = rng.standard_normal((2, n, n))
    gx, gy = oracle.grad(u, h)
    lhs = np.sum(gx * px + gy * py)
    rhs = -np.sum(u * oracle.div(px, py, h))
    assert abs(lhs - rhs) <= 1e-12 * (1 + abs(lhs))


def test_grad_of_constant_and_ramp():
    """grad 1 = 0; for u = a i + b j: d_x = a/h except 0 on the last row
    (Neumann), d_y = b/h except 0 on the last column."""
    n, h, a, b = 6, 0.5, 2.0, -3.0
    gx, gy = oracle.grad(np.ones((n, n)), h)
    assert np.all(gx == 0) and np.all(gy == 0)
    I, J = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    gx, gy = oracle.grad(a * I + b * J, h)
    ex = np.full((n, n), a / h); ex[-1, :] = 0
    ey = np.full((n, n), b / h); ey[:, -1] = 0
    np.testing.assert_allclose(gx, ex, atol=1e-12)
    np.testing.assert_allclose(gy, ey, atol=1e-12)


@pytest.mark.parametrize("n", [5, 12])
def test_neumann_laplacian_spectrum_via_dct(n):
    """-div grad is the Neumann 5-point Laplacian, diagonalised by the DCT-II with
    eigenvalues 4 sin^2(pi k/(2n)) + 4 sin^2(pi l/(2n)) (over h^2).  scipy's DCT is
    an independent library routine."""
    h = 1.0
    u = np.random.default_rng(3).standard_normal((n, n))
    gx, gy = oracle.grad(u, h)
    lap = -oracle.div(gx, gy, h)
    k = np.arange(n)
    lam = 4 * np.sin(np.pi * k / (2 * n)) ** 2
    ref = scipy.fft.idctn((lam[:, None] + lam[None, :]) * scipy.fft.dctn(u, norm="ortho"), norm="ortho")
    np.testing.assert_allclose(lap, ref, atol=1e-12)
    # hence ||grad||^2 = max eigenvalue < 8/h^2 (Sec. 3.1)
    assert (2 * lam.max()) < 8


@pytest.mark.parametrize("n", [6, 9, 16])
def test_periodic_laplacian_symbol(n):
    """F^{-1}(L F(u)) with L = 4 sin^2(pi i/n) + 4 sin^2(pi j/n) is the periodic
    stencil [[0,-1,0],[-1,4,-1],[0,-1,0]] applied by circular shifts (reading P6:
    the second term has j)."""
    u = np.random.default_rng(n).standard_normal((n, n))
    ref = 4 * u - np.roll(u, 1, 0) - np.roll(u, -1, 0) - np.roll(u, 1, 1) - np.roll(u, -1, 1)
    got = np.real(np.fft.ifft2(oracle.lap_symbol(n) * np.fft.fft2(u)))
    np.testing.assert_allclose(got, ref, atol=1e-11)


def test_freq_norm_values():
    """||xi||_eps on the DFT grid: eps at the mean mode; 2 pi/n at the first
    harmonic; pi (the Nyquist frequency) at index n/2; symmetric under i -> n-i."""
    n, eps = 8, 0.1
    F = oracle.freq_norm(n, eps)
    assert F[0, 0] == pytest.approx(eps)
    assert F[1, 0] == pytest.approx(np.hypot(2 * np.pi / n, eps))
    assert F[n // 2, 0] == pytest.approx(np.hypot(np.pi, eps))
    np.testing.assert_allclose(F[1:, :], F[:0:-1, :])
    np.testing.assert_allclose(F, F.T)


def _dense(op, shape_in):
    size = int(np.prod(shape_in))
    cols = [op(e.reshape(shape_in)).ravel() for e in np.eye(size)]
    return np.stack(cols, 1)


def test_power_beta_is_operator_norm():
    """beta from 50 power steps vs the 2-norm of the dense R_h (LAPACK SVD)."""
    geo = Geometry(8, 10, 13)
    A = _dense(lambda x: oracle.rh_forward(x, geo), (8, 8))
    true = np.linalg.norm(A, 2)
    beta = oracle.power_beta(geo, 50)
    assert beta <= true * (1 + 1e-12)
    assert beta == pytest.approx(true, rel=1e-3)


def test_preconditioner_dominates_T():
    """M - T >= 0 for the Alg. 4 preconditioner with c from the power iteration:
    the smallest eigenvalue of the dense M - T is >= 0 (Sec. 4.3: the condition for
    PDRQ); c / margin approximates the top generalised eigenvalue of
    (Rt^* Rt, Mt) computed by LAPACK."""
    n = 8
    geo = Geometry(n, 12, 13)
    sigma, tau, eps = 1.0, 1 / np.sqrt(8), np.pi / n
    beta = oracle.power_beta(geo, 50)
    c = oracle.power_c(geo, beta, eps, 100)
    A = _dense(lambda x: oracle.rh_forward(x, geo), (n, n)) / beta
    G = _dense(lambda x: -oracle.div(*oracle.grad(x)), (n, n))          # -Delta_h
    T = sigma ** 2 * (A.T @ A + tau ** 2 * G)
    sym = oracle.precond_symbol(n, sigma, tau, c, eps)
    Minv = _dense(lambda x: oracle.precond_apply(x, sym), (n, n))
    Minv = 0.5 * (Minv + Minv.T)
    M = np.linalg.inv(Minv)
    ev = np.linalg.eigvalsh(0.5 * (M + M.T) - T)
    assert ev.min() >= -1e-9 * np.abs(ev).max()
    Mt = np.linalg.inv(_dense(lambda x: np.real(np.fft.ifft2(np.fft.fft2(x) * oracle.freq_norm(n, eps))), (n, n)))
    lmax = scipy.linalg.eigh(A.T @ A, 0.5 * (Mt + Mt.T), eigvals_only=True).max()
    assert c / 1.05 == pytest.approx(lmax, rel=1e-3)


def test_preconditioner_symmetric_positive():
    n = 10
    sym = oracle.precond_symbol(n, 1.3, 0.4, 2.0, 0.2)
    rng = np.random.default_rng(0)
    y, z = rng.standard_normal((2, n, n))
    a = np.sum(oracle.precond_apply(y, sym) * z)
    b = np.sum(y * oracle.precond_apply(z, sym))
    assert a == pytest.approx(b, rel=1e-12)
    assert np.sum(oracle.precond_apply(y, sym) * y) > 0
