"""Pins of the oracle's impulse-response preconditioner (Sec. "Impulse response
preconditioners"): the kernel against R_h^* R_h built as a dense matrix, its symmetry, the
condition M - T >= 0 that PDRQ needs, and Alg. 4 with it reaching the minimiser that
Alg. 1 finds."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import Geometry
from paper_1810_03275_gb300 import phantom


def _dense(op, shape):
    cols = [op(e.reshape(shape)).ravel() for e in np.eye(int(np.prod(shape)))]
    return np.stack(cols, 1)


def test_kernel_is_the_centre_column_of_RtR_point_symmetrised():
    """k is column (n/2, n/2) of the dense R_h^T R_h, moved to the origin and averaged
    with its point reflection; its DFT is real; the floor only touches values near 0."""
    for n in (8, 9):
        geo = Geometry(n, 14, 15)
        A = _dense(lambda x: oracle.rh_forward(x, geo), (n, n))
        c = n // 2
        col = (A.T @ A)[:, c * n + c].reshape(n, n)
        kt = np.roll(col, (-c, -c), axis=(0, 1))
        refl = kt[(-np.arange(n)) % n][:, (-np.arange(n)) % n]
        k = 0.5 * (kt + refl)
        F = np.fft.fft2(k)
        assert np.abs(F.imag).max() < 1e-12 * np.abs(F.real).max()
        s = oracle.impulse_response_kernel_dft(geo, floor=-np.inf)
        np.testing.assert_allclose(s, F.real, rtol=0, atol=1e-12 * np.abs(F.real).max())
        s_floor = oracle.impulse_response_kernel_dft(geo)
        assert s_floor.min() > 0 and s_floor.max() == pytest.approx(F.real.max())


def test_impulse_preconditioner_dominates_T():
    """M - T >= 0 with M = sigma^2 c S + (sigma tau)^2 (-Delta_p), S the convolution with
    the kernel, c from the power iteration on S^{-1/2} Rt^* Rt S^{-1/2}; c / margin equals
    the top generalised eigenvalue of (Rt^* Rt, S) computed by LAPACK."""
    n = 8
    geo = Geometry(n, 12, 13)
    sigma, tau, eps = 1.0, 1 / np.sqrt(8), np.pi / n
    beta = oracle.power_beta(geo, 50)
    s = oracle.impulse_response_kernel_dft(geo)
    c = oracle.power_c(geo, beta, eps, 200, s=s)
    A = _dense(lambda x: oracle.rh_forward(x, geo), (n, n)) / beta
    G = _dense(lambda x: -oracle.div(*oracle.grad(x)), (n, n))
    T = sigma ** 2 * (A.T @ A + tau ** 2 * G)
    sym = oracle.precond_symbol_from(n, sigma, tau, c, s)
    Minv = _dense(lambda x: oracle.precond_apply(x, sym), (n, n))
    M = np.linalg.inv(0.5 * (Minv + Minv.T))
    ev = np.linalg.eigvalsh(0.5 * (M + M.T) - T)
    assert ev.min() >= -1e-9 * np.abs(ev).max()
    S = _dense(lambda x: np.real(np.fft.ifft2(np.fft.fft2(x) * s)), (n, n))
    lmax = scipy.linalg.eigh(A.T @ A, 0.5 * (S + S.T), eigvals_only=True).max()
    assert c / 1.05 == pytest.approx(lmax, rel=1e-3)


def test_inverse_norm_is_the_generic_symbol_with_s_one_over_norm():
    n = 12
    s = 1.0 / oracle.freq_norm(n, 0.3)
    np.testing.assert_allclose(oracle.precond_symbol_from(n, 0.9, 0.4, 1.7, s),
                               oracle.precond_symbol(n, 0.9, 0.4, 1.7, 0.3), rtol=1e-13)
    np.testing.assert_allclose(oracle.precond_symbol_from(n, 0.9, 0.4, 1.7, s, nonneg=True),
                               oracle.precond_symbol_nonneg(n, 0.9, 0.4, 1.7, 0.3), rtol=1e-13)


def test_alg4_with_impulse_preconditioner_reaches_the_minimiser():
    n, N, M = 12, 20, 19
    geo = Geometry(n, N, M)
    ph = phantom.random_phantom(n, 3, 7, n_metal=1, metal_radius=(1.5, 2.0), metal_value=3.0)
    truth = phantom.rasterize(ph)
    f = oracle.rh_forward(truth, geo) + 0.05 * np.random.default_rng(7).uniform(-1, 1, (N, M))
    mask = (oracle.rh_forward(phantom.rasterize(ph, "metal"), geo) > 0).astype(np.uint8)
    desc = oracle.make_descriptors(f, mask, 0.1)
    alpha, eps, tau = 1.0, np.pi / n, 1 / np.sqrt(8)
    beta = oracle.power_beta(geo, 100)
    s = oracle.impulse_response_kernel_dft(geo)
    c = oracle.power_c(geo, beta, eps, 100, s=s)
    sym = oracle.precond_symbol_from(n, 1.0, tau, c, s)
    st = oracle.pdrq_solve(geo, desc, alpha, 6000, sigma=1.0, tau=tau, eps=eps, beta=beta, c=c, symbol=sym)
    u_cp = oracle.cp_solve(geo, desc, alpha, 20000, beta=beta)
    # (slower than the inverse-norm preconditioner here: 1.5e-2 after 3000 iterations vs 3e-12)
    assert np.linalg.norm(st.u - u_cp) / np.linalg.norm(u_cp) < 1e-5
