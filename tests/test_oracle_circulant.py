"""Pins of the oracle's circulant (Sec. "Circulant matrix preconditioner") and Richardson
(Sec. "Suitable Preconditioners") preconditioners: the Laplace column in closed form, the
1-D DFT application against a dense circulant solve built from a dense R_h^T R_h column,
M - T >= 0 and c against LAPACK, and Alg. 4 with each preconditioner reaching the
minimiser that Alg. 1 finds."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import Geometry
from paper_1810_03275_gb300 import phantom


def _dense(op, n):
    """Matrix of op on the flattened image (t = i + n j)."""
    cols = []
    for t in range(n * n):
        e = np.zeros(n * n)
        e[t] = 1.0
        cols.append(oracle.flatten(op(oracle.unflatten(e, n))))
    return np.stack(cols, 1)


@pytest.mark.parametrize("n,h", [(6, 1.0), (7, 1.0), (8, 0.7)])
def test_laplace_column_closed_form(n, h):
    """-Delta_h at the centre is the 5-point stencil; flattened with t = i + n j its
    neighbours sit at +-1 and +-n, so F_{h,1}(kappa_Delta)_k = (4 - 2 cos(2 pi k / n^2)
    - 2 cos(2 pi k / n)) / h^2."""
    k = np.arange(n * n)
    ref = (4 - 2 * np.cos(2 * np.pi * k / (n * n)) - 2 * np.cos(2 * np.pi * k / n)) / (h * h)
    np.testing.assert_allclose(oracle.circulant_laplace_dft(n, h), ref, atol=1e-12)


@pytest.mark.parametrize("n", [8, 9])
def test_apply_equals_dense_circulant_solve(n):
    """M^{-1} y through F_{h,1} equals the dense solve with M = sigma^2 c C(k) +
    (sigma tau)^2 C(kappa), C(.) the circulant with that first column, k the column of
    the dense R_h^T R_h at the centre pixel rolled to index 0 and averaged with its
    reflection (floor disabled)."""
    geo = Geometry(n, 14, 15)
    cols = []
    for t in range(n * n):
        e = np.zeros(n * n)
        e[t] = 1.0
        cols.append(oracle.rh_forward(oracle.unflatten(e, n), geo).ravel())
    A = np.stack(cols, 1)
    p = n // 2 + n * (n // 2)
    col = (A.T @ A)[:, p]
    kt = np.array([col[(t + p) % (n * n)] for t in range(n * n)])
    k = np.array([0.5 * (kt[t] + kt[(n * n - t) % (n * n)]) for t in range(n * n)])
    np.testing.assert_allclose(oracle.circulant_first_column(
        oracle.unflatten(col, n)), k, atol=1e-13 * np.abs(k).max())
    s1 = oracle.circulant_kernel_dft(geo, floor=-np.inf)
    lap1 = oracle.circulant_laplace_dft(n)
    kd = np.zeros(n * n)
    kd[0], kd[1], kd[-1], kd[n], kd[-n] = 4.0, -1.0, -1.0, -1.0, -1.0
    sigma, tau, c = 0.9, 0.35, 1.7
    Mdense = sigma ** 2 * c * scipy.linalg.circulant(k) + (sigma * tau) ** 2 * scipy.linalg.circulant(kd)
    y = np.random.default_rng(4).standard_normal((n, n))
    ref = oracle.unflatten(np.linalg.solve(Mdense, oracle.flatten(y)), n)
    got = oracle.precond_apply_circulant(y, oracle.precond_symbol_circulant(n, sigma, tau, c, s1, lap1))
    np.testing.assert_allclose(got, ref, atol=1e-10 * np.abs(ref).max())
    ref5 = oracle.unflatten(np.linalg.solve(np.eye(n * n) + Mdense, oracle.flatten(y)), n)
    got5 = oracle.precond_apply_circulant(y, oracle.precond_symbol_circulant(n, sigma, tau, c, s1, lap1, True))
    np.testing.assert_allclose(got5, ref5, atol=1e-10 * np.abs(ref5).max())


def test_circulant_preconditioner_dominates_T():
    """M - T >= 0 with the floored kernel and c from the power iteration on
    S^{-1/2} Rt^* Rt S^{-1/2}; c / margin is the top generalised eigenvalue of
    (Rt^* Rt, S) from LAPACK; the Laplace circulant alone dominates -Delta_h."""
    n = 8
    geo = Geometry(n, 12, 13)
    sigma, tau = 1.0, 1 / np.sqrt(8)
    beta = oracle.power_beta(geo, 50)
    s1 = oracle.circulant_kernel_dft(geo)
    lap1 = oracle.circulant_laplace_dft(n)
    c = oracle.power_c(geo, beta, 0.1, 300, s=s1, circulant=True)
    cols = []
    for t in range(n * n):
        e = np.zeros(n * n)
        e[t] = 1.0
        cols.append(oracle.rh_forward(oracle.unflatten(e, n), geo).ravel())
    A = np.stack(cols, 1) / beta
    G = _dense(lambda x: -oracle.div(*oracle.grad(x)), n)
    T = sigma ** 2 * (A.T @ A + tau ** 2 * G)
    Minv = _dense(lambda x: oracle.precond_apply_circulant(
        x, oracle.precond_symbol_circulant(n, sigma, tau, c, s1, lap1)), n)
    M = np.linalg.inv(0.5 * (Minv + Minv.T))
    ev = np.linalg.eigvalsh(0.5 * (M + M.T) - T)
    assert ev.min() >= -1e-9 * np.abs(ev).max()
    S = _dense(lambda x: oracle.precond_apply_circulant(x, s1), n)
    lmax = scipy.linalg.eigh(A.T @ A, 0.5 * (S + S.T), eigvals_only=True).max()
    assert c / 1.05 == pytest.approx(lmax, rel=1e-3)
    CL = _dense(lambda x: oracle.precond_apply_circulant(x, lap1), n)
    assert np.linalg.eigvalsh(0.5 * (CL + CL.T) - G).min() > -1e-10


def test_richardson_dominates_T():
    """m = sigma^2 c + 8 (sigma tau)^2 / h^2 >= ||T|| (LAPACK eigenvalues), c / margin =
    ||Rt||^2 (LAPACK) from the power iteration with S = id."""
    n, h = 8, 0.8
    geo = Geometry(n, 12, 13, h=h)
    sigma, tau = 0.9, 0.4
    beta = oracle.power_beta(geo, 50)
    c = oracle.power_c(geo, beta, 0.1, 200, s=np.ones((n, n)))
    cols = []
    for t in range(n * n):
        e = np.zeros(n * n)
        e[t] = 1.0
        cols.append(oracle.rh_forward(oracle.unflatten(e, n), geo).ravel())
    A = np.stack(cols, 1) / beta
    assert c / 1.05 == pytest.approx(np.linalg.norm(A, 2) ** 2, rel=1e-6)
    G = _dense(lambda x: -oracle.div(*oracle.grad(x, h), h), n)
    T = sigma ** 2 * (A.T @ A + tau ** 2 * G)
    m = oracle.richardson_m(sigma, tau, c, h)
    assert np.linalg.eigvalsh(m * np.eye(n * n) - T).min() >= 0


def _problem(n=12, N=20, M=19):
    geo = Geometry(n, N, M)
    ph = phantom.random_phantom(n, 3, 7, n_metal=1, metal_radius=(1.5, 2.0), metal_value=3.0)
    truth = phantom.rasterize(ph)
    f = oracle.rh_forward(truth, geo) + 0.05 * np.random.default_rng(7).uniform(-1, 1, (N, M))
    mask = (oracle.rh_forward(phantom.rasterize(ph, "metal"), geo) > 0).astype(np.uint8)
    return geo, oracle.make_descriptors(f, mask, 0.1)


def test_alg4_with_circulant_and_richardson_reaches_the_minimiser():
    geo, desc = _problem()
    n = geo.n
    alpha, eps, tau = 1.0, np.pi / n, 1 / np.sqrt(8)
    beta = oracle.power_beta(geo, 100)
    u_cp = oracle.cp_solve(geo, desc, alpha, 20000, beta=beta)
    s1 = oracle.circulant_kernel_dft(geo)
    c = oracle.power_c(geo, beta, eps, 100, s=s1, circulant=True)
    sym = oracle.precond_symbol_circulant(n, 1.0, tau, c, s1, oracle.circulant_laplace_dft(n))
    st = oracle.pdrq_solve(geo, desc, alpha, 6000, sigma=1.0, tau=tau, eps=eps, beta=beta, c=c, symbol=sym,
                           circulant=True)
    assert np.linalg.norm(st.u - u_cp) / np.linalg.norm(u_cp) < 1e-5
    c = oracle.power_c(geo, beta, eps, 100, s=np.ones((n, n)))
    sym = np.full((n, n), 1.0 / oracle.richardson_m(1.0, tau, c))
    st = oracle.pdrq_solve(geo, desc, alpha, 6000, sigma=1.0, tau=tau, eps=eps, beta=beta, c=c, symbol=sym)
    assert np.linalg.norm(st.u - u_cp) / np.linalg.norm(u_cp) < 1e-5
