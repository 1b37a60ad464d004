"""Pins of the oracle's Alg. 3 (PDRQS2, unconstrained problem (U_h)): the alpha = 0
reduction to the preconditioned Landweber iteration (dense matrices) heading to the LAPACK
lstsq solution, the minimiser that Alg. 1 finds with the
Fenchel-Young gap and ||K^* t|| vanishing, and M - T >= 0 for Alg. 3's T = sigma
Rt^* Rt + (sigma tau)^2 (-Delta_h) with the symbol's sigma c."""
import numpy as np

import oracle
from oracle import Geometry
from paper_1810_03275_gb300 import phantom


def _dense(op, shape):
    cols = [op(e.reshape(shape)).ravel() for e in np.eye(int(np.prod(shape)))]
    return np.stack(cols, 1)


def test_alpha_zero_reduces_to_preconditioned_landweber():
    """With alpha = 0 the TV dual cancels the Laplacian term from the second iteration on
    (t2 = 0, so bar v2 = -sigma tau grad u), and Alg. 3 becomes the preconditioned
    Landweber iteration u <- u + sigma M^{-1} Rt^*(ft - Rt u) for the least-squares
    problem; its iterates, computed here with dense matrices, match, and both approach
    the LAPACK lstsq solution."""
    n, N, M = 8, 12, 13
    geo = Geometry(n, N, M)
    A = np.stack([oracle.rh_forward(e.reshape(n, n), geo).ravel() for e in np.eye(n * n)], 1)
    u0 = np.random.default_rng(2).uniform(0, 1, (n, n))
    f = oracle.rh_forward(u0, geo) + 0.01 * np.random.default_rng(3).standard_normal((N, M))
    sigma, eps, tau = 0.5, np.pi / n, 1 / np.sqrt(8)
    beta = oracle.power_beta(geo, 60)
    c = oracle.power_c(geo, beta, eps, 60)
    sym = oracle.precond_symbol(n, sigma, tau, c / sigma, eps)
    Minv = _dense(lambda x: oracle.precond_apply(x, sym), (n, n))
    At, ft = A / beta, f.ravel() / beta
    st = oracle.pdrq2_solve(geo, f, 0.0, 1, sigma=sigma, tau=tau, eps=eps, beta=beta, c=c)
    u = st.u.ravel()
    np.testing.assert_allclose(u, sigma * Minv @ (At.T @ ft), rtol=1e-12, atol=1e-14)
    for _ in range(30):
        u = u + sigma * Minv @ (At.T @ (ft - At @ u))
    st = oracle.pdrq2_solve(geo, f, 0.0, 30, sigma=sigma, tau=tau, eps=eps, beta=beta, c=c, state=st)
    np.testing.assert_allclose(st.u.ravel(), u, rtol=1e-10, atol=1e-12)
    u_ls = np.linalg.lstsq(A, f.ravel(), rcond=None)[0]
    e0 = np.linalg.norm(u_ls)
    st = oracle.pdrq2_solve(geo, f, 0.0, 500, sigma=sigma, tau=tau, eps=eps, beta=beta, c=c, state=st)
    assert np.linalg.norm(st.u.ravel() - u_ls) < 0.25 * e0


def test_reaches_the_cp_minimiser_with_vanishing_gap():
    n, N, M = 12, 20, 19
    geo = Geometry(n, N, M)
    truth = phantom.rasterize(phantom.random_phantom(n, 3, 7))
    f = oracle.rh_forward(truth, geo) + 0.05 * np.random.default_rng(7).standard_normal((N, M))
    desc = oracle.make_descriptors(f, None, -1.0)
    alpha, eps, tau = 1.0, np.pi / n, 1 / np.sqrt(8)
    beta = oracle.power_beta(geo, 100)
    c = oracle.power_c(geo, beta, eps, 100)
    st = oracle.pdrq2_solve(geo, f, alpha, 3000, sigma=1.0, tau=tau, eps=eps, beta=beta, c=c)
    u_cp = oracle.cp_solve(geo, desc, alpha, 20000, beta=beta)
    assert np.linalg.norm(st.u - u_cp) / np.linalg.norm(u_cp) < 1e-5
    d = oracle.diagnostics(geo, desc, alpha, st.u, beta=beta, tau=tau, t1=st.t1, t2x=st.t2x, t2y=st.t2y)
    assert abs(d["gap"]) < 1e-6 * d["objective"]
    assert d["dual_residual"] < 1e-6


def test_preconditioner_dominates_alg3_T():
    n = 8
    geo = Geometry(n, 12, 13)
    sigma, tau, eps = 0.6, 1 / np.sqrt(8), np.pi / n
    beta = oracle.power_beta(geo, 50)
    c = oracle.power_c(geo, beta, eps, 200)
    A = _dense(lambda x: oracle.rh_forward(x, geo), (n, n)) / beta
    G = _dense(lambda x: -oracle.div(*oracle.grad(x)), (n, n))
    T = sigma * A.T @ A + (sigma * tau) ** 2 * G
    sym = oracle.precond_symbol(n, sigma, tau, c / sigma, eps)
    Minv = _dense(lambda x: oracle.precond_apply(x, sym), (n, n))
    M = np.linalg.inv(0.5 * (Minv + Minv.T))
    ev = np.linalg.eigvalsh(0.5 * (M + M.T) - T)
    assert ev.min() >= -1e-9 * np.abs(ev).max()
