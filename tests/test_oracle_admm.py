"""Pins of the oracle's ADMM with PCG inner solves (Sec. "Alternating Direction Method of
Multipliers"): PCG against a dense LAPACK solve and the one-step steepest-descent closed
form, the soft-thresholding lemma against numerical minimisation, and ADMM reaching the
minimiser that Alg. 1 finds with z = K u at the limit and its multipliers closing the
saddle problem's gap."""
import numpy as np
import pytest
import scipy.optimize

import oracle
from oracle import Geometry
from paper_1810_03275_gb300 import phantom


def _dense(op, n):
    return np.stack([op(e.reshape(n, n)).ravel() for e in np.eye(n * n)], 1)


def test_pcg_against_dense_solve():
    n = 6
    geo = Geometry(n, 10, 11)
    tau = 0.4
    A = lambda x: oracle.rh_adjoint(oracle.rh_forward(x, geo), geo) - tau ** 2 * oracle.div(*oracle.grad(x))
    sym = oracle.precond_symbol(n, 1.0, tau, 3.0, 0.5)
    Minv = lambda y: oracle.precond_apply(y, sym)
    rng = np.random.default_rng(0)
    b = rng.standard_normal((n, n))
    x0 = rng.standard_normal((n, n))
    ref = np.linalg.solve(_dense(A, n), b.ravel()).reshape(n, n)
    np.testing.assert_allclose(oracle.pcg(A, b, x0, n * n, Minv), ref, rtol=0, atol=1e-8 * np.abs(ref).max())
    # one step: x1 = x0 + (r.z / z.Az) z with r = b - A x0, z = M^{-1} r
    r = b - A(x0)
    z = Minv(r)
    x1 = x0 + (np.sum(r * z) / np.sum(z * A(z))) * z
    np.testing.assert_allclose(oracle.pcg(A, b, x0, 1, Minv), x1, rtol=1e-12, atol=1e-13)


def test_soft_threshold_is_the_prox_of_the_norm():
    rng = np.random.default_rng(1)
    for _ in range(20):
        u = rng.standard_normal(2) * rng.choice([0.1, 1.0, 3.0])
        t = rng.uniform(0.05, 2.0)
        obj = lambda x: 0.5 * np.sum((x - u) ** 2) + t * np.sqrt(np.sum(x * x) + 1e-300)
        best = min((scipy.optimize.minimize(obj, x0, method="Nelder-Mead",
                                            options=dict(xatol=1e-12, fatol=1e-14, maxiter=4000))
                    for x0 in (u, np.zeros(2) + 1e-9, -u)), key=lambda r: r.fun)
        gx, gy = oracle.soft_threshold2(np.array([u[0]]), np.array([u[1]]), t)
        assert obj(np.array([gx[0], gy[0]])) <= best.fun + 1e-10
        if np.linalg.norm(u) <= t:
            assert gx[0] == 0.0 and gy[0] == 0.0


def test_admm_reaches_the_cp_minimiser():
    n, N, M = 12, 20, 19
    geo = Geometry(n, N, M)
    truth = phantom.rasterize(phantom.random_phantom(n, 3, 7))
    f = oracle.rh_forward(truth, geo) + 0.05 * np.random.default_rng(7).standard_normal((N, M))
    desc = oracle.make_descriptors(f, None, -1.0)
    alpha, eps, tau = 1.0, np.pi / n, 1 / np.sqrt(8)
    beta = oracle.power_beta(geo, 100)
    c = oracle.power_c(geo, beta, eps, 100)
    u_cp = oracle.cp_solve(geo, desc, alpha, 20000, beta=beta)
    st = oracle.admm_solve(geo, f, alpha, 2500, mu=1.0, tau=tau, cg_iters=2, beta=beta,
                           minv_symbol=oracle.precond_symbol(n, 1.0, tau, c, eps))
    assert np.linalg.norm(st.u - u_cp) / np.linalg.norm(u_cp) < 2e-6
    gx, gy = oracle.grad(st.u)
    assert np.abs(st.w - st.Ru).max() < 1e-8 and np.abs(st.vx - gx).max() < 1e-6
    # the multipliers are the saddle problem's duals: t1 = Rt u - ft, t2 = mu tau eta_v
    d = oracle.diagnostics(geo, desc, alpha, st.u, beta=beta, tau=tau, t1=st.Ru - f / beta,
                           t2x=tau * st.evx, t2y=tau * st.evy)
    assert abs(d["gap"]) < 1e-7 * d["objective"] and d["dual_residual"] < 1e-7
