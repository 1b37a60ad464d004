"""Pins of the oracle's Alg. 4 (PDRQS1) against facts that do not come from it:
the unique minimiser of (C_h) found by Alg. 1 (Chambolle-Pock, unpreconditioned),
the least-squares solution from LAPACK, and the optimality conditions."""
import numpy as np
import pytest

import oracle
from oracle import Geometry
from paper_1810_03275_gb300 import phantom


def _feasible_problem(n=12, N=20, M=19, seed=7, noise=0.05, delta=0.1):
    """Data from the discrete model plus bounded noise |e| <= noise < delta, so the
    delta-ball and the metal-trace constraints are feasible (the truth is feasible)."""
    geo = Geometry(n, N, M)
    ph = phantom.random_phantom(n, 3, seed, n_metal=1, metal_radius=(1.5, 2.0), metal_value=3.0)
    truth = phantom.rasterize(ph)
    f = oracle.rh_forward(truth, geo)
    f = f + noise * np.random.default_rng(seed).uniform(-1, 1, f.shape)
    mask = (oracle.rh_forward(phantom.rasterize(ph, "metal"), geo) > 0).astype(np.uint8)
    return geo, f, mask, oracle.make_descriptors(f, mask, delta)


@pytest.mark.slow
def test_pdrq_and_chambolle_pock_reach_the_same_minimiser():
    geo, f, mask, desc = _feasible_problem()
    alpha, eps, tau = 1.0, np.pi / geo.n, 1 / np.sqrt(8)
    beta = oracle.power_beta(geo, 100)
    c = oracle.power_c(geo, beta, eps, 100)
    st = oracle.pdrq_solve(geo, desc, alpha, 3000, sigma=1.0, tau=tau, eps=eps, beta=beta, c=c)
    u_cp = oracle.cp_solve(geo, desc, alpha, 20000, beta=beta)
    assert np.linalg.norm(st.u - u_cp) / np.linalg.norm(u_cp) < 1e-4
    d = oracle.diagnostics(geo, desc, alpha, st.u, beta=beta, tau=tau, t1=st.t1, t2x=st.t2x, t2y=st.t2y)
    assert d["violation"] < 1e-6                       # R u >= C on the trace, |R u - f| <= delta off it
    assert abs(d["gap"]) < 1e-6 * d["objective"]       # Fenchel-Young gap of the saddle problem
    assert d["dual_residual"] < 1e-6                   # K^* t = 0 (F = 0)


def test_least_squares_limit():
    """alpha = 0, no trace, no box: (C_h) is least squares; with R_h injective the
    minimiser is the LAPACK lstsq solution."""
    n, N, M = 8, 12, 13
    geo = Geometry(n, N, M)
    A = np.stack([oracle.rh_forward(e.reshape(n, n), geo).ravel() for e in np.eye(n * n)], 1)
    assert np.linalg.matrix_rank(A) == n * n
    u0 = np.random.default_rng(2).uniform(0, 1, (n, n))
    f = oracle.rh_forward(u0, geo) + 0.01 * np.random.default_rng(3).standard_normal((N, M))
    desc = oracle.make_descriptors(f, None, -1.0)
    eps, tau = np.pi / n, 1 / np.sqrt(8)
    beta = oracle.power_beta(geo, 60)
    c = oracle.power_c(geo, beta, eps, 60)
    st = oracle.pdrq_solve(geo, desc, 0.0, 4000, sigma=0.01, tau=tau, eps=eps, beta=beta, c=c)
    u_ls = np.linalg.lstsq(A, f.ravel(), rcond=None)[0].reshape(n, n)
    assert np.linalg.norm(st.u - u_ls) / np.linalg.norm(u_ls) < 1e-8


def test_resume_equals_continuous_run():
    """Running k1 then k2 iterations from the saved state equals k1 + k2 in one go."""
    geo, f, mask, desc = _feasible_problem(n=8, N=10, M=13)
    kw = dict(sigma=1.0, tau=0.4, eps=0.3, beta=5.0, c=0.5)
    a = oracle.pdrq_solve(geo, desc, 0.5, 7, **kw)
    b = oracle.pdrq_solve(geo, desc, 0.5, 4, **kw)
    b = oracle.pdrq_solve(geo, desc, 0.5, 3, state=b, **kw)
    np.testing.assert_array_equal(a.u, b.u)
    np.testing.assert_array_equal(a.v1b, b.v1b)
    assert a.k == b.k == 7


def test_first_iterate_from_zero():
    """From u = 0, v = 0 the first u_tmp is 0, so u_1 = 0; the first dual step then
    sees only the data: v1 = 0 and t1 = prox(0).  Hence after one iteration
    v1b = prox_{sigma g*}(0), which for the unconstrained quadratic is -sigma f/(1+sigma)/beta."""
    geo = Geometry(6, 5, 9)
    f = np.random.default_rng(3).uniform(0, 2, (5, 9))
    desc = oracle.make_descriptors(f, None, -1.0)
    beta, sigma = 2.0, 0.7
    st = oracle.pdrq_solve(geo, desc, 0.3, 1, sigma=sigma, tau=0.5, eps=0.2, beta=beta, c=1.0)
    assert np.all(st.u == 0)
    np.testing.assert_allclose(st.v1b, -sigma * (f / beta) / (1 + sigma), rtol=1e-14)


def test_objective_converges_to_the_minimiser_value():
    """The thesis's convergence record is the objective of (C_h) along the iterates: on a
    small feasible problem it approaches the value at the Chambolle-Pock minimiser, with the
    distance shrinking by orders of magnitude from 30 to 300 to 1500 iterations and the
    iterates becoming feasible."""
    geo, f, mask, desc = _feasible_problem(n=8, N=12, M=13, seed=3)
    alpha, eps, tau = 0.5, np.pi / geo.n, 1 / np.sqrt(8)
    beta = oracle.power_beta(geo, 60)
    c = oracle.power_c(geo, beta, eps, 60)
    u_cp = oracle.cp_solve(geo, desc, alpha, 20000, beta=beta)
    ref = oracle.diagnostics(geo, desc, alpha, u_cp, beta=beta)["objective"]
    errs, viol = [], []
    st = None
    done = 0
    for k in (30, 300, 1500):
        st = oracle.pdrq_solve(geo, desc, alpha, k - done, sigma=1.0, tau=tau, eps=eps, beta=beta, c=c, state=st)
        done = k
        d = oracle.diagnostics(geo, desc, alpha, st.u, beta=beta)
        errs.append(abs(d["objective"] - ref) / ref)
        viol.append(d["violation"])
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 1e-6 and errs[2] < 1e-3 * errs[0]
    assert viol[2] < 1e-6
