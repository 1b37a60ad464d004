"""Pins of the oracle's Alg. 5 (PDRQS1 with the non-negativity constraint u >= 0) against
facts that do not come from it: the operator M it preconditions with (built here in the
image domain with the periodic 5-point stencil), the minimiser of the constrained problem
found by Alg. 1 with a projected primal step, and Alg. 4's minimiser where the constraint
is inactive."""
import numpy as np
import pytest

import oracle
from oracle import Geometry
from paper_1810_03275_gb300 import phantom


def _lap_periodic(u):
    """Periodic 5-point Laplacian, written out (the stencil, not its symbol)."""
    return (np.roll(u, 1, 0) + np.roll(u, -1, 0) + np.roll(u, 1, 1) + np.roll(u, -1, 1) - 4.0 * u)


@pytest.mark.parametrize("n", [8, 12, 16])
def test_nonneg_symbol_inverts_M(n):
    """M u = u + c sigma^2 F^{-1}(F(u)/||xi||_eps) - (sigma tau)^2 Delta_p u; its inverse
    is the Fourier multiplier of Alg. 5."""
    sigma, tau, c, eps = 0.9, 0.35, 1.7, np.pi / n
    y = np.random.default_rng(n).standard_normal((n, n))
    nrm = oracle.freq_norm(n, eps)
    My = y + c * sigma ** 2 * np.real(np.fft.ifft2(np.fft.fft2(y) / nrm)) - (sigma * tau) ** 2 * _lap_periodic(y)
    m5 = oracle.precond_symbol_nonneg(n, sigma, tau, c, eps)
    np.testing.assert_allclose(oracle.precond_apply(My, m5), y, rtol=0, atol=1e-12 * np.abs(y).max())


def _noisy_problem(n=12, N=20, M=19, seed=7, noise=0.3, offset=0.0):
    geo = Geometry(n, N, M)
    truth = phantom.rasterize(phantom.random_phantom(n, 3, seed, n_metal=0)) + offset
    f = oracle.rh_forward(truth, geo) + noise * np.random.default_rng(seed).standard_normal((N, M))
    return geo, f, oracle.make_descriptors(f, None, -1.0)


def test_pdrq5_reaches_the_projected_chambolle_pock_minimiser():
    """Heavy noise, small alpha: the unconstrained minimiser dips below zero, so u >= 0 is
    active; Alg. 5 must land on the constrained minimiser (Alg. 1 with the projection onto
    u >= 0 in its primal step) and differ from Alg. 4's."""
    geo, f, desc = _noisy_problem()
    alpha, eps, tau = 0.05, np.pi / geo.n, 1 / np.sqrt(8)
    beta = oracle.power_beta(geo, 100)
    c = oracle.power_c(geo, beta, eps, 100)
    kw = dict(sigma=1.0, tau=tau, eps=eps, beta=beta, c=c)
    u5 = oracle.pdrq5_solve(geo, desc, alpha, 3000, **kw).u
    u4 = oracle.pdrq_solve(geo, desc, alpha, 3000, **kw).u
    ucp = oracle.cp_solve(geo, desc, alpha, 20000, beta=beta, nonneg=True)
    assert u4.min() < -0.1 and np.count_nonzero(ucp == 0) > 10      # the constraint is active
    assert np.linalg.norm(u5 - ucp) / np.linalg.norm(ucp) < 1e-5
    assert u5.min() > -1e-8
    assert np.linalg.norm(u4 - ucp) / np.linalg.norm(ucp) > 0.1


def test_pdrq5_equals_pdrq4_when_the_constraint_is_inactive():
    """Positive truth on a raised background, little noise: the unconstrained minimiser
    (Alg. 1) is already >= 0, so it also solves the constrained problem, and Alg. 5
    reaches it (more slowly than Alg. 4: its M carries the extra identity)."""
    geo, f, desc = _noisy_problem(noise=0.01, offset=1.0)
    alpha, eps, tau = 0.05, np.pi / geo.n, 1 / np.sqrt(8)
    beta = oracle.power_beta(geo, 100)
    c = oracle.power_c(geo, beta, eps, 100)
    kw = dict(sigma=1.0, tau=tau, eps=eps, beta=beta, c=c)
    ucp = oracle.cp_solve(geo, desc, alpha, 20000, beta=beta)
    u5 = oracle.pdrq5_solve(geo, desc, alpha, 8000, **kw).u
    assert ucp.min() > 0.5
    assert np.linalg.norm(u5 - ucp) / np.linalg.norm(ucp) < 2e-5


def test_pdrq5_resume_equals_continuous_run():
    geo, f, desc = _noisy_problem(n=8, N=10, M=13)
    kw = dict(sigma=1.0, tau=0.4, eps=0.3, beta=5.0, c=0.5)
    a = oracle.pdrq5_solve(geo, desc, 0.5, 7, **kw)
    b = oracle.pdrq5_solve(geo, desc, 0.5, 4, **kw)
    b = oracle.pdrq5_solve(geo, desc, 0.5, 3, state=b, **kw)
    np.testing.assert_array_equal(a.u, b.u)
    np.testing.assert_array_equal(a.ub, b.ub)
