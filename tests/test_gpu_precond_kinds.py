"""GPU parity of the alternative preconditioners (params.precond): 1 = impulse response
(Sec. "Impulse response preconditioners"), 2 = circulant (Sec. "Circulant matrix
preconditioner", 1-D DFT of length n^2 on the flattened image), 3 = Richardson (Sec.
"Suitable Preconditioners"), with the oracle: the multiplier through precond_apply, c from
the solve's own power iteration, Alg. 4 iterates at fixed (beta, c), the FP32 benchmark
geometry, and the refusals (batches with the kinds: tests/test_gpu_batch.py)."""
import numpy as np
import pytest

import oracle
from gpu_common import rel_l2, to_dev, to_np
from paper_1810_03275_gb300 import phantom

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ct():
    from paper_1810_03275_gb300 import ctrecon
    return ctrecon


def _oracle_precond(geo, kind, sigma, tau, c, nonneg=False):
    """(apply M^{-1}, symbol, circulant flag, s for power_c) of the oracle for one kind."""
    n = geo.n
    if kind == 1:
        s = oracle.impulse_response_kernel_dft(geo)
        sym = oracle.precond_symbol_from(n, sigma, tau, c, s, nonneg)
        return (lambda y: oracle.precond_apply(y, sym)), sym, False, s
    if kind == 2:
        s = oracle.circulant_kernel_dft(geo)
        sym = oracle.precond_symbol_circulant(n, sigma, tau, c, s, oracle.circulant_laplace_dft(n, geo.h), nonneg)
        return (lambda y: oracle.precond_apply_circulant(y, sym)), sym, True, s
    m = oracle.richardson_m(sigma, tau, c, geo.h, nonneg)
    sym = np.full((n, n), 1.0 / m)
    return (lambda y: y / m), sym, False, np.ones((n, n))


@pytest.mark.parametrize("kind", [1, 2, 3])
@pytest.mark.parametrize("n,N,M,h,dtype,tol", [(64, 90, 95, 1.0, "f64", 1e-10), (48, 37, 71, 1.0, "f32", 2e-5),
                                               (96, 120, 137, 0.8, "f32", 2e-5), (27, 30, 41, 1.0, "f64", 1e-10),
                                               (81, 44, 117, 1.0, "f32", 2e-5)])
def test_symbol_through_precond_apply(ct, kind, n, N, M, h, dtype, tol):
    """M^{-1} y for a random y against the oracle's preconditioner of the same kind, with
    and without the identity of Alg. 5; precond = 0 is unchanged afterwards."""
    geo = oracle.Geometry(n, N, M, h=h)
    plan = ct.Plan(n, N, M, h=h, dtype=dtype)
    y = np.random.default_rng(1).standard_normal((n, n))
    for nonneg in (0, 1):
        prm = ct.default_params(sigma=0.9, tau=0.35, c=1.7, eps=np.pi / n, precond=kind, nonneg=nonneg)
        got = to_np(plan.precond_apply(to_dev(y, plan.torch_dtype), prm))
        ref = _oracle_precond(geo, kind, 0.9, 0.35, 1.7, bool(nonneg))[0](y)
        assert rel_l2(got, ref) < tol, (nonneg, rel_l2(got, ref))
    prm0 = ct.default_params(sigma=0.9, tau=0.35, c=1.7, eps=np.pi / n)
    got = to_np(plan.precond_apply(to_dev(y, plan.torch_dtype), prm0))
    assert rel_l2(got, oracle.precond_apply(y, oracle.precond_symbol(n, 0.9, 0.35, 1.7, np.pi / n))) < tol


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_iterates_and_c_match_oracle(ct, kind):
    """64 x 64, 90 angles, metal trace, FP64: c from the solve's power iteration on
    S^{-1/2} Rt^* Rt S^{-1/2} and u after 1, 10 and 100 iterations of Alg. 4 with each
    preconditioner match the oracle."""
    import torch
    pr = phantom.make_problem("t", 64, 90, 95, seed=3, n_ellipses=4, n_metal=2, noise="gaussian", alpha=0.05)
    geo = oracle.Geometry(64, 90, 95, theta=pr.theta)
    eps, tau = np.pi / 64, 1 / np.sqrt(8)
    beta = oracle.power_beta(geo, 30)
    _, _, circ, s = _oracle_precond(geo, kind, 1.0, tau, 1.0)
    c_ref = oracle.power_c(geo, beta, eps, 30, s=s, circulant=circ)
    plan = ct.Plan(64, 90, 95, angles=pr.theta, dtype="f64")
    f = to_dev(pr.f, torch.float64)
    mask = torch.as_tensor(pr.mask, device="cuda")
    prm = ct.default_params(beta=beta, eps=eps, precond=kind, power_iters=30)
    _, d = plan.tv_pd_solve(f, mask, pr.alpha, pr.delta, 1, params=prm)
    assert d["c"] == pytest.approx(c_ref, rel=1e-10)
    desc = oracle.make_descriptors(pr.f, pr.mask, pr.delta)
    _, sym, circ, _ = _oracle_precond(geo, kind, 1.0, tau, c_ref)
    prm = ct.default_params(beta=beta, c=c_ref, eps=eps, precond=kind)
    for k in (1, 10, 100):
        ref = oracle.pdrq_solve(geo, desc, pr.alpha, k, sigma=1.0, tau=tau, eps=eps, beta=beta, c=c_ref,
                                symbol=sym, circulant=circ)
        u, _ = plan.tv_pd_solve(f, mask, pr.alpha, pr.delta, k, params=prm)
        assert rel_l2(to_np(u), ref.u) < 1e-9, (k, rel_l2(to_np(u), ref.u))


@pytest.mark.parametrize("kind", [1, 2])
def test_benchmark_geometry_fp32(ct, kind):
    """512 x 512, 720 x 729 (symmetric projector path): the symbol matches the oracle's on
    the FP32 plan, and 3 iterations with it match the oracle's Alg. 4."""
    import torch
    pr = phantom.config_mar_fp32()
    geo = oracle.Geometry(pr.n, pr.n_angles, pr.n_bins, theta=pr.theta)
    plan = ct.Plan(pr.n, pr.n_angles, pr.n_bins, angles=pr.theta)
    y = np.random.default_rng(2).standard_normal((pr.n, pr.n))
    prm = ct.default_params(sigma=1.0, c=2.0, precond=kind)
    apply, sym, circ, _ = _oracle_precond(geo, kind, 1.0, prm.tau, 2.0)
    got = to_np(plan.precond_apply(to_dev(y, torch.float32), prm))
    assert rel_l2(got, apply(y)) < 1e-4
    beta = plan.power_beta(30)
    prm = ct.default_params(beta=beta, c=2.0, precond=kind)
    desc = oracle.make_descriptors(pr.f, pr.mask, pr.delta)
    st = oracle.pdrq_solve(geo, desc, pr.alpha, 3, sigma=1.0, tau=prm.tau, eps=np.pi / pr.n, beta=beta, c=2.0,
                           symbol=sym, circulant=circ)
    u, _ = plan.tv_pd_solve(to_dev(pr.f, torch.float32), torch.as_tensor(pr.mask, device="cuda"), pr.alpha,
                            pr.delta, 3, params=prm)
    assert rel_l2(to_np(u), st.u) < 1e-4


def test_refusals(ct):
    import torch
    with pytest.raises(Exception, match="precond"):
        ct.Plan(32, 20, 47).tv_pd_solve(torch.zeros((20, 47), device="cuda"), None, 0.1, 0.1, 2,
                                        params=ct.default_params(precond=4))
    batch = ct.Batch([dict(n=32, n_angles=20, n_bins=47)])
    with pytest.raises(Exception, match="precond"):
        batch.solve([torch.zeros((20, 47), device="cuda")], [None], [0.1], [-1.0], 2,
                    params=ct.default_params(precond=5))
