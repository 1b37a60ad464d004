"""GPU ADMM with PCG inner solves (tv_admm_solve through the C ABI) against the oracle's
ADMM: iterates at fixed (beta, c) on both projector paths and with the circulant
preconditioner of the original method, the solve's own power iterations and its
diagnostics, and the argument errors."""
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


def _problem(n, N, M, kind, seed=6):
    pr = phantom.make_problem("admm", n, N, M, seed=seed, n_ellipses=4, n_metal=0, noise="gaussian", alpha=0.05)
    th = pr.theta if kind == "uniform" else np.random.default_rng(seed).uniform(0, np.pi, N)
    f = pr.f if kind == "uniform" else oracle.rh_forward(pr.truth, oracle.Geometry(n, N, M, theta=th))
    return th, f, pr.alpha


@pytest.mark.parametrize("kind", ["uniform", "random"])
@pytest.mark.parametrize("dtype,tol,cg", [("f64", 1e-9, 2), ("f64", 1e-9, 3), ("f32", 1e-4, 2)])
def test_iterates_match_oracle(ct, kind, dtype, tol, cg):
    n, N, M = 64, 92, 95
    th, f, alpha = _problem(n, N, M, kind)
    geo = oracle.Geometry(n, N, M, theta=th)
    eps, tau, mu = np.pi / n, 1 / np.sqrt(8), 0.7
    beta = oracle.power_beta(geo, 30)
    c = oracle.power_c(geo, beta, eps, 30)
    sym = oracle.precond_symbol(n, 1.0, tau, c, eps)
    plan = ct.Plan(n, N, M, angles=th, dtype=dtype)
    prm = ct.default_params(beta=beta, c=c, eps=eps, graph_block=3)
    fd = to_dev(f, plan.torch_dtype)
    for k in (1, 5, 30):
        ref = oracle.admm_solve(geo, f, alpha, k, mu=mu, tau=tau, cg_iters=cg, beta=beta, minv_symbol=sym)
        got, d = plan.tv_admm_solve(fd, alpha, k, mu=mu, cg_iters=cg, params=prm)
        assert rel_l2(to_np(got), ref.u) < tol, (k, rel_l2(to_np(got), ref.u))
        assert d["iters_done"] == k


def test_circulant_preconditioned_pcg(ct):
    n, N, M = 48, 60, 71
    th, f, alpha = _problem(n, N, M, "uniform")
    geo = oracle.Geometry(n, N, M, theta=th)
    tau, c = 1 / np.sqrt(8), 1.4
    beta = oracle.power_beta(geo, 30)
    sym = oracle.precond_symbol_circulant(n, 1.0, tau, c, oracle.circulant_kernel_dft(geo),
                                          oracle.circulant_laplace_dft(n))
    plan = ct.Plan(n, N, M, angles=th, dtype="f64")
    ref = oracle.admm_solve(geo, f, alpha, 10, mu=1.0, tau=tau, cg_iters=3, beta=beta, minv_symbol=sym,
                            circulant=True)
    got, _ = plan.tv_admm_solve(to_dev(f, plan.torch_dtype), alpha, 10, mu=1.0, cg_iters=3,
                                params=ct.default_params(beta=beta, c=c, precond=2))
    assert rel_l2(to_np(got), ref.u) < 1e-9


def test_power_iterations_and_diagnostics(ct):
    import torch
    n, N, M = 64, 90, 95
    th, f, alpha = _problem(n, N, M, "uniform")
    geo = oracle.Geometry(n, N, M, theta=th)
    eps, tau, mu = np.pi / n, 1 / np.sqrt(8), 1.0
    beta = oracle.power_beta(geo, 40)
    c = oracle.power_c(geo, beta, eps, 40)
    plan = ct.Plan(n, N, M, angles=th, dtype="f64")
    u, d = plan.tv_admm_solve(to_dev(f, torch.float64), alpha, 40, mu=mu, cg_iters=2,
                              params=ct.default_params(power_iters=40))
    assert d["beta"] == pytest.approx(beta, rel=1e-12) and d["c"] == pytest.approx(c, rel=1e-10)
    ref = oracle.admm_solve(geo, f, alpha, 40, mu=mu, tau=tau, cg_iters=2, beta=beta,
                            minv_symbol=oracle.precond_symbol(n, 1.0, tau, c, eps))
    assert rel_l2(to_np(u), ref.u) < 1e-9
    desc = oracle.make_descriptors(f, None, -1.0)
    dr = oracle.diagnostics(geo, desc, alpha, ref.u, beta=beta, tau=tau, t1=ref.Ru - f / beta,
                            t2x=mu * tau * ref.evx, t2y=mu * tau * ref.evy)
    for key in ("objective", "tv", "data_fit"):
        assert d[key] == pytest.approx(dr[key], rel=1e-9), key
    assert d["gap"] == pytest.approx(dr["gap"], rel=1e-6, abs=1e-9)
    assert d["dual_residual"] == pytest.approx(dr["dual_residual"], rel=1e-6)


def test_argument_errors(ct):
    import torch
    plan = ct.Plan(32, 20, 47)
    f = torch.zeros((20, 47), device="cuda")
    for kw in (dict(mu=0.0), dict(mu=float("inf")), dict(cg_iters=0), dict(cg_iters=65)):
        with pytest.raises(ct.CtrError):
            plan.tv_admm_solve(f, 0.1, 2, **kw)
    with pytest.raises(ct.CtrError):
        ct.Plan(32, 20, 47, dtype="bf16").tv_admm_solve(f, 0.1, 2)
    with pytest.raises(ct.CtrError):
        plan.tv_admm_solve(f, 0.1, 2, params=ct.default_params(nonneg=1))
