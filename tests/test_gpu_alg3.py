"""GPU Alg. 3 (PDRQS2 for the unconstrained problem (U_h), tv_pdrq2_solve through the C
ABI): iterates against the oracle's Alg. 3 at fixed (beta, c) on both projector paths and
with the alternative preconditioners, the solve's own power iterations and diagnostics,
the BF16 plan against the FP32 one, and the refusal of nonneg."""
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


def _problem(n, N, M, kind, seed=5):
    pr = phantom.make_problem("a3", n, N, M, seed=seed, n_ellipses=4, n_metal=0, noise="gaussian", alpha=0.05)
    th = pr.theta if kind == "uniform" else np.random.default_rng(seed).uniform(0, np.pi, N)
    f = pr.f if kind == "uniform" else oracle.rh_forward(pr.truth, oracle.Geometry(n, N, M, theta=th))
    return th, f, pr.alpha


@pytest.mark.parametrize("kind", ["uniform", "random"])
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-9), ("f32", 1e-5)])
def test_iterates_match_oracle(ct, kind, dtype, tol):
    n, N, M = 64, 92, 95
    th, f, alpha = _problem(n, N, M, kind)
    geo = oracle.Geometry(n, N, M, theta=th)
    eps, tau, sigma = np.pi / n, 1 / np.sqrt(8), 0.8
    beta = oracle.power_beta(geo, 30)
    c = oracle.power_c(geo, beta, eps, 30)
    plan = ct.Plan(n, N, M, angles=th, dtype=dtype)
    prm = ct.default_params(beta=beta, c=c, sigma=sigma, eps=eps, graph_block=4)
    fd = to_dev(f, plan.torch_dtype)
    for k in (1, 10, 100):
        ref = oracle.pdrq2_solve(geo, f, alpha, k, sigma=sigma, tau=tau, eps=eps, beta=beta, c=c)
        got, d = plan.tv_pdrq2_solve(fd, alpha, k, params=prm)
        assert rel_l2(to_np(got), ref.u) < tol, (k, rel_l2(to_np(got), ref.u))
        assert d["iters_done"] == k


@pytest.mark.parametrize("precond", [1, 2, 3])
def test_alternative_preconditioners(ct, precond):
    n, N, M = 48, 60, 71
    th, f, alpha = _problem(n, N, M, "uniform")
    geo = oracle.Geometry(n, N, M, theta=th)
    eps, tau, sigma, c = np.pi / n, 1 / np.sqrt(8), 0.7, 1.3
    beta = oracle.power_beta(geo, 30)
    if precond == 1:
        sym = oracle.precond_symbol_from(n, sigma, tau, c / sigma, oracle.impulse_response_kernel_dft(geo))
    elif precond == 2:
        sym = oracle.precond_symbol_circulant(n, sigma, tau, c / sigma, oracle.circulant_kernel_dft(geo),
                                              oracle.circulant_laplace_dft(n))
    else:
        sym = np.full((n, n), 1.0 / oracle.richardson_m(sigma, tau, c / sigma))
    plan = ct.Plan(n, N, M, angles=th, dtype="f64")
    prm = ct.default_params(beta=beta, c=c, sigma=sigma, eps=eps, precond=precond)
    ref = oracle.pdrq2_solve(geo, f, alpha, 20, sigma=sigma, tau=tau, eps=eps, beta=beta, c=c, symbol=sym,
                             circulant=precond == 2)
    got, _ = plan.tv_pdrq2_solve(to_dev(f, plan.torch_dtype), alpha, 20, params=prm)
    assert rel_l2(to_np(got), ref.u) < 1e-9


def test_power_iterations_and_diagnostics(ct):
    """beta and c from the solve's own power iterations; objective, gap and dual residual
    against the oracle's diagnostics with the unconstrained descriptors."""
    import torch
    n, N, M = 64, 90, 95
    th, f, alpha = _problem(n, N, M, "uniform")
    geo = oracle.Geometry(n, N, M, theta=th)
    eps, tau = np.pi / n, 1 / np.sqrt(8)
    beta = oracle.power_beta(geo, 40)
    c = oracle.power_c(geo, beta, eps, 40)
    plan = ct.Plan(n, N, M, angles=th, dtype="f64")
    u, d = plan.tv_pdrq2_solve(to_dev(f, torch.float64), alpha, 60, params=ct.default_params(power_iters=40))
    assert d["beta"] == pytest.approx(beta, rel=1e-12) and d["c"] == pytest.approx(c, rel=1e-10)
    ref = oracle.pdrq2_solve(geo, f, alpha, 60, sigma=1.0, tau=tau, eps=eps, beta=beta, c=c)
    assert rel_l2(to_np(u), ref.u) < 1e-9
    desc = oracle.make_descriptors(f, None, -1.0)
    dr = oracle.diagnostics(geo, desc, alpha, ref.u, beta=beta, tau=tau, t1=ref.t1, t2x=ref.t2x, t2y=ref.t2y)
    for key in ("objective", "tv", "data_fit"):
        assert d[key] == pytest.approx(dr[key], rel=1e-9), key
    assert d["gap"] == pytest.approx(dr["gap"], rel=1e-6, abs=1e-9)
    assert d["dual_residual"] == pytest.approx(dr["dual_residual"], rel=1e-6)


def test_bf16_plan_and_refusal(ct):
    """The BF16 plan (bfloat16 projector operands) stays within 2e-2 of the FP32 plan
    after 30 iterations; nonneg is refused."""
    import torch
    n, N, M = 96, 120, 137
    th, f, alpha = _problem(n, N, M, "uniform")
    p32 = ct.Plan(n, N, M, angles=th)
    p16 = ct.Plan(n, N, M, angles=th, dtype="bf16")
    beta = p32.power_beta(30)
    prm = ct.default_params(beta=beta, c=1.2)
    fd = to_dev(f, torch.float32)
    u32, _ = p32.tv_pdrq2_solve(fd, alpha, 30, params=prm)
    u16, _ = p16.tv_pdrq2_solve(fd, alpha, 30, params=prm)
    assert rel_l2(to_np(u16), to_np(u32)) < 2e-2
    with pytest.raises(Exception, match="nonneg"):
        p32.tv_pdrq2_solve(fd, alpha, 3, params=ct.default_params(nonneg=1))


def test_thesis_comparison_of_preconditioners(ct):
    """The thesis's comparison on the unconstrained problem: after the same number of
    iterations the objective of Alg. 3 with the inverse-norm preconditioner is closer to
    the minimum than with Richardson, which is closer than Alg. 1 (Chambolle-Pock).
    The minimum is taken from 4000 iterations of Alg. 3; relative objective excess
    (FP64, 64 x 64, 92 views)."""
    import torch
    n, N, M = 64, 92, 95
    th, f, alpha = _problem(n, N, M, "uniform")
    plan = ct.Plan(n, N, M, angles=th, dtype="f64")
    fd = to_dev(f, torch.float64)
    beta = plan.power_beta(50)
    prm = ct.default_params(beta=beta)
    _, d = plan.tv_pdrq2_solve(fd, alpha, 4000, params=prm)
    e_min = d["objective"]
    ex = {}
    for k in (100, 300):
        _, a = plan.tv_pdrq2_solve(fd, alpha, k, params=prm)
        _, r = plan.tv_pdrq2_solve(fd, alpha, k, params=ct.default_params(beta=beta, precond=3))
        _, cp = plan.tv_cp_solve(fd, None, alpha, -1.0, k, params=prm)
        ex[k] = [(x["objective"] - e_min) / e_min for x in (a, r, cp)]
        assert 0 <= ex[k][0] < ex[k][1] < ex[k][2], (k, ex[k])
    assert ex[300][0] < 0.5 * ex[100][0]
