"""GPU Alg. 1 (Chambolle-Pock, tv_cp_solve through the C ABI), the unpreconditioned
baseline of the thesis: iterates against the oracle's Alg. 1 at fixed steps on both
projector paths, and the comparison the thesis makes, Alg. 4 converging faster per
iteration than Alg. 1 on the same problem."""
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


def _problem(n, N, M, kind, seed=11):
    pr = phantom.make_problem("cp", n, N, M, seed=seed, n_ellipses=4, n_metal=1, noise="gaussian", alpha=0.05)
    th = pr.theta if kind == "uniform" else np.random.default_rng(seed).uniform(0, np.pi, N)
    f = pr.f if kind == "uniform" else oracle.rh_forward(pr.truth, oracle.Geometry(n, N, M, theta=th))
    return th, f, pr.mask, pr.alpha, pr.delta


@pytest.mark.parametrize("kind", ["uniform", "random"])
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-9), ("f32", 1e-5)])
def test_cp_iterates_match_oracle(ct, kind, dtype, tol):
    """n = 40 is not of the form 2^a 3^b: Alg. 1 needs no FFT and takes it."""
    import torch
    n, N, M = 40, 48, 59
    th, f, mask, alpha, delta = _problem(n, N, M, kind)
    geo = oracle.Geometry(n, N, M, theta=th)
    desc = oracle.make_descriptors(f, mask, delta)
    beta = oracle.power_beta(geo, 30)
    sp, sd = 0.25, 0.3
    plan = ct.Plan(n, N, M, angles=th, dtype=dtype)
    prm = ct.default_params(beta=beta, graph_block=4)
    fd = to_dev(f, plan.torch_dtype)
    md = torch.as_tensor(mask, device="cuda")
    for k in (1, 10, 100):
        ref = oracle.cp_solve(geo, desc, alpha, k, beta=beta, sigma=sp, tau=sd)
        got, d = plan.tv_cp_solve(fd, md, alpha, delta, k, sigma_p=sp, tau_d=sd, params=prm)
        assert rel_l2(to_np(got), ref) < tol, (k, rel_l2(to_np(got), ref))
        assert np.isfinite(d["gap"]) and d["iters_done"] == k


def test_preconditioned_alg4_beats_alg1_per_iteration(ct):
    """Sec. 4 / the thesis's comparison: on the 64 x 64 configuration with metal, after
    the same number of iterations Alg. 4 is closer to the minimiser than Alg. 1 (default
    steps), measured against a long Alg. 4 run (measured: 0.20 vs 0.27 after 100)."""
    import torch
    n, N, M = 64, 90, 95
    th, f, mask, alpha, delta = _problem(n, N, M, "uniform")
    plan = ct.Plan(n, N, M, angles=th, dtype="f64")
    fd = to_dev(f, torch.float64)
    md = torch.as_tensor(mask, device="cuda")
    beta = plan.power_beta(50)
    prm = ct.default_params(beta=beta)
    u_star, _ = plan.tv_pd_solve(fd, md, alpha, delta, 5000, params=prm)
    u_star = to_np(u_star)
    for k in (100, 300):
        u4, _ = plan.tv_pd_solve(fd, md, alpha, delta, k, params=prm)
        u1, _ = plan.tv_cp_solve(fd, md, alpha, delta, k, params=prm)
        e4, e1 = rel_l2(to_np(u4), u_star), rel_l2(to_np(u1), u_star)
        assert e4 < 0.9 * e1, (k, e4, e1)


def test_cp_refuses_bf16(ct):
    import torch
    plan = ct.Plan(32, 20, 47, dtype="bf16")
    with pytest.raises(Exception, match="FP32 and FP64"):
        plan.tv_cp_solve(torch.zeros((20, 47), device="cuda"), None, 0.1, -1.0, 2)
