"""GPU parity of grad/div, the Fourier preconditioner and the power iterations."""
import numpy as np
import pytest

import oracle
from gpu_common import TOL, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ct():
    from paper_1810_03275_gb300 import ctrecon
    return ctrecon


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("n,h", [(1, 1.0), (2, 1.0), (37, 1.0), (64, 0.5)])
def test_grad_div(ct, n, h, dtype):
    plan = ct.Plan(n, 3, 5, h=h, dtype=dtype)
    rng = np.random.default_rng(n)
    u = rng.standard_normal((n, n))
    p = rng.standard_normal((2, n, n))
    gx, gy = oracle.grad(u, h)
    got = to_np(plan.grad(to_dev(u, plan.torch_dtype)))
    assert rel_l2(got, np.stack([gx, gy])) < TOL[dtype]
    got = to_np(plan.div(to_dev(p, plan.torch_dtype)))
    ref = oracle.div(p[0], p[1], h)
    assert rel_l2(got, ref) < TOL[dtype] or np.abs(ref).max() == 0


@pytest.mark.parametrize("dtype,n", [("f64", 64), ("f32", 64), ("f32", 48), ("f32", 384), ("f32", 512),
                                     ("f64", 27), ("f32", 1), ("f32", 2048), ("f32", 81), ("f64", 3),
                                     ("f32", 6), ("f64", 1024), ("f32", 256), ("f32", 1024)])
def test_precond_apply(ct, n, dtype):
    """M^{-1} y of Alg. 4 vs numpy's FFT on the oracle's symbol (radix 2, 3, 4 paths; the
    real-input form with paired rows and n/2 + 1 columns, odd n included)."""
    plan = ct.Plan(n, 4, 5, dtype=dtype)
    sigma, tau, c, eps = 1.3, 0.35, 0.7, np.pi / n
    prm = ct.default_params(sigma=sigma, tau=tau, c=c, eps=eps)
    y = np.random.default_rng(n).standard_normal((n, n))
    got = to_np(plan.precond_apply(to_dev(y, plan.torch_dtype), prm))
    ref = oracle.precond_apply(y, oracle.precond_symbol(n, sigma, tau, c, eps))
    assert rel_l2(got, ref) < (2e-6 if dtype == "f32" else 1e-12)


def test_plans_of_different_sizes_coexist(ct):
    """Kernel shared-memory limits are process-wide: creating a smaller plan after a
    larger one must not break the larger plan's launches (regression)."""
    big = ct.Plan(2048, 4, 5)
    ct.Plan(768, 4, 5)
    ct.Plan(1024, 4, 5)
    prm = ct.default_params(c=1.0, eps=0.01)
    y = np.random.default_rng(0).standard_normal((2048, 2048))
    got = to_np(big.precond_apply(to_dev(y, big.torch_dtype), prm))
    ref = oracle.precond_apply(y, oracle.precond_symbol(2048, 1.0, prm.tau, 1.0, 0.01))
    assert rel_l2(got, ref) < 2e-6


def test_precond_rejects_other_sizes(ct):
    plan = ct.Plan(10, 4, 5)
    with pytest.raises(ct.CtrError) as e:
        plan.precond_apply(to_dev(np.zeros((10, 10)), plan.torch_dtype), ct.default_params(c=1.0))
    assert e.value.status == -6


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_power_iterations(ct, dtype):
    """beta and lambda_max from the GPU power iterations follow the oracle's
    (same start vector, same step count)."""
    n, N, M = 32, 40, 47
    plan = ct.Plan(n, N, M, dtype=dtype)
    geo = oracle.Geometry(n, N, M)
    beta_ref = oracle.power_beta(geo, 30)
    beta = plan.power_beta(30)
    assert beta == pytest.approx(beta_ref, rel=1e-6 if dtype == "f32" else 1e-12)
    eps = np.pi / n
    lam_ref = oracle.power_c(geo, beta_ref, eps, 30, margin=1.0)
    lam = plan.power_lambda(beta_ref, eps, 30)
    assert lam == pytest.approx(lam_ref, rel=1e-5 if dtype == "f32" else 1e-11)


@pytest.mark.parametrize("n", [256, 512, 1024])
def test_fft_forms_agree(ct, n):
    """The warp-level preconditioner passes (form 0: one warp per row pair / column, the
    four-step factorisation n = 32 x n/32) against the CTA-level Stockham passes (form 1)
    and the oracle: precond_apply, and a few Alg. 4 iterations (the fused fold of the
    backprojection into the first pass, u += in the last) on FP32 and BF16 plans."""
    import torch
    sigma, tau, c, eps = 1.3, 0.35, 0.7, np.pi / n
    prm = ct.default_params(sigma=sigma, tau=tau, c=c, eps=eps)
    plan = ct.Plan(n, 4, 5)
    assert plan.fft_form == 0
    y = np.random.default_rng(n + 1).standard_normal((n, n))
    a = to_np(plan.precond_apply(to_dev(y, torch.float32), prm))
    plan.set_fft_form(1)
    assert plan.fft_form == 1
    b = to_np(plan.precond_apply(to_dev(y, torch.float32), prm))
    ref = oracle.precond_apply(y, oracle.precond_symbol(n, sigma, tau, c, eps))
    assert rel_l2(a, ref) < 2e-6
    assert rel_l2(a, b) < 2e-6
    with pytest.raises(ct.CtrError):
        plan.set_fft_form(2)
    N = max(8, n // 4)
    M = int(np.ceil(np.sqrt(2) * n))
    th = np.arange(N) * (np.pi / N)
    rng = np.random.default_rng(n)
    f = rng.standard_normal((N, M)).astype(np.float32)
    mask = (rng.random((N, M)) < 0.05).astype(np.uint8)
    for dtype in ("f32", "bf16"):
        us = []
        for form in (0, 1):
            pl = ct.Plan(n, N, M, angles=th, dtype=dtype)
            pl.set_fft_form(form)
            p2 = ct.default_params(beta=float(M), c=1.0, eps=np.pi / n)
            u, _ = pl.tv_pd_solve(to_dev(f, torch.float32), torch.as_tensor(mask, device="cuda"), 0.3, 0.05, 6,
                                  params=p2)
            us.append(to_np(u))
        assert rel_l2(us[0], us[1]) < (2e-6 if dtype == "f32" else 2e-3), dtype


def test_precond_apply_largest_image(ct):
    """M^{-1} y at 4096 x 4096 (the CTA-level passes in real-input form) against numpy's FFT
    on the oracle's symbol."""
    import torch
    n = 4096
    plan = ct.Plan(n, 4, 5)
    sigma, tau, c, eps = 1.3, 0.35, 0.7, np.pi / n
    prm = ct.default_params(sigma=sigma, tau=tau, c=c, eps=eps)
    y = np.random.default_rng(n).standard_normal((n, n))
    got = to_np(plan.precond_apply(to_dev(y, torch.float32), prm))
    ref = oracle.precond_apply(y, oracle.precond_symbol(n, sigma, tau, c, eps))
    assert rel_l2(got, ref) < 2e-6
