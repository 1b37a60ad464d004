"""The differentiable form: R_h / R_h^* as autograd Functions, and K unrolled
iterations of Alg. 4 differentiated by the library's reverse-mode kernels
(tv_pd_vjp_step) with checkpoints every few iterates.  Gradients with respect to the
data f and alpha are checked against the FP64 oracle's reverse mode (itself pinned by
finite differences) and against FP64 central differences of the GPU forward."""
import numpy as np
import pytest

import oracle
from gpu_common import rel_l2, to_dev, to_np
from paper_1810_03275_gb300 import phantom

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_1810_03275_gb300 import autograd, ctrecon
    return ctrecon, autograd


def test_radon_functions_are_adjoint_pairs(mods):
    import torch
    ct, ag = mods
    plan = ct.Plan(40, 30, 57)
    u = torch.randn((40, 40), device="cuda", requires_grad=True)
    g = torch.randn((30, 57), device="cuda")
    (ag.radon(u, plan) * g).sum().backward()
    assert rel_l2(to_np(u.grad), to_np(plan.rh_adjoint(g))) < 1e-6
    gg = g.clone().requires_grad_(True)
    w = torch.randn((40, 40), device="cuda")
    (ag.backproject(gg, plan) * w).sum().backward()
    assert rel_l2(to_np(gg.grad), to_np(plan.rh_forward(w))) < 1e-6


def _setup(ct, dtype, n=32, N=40, M=47, metal=True, seed=4):
    import torch
    pr = phantom.make_problem("ag", n, N, M, seed=seed, n_ellipses=3, n_metal=1 if metal else 0, noise="gaussian",
                              alpha=0.2)
    geo = oracle.Geometry(n, N, M, theta=pr.theta)
    beta = oracle.power_beta(geo, 30)
    eps = np.pi / n
    c = oracle.power_c(geo, beta, eps, 30)
    plan = ct.Plan(n, N, M, angles=pr.theta, dtype=dtype)
    prm = ct.default_params(beta=beta, c=c, eps=eps)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    mask = torch.as_tensor(pr.mask, device="cuda") if metal else None
    return pr, geo, plan, prm, tdt, mask, dict(sigma=1.0, tau=prm.tau, eps=eps, beta=beta, c=c)


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-9), ("f32", 1e-4)])
def test_unrolled_gradient_matches_oracle(mods, dtype, tol):
    import torch
    ct, ag = mods
    pr, geo, plan, prm, tdt, mask, kw = _setup(ct, dtype)
    K, delta = 10, 2.0 * pr.delta
    f = to_dev(pr.f, tdt).requires_grad_(True)
    alpha = torch.tensor(pr.alpha, dtype=torch.float64, requires_grad=True)
    u = ag.unrolled_pdrq(f, alpha, plan, mask, delta, iters=K, ckpt=3, params=prm)
    truth = to_dev(pr.truth, tdt)
    ((u - truth) ** 2).sum().backward()
    uK = oracle.pdrq_solve(geo, oracle.make_descriptors(pr.f, pr.mask, delta), pr.alpha, K, **kw).u
    assert rel_l2(to_np(u), uK) < (1e-9 if dtype == "f64" else 1e-5)
    df, dalpha = oracle.pdrq_grad(geo, pr.f, pr.mask, delta, pr.alpha, K, 2.0 * (uK - pr.truth), **kw)
    assert rel_l2(to_np(f.grad), df) < tol
    assert float(alpha.grad) == pytest.approx(dalpha, rel=tol * 10, abs=1e-12)


def test_unrolled_gradient_matches_finite_differences_fp64(mods):
    """FP64 GPU: directional derivatives of ||u_K - u_true||^2 along random data
    directions and along alpha vs central differences with h = 1e-6."""
    import torch
    ct, ag = mods
    pr, geo, plan, prm, tdt, mask, kw = _setup(ct, "f64", seed=6)
    K, delta = 8, -1.0
    truth = to_dev(pr.truth, tdt)

    def loss(fv, av):
        with torch.no_grad():
            u = ag.unrolled_pdrq(fv, torch.tensor(av, dtype=torch.float64), plan, mask, delta, iters=K, ckpt=4,
                                 params=prm)
            return float(((u - truth) ** 2).sum())

    f = to_dev(pr.f, tdt).requires_grad_(True)
    alpha = torch.tensor(pr.alpha, dtype=torch.float64, requires_grad=True)
    u = ag.unrolled_pdrq(f, alpha, plan, mask, delta, iters=K, ckpt=4, params=prm)
    ((u - truth) ** 2).sum().backward()
    h = 1e-6
    for s in range(2):
        d = to_dev(np.random.default_rng(s).standard_normal(pr.f.shape), tdt)
        fd = (loss(f.detach() + h * d, pr.alpha) - loss(f.detach() - h * d, pr.alpha)) / (2 * h)
        assert float((f.grad * d).sum()) == pytest.approx(fd, rel=1e-5)
    fd = (loss(f.detach(), pr.alpha + h) - loss(f.detach(), pr.alpha - h)) / (2 * h)
    assert float(alpha.grad) == pytest.approx(fd, rel=1e-5)


def test_differentiation_configuration(mods):
    """Batch of 16 phantoms of 256 x 256, 360 angles, 363 bins, FP32; K = 20 unrolled
    iterations with checkpoints every 5; gradient of ||u_K - u_true||^2 with respect to
    f and alpha for every slice; slice 0 checked against the FP64 oracle's gradient."""
    import torch
    ct, ag = mods
    n, N, M, K = 256, 360, 363, 20
    probs = [phantom.make_problem(f"d{i}", n, N, M, seed=40 + i, n_ellipses=4, n_metal=1, noise="poisson", alpha=0.3)
             for i in range(16)]
    plan = ct.Plan(n, N, M, angles=probs[0].theta)
    prm = ag.fixed_scaling(plan)
    grads = []
    for p in probs:
        f = to_dev(p.f, torch.float32).requires_grad_(True)
        alpha = torch.tensor(p.alpha, dtype=torch.float64, requires_grad=True)
        mask = torch.as_tensor(p.mask, device="cuda")
        u = ag.unrolled_pdrq(f, alpha, plan, mask, p.delta, iters=K, ckpt=5, params=prm)
        ((u - to_dev(p.truth, torch.float32)) ** 2).sum().backward()
        assert torch.isfinite(f.grad).all() and np.isfinite(float(alpha.grad))
        grads.append((to_np(f.grad), float(alpha.grad), to_np(u)))
    p = probs[0]
    geo = oracle.Geometry(n, N, M, theta=p.theta)
    kw = dict(sigma=1.0, tau=prm.tau, eps=prm.eps, beta=prm.beta, c=prm.c)
    uK = oracle.pdrq_solve(geo, oracle.make_descriptors(p.f, p.mask, p.delta), p.alpha, K, **kw).u
    assert rel_l2(grads[0][2], uK) < 1e-5
    df, dalpha = oracle.pdrq_grad(geo, p.f, p.mask, p.delta, p.alpha, K, 2.0 * (grads[0][2] - p.truth), **kw)
    e = rel_l2(grads[0][0], df)
    print(f"256^2 K=20 FP32 gradient vs FP64 oracle: rel_l2(df) {e:.2e}, dalpha {grads[0][1]:.6e} vs {dalpha:.6e}")
    # stated FP32 bound (measured 8.3e-4: FP32 rounding carried back through 20
    # iterations); the FP64 GPU path below matches the oracle to 1e-8
    assert e < 2e-3
    assert grads[0][1] == pytest.approx(dalpha, rel=1e-4)
    p64 = ct.Plan(n, N, M, angles=p.theta, dtype="f64")
    f = to_dev(p.f, torch.float64).requires_grad_(True)
    alpha = torch.tensor(p.alpha, dtype=torch.float64, requires_grad=True)
    u = ag.unrolled_pdrq(f, alpha, p64, torch.as_tensor(p.mask, device="cuda"), p.delta, iters=K, ckpt=5,
                         params=prm)
    ((u - to_dev(p.truth, torch.float64)) ** 2).sum().backward()
    df64, _ = oracle.pdrq_grad(geo, p.f, p.mask, p.delta, p.alpha, K, 2.0 * (to_np(u) - p.truth), **kw)
    assert rel_l2(to_np(f.grad), df64) < 1e-8
    assert float(alpha.grad) == pytest.approx(dalpha, rel=1e-6)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_vjp_segment_equals_step_by_step(mods, dtype):
    """tv_pd_vjp_segment (replay and reverse on the device) gives the same cotangents as
    replaying with tv_pd_solve_state and calling tv_pd_vjp_step per iteration."""
    import torch
    ct, ag = mods
    pr = phantom.make_problem("seg", 64, 90, 95, seed=8, n_ellipses=4, n_metal=1, noise="gaussian", alpha=0.05)
    plan = ct.Plan(64, 90, 95, angles=pr.theta, dtype=dtype)
    prm = ag.fixed_scaling(plan, power_iters=20)
    dt = plan.torch_dtype
    f = to_dev(pr.f, dt)
    mask = torch.as_tensor(pr.mask, device="cuda")
    st0 = plan.new_state()
    plan.tv_pd_solve_state(f, mask, pr.alpha, pr.delta, 3, prm, st0)      # a non-zero checkpoint
    L = 4
    rng = np.random.default_rng(1)
    seeds = [to_dev(rng.standard_normal(s), dt) for s in ((64, 64), (90, 95), (2, 64, 64))]
    outs = []
    for mode in ("step", "segment"):
        bu, b1, b2 = (x.clone() for x in seeds)
        gf = torch.zeros((90, 95), dtype=dt, device="cuda")
        ga = torch.zeros(1, dtype=torch.float64, device="cuda")
        if mode == "step":
            states = [{k: v.clone() for k, v in st0.items()}]
            for _ in range(L):
                nxt = {k: v.clone() for k, v in states[-1].items()}
                plan.tv_pd_solve_state(f, mask, pr.alpha, pr.delta, 1, prm, nxt)
                states.append(nxt)
            for k in reversed(range(L)):
                plan.tv_pd_vjp_step(f, mask, pr.alpha, pr.delta, prm, states[k], states[k + 1], bu, b1, b2, gf, ga)
        else:
            plan.tv_pd_vjp_segment(f, mask, pr.alpha, pr.delta, prm, st0, L, plan.vjp_workspace(L), bu, b1, b2, gf,
                                   ga)
        outs.append([to_np(x) for x in (bu, b1, b2, gf)] + [float(ga)])
    for a, b in zip(outs[0][:4], outs[1][:4]):
        np.testing.assert_array_equal(a, b)
    assert outs[0][4] == outs[1][4]
