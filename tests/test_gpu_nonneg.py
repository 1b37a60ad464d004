"""GPU parity of Alg. 5 (PDRQS1 with the non-negativity constraint u >= 0, params.nonneg = 1)
with the oracle: iterates at fixed (beta, c) on both projector paths, the preconditioner
symbol through precond_apply, resume through the state's bar u, the constraint holding
at the end of a long solve, and the entry points that refuse it."""
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
    """Noisy data (5 % Gaussian), small alpha: the unconstrained iterates go negative,
    so the constraint is active."""
    pr = phantom.make_problem("nn", n, N, M, seed=seed, n_ellipses=4, n_metal=1, noise="gaussian", alpha=0.02)
    th = pr.theta if kind == "uniform" else np.random.default_rng(seed).uniform(0, np.pi, N)
    f = pr.f
    if kind != "uniform":
        geo = oracle.Geometry(n, N, M, theta=th)
        f = oracle.rh_forward(pr.truth, geo)
    f = f + 0.05 * np.abs(f).max() * np.random.default_rng(seed + 1).standard_normal(f.shape)
    return th, f, pr.mask, pr.alpha, pr.delta


def _alg4_min(n, N, M, kind, iters=150):
    th, f, mask, alpha, delta = _problem(n, N, M, kind)
    geo = oracle.Geometry(n, N, M, theta=th)
    eps = np.pi / n
    beta = oracle.power_beta(geo, 30)
    c = oracle.power_c(geo, beta, eps, 30)
    u = oracle.pdrq_solve(geo, oracle.make_descriptors(f, mask, delta), alpha, iters, sigma=1.0,
                          tau=1 / np.sqrt(8), eps=eps, beta=beta, c=c).u
    return u.min() / np.abs(u).max()


def _run(ct, n, N, M, kind, dtype, iters_list):
    th, f, mask, alpha, delta = _problem(n, N, M, kind)
    geo = oracle.Geometry(n, N, M, theta=th)
    desc = oracle.make_descriptors(f, mask, delta)
    sigma, tau, eps = 1.0, 1 / np.sqrt(8), np.pi / n
    beta = oracle.power_beta(geo, 30)
    c = oracle.power_c(geo, beta, eps, 30)
    plan = ct.Plan(n, N, M, angles=th, dtype=dtype)
    prm = ct.default_params(sigma=sigma, tau=tau, eps=eps, beta=beta, c=c, graph_block=4, nonneg=1)
    dev = [to_dev(x, plan.torch_dtype) for x in desc]
    state = plan.new_state()
    st, done, out = None, 0, []
    for k in iters_list:
        st = oracle.pdrq5_solve(geo, desc, alpha, k - done, sigma=sigma, tau=tau, eps=eps, beta=beta, c=c, state=st)
        plan.tv_pd_run(*dev, alpha, k - done, params=prm, state=state)
        out.append((k, st.copy(), {kk: to_np(v) for kk, v in state.items()}))
        done = k
    return out, plan


@pytest.mark.parametrize("kind", ["uniform", "random"])
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-9), ("f32", 1e-5)])
def test_alg5_iterates_match_oracle(ct, kind, dtype, tol):
    """u, bar u, R u and both duals after 1, 10 and 150 iterations; uniform angles take the
    symmetric projector path (FP32), random angles the per-angle path."""
    res, plan = _run(ct, 48, 60, 71, kind, dtype, [1, 10, 150])
    if dtype == "f32":
        assert (plan.symmetric_jobs > 0) == (kind == "uniform")
    for k, ref, got in res:
        b = tol
        assert rel_l2(got["u"], ref.u) < b, (k, rel_l2(got["u"], ref.u))
        if k > 1:
            assert rel_l2(got["ub"], ref.ub) < b, (k, rel_l2(got["ub"], ref.ub))
        assert rel_l2(got["Ru"], ref.Ru) < b
        assert rel_l2(got["v1b"], ref.v1b) < b
        assert rel_l2(got["v2b"], np.stack([ref.v2bx, ref.v2by])) < b
    # the constraint is active: the oracle's Alg. 4 on the same data goes clearly negative
    assert _alg4_min(48, 60, 71, kind) < -0.1


def test_alg5_preconditioner_symbol(ct):
    import torch
    n = 36
    plan = ct.Plan(n, 30, 53, dtype="f64")
    y = np.random.default_rng(2).standard_normal((n, n))
    prm = ct.default_params(sigma=0.8, tau=0.3, eps=0.2, c=1.3, nonneg=1)
    got = to_np(plan.precond_apply(to_dev(y, torch.float64), prm))
    ref = oracle.precond_apply(y, oracle.precond_symbol_nonneg(n, 0.8, 0.3, 1.3, 0.2))
    assert rel_l2(got, ref) < 1e-12
    prm4 = ct.default_params(sigma=0.8, tau=0.3, eps=0.2, c=1.3)
    assert rel_l2(to_np(plan.precond_apply(to_dev(y, torch.float64), prm4)), ref) > 1e-3


def test_alg5_resume_equals_continuous_run(ct):
    """Running 9 then 6 iterations through the state (bar u included) equals 15 at once."""
    res_a, _ = _run(ct, 32, 40, 47, "uniform", "f64", [15])
    res_b, _ = _run(ct, 32, 40, 47, "uniform", "f64", [9, 15])
    a, b = res_a[-1][2], res_b[-1][2]
    for key in ("u", "ub", "v1b", "v2b"):
        assert rel_l2(b[key], a[key]) < 1e-12, key


def test_alg5_solution_is_nonnegative(ct):
    """A long FP32 solve through tv_pd_solve ends with u >= 0 up to the solver's
    tolerance, where Alg. 4 on the same data leaves clearly negative pixels."""
    import torch
    n, N, M = 64, 90, 95
    th, f, mask, alpha, delta = _problem(n, N, M, "uniform")
    plan = ct.Plan(n, N, M, angles=th)
    fd = to_dev(f, torch.float32)
    md = torch.as_tensor(mask, device="cuda")
    u5, d5 = plan.tv_pd_solve(fd, md, alpha, delta, 3000, params=ct.default_params(nonneg=1))
    u4, _ = plan.tv_pd_solve(fd, md, alpha, delta, 3000)
    u5, u4 = to_np(u5), to_np(u4)
    scale = np.abs(u4).max()
    assert u4.min() < -0.02 * scale
    assert u5.min() > -1e-3 * scale
    assert np.isnan(d5["gap"]) and np.isfinite(d5["objective"])


def test_alg5_refused_where_not_covered(ct):
    import torch
    plan = ct.Plan(32, 20, 47)
    with pytest.raises(Exception, match="nonneg"):
        plan.tv_pd_solve(torch.zeros((20, 47), device="cuda"), None, 0.1, -1.0, 2,
                         params=ct.default_params(nonneg=2))
    batch = ct.Batch([dict(n=32, n_angles=20, n_bins=47)])
    with pytest.raises(Exception, match="nonneg"):
        batch.solve([torch.zeros((20, 47), device="cuda")], [None], [0.1], [-1.0], 2,
                    params=ct.default_params(nonneg=3))


def test_alg5_at_a_warp_fft_size(ct):
    """Alg. 5 on a 256 x 256 FP32 plan (symmetric path, warp-level preconditioner passes whose
    first pass folds the partial planes with the u >= 0 epilogue): iterates after 1 and 10
    iterations equal the oracle's."""
    res, plan = _run(ct, 256, 90, 363, "uniform", "f32", [1, 10])
    assert plan.symmetric_jobs > 0 and plan.fft_form == 0
    for k, ref, got in res:
        assert rel_l2(got["u"], ref.u) < 1e-5, (k, rel_l2(got["u"], ref.u))
        if k > 1:
            assert rel_l2(got["ub"], ref.ub) < 1e-5
        assert rel_l2(got["v1b"], ref.v1b) < 1e-5
