"""GPU parity of Alg. 4 (tv_pd_run / tv_pd_solve through the C ABI) with the oracle:
per-iterate agreement at fixed (beta, c), the end-to-end 64 x 64 FP64 solve, edge
cases, argument errors, and properties of the 512 x 512 benchmark solve."""
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


def _run_both(ct, n, N, M, dtype, iters_list, *, metal=True, delta=None, alpha=0.05, seed=3, graph_block=4):
    pr = phantom.make_problem("t", n, N, M, seed=seed, n_ellipses=4, n_metal=2 if metal else 0,
                              noise="gaussian", alpha=alpha)
    if delta is None:
        delta = pr.delta
    geo = oracle.Geometry(n, N, M, theta=pr.theta)
    desc = oracle.make_descriptors(pr.f, pr.mask, delta)
    sigma, tau, eps = 1.0, 1 / np.sqrt(8), np.pi / n
    beta = oracle.power_beta(geo, 30)
    c = oracle.power_c(geo, beta, eps, 30)
    plan = ct.Plan(n, N, M, angles=pr.theta, dtype=dtype)
    prm = ct.default_params(sigma=sigma, tau=tau, eps=eps, beta=beta, c=c, graph_block=graph_block)
    dev = [to_dev(x, plan.torch_dtype) for x in desc]
    state = plan.new_state()
    st = None
    out = []
    done = 0
    for k in iters_list:
        st = oracle.pdrq_solve(geo, desc, pr.alpha, k - done, sigma=sigma, tau=tau, eps=eps, beta=beta, c=c, state=st)
        plan.tv_pd_run(*dev, pr.alpha, k - done, params=prm, state=state)
        out.append((k, st.copy(), {kk: to_np(v) for kk, v in state.items()}))
        done = k
    return out, plan, geo, desc


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-9), ("f32", 1e-5)])
def test_iterates_match_oracle(ct, dtype, tol):
    """u_k, R u_k and the duals after 1, 10 and 200 iterations on the 64 x 64, 90-angle
    geometry with metal-trace constraints (graph-captured blocks of 4 iterations)."""
    res, *_ = _run_both(ct, 64, 90, 95, dtype, [1, 10, 200])
    for k, ref, got in res:
        assert rel_l2(got["u"], ref.u) < tol, (k, rel_l2(got["u"], ref.u))
        assert rel_l2(got["Ru"], ref.Ru) < tol
        assert rel_l2(got["v1b"], ref.v1b) < tol
        v2 = np.stack([ref.v2bx, ref.v2by])
        assert rel_l2(got["v2b"], v2) < tol, (k, rel_l2(got["v2b"], v2))


def test_ragged_and_radix3_sizes(ct):
    """n = 48 (radix-3 FFT, ragged tiles), odd M, no metal, no box (delta < 0)."""
    res, *_ = _run_both(ct, 48, 37, 71, "f32", [5, 30], metal=False, delta=-1.0)
    for k, ref, got in res:
        assert rel_l2(got["u"], ref.u) < 1e-5, k


def test_end_to_end_fp64_configuration(ct):
    """The 64 x 64 FP64 configuration (6 ellipses, 90 angles, 95 bins, 1 % noise,
    alpha = 0.01, delta = 3 sigma, 200 iterations) solved by tv_pd_solve with its own
    power iterations vs the oracle's full pipeline."""
    import torch
    pr = phantom.config_plain_fp64()
    geo = oracle.Geometry(pr.n, pr.n_angles, pr.n_bins, theta=pr.theta)
    eps = np.pi / pr.n
    beta = oracle.power_beta(geo, 50)
    c = 1.05 * oracle.power_c(geo, beta, eps, 50, margin=1.0)
    desc = oracle.make_descriptors(pr.f, pr.mask, pr.delta)
    ref = oracle.pdrq_solve(geo, desc, pr.alpha, pr.iters, sigma=1.0, tau=1 / np.sqrt(8), eps=eps, beta=beta, c=c)
    plan = ct.Plan(pr.n, pr.n_angles, pr.n_bins, angles=pr.theta, dtype="f64")
    u, diag = plan.tv_pd_solve(to_dev(pr.f, torch.float64), None, pr.alpha, pr.delta, pr.iters)
    assert diag["beta"] == pytest.approx(beta, rel=1e-12)
    assert diag["c"] == pytest.approx(c, rel=1e-10)
    assert rel_l2(to_np(u), ref.u) < 1e-9
    d = oracle.diagnostics(geo, desc, pr.alpha, ref.u, beta=beta, tau=1 / np.sqrt(8), t1=ref.t1, t2x=ref.t2x, t2y=ref.t2y)
    for key in ("objective", "tv", "data_fit"):
        assert diag[key] == pytest.approx(d[key], rel=1e-9), key
    assert diag["violation"] == pytest.approx(d["violation"], rel=1e-6, abs=1e-9)
    assert diag["gap"] == pytest.approx(d["gap"], rel=1e-6, abs=1e-9)
    assert diag["dual_residual"] == pytest.approx(d["dual_residual"], rel=1e-6)


def test_edge_cases(ct):
    """alpha = 0, delta = 0 (hard data constraint), the whole sinogram on the metal
    trace, zero iterations, and a single-angle geometry."""
    import torch
    n, N, M = 24, 20, 35
    rng = np.random.default_rng(5)
    geo = oracle.Geometry(n, N, M)
    f = oracle.rh_forward(rng.uniform(0, 1, (n, n)), geo)
    plan = ct.Plan(n, N, M, dtype="f64")
    beta = oracle.power_beta(geo, 20)
    c = oracle.power_c(geo, beta, np.pi / n, 20)
    prm = ct.default_params(beta=beta, c=c, eps=np.pi / n, graph_block=0)
    for alpha, delta, mask in [(0.0, 0.5, None), (0.1, 0.0, None), (0.1, 0.5, np.ones((N, M), np.uint8))]:
        desc = oracle.make_descriptors(f, mask, delta)
        ref = oracle.pdrq_solve(geo, desc, alpha, 15, sigma=1.0, tau=1 / np.sqrt(8), eps=np.pi / n, beta=beta, c=c)
        m = None if mask is None else torch.as_tensor(mask, device="cuda")
        u, _ = plan.tv_pd_solve(to_dev(f, torch.float64), m, alpha, delta, 15, params=prm)
        assert rel_l2(to_np(u), ref.u) < 1e-10
    u, d = plan.tv_pd_solve(to_dev(f, torch.float64), None, 0.1, 0.5, 0, params=prm)
    assert float(u.abs().max()) == 0.0 and d["iters_done"] == 0
    p1 = ct.Plan(16, 1, 23)
    g = p1.rh_forward(torch.ones((16, 16), device="cuda"))
    assert float(g.sum()) == pytest.approx(256.0, rel=1e-6)


def test_argument_errors(ct):
    import torch
    plan = ct.Plan(16, 8, 23)
    f = torch.zeros((8, 23), device="cuda")
    with pytest.raises(ct.CtrError) as e:
        plan.tv_pd_solve(f, None, -1.0, 0.1, 3)
    assert e.value.status == -1
    with pytest.raises(ct.CtrError):
        plan.tv_pd_solve(f, None, 0.1, float("nan"), 3)
    with pytest.raises(ct.CtrError):
        plan.tv_pd_solve(f, None, 0.1, 0.1, -2)
    with pytest.raises(ct.CtrError):
        plan.tv_pd_solve(f, None, 0.1, 0.1, 3, params=ct.default_params(sigma=0.0))
    with pytest.raises(ct.CtrError):
        ct.Plan(0, 8, 23)
    with pytest.raises(ct.CtrError):
        ct.Plan(16, 8, 23, h=1.0, ds=3.0)
    with pytest.raises(TypeError):
        plan.rh_forward(torch.zeros((16, 16), device="cuda", dtype=torch.float64))


def test_benchmark_configuration_properties(ct):
    """512 x 512, 720 x 729, metal trace, Poisson data: two iterations agree with the
    oracle; after the full 500 iterations the result is finite, the objective and the
    trace violation fell, and the reconstruction beats the data's noise floor."""
    import torch
    pr = phantom.config_mar_fp32()
    geo = oracle.Geometry(pr.n, pr.n_angles, pr.n_bins, theta=pr.theta)
    plan = ct.Plan(pr.n, pr.n_angles, pr.n_bins, angles=pr.theta)
    f = to_dev(pr.f, torch.float32)
    mask = torch.as_tensor(pr.mask, device="cuda")
    beta = plan.power_beta(50)
    lam = plan.power_lambda(beta, np.pi / pr.n, 50)
    prm = ct.default_params(beta=beta, c=1.05 * lam)
    desc = oracle.make_descriptors(pr.f, pr.mask, pr.delta)
    ref = oracle.pdrq_solve(geo, desc, pr.alpha, 2, sigma=1.0, tau=1 / np.sqrt(8), eps=np.pi / pr.n, beta=beta,
                            c=1.05 * lam)
    u2, _ = plan.tv_pd_solve(f, mask, pr.alpha, pr.delta, 2, params=prm)
    assert rel_l2(to_np(u2), ref.u) < 1e-5
    u, d = plan.tv_pd_solve(f, mask, pr.alpha, pr.delta, pr.iters, params=prm)
    un = to_np(u)
    assert np.all(np.isfinite(un))
    d0 = oracle.diagnostics(geo, desc, pr.alpha, np.zeros((pr.n, pr.n)))
    assert d["objective"] < 0.05 * d0["objective"]
    assert d["violation"] < 0.2 * d0["violation"]
    assert d["rel_change"] < 1e-2


@pytest.mark.parametrize("n,N,M", [(64, 91, 95), (96, 121, 137), (256, 181, 363)])
def test_odd_view_count_pair_jobs(ct, n, N, M):
    """Odd view counts on [0, pi): every angle but 0 pairs only with its mirror pi - theta,
    so the symmetric path runs (N + 1) / 2 pair jobs (two live channels each).  Iterates after
    1 and 20 FP32 iterations equal the oracle's."""
    res, plan, *_ = _run_both(ct, n, N, M, "f32", [1, 20])
    assert plan.symmetric_jobs == (N + 1) // 2
    for k, ref, got in res:
        assert rel_l2(got["u"], ref.u) < 1e-5, (k, rel_l2(got["u"], ref.u))
        assert rel_l2(got["Ru"], ref.Ru) < 1e-5
        assert rel_l2(got["v1b"], ref.v1b) < 1e-5
