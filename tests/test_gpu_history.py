"""The diagnostics cadence (params.check_every): every k-th iteration the solve records
the objective, data fit, TV, constraint violation, Fenchel-Young gap, dual residual and
relative change on the device, and ctr_plan_history returns them -- the convergence
record of the thesis's Sec. 5 (objective against the iteration count).  Each record is
compared with the oracle's diagnostics() of its own Alg. 4 run at the same iterate;
stop_tol ends the solve at the first check whose relative change is small enough."""
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


def _oracle_history(geo, desc, alpha, iters, every, kw, nonneg=False):
    """diagnostics() of the oracle's iterate after every `every` iterations, with the
    relative change ||u_k - u_{k-1}|| / ||u_k|| of the last step."""
    out = []
    prev = {"u": np.zeros(geo.image_shape)}

    def cb(st):
        if st.k % every == 0:
            d = oracle.diagnostics(geo, desc, alpha, st.u, beta=kw["beta"], tau=kw["tau"], t1=st.t1, t2x=st.t2x,
                                   t2y=st.t2y)
            nu = np.linalg.norm(st.u)
            d["rel_change"] = float(np.linalg.norm(st.u - prev["u"]) / nu) if nu > 0 else 0.0
            d["iters_done"] = st.k
            out.append(d)
        prev["u"] = st.u.copy()

    oracle.pdrq_solve(geo, desc, alpha, iters, callback=cb, **kw)
    return out


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-9), ("f32", 1e-4)])
def test_history_matches_oracle_diagnostics(ct, dtype, tol):
    """48 x 48, 60 angles, metal trace and data box, 60 iterations checked every 7 (the
    last 4 iterations after the 8th check run without one), graph blocks of 4."""
    import torch
    pr = phantom.make_problem("h", 48, 60, 71, seed=13, n_ellipses=4, n_metal=2, noise="gaussian", alpha=0.05)
    geo = oracle.Geometry(pr.n, pr.n_angles, pr.n_bins, theta=pr.theta)
    eps, tau = np.pi / pr.n, 1 / np.sqrt(8)
    beta = oracle.power_beta(geo, 30)
    c = oracle.power_c(geo, beta, eps, 30)
    desc = oracle.make_descriptors(pr.f, pr.mask, pr.delta)
    kw = dict(sigma=1.0, tau=tau, eps=eps, beta=beta, c=c)
    iters, every = 60, 7
    ref = _oracle_history(geo, desc, pr.alpha, iters, every, kw)
    plan = ct.Plan(pr.n, pr.n_angles, pr.n_bins, angles=pr.theta, dtype=dtype)
    prm = ct.default_params(beta=beta, c=c, eps=eps, graph_block=4, check_every=every)
    u, d = plan.tv_pd_solve(to_dev(pr.f, plan.torch_dtype), torch.as_tensor(pr.mask, device="cuda"), pr.alpha,
                            pr.delta, iters, params=prm)
    hist = plan.history()
    assert len(hist) == len(ref) == iters // every
    for got, want in zip(hist, ref):
        assert got["iters_done"] == want["iters_done"]
        assert got["beta"] == beta and got["c"] == c
        for key in ("objective", "data_fit", "tv", "dual_residual", "rel_change"):
            assert got[key] == pytest.approx(want[key], rel=tol), (want["iters_done"], key, got[key], want[key])
        scale = max(abs(want["objective"]) / beta ** 2, 1e-12)
        assert abs(got["gap"] - want["gap"]) <= tol * scale + 1e-12, (want["iters_done"], got["gap"], want["gap"])
        vrel = 1e-6 if dtype == "f64" else 1e-3
        assert got["violation"] == pytest.approx(want["violation"], rel=vrel, abs=tol * pr.delta)
    # the solve itself is unchanged by the checks
    u0, d0 = plan.tv_pd_solve(to_dev(pr.f, plan.torch_dtype), torch.as_tensor(pr.mask, device="cuda"), pr.alpha,
                              pr.delta, iters, params=ct.default_params(beta=beta, c=c, eps=eps, graph_block=4))
    assert torch.equal(u, u0)
    assert d["objective"] == d0["objective"] and d["iters_done"] == iters
    assert plan.history() == []            # a solve without checks leaves no records


def test_history_of_alg5_and_alg3(ct):
    """Alg. 5 records NaN for the gap and the dual residual (they belong to Alg. 4's saddle
    problem); Alg. 3 records objectives that equal its final diagnostics at the end."""
    import torch
    pr = phantom.make_problem("h5", 32, 40, 47, seed=3, n_ellipses=3, n_metal=1, noise="gaussian", alpha=0.05)
    plan = ct.Plan(pr.n, pr.n_angles, pr.n_bins, angles=pr.theta, dtype="f64")
    f = to_dev(pr.f, torch.float64)
    prm = ct.default_params(check_every=5, nonneg=1, graph_block=2)
    _, d = plan.tv_pd_solve(f, None, pr.alpha, pr.delta, 20, params=prm)
    hist = plan.history()
    assert len(hist) == 4 and all(np.isnan(h["gap"]) and np.isnan(h["dual_residual"]) for h in hist)
    assert hist[-1]["objective"] == pytest.approx(d["objective"], rel=1e-12)
    _, d3 = plan.tv_pdrq2_solve(f, pr.alpha, 20, params=ct.default_params(check_every=10))
    h3 = plan.history()
    assert [h["iters_done"] for h in h3] == [10, 20]
    assert h3[-1]["objective"] == pytest.approx(d3["objective"], rel=1e-12)
    assert h3[-1]["gap"] == pytest.approx(d3["gap"], rel=1e-9, abs=1e-14)


def test_stop_tol_ends_the_solve_early(ct):
    """With stop_tol the solve stops at the first check whose relative change is below it;
    the result equals a solve of exactly that many iterations."""
    import torch
    pr = phantom.make_problem("st", 32, 40, 47, seed=4, n_ellipses=3, n_metal=0, noise="gaussian", alpha=0.05)
    plan = ct.Plan(pr.n, pr.n_angles, pr.n_bins, angles=pr.theta, dtype="f64")
    f = to_dev(pr.f, torch.float64)
    base = dict(beta=plan.power_beta(30), graph_block=3)
    _, full = plan.tv_pd_solve(f, None, pr.alpha, pr.delta, 400, params=ct.default_params(check_every=10, **base))
    hist = plan.history()
    tol = hist[5]["rel_change"] * 1.0000001       # reached at the 6th check (rel_change need not be monotone)
    first = next(h["iters_done"] for h in hist if h["rel_change"] <= tol)
    u, d = plan.tv_pd_solve(f, None, pr.alpha, pr.delta, 400,
                            params=ct.default_params(check_every=10, stop_tol=tol, **base))
    assert d["iters_done"] == first < 400
    assert len(plan.history()) == first // 10
    u2, _ = plan.tv_pd_solve(f, None, pr.alpha, pr.delta, first, params=ct.default_params(**base))
    assert rel_l2(to_np(u), to_np(u2)) < 1e-12


def test_cadence_argument_errors(ct):
    import torch
    plan = ct.Plan(16, 8, 23)
    f = torch.zeros((8, 23), device="cuda")
    with pytest.raises(ct.CtrError) as e:                       # stop_tol needs checks
        plan.tv_pd_solve(f, None, 0.1, 0.1, 3, params=ct.default_params(stop_tol=1e-3))
    assert e.value.status == -1
    with pytest.raises(ct.CtrError) as e:                       # more checks than records
        plan.tv_pd_solve(f, None, 0.1, 0.1, 4097, params=ct.default_params(check_every=1))
    assert e.value.status == -1
    with pytest.raises(ct.CtrError) as e:                       # Alg. 1 has no cadence
        plan.tv_cp_solve(f, None, 0.1, 0.1, 3, params=ct.default_params(check_every=1))
    assert e.value.status == -6
    with pytest.raises(ct.CtrError) as e:
        plan.tv_admm_solve(f, 0.1, 3, params=ct.default_params(check_every=1))
    assert e.value.status == -6
