"""The batched form: many slices of uneven size and view count solved together, one
launch per stage of each iteration over all slices, graph-captured, with the
project-written autotuner choosing the backprojection's angle split.

Parity: each slice of a batch equals the same slice solved alone by tv_pd_solve
(same kernels, same arithmetic) and the FP64 oracle within the FP32 bar."""
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


def _slices():
    # uneven sizes (radix 2 and 3), view counts and bins; one with no metal
    spec = [(32, 40, 46, 1), (48, 25, 69, 2), (64, 90, 91, 0), (96, 57, 136, 2), (24, 33, 34, 1)]
    probs = [phantom.make_problem(f"s{i}", n, N, M, seed=20 + i, n_ellipses=3, n_metal=m, noise="gaussian",
                                  alpha=0.05 * (i + 1)) for i, (n, N, M, m) in enumerate(spec)]
    # slices 1 and 4: angles offset from the uniform grid (no symmetric images: per-angle path)
    for i in (1, 4):
        probs[i].theta = probs[i].theta + 0.013
    return probs


def test_batch_matches_single_slices_and_oracle(ct):
    import torch
    probs = _slices()
    batch = ct.Batch([dict(n=p.n, n_angles=p.n_angles, n_bins=p.n_bins, angles=p.theta) for p in probs])
    fs = [to_dev(p.f, torch.float32) for p in probs]
    ms = [torch.as_tensor(p.mask, device="cuda") for p in probs]
    # uniform angle sets take the symmetric path (slice 3, odd, as pair jobs), offset sets the
    # per-angle path: both in one batch
    assert [pl.symmetric_jobs > 0 for pl in batch.plans] == [True, False, True, True, False]
    betas, cs = [], []
    for p in probs:
        geo = oracle.Geometry(p.n, p.n_angles, p.n_bins, theta=p.theta)
        b = oracle.power_beta(geo, 30)
        betas.append(b)
        cs.append(oracle.power_c(geo, b, np.pi / p.n, 30))
    iters = 40
    prm = ct.default_params(graph_block=8)
    us, diags = batch.solve(fs, ms, [p.alpha for p in probs], [p.delta for p in probs], iters, params=prm,
                            betas=betas, cs=cs)
    for i, p in enumerate(probs):
        plan = ct.Plan(p.n, p.n_angles, p.n_bins, angles=p.theta)
        plan.set_bp_groups(batch.plans[i].bp_groups)
        u1, d1 = plan.tv_pd_solve(fs[i], ms[i], p.alpha, p.delta, iters,
                                  params=ct.default_params(beta=betas[i], c=cs[i], graph_block=8))
        # same kernel bodies; FP32 contraction may differ between the two compiled
        # instances, so agreement is to FP32 rounding, not bit for bit
        assert rel_l2(to_np(us[i]), to_np(u1)) < 2e-6, i
        assert diags[i]["objective"] == pytest.approx(d1["objective"], rel=1e-5)
        geo = oracle.Geometry(p.n, p.n_angles, p.n_bins, theta=p.theta)
        desc = oracle.make_descriptors(p.f, p.mask, p.delta)
        ref = oracle.pdrq_solve(geo, desc, p.alpha, iters, sigma=1.0, tau=1 / np.sqrt(8), eps=np.pi / p.n,
                                beta=betas[i], c=cs[i])
        assert rel_l2(to_np(us[i]), ref.u) < 1e-5, i
    # one launch per stage per iteration, plus per-slice set-up and the last iteration
    assert batch.launch_count > 0


def test_batch_power_iterations_and_single_slice(ct):
    """Without betas/cs the batch runs each slice's power iterations; a batch of one
    slice equals tv_pd_solve."""
    import torch
    p = _slices()[1]
    batch = ct.Batch([dict(n=p.n, n_angles=p.n_angles, n_bins=p.n_bins, angles=p.theta)])
    f = to_dev(p.f, torch.float32)
    m = torch.as_tensor(p.mask, device="cuda")
    us, diags = batch.solve([f], [m], [p.alpha], [p.delta], 30)
    plan = ct.Plan(p.n, p.n_angles, p.n_bins, angles=p.theta)
    plan.set_bp_groups(batch.plans[0].bp_groups)
    u1, d1 = plan.tv_pd_solve(f, m, p.alpha, p.delta, 30)
    assert diags[0]["beta"] == d1["beta"] and diags[0]["c"] == d1["c"]
    assert rel_l2(to_np(us[0]), to_np(u1)) < 2e-6


def test_autotuner_keeps_results(ct, tmp_path, monkeypatch):
    """The tuner picks an angle split by timing; results stay within FP32 rounding of
    the oracle whatever it picks, and the choice is cached."""
    import torch
    from paper_1810_03275_gb300 import autotune
    monkeypatch.setenv("CTR_TUNE_CACHE", str(tmp_path / "tune.json"))
    n, N, M = 256, 180, 363
    plan = ct.Plan(n, N, M)
    G = autotune.tune_plan(plan, reps=2)
    assert plan.bp_groups == G
    geo = oracle.Geometry(n, N, M)
    g = np.random.default_rng(0).standard_normal((N, M))
    got = to_np(plan.rh_adjoint(to_dev(g, torch.float32)))
    assert rel_l2(got, oracle.rh_adjoint(g, geo)) < 1e-5
    assert autotune.tune_plan(ct.Plan(n, N, M), reps=2) == G          # from the cache
    probs = _slices()
    batch = ct.Batch([dict(n=p.n, n_angles=p.n_angles, n_bins=p.n_bins, angles=p.theta) for p in probs])
    fs = [to_dev(p.f, torch.float32) for p in probs]
    pol = autotune.tune_batch(batch, fs, None, [p.alpha for p in probs], [p.delta for p in probs], iters=3)
    assert pol in (None, 1, 2, 4)


def test_batch_rejects_bad_input(ct):
    with pytest.raises(ct.CtrError):
        ct.Batch([dict(n=10, n_angles=8, n_bins=15)])            # n not 2^a 3^b
    with pytest.raises(ct.CtrError):
        ct.Batch([dict(n=16, n_angles=8, n_bins=23, h=1.0, ds=2.0)])


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_batch_with_other_preconditioners(ct, kind):
    """params.precond = 1 (impulse response), 2 (circulant, twisted column pass in the
    batched stage), 3 (Richardson): each slice equals the same slice solved alone with
    that kind (β, c from the slices' own power iterations, which read the kind), and the
    oracle's Alg. 4 with that kind's multiplier."""
    import torch
    probs = _slices()[:4]
    batch = ct.Batch([dict(n=p.n, n_angles=p.n_angles, n_bins=p.n_bins, angles=p.theta) for p in probs])
    fs = [to_dev(p.f, torch.float32) for p in probs]
    ms = [torch.as_tensor(p.mask, device="cuda") for p in probs]
    iters = 25
    prm = ct.default_params(graph_block=8, precond=kind, power_iters=25)
    us, diags = batch.solve(fs, ms, [p.alpha for p in probs], [p.delta for p in probs], iters, params=prm)
    for i, p in enumerate(probs):
        plan = ct.Plan(p.n, p.n_angles, p.n_bins, angles=p.theta)
        plan.set_bp_groups(batch.plans[i].bp_groups)
        u1, d1 = plan.tv_pd_solve(fs[i], ms[i], p.alpha, p.delta, iters, params=prm)
        assert diags[i]["c"] == pytest.approx(d1["c"], rel=1e-6) and diags[i]["beta"] == pytest.approx(d1["beta"], rel=1e-6)
        assert rel_l2(to_np(us[i]), to_np(u1)) < 2e-6, i
        geo = oracle.Geometry(p.n, p.n_angles, p.n_bins, theta=p.theta)
        tau, c = 1 / np.sqrt(8), d1["c"]
        if kind == 1:
            sym, circ = oracle.precond_symbol_from(p.n, 1.0, tau, c, oracle.impulse_response_kernel_dft(geo)), False
        elif kind == 2:
            sym = oracle.precond_symbol_circulant(p.n, 1.0, tau, c, oracle.circulant_kernel_dft(geo),
                                                  oracle.circulant_laplace_dft(p.n))
            circ = True
        else:
            sym, circ = np.full((p.n, p.n), 1.0 / oracle.richardson_m(1.0, tau, c)), False
        ref = oracle.pdrq_solve(geo, oracle.make_descriptors(p.f, p.mask, p.delta), p.alpha, iters, sigma=1.0,
                                tau=tau, eps=np.pi / p.n, beta=d1["beta"], c=c, symbol=sym, circulant=circ)
        assert rel_l2(to_np(us[i]), ref.u) < 1e-5, i


def test_batch_alg5(ct):
    """params.nonneg = 1 in a batch (symmetric and per-angle slices): each slice equals
    the same slice solved alone by Alg. 5 and the oracle's Alg. 5; gap and dual residual
    are NaN as for single solves."""
    import torch
    probs = _slices()[:4]
    batch = ct.Batch([dict(n=p.n, n_angles=p.n_angles, n_bins=p.n_bins, angles=p.theta) for p in probs])
    fs = [to_dev(p.f, torch.float32) for p in probs]
    ms = [torch.as_tensor(p.mask, device="cuda") for p in probs]
    iters = 30
    prm = ct.default_params(graph_block=8, nonneg=1, power_iters=25)
    us, diags = batch.solve(fs, ms, [p.alpha for p in probs], [p.delta for p in probs], iters, params=prm)
    for i, p in enumerate(probs):
        plan = ct.Plan(p.n, p.n_angles, p.n_bins, angles=p.theta)
        plan.set_bp_groups(batch.plans[i].bp_groups)
        u1, d1 = plan.tv_pd_solve(fs[i], ms[i], p.alpha, p.delta, iters, params=prm)
        assert rel_l2(to_np(us[i]), to_np(u1)) < 2e-6, i
        assert np.isnan(diags[i]["gap"]) and np.isfinite(diags[i]["objective"])
        geo = oracle.Geometry(p.n, p.n_angles, p.n_bins, theta=p.theta)
        ref = oracle.pdrq5_solve(geo, oracle.make_descriptors(p.f, p.mask, p.delta), p.alpha, iters, sigma=1.0,
                                 tau=1 / np.sqrt(8), eps=np.pi / p.n, beta=d1["beta"], c=d1["c"])
        assert rel_l2(to_np(us[i]), ref.u) < 1e-5, i


def test_persistent_iteration_matches_staged_form(ct):
    """mode 1 (one persistent cooperative launch per iteration, stages separated by grid
    barriers) gives the same slices as mode 0 (one launch per stage) and the oracle; one
    launch per iteration."""
    import torch
    probs = _slices()
    batch = ct.Batch([dict(n=p.n, n_angles=p.n_angles, n_bins=p.n_bins, angles=p.theta) for p in probs])
    assert batch.mode == 0 and batch.persistent_ctas > 0
    fs = [to_dev(p.f, torch.float32) for p in probs]
    ms = [torch.as_tensor(p.mask, device="cuda") for p in probs]
    betas, cs = [], []
    for p in probs:
        geo = oracle.Geometry(p.n, p.n_angles, p.n_bins, theta=p.theta)
        b = oracle.power_beta(geo, 30)
        betas.append(b)
        cs.append(oracle.power_c(geo, b, np.pi / p.n, 30))
    iters = 25
    al, de = [p.alpha for p in probs], [p.delta for p in probs]
    u0, d0 = batch.solve(fs, ms, al, de, iters, params=ct.default_params(graph_block=8), betas=betas, cs=cs)
    batch.set_mode(1)
    l0 = batch.launch_count
    u1, d1 = batch.solve(fs, ms, al, de, iters, params=ct.default_params(graph_block=8), betas=betas, cs=cs)
    assert batch.mode == 1
    for i, p in enumerate(probs):
        assert rel_l2(to_np(u1[i]), to_np(u0[i])) < 2e-6, i
        assert d1[i]["objective"] == pytest.approx(d0[i]["objective"], rel=1e-5)
        geo = oracle.Geometry(p.n, p.n_angles, p.n_bins, theta=p.theta)
        ref = oracle.pdrq_solve(geo, oracle.make_descriptors(p.f, p.mask, p.delta), p.alpha, iters, sigma=1.0,
                                tau=1 / np.sqrt(8), eps=np.pi / p.n, beta=betas[i], c=cs[i])
        assert rel_l2(to_np(u1[i]), ref.u) < 1e-5, i
    batch.set_mode(0)
    assert batch.mode == 0


def test_persistent_grid_barrier_gives_up(ct):
    """With a spin limit of 0 every grid barrier gives up at once: the launch ends early,
    the status word is set and the solve reports CTR_ETIMEOUT; the next solve (normal
    limit) is unaffected."""
    import torch
    probs = _slices()[:3]
    batch = ct.Batch([dict(n=p.n, n_angles=p.n_angles, n_bins=p.n_bins, angles=p.theta) for p in probs])
    fs = [to_dev(p.f, torch.float32) for p in probs]
    al, de = [p.alpha for p in probs], [p.delta for p in probs]
    kw = dict(params=ct.default_params(), betas=[30.0] * 3, cs=[1.0] * 3)
    ref, _ = batch.solve(fs, None, al, de, 6, **kw)
    batch.set_mode(1, spin_limit=0)
    with pytest.raises(ct.CtrError) as e:
        batch.solve(fs, None, al, de, 6, **kw)
    assert e.value.status == -4
    batch.set_mode(1)
    got, _ = batch.solve(fs, None, al, de, 6, **kw)
    for a, b in zip(got, ref):
        assert rel_l2(to_np(a), to_np(b)) < 2e-6
    with pytest.raises(ct.CtrError):
        batch.set_mode(2)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_forward_shape_variants_agree(ct, dtype):
    """The symmetric forward projector's launch shape (adjacent jobs per CTA, warps per job)
    is a runtime choice among compiled instances: every shape matches the oracle (on the
    BF16 plan, for the rounded input), and the autotuner sets one of them."""
    import torch
    n, N, M = 96, 120, 137
    plan = ct.Plan(n, N, M, dtype=dtype)
    assert plan.fwd_shape == (1, 4)
    u = torch.randn((n, n), device="cuda").to(plan.op_dtype)
    ref = oracle.rh_forward(u.double().cpu().numpy(), oracle.Geometry(n, N, M))
    outs = {}
    for shp in plan.FWD_SHAPES:
        plan.set_fwd_shape(*shp)
        assert plan.fwd_shape == shp
        outs[shp] = to_np(plan.rh_forward(u))
        assert rel_l2(outs[shp], ref) < 1e-5, shp
    assert rel_l2(outs[(1, 2)], outs[(4, 2)]) < 2e-6
    with pytest.raises(ct.CtrError):
        plan.set_fwd_shape(3, 4)
    with pytest.raises(ct.CtrError):
        ct.Plan(n, N, M, dtype="f64").set_fwd_shape(1, 2)


def test_autotuner_picks_forward_shape(ct, tmp_path, monkeypatch):
    from paper_1810_03275_gb300 import autotune
    monkeypatch.setenv("CTR_TUNE_CACHE", str(tmp_path / "tune.json"))
    plan = ct.Plan(256, 180, 363)
    autotune.tune_plan(plan, reps=2)
    assert plan.fwd_shape in plan.FWD_SHAPES
    shp = plan.fwd_shape
    other = ct.Plan(256, 180, 363)
    autotune.tune_plan(other, reps=2)                    # from the cache
    assert other.fwd_shape == shp


def test_solve_tuner_keeps_results(ct, tmp_path, monkeypatch):
    """The solve-level tuner (split and forward shape timed on Alg. 4 itself) leaves the
    iterates within FP32 rounding of the oracle."""
    import torch
    from paper_1810_03275_gb300 import autotune
    monkeypatch.setenv("CTR_TUNE_CACHE", str(tmp_path / "tune.json"))
    p = phantom.make_problem("ts", 96, 120, 137, seed=7, n_ellipses=4, n_metal=1, noise="gaussian", alpha=0.05)
    plan = ct.Plan(p.n, p.n_angles, p.n_bins, angles=p.theta)
    geo = oracle.Geometry(p.n, p.n_angles, p.n_bins, theta=p.theta)
    beta = oracle.power_beta(geo, 20)
    c = oracle.power_c(geo, beta, np.pi / p.n, 20)
    prm = ct.default_params(beta=beta, c=c)
    f, m = to_dev(p.f, torch.float32), torch.as_tensor(p.mask, device="cuda")
    choice = autotune.tune_solve(plan, f, m, p.alpha, p.delta, iters=5, reps=1, params=prm)
    assert choice["bp_groups"] == plan.bp_groups and tuple(choice["fwd_shape"]) == plan.fwd_shape
    u, _ = plan.tv_pd_solve(f, m, p.alpha, p.delta, 20, params=prm)
    ref = oracle.pdrq_solve(geo, oracle.make_descriptors(p.f, p.mask, p.delta), p.alpha, 20, sigma=1.0,
                            tau=1 / np.sqrt(8), eps=np.pi / p.n, beta=beta, c=c)
    assert rel_l2(to_np(u), ref.u) < 1e-5
