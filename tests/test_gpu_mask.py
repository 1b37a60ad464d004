"""GPU metal-trace estimation (ctr_metal_trace) and the metal-artifact pipeline
(tv_mar_solve) against the oracle: marks bit-exact, the trace bit-exact except at bins
whose projected mark value lies within the projector's rounding of the tolerance, the
BF16 plan equal to the FP32 one, and the pipeline equal to its three stages run one by
one, with the estimated trace covering the true one."""
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


def _image(n, seed):
    """A metal phantom plus noise, kept 1e-3 away from the threshold 2.0."""
    ph = phantom.random_phantom(n, 4, seed, n_metal=2, metal_value=3.0)
    u = phantom.rasterize(ph) + 0.05 * np.random.default_rng(seed).standard_normal((n, n))
    u[np.abs(u - 2.0) < 1e-3] = 2.0 + 1e-3
    return u


def _compare_trace(got, u, geo, radius, tol, band):
    marked, ref = oracle.metal_trace_estimate(u, geo, 2.0, radius, tol)
    proj = oracle.rh_forward(marked.astype(np.float64), geo)
    sure = np.abs(proj - tol) > band
    assert sure.mean() > 0.99
    np.testing.assert_array_equal(got[sure], ref[sure])
    return marked, ref


@pytest.mark.parametrize("n,N,M,dtype,band,radius", [(64, 90, 95, "f64", 1e-9, 5), (64, 90, 95, "f32", 1e-5, 5),
                                                     (48, 37, 71, "f32", 1e-5, 0), (96, 41, 137, "f64", 1e-9, 3)])
def test_trace_matches_oracle(ct, n, N, M, dtype, band, radius):
    geo = oracle.Geometry(n, N, M)
    plan = ct.Plan(n, N, M, dtype=dtype)
    u = _image(n, 3)
    trace, marks = plan.metal_trace(to_dev(u, plan.torch_dtype), 2.0, radius, 1e-3, want_marks=True)
    marked, _ = _compare_trace(to_np(trace), u, geo, radius, 1e-3, band)
    np.testing.assert_array_equal(to_np(marks), marked)


def test_benchmark_geometry_and_bf16(ct):
    """512 x 512, 720 x 729 (symmetric projector path), FP32 and BF16 plans."""
    import torch
    pr = phantom.config_mar_fp32()
    geo = oracle.Geometry(pr.n, pr.n_angles, pr.n_bins, theta=pr.theta)
    u = _image(pr.n, 9)
    p32 = ct.Plan(pr.n, pr.n_angles, pr.n_bins, angles=pr.theta)
    t32 = p32.metal_trace(to_dev(u, torch.float32), 2.0, 5, 1e-3)
    _compare_trace(to_np(t32), u, geo, 5, 1e-3, 1e-4)
    p16 = ct.Plan(pr.n, pr.n_angles, pr.n_bins, angles=pr.theta, dtype="bf16")
    t16 = p16.metal_trace(to_dev(u, torch.float32), 2.0, 5, 1e-3)
    assert (to_np(t16) != to_np(t32)).mean() < 1e-4


def test_pipeline_equals_its_stages_and_finds_the_trace(ct):
    import torch
    pr = phantom.make_problem("mar", 64, 90, 95, seed=4, n_ellipses=4, n_metal=2, noise="gaussian", alpha=0.02)
    plan = ct.Plan(64, 90, 95, angles=pr.theta, dtype="f64")
    f = to_dev(pr.f, torch.float64)
    prm = ct.default_params(power_iters=30)
    u, trace, d = plan.tv_mar_solve(f, pr.alpha, pr.delta, 2.0, 150, 100, radius=2, proj_tol=1e-3, params=prm)
    u3, d3 = plan.tv_pdrq2_solve(f, pr.alpha, 150, params=prm)
    t3 = plan.metal_trace(u3, 2.0, 2, 1e-3)
    assert torch.equal(t3, trace)
    u4, d4 = plan.tv_pd_solve(f, t3, pr.alpha, pr.delta, 100,
                              params=ct.default_params(beta=d3["beta"], c=d3["c"]))
    assert rel_l2(to_np(u), to_np(u4)) < 1e-12 and d["objective"] == pytest.approx(d4["objective"], rel=1e-12)
    true = pr.mask.astype(bool)
    est = to_np(trace).astype(bool)
    assert (est & true).sum() >= 0.95 * true.sum()
    assert est.sum() < 2.0 * true.sum()


def test_argument_errors(ct):
    import torch
    plan = ct.Plan(16, 8, 23)
    u = torch.zeros((16, 16), device="cuda")
    for kw in (dict(radius=-1), dict(radius=65), dict(proj_tol=-1.0)):
        with pytest.raises(ct.CtrError):
            plan.metal_trace(u, 1.0, **kw)
    with pytest.raises(ct.CtrError):
        plan.metal_trace(u, float("nan"))
    with pytest.raises(TypeError):
        plan.metal_trace(u.double(), 1.0)
