"""GPU detector-axis ramp filter (ctr_ramp_filter) and filtered backprojection (ctr_fbp)
against the oracle: per-view linear Ram-Lak convolution and FBP on several geometries
(incl. one bin, odd bin counts, ds != 1, the 512 x 512 / 720 x 729 workload on the
symmetric projector path), the BF16 plan against the FP32 one, and the FBP of exact disk
chord lengths reconstructing the disk."""
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


@pytest.mark.parametrize("n,N,M,ds,dtype,tol", [(64, 90, 95, 1.0, "f64", 1e-10), (64, 90, 95, 1.0, "f32", 1e-5),
                                                (48, 37, 1, 1.0, "f64", 1e-10), (96, 41, 137, 1.3, "f64", 1e-10),
                                                (40, 12, 23, 1.0, "f32", 1e-5)])
def test_ramp_and_fbp_match_oracle(ct, n, N, M, ds, dtype, tol):
    geo = oracle.Geometry(n, N, M, ds=ds)
    plan = ct.Plan(n, N, M, ds=ds, dtype=dtype)
    g = np.random.default_rng(M).standard_normal((N, M))
    y = to_np(plan.ramp_filter(to_dev(g, plan.torch_dtype)))
    assert rel_l2(y, oracle.ramp_filter(g, ds)) < tol
    u = to_np(plan.fbp(to_dev(g, plan.torch_dtype)))
    assert rel_l2(u, oracle.fbp(g, geo)) < tol


def test_benchmark_geometry_disk_and_bf16(ct):
    """512 x 512, 720 views, 729 bins (L = 1458): parity on random data, the disk of radius
    150 reconstructed to within 1 % in the mean, BF16 within 1e-2 of FP32."""
    import torch
    pr = phantom.config_mar_fp32()
    geo = oracle.Geometry(pr.n, pr.n_angles, pr.n_bins, theta=pr.theta)
    p32 = ct.Plan(pr.n, pr.n_angles, pr.n_bins, angles=pr.theta)
    g = np.random.default_rng(3).standard_normal((pr.n_angles, pr.n_bins))
    assert rel_l2(to_np(p32.fbp(to_dev(g, torch.float32))), oracle.fbp(g, geo)) < 1e-5
    r = 150.0
    s = phantom.bin_centres(pr.n_bins)
    chord = np.tile(2.0 * np.sqrt(np.maximum(r * r - s * s, 0.0)), (pr.n_angles, 1))
    u = to_np(p32.fbp(to_dev(chord, torch.float32)))
    x = phantom.pixel_centres(pr.n)
    R = np.hypot(*np.meshgrid(x, x, indexing="ij"))
    assert abs(u[R < r - 3].mean() - 1.0) < 0.01 and abs(u[(R > r + 3) & (R < 240)].mean()) < 0.01
    p16 = ct.Plan(pr.n, pr.n_angles, pr.n_bins, angles=pr.theta, dtype="bf16")
    u16 = to_np(p16.fbp(to_dev(chord, torch.float32)))
    assert rel_l2(u16, u) < 1e-2


def test_over_long_detector_is_refused(ct):
    """One padded FP64 view of 2 * 3000 - 1 points does not fit a CTA: CTR_EUNSUPPORTED,
    and the plan stays usable."""
    import torch
    plan = ct.Plan(32, 4, 3000, dtype="f64")
    g = torch.zeros((4, 3000), dtype=torch.float64, device="cuda")
    with pytest.raises(ct.CtrError) as e:
        plan.ramp_filter(g)
    assert e.value.status == -6
    assert float(plan.rh_adjoint(g).abs().max()) == 0.0
