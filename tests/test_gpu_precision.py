"""The precision workload against its FP64 reference: 2048 x 2048, 2048 views on [0, pi),
2897 bins, 6 metal disks, 1e5-photon Poisson data, 300 iterations of Alg. 4.  The reference
(tests/golden/precision_2048_reference.npz) is the central 512 x 512 crop of the FP64
oracle's iterate, written once by tests/golden/make_precision_reference.py (oracle and
input generator only) with its beta and c.  The GPU solves the regenerated problem with
the same beta and c in FP32 and in the BF16 form; the crop is compared element by element:
FP32 within the 1e-5 relative bar, BF16 within its stated bound (relative l2 <= 1e-3,
PSNR >= 70 dB), and the maximum error of each is reported."""
import importlib.util
import json
import os

import numpy as np
import pytest

from gpu_common import rel_l2, to_dev, to_np
from paper_1810_03275_gb300 import phantom

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
REF = os.path.join(HERE, "golden", "precision_2048_reference.npz")


def _maker():
    spec = importlib.util.spec_from_file_location("make_precision_reference",
                                                  os.path.join(HERE, "golden", "make_precision_reference.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _psnr(got, ref):
    peak = float(np.max(np.abs(ref)))
    mse = float(np.mean((got - ref) ** 2))
    return 10 * np.log10(peak * peak / mse) if mse > 0 else np.inf


@pytest.fixture(scope="module")
def reference():
    z = np.load(REF)
    meta = json.loads(str(z["meta"]))
    return z["u_crop"].astype(np.float64), meta


@pytest.fixture(scope="module")
def problem(reference):
    _, meta = reference
    pr = phantom.config_bf16_2048(seed=meta["seed"])
    fp = _maker().input_fingerprint(pr)
    want = meta["inputs"]
    for key in ("f_sum", "f_sumsq", "f_max", "f_min", "delta"):
        assert fp[key] == pytest.approx(want[key], rel=1e-12, abs=1e-12), (key, "regenerated inputs differ")
    assert fp["mask_sum"] == want["mask_sum"]
    np.testing.assert_allclose(fp["f_samples"], want["f_samples"], rtol=1e-12, atol=1e-12)
    return pr


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_precision_workload_against_fp64_reference(reference, problem, dtype):
    import torch
    from paper_1810_03275_gb300 import ctrecon as ct
    ref, meta = reference
    pr = problem
    a, b = meta["crop"]
    plan = ct.Plan(pr.n, pr.n_angles, pr.n_bins, angles=pr.theta, dtype=dtype)
    prm = ct.default_params(beta=meta["beta"], c=meta["c"], eps=meta["eps"], tau=meta["tau"], sigma=meta["sigma"])
    u, d = plan.tv_pd_solve(to_dev(pr.f, torch.float32), torch.as_tensor(pr.mask, device="cuda"), pr.alpha,
                            pr.delta, meta["iters"], params=prm)
    got = to_np(u)[a:b, a:b]
    e = rel_l2(got, ref)
    emax = float(np.max(np.abs(got - ref)))
    p = _psnr(got, ref)
    print(f"2048^2 precision workload, {dtype} vs FP64 reference crop: rel_l2 {e:.3e}, max abs {emax:.3e} "
          f"(max |u| {np.abs(ref).max():.3f}), PSNR {p:.1f} dB; objective {d['objective']:.9g} vs "
          f"{meta['diagnostics']['objective']:.9g}")
    assert np.all(np.isfinite(got))
    if dtype == "f32":
        assert e < 1e-5
        assert d["objective"] == pytest.approx(meta["diagnostics"]["objective"], rel=1e-5)
    else:
        assert e < 1e-3
        assert p >= 70.0
