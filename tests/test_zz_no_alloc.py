"""precond_apply_static: the preconditioner for callers that cannot allocate device
memory (their host application owns a fixed device pool and forbids cudaMalloc /
cudaFree after start-up).  Called through the C ABI with caller-owned buffers and
compared with the plan-based precond_apply, twice in a row (the static scratch is
shared and keeps the previous call's contents).  This file is collected last."""
import ctypes

import numpy as np
import pytest

from gpu_common import rel_l2

pytestmark = pytest.mark.gpu


def _call_static(lib, y, sigma, tau, c, eps, x, stream):
    return lib.precond_apply_static(int(y.shape[0]), sigma, tau, c, eps, ctypes.c_void_p(y.data_ptr()),
                                    ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(stream))


@pytest.mark.parametrize("n", [384, 64, 1024])
def test_static_scratch_matches_plan_based_preconditioner(n):
    import torch
    from paper_1810_03275_gb300 import ctrecon as ct
    lib = ct.load()
    plan = ct.Plan(n, 4, 5)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(n)
    cases = [(1.0, 8 ** -0.5, 0.7, np.pi / n), (0.6, 0.3, 2.5, 0.05)]
    outs = []
    for k, (sigma, tau, c, eps) in enumerate(cases):          # two calls in a row
        y = torch.as_tensor(rng.standard_normal((n, n)), dtype=torch.float32, device="cuda")
        x = torch.full((n, n), float("nan"), dtype=torch.float32, device="cuda")
        assert _call_static(lib, y, sigma, tau, c, eps, x, stream) == 0, lib.ctr_last_error()
        ref = plan.precond_apply(y, ct.default_params(sigma=sigma, tau=tau, c=c, eps=eps))
        torch.cuda.synchronize()
        outs.append(x.double().cpu().numpy())
        assert rel_l2(outs[-1], ref.double().cpu().numpy()) < 2e-6
    assert not np.allclose(outs[0], outs[1])


def test_static_scratch_rejects_oversized_images():
    import torch
    from paper_1810_03275_gb300 import ctrecon as ct
    lib = ct.load()
    y = torch.zeros((1, 1), dtype=torch.float32, device="cuda")
    st = lib.precond_apply_static(2048, 1.0, 0.35, 1.0, 0.1, ctypes.c_void_p(y.data_ptr()),
                                  ctypes.c_void_p(y.data_ptr()), None)
    assert st == -1
    assert b"1024" in lib.ctr_last_error()
