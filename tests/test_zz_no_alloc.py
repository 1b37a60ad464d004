"""precond_apply_static: the preconditioner for callers that cannot allocate device
memory (their host application owns a fixed device pool and forbids cudaMalloc /
cudaFree after start-up).  Called through the C ABI with caller-owned buffers and
compared with the FP64 oracle's preconditioner and with the plan-based
precond_apply, twice in a row (the static scratch is shared and keeps the previous
call's contents).  This file is collected last."""
import ctypes

import numpy as np
import pytest

import oracle
from gpu_common import rel_l2

pytestmark = pytest.mark.gpu


def _call_static(lib, y, sigma, tau, c, eps, x, stream, n=None):
    return lib.precond_apply_static(int(y.shape[0]) if n is None else n, sigma, tau, c, eps,
                                    ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                    ctypes.c_void_p(stream))


@pytest.mark.parametrize("n", [384, 64, 1024])
def test_static_scratch_matches_oracle_and_plan_based_preconditioner(n):
    import torch
    from paper_1810_03275_gb300 import ctrecon as ct
    lib = ct.load()
    plan = ct.Plan(n, 4, 5)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(n)
    cases = [(1.0, 8 ** -0.5, 0.7, np.pi / n), (0.6, 0.3, 2.5, 0.05)]
    for sigma, tau, c, eps in cases:          # two calls in a row
        y_np = rng.standard_normal((n, n))
        y = torch.as_tensor(y_np, dtype=torch.float32, device="cuda")
        x = torch.full((n, n), float("nan"), dtype=torch.float32, device="cuda")
        assert _call_static(lib, y, sigma, tau, c, eps, x, stream) == 0, lib.ctr_last_error()
        ref = plan.precond_apply(y, ct.default_params(sigma=sigma, tau=tau, c=c, eps=eps))
        torch.cuda.synchronize()
        got = x.double().cpu().numpy()
        want = oracle.precond_apply(y.double().cpu().numpy(), oracle.precond_symbol(n, sigma, tau, c, eps))
        assert rel_l2(got, want) < 1e-5
        assert rel_l2(got, ref.double().cpu().numpy()) < 2e-6


def test_small_call_after_large_call_sees_no_stale_scratch():
    """A 1024 x 1024 call fills the whole scratch; a 64 x 64 call right after it (same
    input as a 64 x 64 call made first) must give the same result bit for bit."""
    import torch
    from paper_1810_03275_gb300 import ctrecon as ct
    lib = ct.load()
    stream = torch.cuda.current_stream().cuda_stream
    prm = (0.9, 0.3, 1.7, np.pi / 64)
    y64 = torch.as_tensor(np.random.default_rng(7).standard_normal((64, 64)), dtype=torch.float32, device="cuda")
    first = torch.empty_like(y64)
    assert _call_static(lib, y64, *prm, first, stream) == 0, lib.ctr_last_error()
    big = torch.as_tensor(np.random.default_rng(8).standard_normal((1024, 1024)), dtype=torch.float32, device="cuda")
    xbig = torch.empty_like(big)
    assert _call_static(lib, big, 1.0, 0.35, 0.5, 0.01, xbig, stream) == 0, lib.ctr_last_error()
    again = torch.empty_like(y64)
    assert _call_static(lib, y64, *prm, again, stream) == 0, lib.ctr_last_error()
    torch.cuda.synchronize()
    assert torch.equal(first, again)
    want = oracle.precond_apply(y64.double().cpu().numpy(), oracle.precond_symbol(64, *prm))
    assert rel_l2(again.double().cpu().numpy(), want) < 1e-5


def test_static_scratch_rejects_oversized_images():
    import torch
    from paper_1810_03275_gb300 import ctrecon as ct
    lib = ct.load()
    y = torch.zeros((1, 1), dtype=torch.float32, device="cuda")
    st = lib.precond_apply_static(2048, 1.0, 0.35, 1.0, 0.1, ctypes.c_void_p(y.data_ptr()),
                                  ctypes.c_void_p(y.data_ptr()), None)
    assert st == -1
    assert b"1024" in lib.ctr_last_error()


def test_static_entry_rejects_host_buffers():
    """A host pointer is refused before anything is launched (pointer attributes, no
    allocation); the binding refuses a mismatched output tensor."""
    import torch
    from paper_1810_03275_gb300 import ctrecon as ct
    lib = ct.load()
    yd = torch.zeros((16, 16), dtype=torch.float32, device="cuda")
    yh = torch.zeros((16, 16), dtype=torch.float32)
    st = lib.precond_apply_static(16, 1.0, 0.35, 1.0, 0.1, ctypes.c_void_p(yh.data_ptr()),
                                  ctypes.c_void_p(yd.data_ptr()), None)
    assert st == -1 and b"device memory" in lib.ctr_last_error()
    st = lib.precond_apply_static(16, 1.0, 0.35, 1.0, 0.1, ctypes.c_void_p(yd.data_ptr()),
                                  ctypes.c_void_p(yh.data_ptr()), None)
    assert st == -1
    with pytest.raises(TypeError):
        ct.precond_apply_static(yd, 1.0, 0.35, 1.0, 0.1, x=torch.zeros((8, 8), device="cuda"))
    with pytest.raises(TypeError):
        ct.precond_apply_static(yd, 1.0, 0.35, 1.0, 0.1, x=yh)
