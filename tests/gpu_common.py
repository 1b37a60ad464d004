"""Helpers shared by the GPU parity tests (plans, conversions, error metrics)."""
import numpy as np


def rel_l2(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (den if den > 0 else 1.0))


def rel_max(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.max(np.abs(ref))
    return float(np.max(np.abs(got - ref)) / (den if den > 0 else 1.0))


def to_dev(x, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda").contiguous()


def to_np(t):
    return t.detach().double().cpu().numpy()


# Tolerances: FP32 results within 1e-5 relative (l2) of the FP64 oracle; FP64 GPU
# results within 1e-10 (the fixed-point geometry quantises p to 2^-48 bins).
TOL = {"f32": 1e-5, "f64": 1e-10}
