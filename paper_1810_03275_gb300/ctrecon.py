"""Thin Python binding of libctrecon (include/ctrecon.h): argument marshalling only.

Every operation runs in the library's CUDA kernels; tensors are PyTorch CUDA
tensors used as device buffers, and the current torch stream is passed through.
Loading fails loudly if the library has not been built (run
``python -c "import __graft_entry__ as g; g.build()"``) -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libctrecon.so")
_lock = threading.Lock()
_lib = None

CTR_OK = 0
CTR_F32, CTR_F64, CTR_BF16 = 0, 1, 2
_STATUS = {0: "CTR_OK", -1: "CTR_EINVAL", -2: "CTR_ENOMEM", -3: "CTR_ECUDA", -4: "CTR_ETIMEOUT",
           -5: "CTR_ENUMERIC", -6: "CTR_EUNSUPPORTED"}


class CtrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Geometry(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("n_angles", ctypes.c_int), ("n_bins", ctypes.c_int),
                ("h", ctypes.c_double), ("ds", ctypes.c_double),
                ("angles_host", ctypes.POINTER(ctypes.c_double))]


class Params(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("tau", ctypes.c_double), ("eps", ctypes.c_double),
                ("c", ctypes.c_double), ("beta", ctypes.c_double), ("power_iters", ctypes.c_int),
                ("c_margin", ctypes.c_double), ("trace_ratio", ctypes.c_double),
                ("check_every", ctypes.c_int), ("graph_block", ctypes.c_int), ("nonneg", ctypes.c_int),
                ("precond", ctypes.c_int), ("stop_tol", ctypes.c_double)]


class Diag(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("c", ctypes.c_double), ("objective", ctypes.c_double),
                ("data_fit", ctypes.c_double), ("tv", ctypes.c_double), ("violation", ctypes.c_double),
                ("gap", ctypes.c_double), ("dual_residual", ctypes.c_double),
                ("rel_change", ctypes.c_double), ("iters_done", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class State(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("Ru", ctypes.c_void_p), ("v1b", ctypes.c_void_p), ("v2b", ctypes.c_void_p),
                ("ub", ctypes.c_void_p)]


EXPORTS = ["ctr_plan_create", "ctr_plan_destroy", "ctr_default_params", "ctr_last_error", "ctr_plan_device_bytes",
           "ctr_plan_launch_count", "ctr_plan_symmetric_jobs", "rh_forward", "rh_forward_t", "rh_adjoint", "precond_apply", "tv_pd_solve", "tv_pd_run", "ctr_power_beta",
           "ctr_power_lambda", "ctr_grad", "ctr_div", "precond_apply_static", "ctr_plan_set_bp_groups",
           "ctr_plan_get_bp_groups", "ctr_batch_create", "ctr_batch_destroy", "ctr_batch_plan", "ctr_batch_retune",
           "ctr_batch_launch_count", "tv_pd_solve_batched", "tv_pd_solve_state", "tv_pd_vjp_step",
           "tv_cp_solve", "tv_pdrq2_solve", "ctr_metal_trace", "tv_mar_solve",
           "tv_admm_solve", "ctr_ramp_filter", "ctr_fbp", "tv_pd_vjp_segment", "ctr_plan_history",
           "ctr_fp32_fma_rate", "ctr_batch_set_mode", "ctr_batch_get_mode", "ctr_batch_persistent_ctas",
           "ctr_plan_set_fwd_shape", "ctr_plan_get_fwd_shape", "ctr_plan_set_fft_form", "ctr_plan_get_fft_form",
           "ctr_plan_set_launch_overlap", "ctr_plan_get_launch_overlap"]


def load(path: str = LIB_PATH):
    """Load libctrecon.so and declare its signatures (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libctrecon.so not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        vp, P = ctypes.c_void_p, ctypes.POINTER
        lib.ctr_plan_create.argtypes = [P(Geometry), ctypes.c_int, P(vp)]
        lib.ctr_plan_destroy.argtypes = [vp]
        lib.ctr_plan_destroy.restype = None
        lib.ctr_default_params.argtypes = [P(Params)]
        lib.ctr_default_params.restype = None
        lib.ctr_last_error.restype = ctypes.c_char_p
        lib.ctr_plan_device_bytes.argtypes = [vp]
        lib.ctr_plan_device_bytes.restype = ctypes.c_size_t
        lib.rh_forward.argtypes = [vp, vp, vp, vp]
        lib.rh_adjoint.argtypes = [vp, vp, vp, vp]
        lib.rh_forward_t.argtypes = [vp, vp, vp, vp, vp]
        lib.rh_forward_t.restype = ctypes.c_int
        lib.ctr_plan_launch_count.argtypes = [vp]
        lib.ctr_plan_launch_count.restype = ctypes.c_ulonglong
        lib.ctr_plan_symmetric_jobs.argtypes = [vp]
        lib.ctr_plan_symmetric_jobs.restype = ctypes.c_int
        lib.precond_apply.argtypes = [vp, P(Params), vp, vp, vp]
        lib.tv_pd_solve.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, P(Params), vp,
                                    P(Diag), vp]
        lib.tv_pd_run.argtypes = [vp, vp, vp, vp, vp, ctypes.c_double, ctypes.c_int, P(Params), P(State), vp,
                                  P(Diag), vp]
        lib.tv_cp_solve.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, P(Params), vp, P(Diag), vp]
        lib.tv_pdrq2_solve.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int, P(Params), vp, P(Diag), vp]
        lib.ctr_metal_trace.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int, ctypes.c_double, vp, vp, vp]
        lib.ctr_ramp_filter.argtypes = [vp, vp, vp, vp]
        lib.ctr_fbp.argtypes = [vp, vp, vp, vp]
        lib.tv_admm_solve.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                      P(Params), vp, P(Diag), vp]
        lib.tv_mar_solve.argtypes = [vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_int, P(Params), vp, vp, P(Diag), vp]
        lib.ctr_power_beta.argtypes = [vp, ctypes.c_int, P(ctypes.c_double), vp]
        lib.ctr_power_lambda.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, P(ctypes.c_double), vp]
        lib.precond_apply_static.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, vp, vp, vp]
        lib.precond_apply_static.restype = ctypes.c_int
        lib.ctr_plan_set_bp_groups.argtypes = [vp, ctypes.c_int]
        lib.ctr_plan_set_bp_groups.restype = ctypes.c_int
        lib.ctr_plan_get_bp_groups.argtypes = [vp]
        lib.ctr_plan_get_bp_groups.restype = ctypes.c_int
        lib.ctr_batch_create.argtypes = [P(Geometry), ctypes.c_int, P(vp)]
        lib.ctr_batch_create.restype = ctypes.c_int
        lib.ctr_batch_destroy.argtypes = [vp]
        lib.ctr_batch_destroy.restype = None
        lib.ctr_batch_plan.argtypes = [vp, ctypes.c_int]
        lib.ctr_batch_plan.restype = vp
        lib.ctr_batch_retune.argtypes = [vp]
        lib.ctr_batch_retune.restype = ctypes.c_int
        lib.ctr_batch_launch_count.argtypes = [vp]
        lib.ctr_batch_launch_count.restype = ctypes.c_ulonglong
        lib.tv_pd_solve_batched.argtypes = [vp, P(vp), P(vp), P(ctypes.c_double), P(ctypes.c_double), ctypes.c_int,
                                            P(Params), P(ctypes.c_double), P(ctypes.c_double), P(vp), P(Diag), vp]
        lib.tv_pd_solve_batched.restype = ctypes.c_int
        lib.tv_pd_solve_state.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, P(Params),
                                          P(State), P(Diag), vp]
        lib.tv_pd_solve_state.restype = ctypes.c_int
        lib.tv_pd_vjp_step.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_double, P(Params), P(State), P(State),
                                       vp, vp, vp, vp, vp, vp]
        lib.tv_pd_vjp_step.restype = ctypes.c_int
        lib.tv_pd_vjp_segment.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_double, P(Params), P(State),
                                          ctypes.c_int, vp, vp, vp, vp, vp, vp, vp]
        lib.ctr_plan_history.argtypes = [vp, P(Diag), ctypes.c_int, P(ctypes.c_int)]
        lib.ctr_plan_history.restype = ctypes.c_int
        lib.ctr_plan_set_fwd_shape.argtypes = [vp, ctypes.c_int, ctypes.c_int]
        lib.ctr_plan_set_fwd_shape.restype = ctypes.c_int
        lib.ctr_plan_get_fwd_shape.argtypes = [vp, P(ctypes.c_int), P(ctypes.c_int)]
        lib.ctr_plan_get_fwd_shape.restype = ctypes.c_int
        lib.ctr_plan_set_fft_form.argtypes = [vp, ctypes.c_int]
        lib.ctr_plan_set_fft_form.restype = ctypes.c_int
        lib.ctr_plan_get_fft_form.argtypes = [vp]
        lib.ctr_plan_get_fft_form.restype = ctypes.c_int
        lib.ctr_plan_set_launch_overlap.argtypes = [vp, ctypes.c_int]
        lib.ctr_plan_set_launch_overlap.restype = ctypes.c_int
        lib.ctr_plan_get_launch_overlap.argtypes = [vp]
        lib.ctr_plan_get_launch_overlap.restype = ctypes.c_int
        lib.ctr_batch_set_mode.argtypes = [vp, ctypes.c_int, ctypes.c_ulonglong]
        lib.ctr_batch_set_mode.restype = ctypes.c_int
        lib.ctr_batch_get_mode.argtypes = [vp]
        lib.ctr_batch_get_mode.restype = ctypes.c_int
        lib.ctr_batch_persistent_ctas.argtypes = [vp]
        lib.ctr_batch_persistent_ctas.restype = ctypes.c_int
        lib.ctr_fp32_fma_rate.argtypes = [P(ctypes.c_double), vp]
        lib.ctr_fp32_fma_rate.restype = ctypes.c_int
        lib.ctr_grad.argtypes = [vp, vp, vp, vp]
        lib.ctr_div.argtypes = [vp, vp, vp, vp]
        for name in ["ctr_plan_create", "rh_forward", "rh_adjoint", "precond_apply", "tv_pd_solve", "tv_pd_run",
                     "ctr_power_beta", "ctr_power_lambda", "ctr_grad", "ctr_div"]:
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _check(st: int):
    if st != CTR_OK:
        raise CtrError(st, load().ctr_last_error().decode(errors="replace"))


def default_params(**kw) -> Params:
    p = Params()
    load().ctr_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def precond_apply_static(y, sigma: float, tau: float, c: float, eps: float, x=None, stream=None):
    """precond_apply without a plan and without device allocation inside the library
    (static scratch, FP32, n <= 1024): for callers that own all device memory.  Calls
    that overlap on the GPU race on the shared scratch."""
    import torch
    if not isinstance(y, torch.Tensor) or not y.is_cuda or y.dtype != torch.float32 or not y.is_contiguous() \
            or y.dim() != 2 or y.shape[0] != y.shape[1]:
        raise TypeError("y must be a contiguous square float32 CUDA tensor")
    x = torch.empty_like(y) if x is None else x
    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.float32 or not x.is_contiguous() \
            or x.shape != y.shape:
        raise TypeError("x must be a contiguous float32 CUDA tensor of y's shape")
    # the C entry runs on the current device: both buffers must live there
    dev = torch.cuda.current_device()
    if y.device.index != dev or x.device.index != dev:
        raise TypeError(f"x and y must be on the current CUDA device (cuda:{dev})")
    _check(load().precond_apply_static(int(y.shape[0]), float(sigma), float(tau), float(c), float(eps),
                                       ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x.data_ptr()), _stream(stream)))
    return x


def fp32_fma_rate(stream=None) -> float:
    """Measured FP32 FMA ceiling of the current device in FMA/s (ctr_fp32_fma_rate)."""
    out = ctypes.c_double()
    _check(load().ctr_fp32_fma_rate(ctypes.byref(out), _stream(stream)))
    return out.value


def _stream(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """A ctr_plan: geometry tables and device workspace for one (n, angles, bins, dtype)."""

    def __init__(self, n: int, n_angles: int, n_bins: int, angles=None, h: float = 1.0, ds: float = 1.0,
                 dtype: str = "f32"):
        import torch
        lib = load()
        if angles is None:
            angles = np.arange(n_angles, dtype=np.float64) * (np.pi / n_angles)
        self.angles = np.ascontiguousarray(angles, dtype=np.float64)
        self.n, self.n_angles, self.n_bins, self.h, self.ds = n, n_angles, n_bins, h, ds
        self.dtype = dtype
        # compute / input-output dtype, and the storage dtype of the projectors' operands
        self.torch_dtype = {"f32": torch.float32, "f64": torch.float64, "bf16": torch.float32}[dtype]
        self.op_dtype = torch.bfloat16 if dtype == "bf16" else self.torch_dtype
        code = {"f32": CTR_F32, "f64": CTR_F64, "bf16": CTR_BF16}[dtype]
        geo = Geometry(n, n_angles, n_bins, h, ds, self.angles.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        handle = ctypes.c_void_p()
        _check(lib.ctr_plan_create(ctypes.byref(geo), code, ctypes.byref(handle)))
        self._h = handle

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().ctr_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers ---------------------------------------------------------------
    @property
    def device_bytes(self) -> int:
        return int(load().ctr_plan_device_bytes(self._h))

    def _t(self, x, shape, name, dtype=None):
        import torch
        dtype = self.torch_dtype if dtype is None else dtype
        if not isinstance(x, torch.Tensor) or not x.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if x.dtype != dtype:
            raise TypeError(f"{name} must be {dtype}, got {x.dtype}")
        if tuple(x.shape) != tuple(shape) or not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous with shape {shape}, got {tuple(x.shape)}")
        return ctypes.c_void_p(x.data_ptr())

    def empty_image(self, planes: int = 1):
        import torch
        shape = (self.n, self.n) if planes == 1 else (planes, self.n, self.n)
        return torch.empty(shape, dtype=self.torch_dtype, device="cuda")

    def empty_sino(self):
        import torch
        return torch.empty((self.n_angles, self.n_bins), dtype=self.torch_dtype, device="cuda")

    # -- the C ABI -------------------------------------------------------------
    def rh_forward(self, u, g=None, stream=None):
        g = self.empty_sino() if g is None else g
        _check(load().rh_forward(self._h, self._t(u, (self.n, self.n), "u", self.op_dtype),
                                 self._t(g, (self.n_angles, self.n_bins), "g"), _stream(stream)))
        return g

    def rh_forward_t(self, u, uT, g=None, stream=None):
        g = self.empty_sino() if g is None else g
        _check(load().rh_forward_t(self._h, self._t(u, (self.n, self.n), "u", self.op_dtype),
                                   self._t(uT, (self.n, self.n), "uT", self.op_dtype),
                                   self._t(g, (self.n_angles, self.n_bins), "g"), _stream(stream)))
        return g

    def history(self):
        """Diagnostics records of the last solve with params.check_every > 0 (list of dicts,
        one per check, in order)."""
        lib = load()
        count = ctypes.c_int()
        _check(lib.ctr_plan_history(self._h, None, 0, ctypes.byref(count)))
        if count.value == 0:
            return []
        recs = (Diag * count.value)()
        _check(lib.ctr_plan_history(self._h, recs, count.value, ctypes.byref(count)))
        return [r.as_dict() for r in recs]

    @property
    def launch_count(self) -> int:
        return int(load().ctr_plan_launch_count(self._h))

    @property
    def symmetric_jobs(self) -> int:
        """Jobs of the projectors' symmetric path (0: angle-by-angle path)."""
        return int(load().ctr_plan_symmetric_jobs(self._h))

    @property
    def bp_groups(self) -> int:
        return int(load().ctr_plan_get_bp_groups(self._h))

    def set_bp_groups(self, groups: int):
        _check(load().ctr_plan_set_bp_groups(self._h, int(groups)))

    FWD_SHAPES = ((1, 2), (1, 4), (1, 8), (2, 2), (2, 4), (4, 2), (4, 1))

    @property
    def fwd_shape(self):
        """(jobs per CTA, row segments) of the symmetric forward projector ((0, 0): per-angle path)."""
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(load().ctr_plan_get_fwd_shape(self._h, ctypes.byref(a), ctypes.byref(b)))
        return (a.value, b.value)

    def set_fwd_shape(self, jobs_per_cta: int, segments: int):
        _check(load().ctr_plan_set_fwd_shape(self._h, int(jobs_per_cta), int(segments)))

    @property
    def fft_form(self) -> int:
        """Kernels of the preconditioner passes: 0 warp-level (FP32, n = 256/512/1024), 1 CTA-level."""
        return int(load().ctr_plan_get_fft_form(self._h))

    def set_fft_form(self, form: int):
        _check(load().ctr_plan_set_fft_form(self._h, int(form)))

    @property
    def launch_overlap(self) -> int:
        """1: the iteration's kernels use programmatic dependent launch (default), 0: plain stream order."""
        return int(load().ctr_plan_get_launch_overlap(self._h))

    def set_launch_overlap(self, on: int):
        _check(load().ctr_plan_set_launch_overlap(self._h, int(on)))

    def rh_adjoint(self, g, u=None, stream=None):
        u = self.empty_image() if u is None else u
        _check(load().rh_adjoint(self._h, self._t(g, (self.n_angles, self.n_bins), "g", self.op_dtype),
                                 self._t(u, (self.n, self.n), "u"), _stream(stream)))
        return u

    def precond_apply(self, y, params: Params, x=None, stream=None):
        x = self.empty_image() if x is None else x
        _check(load().precond_apply(self._h, ctypes.byref(params), self._t(y, (self.n, self.n), "y"),
                                    self._t(x, (self.n, self.n), "x"), _stream(stream)))
        return x

    def grad(self, u, p=None, stream=None):
        p = self.empty_image(2) if p is None else p
        _check(load().ctr_grad(self._h, self._t(u, (self.n, self.n), "u"), self._t(p, (2, self.n, self.n), "p"),
                               _stream(stream)))
        return p

    def div(self, p, d=None, stream=None):
        d = self.empty_image() if d is None else d
        _check(load().ctr_div(self._h, self._t(p, (2, self.n, self.n), "p"), self._t(d, (self.n, self.n), "d"),
                              _stream(stream)))
        return d

    def power_beta(self, iters: int = 50, stream=None) -> float:
        out = ctypes.c_double()
        _check(load().ctr_power_beta(self._h, iters, ctypes.byref(out), _stream(stream)))
        return out.value

    def power_lambda(self, beta: float, eps: float, iters: int = 50, stream=None) -> float:
        out = ctypes.c_double()
        _check(load().ctr_power_lambda(self._h, beta, eps, iters, ctypes.byref(out), _stream(stream)))
        return out.value

    def tv_pd_solve(self, f, metal_mask, alpha: float, delta: float, iters: int, params: Optional[Params] = None,
                    u_out=None, stream=None):
        """Alg. 4 from u = 0 on problem (C_h); returns (u, diag dict)."""
        import torch
        u_out = self.empty_image() if u_out is None else u_out
        if metal_mask is not None:
            if metal_mask.dtype != torch.uint8 or not metal_mask.is_cuda or not metal_mask.is_contiguous() \
                    or tuple(metal_mask.shape) != (self.n_angles, self.n_bins):
                raise ValueError("metal_mask must be a contiguous CUDA uint8 tensor of the sinogram's shape")
            mptr = ctypes.c_void_p(metal_mask.data_ptr())
        else:
            mptr = ctypes.c_void_p()
        diag = Diag()
        prm = params if params is not None else default_params()
        _check(load().tv_pd_solve(self._h, self._t(f, (self.n_angles, self.n_bins), "f"), mptr, float(alpha),
                                  float(delta), int(iters), ctypes.byref(prm), self._t(u_out, (self.n, self.n), "u_out"),
                                  ctypes.byref(diag), _stream(stream)))
        return u_out, diag.as_dict()

    def tv_cp_solve(self, f, metal_mask, alpha: float, delta: float, iters: int, sigma_p: float = 0.0,
                    tau_d: float = 0.0, params: Optional[Params] = None, u_out=None, stream=None):
        """Alg. 1 (Chambolle-Pock) from u = 0 on problem (C_h); returns (u, diag dict)."""
        u_out = self.empty_image() if u_out is None else u_out
        diag = Diag()
        prm = params if params is not None else default_params()
        _check(load().tv_cp_solve(self._h, self._t(f, (self.n_angles, self.n_bins), "f"), self._mask(metal_mask),
                                  float(alpha), float(delta), int(iters), float(sigma_p), float(tau_d),
                                  ctypes.byref(prm), self._t(u_out, (self.n, self.n), "u_out"), ctypes.byref(diag),
                                  _stream(stream)))
        return u_out, diag.as_dict()

    def ramp_filter(self, g, y=None, stream=None):
        """Detector-axis Ram-Lak filter of each view (linear convolution along the bins)."""
        y = self.empty_sino() if y is None else y
        sino = (self.n_angles, self.n_bins)
        _check(load().ctr_ramp_filter(self._h, self._t(g, sino, "g"), self._t(y, sino, "y"), _stream(stream)))
        return y

    def fbp(self, g, u_out=None, stream=None):
        """Filtered backprojection (pi / N) R_h^*(ramp-filtered g)."""
        u_out = self.empty_image() if u_out is None else u_out
        _check(load().ctr_fbp(self._h, self._t(g, (self.n_angles, self.n_bins), "g"),
                              self._t(u_out, (self.n, self.n), "u_out"), _stream(stream)))
        return u_out

    def metal_trace(self, u, threshold: float, radius: int = 5, proj_tol: float = 1e-6, want_marks: bool = False,
                    stream=None):
        """Metal-trace estimate from a reconstruction u: the sinogram mask (uint8, N x M) of
        the bins that the marks (u > threshold, dilated by a disk of `radius` px) project
        onto; with want_marks also the dilated marks (uint8, n x n)."""
        import torch
        trace = torch.empty((self.n_angles, self.n_bins), dtype=torch.uint8, device="cuda")
        marks = torch.empty((self.n, self.n), dtype=torch.uint8, device="cuda") if want_marks else None
        u_p = self._t(u, (self.n, self.n), "u")
        _check(load().ctr_metal_trace(self._h, u_p, float(threshold), int(radius),
                                      float(proj_tol), ctypes.c_void_p(marks.data_ptr() if marks is not None else 0),
                                      ctypes.c_void_p(trace.data_ptr()), _stream(stream)))
        return (trace, marks) if want_marks else trace

    def tv_admm_solve(self, f, alpha: float, iters: int, mu: float = 1.0, cg_iters: int = 2,
                      params: Optional[Params] = None, u_out=None, stream=None):
        """ADMM with PCG inner solves from u = 0 on the unconstrained problem; returns (u, diag dict)."""
        u_out = self.empty_image() if u_out is None else u_out
        diag = Diag()
        prm = params if params is not None else default_params()
        _check(load().tv_admm_solve(self._h, self._t(f, (self.n_angles, self.n_bins), "f"), float(alpha), int(iters),
                                    float(mu), int(cg_iters), ctypes.byref(prm),
                                    self._t(u_out, (self.n, self.n), "u_out"), ctypes.byref(diag), _stream(stream)))
        return u_out, diag.as_dict()

    def tv_mar_solve(self, f, alpha: float, delta: float, threshold: float, iters_pre: int, iters: int,
                     radius: int = 5, proj_tol: float = 1e-6, params: Optional[Params] = None, u_out=None,
                     stream=None):
        """Alg. 3 pre-reconstruction -> metal trace -> Alg. 4 on (C_h); returns (u, trace, diag dict)."""
        import torch
        u_out = self.empty_image() if u_out is None else u_out
        trace = torch.empty((self.n_angles, self.n_bins), dtype=torch.uint8, device="cuda")
        diag = Diag()
        prm = params if params is not None else default_params()
        _check(load().tv_mar_solve(self._h, self._t(f, (self.n_angles, self.n_bins), "f"), float(alpha),
                                   float(delta), float(threshold), int(radius), float(proj_tol), int(iters_pre),
                                   int(iters), ctypes.byref(prm), ctypes.c_void_p(trace.data_ptr()),
                                   self._t(u_out, (self.n, self.n), "u_out"), ctypes.byref(diag), _stream(stream)))
        return u_out, trace, diag.as_dict()

    def tv_pdrq2_solve(self, f, alpha: float, iters: int, params: Optional[Params] = None, u_out=None,
                       stream=None):
        """Alg. 3 (PDRQS2) from u = 0 on the unconstrained problem (U_h); returns (u, diag dict)."""
        u_out = self.empty_image() if u_out is None else u_out
        diag = Diag()
        prm = params if params is not None else default_params()
        _check(load().tv_pdrq2_solve(self._h, self._t(f, (self.n_angles, self.n_bins), "f"), float(alpha),
                                     int(iters), ctypes.byref(prm), self._t(u_out, (self.n, self.n), "u_out"),
                                     ctypes.byref(diag), _stream(stream)))
        return u_out, diag.as_dict()

    def _state(self, st):
        sino = (self.n_angles, self.n_bins)
        ub = self._t(st["ub"], (self.n, self.n), "ub").value if st.get("ub") is not None else None
        return State(self._t(st["u"], (self.n, self.n), "u").value, self._t(st["Ru"], sino, "Ru").value,
                     self._t(st["v1b"], sino, "v1b").value, self._t(st["v2b"], (2, self.n, self.n), "v2b").value, ub)

    def _mask(self, metal_mask):
        import torch
        if metal_mask is None:
            return ctypes.c_void_p()
        if metal_mask.dtype != torch.uint8 or not metal_mask.is_cuda or not metal_mask.is_contiguous() \
                or tuple(metal_mask.shape) != (self.n_angles, self.n_bins):
            raise ValueError("metal_mask must be a contiguous CUDA uint8 tensor of the sinogram's shape")
        return ctypes.c_void_p(metal_mask.data_ptr())

    def tv_pd_solve_state(self, f, metal_mask, alpha: float, delta: float, iters: int, params: Params, state,
                          stream=None):
        """Continue Alg. 4 from `state` (dict of tensors, updated in place)."""
        st = self._state(state)
        _check(load().tv_pd_solve_state(self._h, self._t(f, (self.n_angles, self.n_bins), "f"),
                                        self._mask(metal_mask), float(alpha), float(delta), int(iters),
                                        ctypes.byref(params), ctypes.byref(st), None, _stream(stream)))
        return state

    def tv_pd_vjp_step(self, f, metal_mask, alpha: float, delta: float, params: Params, s0, s1, bu, b1, b2, gf,
                       galpha, stream=None):
        """Reverse mode of the iteration s0 -> s1 (cotangents bu, b1, b2 updated in place;
        gf and the float64 device scalar galpha accumulate)."""
        import torch
        if galpha.dtype != torch.float64 or not galpha.is_cuda:
            raise TypeError("galpha must be a float64 CUDA tensor")
        a, b = self._state(s0), self._state(s1)
        sino = (self.n_angles, self.n_bins)
        _check(load().tv_pd_vjp_step(self._h, self._t(f, sino, "f"), self._mask(metal_mask), float(alpha),
                                     float(delta), ctypes.byref(params), ctypes.byref(a), ctypes.byref(b),
                                     self._t(bu, (self.n, self.n), "bu"), self._t(b1, sino, "b1"),
                                     self._t(b2, (2, self.n, self.n), "b2"), self._t(gf, sino, "gf"),
                                     ctypes.c_void_p(galpha.data_ptr()), _stream(stream)))

    def vjp_workspace(self, length: int):
        """Device workspace for tv_pd_vjp_segment of up to `length` iterations."""
        import torch
        per = 3 * self.n * self.n + 2 * self.n_angles * self.n_bins
        return torch.empty((length + 1) * per, dtype=self.torch_dtype, device="cuda")

    def tv_pd_vjp_segment(self, f, metal_mask, alpha: float, delta: float, params: Params, s_start, length: int,
                          workspace, bu, b1, b2, gf, galpha, stream=None):
        """Reverse mode of `length` iterations from the checkpoint s_start, replayed and
        reversed on the device (cotangents as tv_pd_vjp_step)."""
        import torch
        if galpha.dtype != torch.float64 or not galpha.is_cuda:
            raise TypeError("galpha must be a float64 CUDA tensor")
        per = 3 * self.n * self.n + 2 * self.n_angles * self.n_bins
        if workspace.dtype != self.torch_dtype or not workspace.is_cuda or workspace.numel() < (length + 1) * per \
                or not workspace.is_contiguous():
            raise ValueError("workspace too small (see vjp_workspace)")
        a = self._state(s_start)
        sino = (self.n_angles, self.n_bins)
        _check(load().tv_pd_vjp_segment(self._h, self._t(f, sino, "f"), self._mask(metal_mask), float(alpha),
                                        float(delta), ctypes.byref(params), ctypes.byref(a), int(length),
                                        ctypes.c_void_p(workspace.data_ptr()), self._t(bu, (self.n, self.n), "bu"),
                                        self._t(b1, sino, "b1"), self._t(b2, (2, self.n, self.n), "b2"),
                                        self._t(gf, sino, "gf"), ctypes.c_void_p(galpha.data_ptr()),
                                        _stream(stream)))

    def new_state(self):
        import torch
        z = dict(device="cuda", dtype=self.torch_dtype)
        return {"u": torch.zeros((self.n, self.n), **z), "Ru": torch.zeros((self.n_angles, self.n_bins), **z),
                "v1b": torch.zeros((self.n_angles, self.n_bins), **z), "v2b": torch.zeros((2, self.n, self.n), **z),
                "ub": torch.zeros((self.n, self.n), **z)}

    def tv_pd_run(self, w, a, lo, hi, alpha: float, iters: int, params: Optional[Params] = None, state=None,
                  u_out=None, want_diag: bool = True, stream=None):
        """General per-bin data term; `state` (dict of tensors, see new_state) is updated in place."""
        sino = (self.n_angles, self.n_bins)
        st = None
        if state is not None:
            st = self._state(state)
        if state is None and u_out is None:
            u_out = self.empty_image()
        diag = Diag()
        prm = params if params is not None else default_params()
        _check(load().tv_pd_run(self._h, self._t(w, sino, "w"), self._t(a, sino, "a"), self._t(lo, sino, "lo"),
                                self._t(hi, sino, "hi"), float(alpha), int(iters), ctypes.byref(prm),
                                ctypes.byref(st) if st is not None else None,
                                self._t(u_out, (self.n, self.n), "u_out") if u_out is not None else None,
                                ctypes.byref(diag) if want_diag else None, _stream(stream)))
        return (u_out if u_out is not None else state["u"]), diag.as_dict()


class _PlanView(Plan):
    """A plan owned by a Batch (not destroyed on its own)."""

    def __init__(self, handle, n, n_angles, n_bins, angles, h, ds):
        import torch
        self._h = ctypes.c_void_p(handle)
        self.angles = angles
        self.n, self.n_angles, self.n_bins, self.h, self.ds = n, n_angles, n_bins, h, ds
        self.dtype = "f32"
        self.torch_dtype = torch.float32
        self.op_dtype = torch.float32

    def close(self):
        self._h = ctypes.c_void_p()


class Batch:
    """Many independent FP32 slices solved together: each stage of an iteration is one
    kernel launch over all slices (ctr_batch in include/ctrecon.h)."""

    def __init__(self, geometries):
        """geometries: iterable of dicts with n, n_angles, n_bins and optional angles, h, ds."""
        lib = load()
        self.geoms = []
        arr = (Geometry * len(geometries))()
        for i, g in enumerate(geometries):
            n, N, M = int(g["n"]), int(g["n_angles"]), int(g["n_bins"])
            ang = g.get("angles")
            ang = np.arange(N, dtype=np.float64) * (np.pi / N) if ang is None else np.ascontiguousarray(ang, np.float64)
            h, ds = float(g.get("h", 1.0)), float(g.get("ds", 1.0))
            self.geoms.append(dict(n=n, n_angles=N, n_bins=M, angles=ang, h=h, ds=ds))
            arr[i] = Geometry(n, N, M, h, ds, ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        handle = ctypes.c_void_p()
        _check(lib.ctr_batch_create(arr, len(geometries), ctypes.byref(handle)))
        self._h = handle
        self.plans = [_PlanView(lib.ctr_batch_plan(handle, i), g["n"], g["n_angles"], g["n_bins"], g["angles"],
                                g["h"], g["ds"]) for i, g in enumerate(self.geoms)]

    def __len__(self):
        return len(self.geoms)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().ctr_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def launch_count(self) -> int:
        return int(load().ctr_batch_launch_count(self._h))

    def retune(self):
        _check(load().ctr_batch_retune(self._h))

    @property
    def mode(self) -> int:
        """0: one launch per stage (graph-captured); 1: one persistent cooperative launch per iteration."""
        return int(load().ctr_batch_get_mode(self._h))

    @property
    def persistent_ctas(self) -> int:
        return int(load().ctr_batch_persistent_ctas(self._h))

    def set_mode(self, mode: int, spin_limit: int = 1 << 26):
        _check(load().ctr_batch_set_mode(self._h, int(mode), int(spin_limit)))

    def solve(self, fs, masks, alphas, deltas, iters: int, params: Optional[Params] = None, betas=None, cs=None,
              u_outs=None, want_diag: bool = True, stream=None):
        """tv_pd_solve for every slice; returns (list of u, list of diag dicts or None)."""
        import torch
        ns = len(self)
        if u_outs is None:
            u_outs = [torch.empty((g["n"], g["n"]), dtype=torch.float32, device="cuda") for g in self.geoms]
        fp = (ctypes.c_void_p * ns)()
        up = (ctypes.c_void_p * ns)()
        mp = (ctypes.c_void_p * ns)()
        for i, g in enumerate(self.geoms):
            fp[i] = self.plans[i]._t(fs[i], (g["n_angles"], g["n_bins"]), f"f[{i}]").value
            up[i] = self.plans[i]._t(u_outs[i], (g["n"], g["n"]), f"u_out[{i}]").value
            m = None if masks is None else masks[i]
            if m is not None:
                if m.dtype != torch.uint8 or not m.is_cuda or tuple(m.shape) != (g["n_angles"], g["n_bins"]):
                    raise ValueError(f"mask[{i}] must be a CUDA uint8 tensor of the sinogram's shape")
                mp[i] = m.data_ptr()
        al = (ctypes.c_double * ns)(*[float(a) for a in alphas])
        de = (ctypes.c_double * ns)(*[float(d) for d in deltas])
        be = (ctypes.c_double * ns)(*[float(b) for b in betas]) if betas is not None else None
        cc = (ctypes.c_double * ns)(*[float(c) for c in cs]) if cs is not None else None
        diags = (Diag * ns)() if want_diag else None
        prm = params if params is not None else default_params()
        _check(load().tv_pd_solve_batched(self._h, fp, mp, al, de, int(iters), ctypes.byref(prm), be, cc, up,
                                          diags, _stream(stream)))
        return u_outs, ([d.as_dict() for d in diags] if want_diag else None)
