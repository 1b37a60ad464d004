"""Differentiable forms: R_h and R_h^* as torch.autograd.Functions (each other's
hand-written adjoint kernels), and K unrolled iterations of Alg. 4 as a function of
the data f and of alpha, with checkpoints every few iterates.

Forward: the iterations run through tv_pd_solve_state in segments of `ckpt`
iterations; the state (u, R u, v1b, v2b) at the start of each segment is kept.
Backward: each segment is replayed one iteration at a time from its checkpoint and
then reversed (tv_pd_vjp_segment: the library's reverse-mode kernels, the states kept in
a device workspace), newest segment first.  beta and c are fixed per plan (they depend on the geometry only).
"""
from __future__ import annotations

import math
from typing import Optional

import torch

from . import ctrecon as ct


class RadonFn(torch.autograd.Function):
    """g = R_h u; the VJP is R_h^* (the exact transpose kernel)."""

    @staticmethod
    def forward(ctx, u, plan):
        ctx.plan = plan
        return plan.rh_forward(u.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.rh_adjoint(g.contiguous()), None


class BackprojFn(torch.autograd.Function):
    """u = R_h^* g; the VJP is R_h."""

    @staticmethod
    def forward(ctx, g, plan):
        ctx.plan = plan
        return plan.rh_adjoint(g.contiguous())

    @staticmethod
    def backward(ctx, u):
        return ctx.plan.rh_forward(u.contiguous()), None


def radon(u, plan):
    return RadonFn.apply(u, plan)


def backproject(g, plan):
    return BackprojFn.apply(g, plan)


def _clone(st):
    return {k: v.clone() for k, v in st.items()}


class UnrolledPDRQ(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, alpha, plan, mask, delta, iters, ckpt, params):
        # alpha is a host scalar of the C ABI: a CPU tensor (or float) costs no device
        # synchronisation; a CUDA tensor is read back once here
        a = float(alpha.detach().item()) if isinstance(alpha, torch.Tensor) else float(alpha)
        f = f.detach().contiguous()
        if params.graph_block > max(ckpt - 1, 0):
            # each segment is ckpt iterations (the last one kept apart for the diagnostics
            # state): capture graphs of ckpt - 1 iterations, which the plan replays from its
            # graph cache on every segment and every later call
            params = ct.Params.from_buffer_copy(params)
            params.graph_block = max(ckpt - 1, 0)
        state = plan.new_state()
        ckpts = []
        done = 0
        while done < iters:
            ckpts.append((done, _clone(state)))
            k = min(ckpt, iters - done)
            plan.tv_pd_solve_state(f, mask, a, delta, k, params, state)
            done += k
        ctx.plan, ctx.mask, ctx.delta, ctx.iters, ctx.params, ctx.alpha = plan, mask, delta, iters, params, a
        ctx.ckpts = ckpts
        ctx.save_for_backward(f)
        ctx.alpha_is_tensor = isinstance(alpha, torch.Tensor)
        return state["u"].clone()

    @staticmethod
    def backward(ctx, gu):
        (f,) = ctx.saved_tensors
        plan, mask, delta, params, a = ctx.plan, ctx.mask, ctx.delta, ctx.params, ctx.alpha
        dt = plan.torch_dtype
        n, N, M = plan.n, plan.n_angles, plan.n_bins
        bu = gu.detach().to(dt).contiguous().clone()
        b1 = torch.zeros((N, M), dtype=dt, device="cuda")
        b2 = torch.zeros((2, n, n), dtype=dt, device="cuda")
        gf = torch.zeros((N, M), dtype=dt, device="cuda")
        galpha = torch.zeros(1, dtype=torch.float64, device="cuda")
        bounds = [k for k, _ in ctx.ckpts] + [ctx.iters]
        ws = plan.vjp_workspace(max(bounds[i + 1] - bounds[i] for i in range(len(ctx.ckpts))))
        for seg in reversed(range(len(ctx.ckpts))):      # each segment replayed and reversed on the device
            start, st0 = ctx.ckpts[seg]
            plan.tv_pd_vjp_segment(f, mask, a, delta, params, st0, bounds[seg + 1] - start, ws, bu, b1, b2, gf,
                                   galpha)
        ga = galpha.to(torch.float64) if ctx.alpha_is_tensor else None
        if ga is not None:
            ga = ga.reshape(()).to(dtype=torch.float64)
        return gf, ga, None, None, None, None, None, None


def fixed_scaling(plan, power_iters: int = 50, margin: float = 1.05, eps: Optional[float] = None) -> ct.Params:
    """Solver parameters with beta and c from the plan's power iterations, computed once."""
    eps = math.pi / plan.n if eps is None else eps
    beta = plan.power_beta(power_iters)
    c = margin * plan.power_lambda(beta, eps, power_iters)
    return ct.default_params(beta=beta, c=c, eps=eps)


def unrolled_pdrq(f, alpha, plan, mask=None, delta: float = -1.0, iters: int = 20, ckpt: int = 5,
                  params: Optional[ct.Params] = None):
    """u_K of K = `iters` iterations of Alg. 4 from zero, differentiable in f and alpha
    (alpha a 0-d float64 tensor to get its gradient).  params must fix beta and c."""
    if params is None:
        params = fixed_scaling(plan)
    if not (params.beta > 0 and params.c > 0):
        raise ValueError("params must fix beta and c (see fixed_scaling)")
    return UnrolledPDRQ.apply(f, alpha, plan, mask, float(delta), int(iters), int(ckpt), params)
