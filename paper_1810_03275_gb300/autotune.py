"""Project-written autotuner for the projectors' launch shapes.

Two runtime choices per plan, both selecting among compiled kernel instances through
the C ABI (results change only in FP32 summation order):
  * the backprojection's angle (or symmetric-job) split into G groups whose partial
    images are summed: more CTAs in flight against an extra fold;
  * the symmetric forward projector's launch shape: adjacent jobs per CTA (their rays
    nearly coincide, so they share the orbit image's lines in L1, which matters where the
    kernel is bound by L2 bandwidth) and warps per job splitting its rows (shorter serial
    marches against a larger reduction).
The best values depend on the image size and view count and, in a batch, on the other
slices.  The tuner times the candidates with CUDA events and keeps the fastest;
results are cached in a JSON file keyed by (device, n, views, bins) for single plans and
by the batch signature for batches.
"""
from __future__ import annotations

import json
import os
import threading
from typing import Dict, Iterable, Optional

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("CTR_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "ctrecon", "tune.json"))


def _load_cache() -> Dict[str, int]:
    try:
        with open(cache_path()) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _store(key: str, value) -> None:
    with _lock:
        d = _load_cache()
        d[key] = value
        path = cache_path()
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(d, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)


def _device_key() -> str:
    import torch
    return torch.cuda.get_device_name().replace(" ", "_")


def _time(fn, reps: int) -> float:
    import torch
    for _ in range(2):
        fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _try_shape(plan, shape) -> bool:
    """Set a forward launch shape; False where the plan does not offer it (the staged
    shape needs its orbit-image window to fit one CTA's shared memory)."""
    from . import ctrecon as ct
    try:
        plan.set_fwd_shape(*shape)
        return True
    except ct.CtrError:
        return False


def tune_plan(plan, candidates: Iterable[int] = (1, 2, 3, 4, 5, 6, 8), reps: int = 5, use_cache: bool = True,
              shapes=None) -> int:
    """Pick the angle-group count of `plan`'s backprojection and, on the symmetric path,
    the forward projector's launch shape; sets both and returns the group count."""
    import torch
    key = f"plan/{_device_key()}/{plan.dtype}/n{plan.n}/N{plan.n_angles}/M{plan.n_bins}"
    if use_cache:
        hit = _load_cache().get(key)
        if hit is not None:
            try:
                hit = hit if isinstance(hit, dict) else {"bp_groups": int(hit)}
                plan.set_bp_groups(int(hit["bp_groups"]))
                if hit.get("fwd_shape") and plan.fwd_shape[0]:
                    plan.set_fwd_shape(*hit["fwd_shape"])
                return int(hit["bp_groups"])
            except Exception:
                pass
    g = torch.randn((plan.n_angles, plan.n_bins), device="cuda").to(plan.op_dtype)
    u = torch.empty((plan.n, plan.n), device="cuda", dtype=plan.torch_dtype)
    best, best_t = plan.bp_groups, None
    for G in candidates:
        try:
            plan.set_bp_groups(G)
        except Exception:
            continue
        t = _time(lambda: plan.rh_adjoint(g, u), reps)
        if best_t is None or t < best_t:
            best, best_t = G, t
    plan.set_bp_groups(best)
    choice = {"bp_groups": best}
    if plan.fwd_shape[0]:
        x = torch.randn((plan.n, plan.n), device="cuda").to(plan.op_dtype)
        xt = x.t().contiguous()
        gs = torch.empty((plan.n_angles, plan.n_bins), device="cuda", dtype=plan.torch_dtype)
        best_s, best_st = plan.fwd_shape, None
        for shp in (shapes or plan.FWD_SHAPES):
            if not _try_shape(plan, shp):
                continue
            t = _time(lambda: plan.rh_forward_t(x, xt, gs), reps)
            if best_st is None or t < best_st:
                best_s, best_st = tuple(shp), t
        plan.set_fwd_shape(*best_s)
        choice["fwd_shape"] = list(best_s)
    _store(key, choice)
    return best


def tune_batch(batch, fs, masks, alphas, deltas, policies: Iterable[Optional[int]] = (None, 1, 2, 4),
               iters: int = 4, betas=None, cs=None, use_cache: bool = True):
    """Pick the batch's angle-split policy: None keeps each slice's size-based default,
    an integer G applies min(G, capacity) to every slice.  Timed on `iters` batched
    iterations with the given data.  Sets the policy, rebuilds the launch tables and
    returns it."""
    from . import ctrecon as ct
    sig = "|".join(f"{g['n']}x{g['n_angles']}x{g['n_bins']}" for g in batch.geoms)
    import hashlib
    key = f"batch/{_device_key()}/{hashlib.sha1(sig.encode()).hexdigest()[:16]}"
    defaults = [p.bp_groups for p in batch.plans]

    def apply(policy):
        for p, d in zip(batch.plans, defaults):
            want = d if policy is None else policy
            for G in (want, want // 2, 2, 1):
                try:
                    p.set_bp_groups(max(1, G))
                    break
                except ct.CtrError:
                    continue
        batch.retune()

    if use_cache:
        hit = _load_cache().get(key, "missing")
        if hit != "missing":
            apply(hit)
            return hit
    if betas is None or cs is None:
        import numpy as np
        betas = [p.power_beta(10) for p in batch.plans]
        cs = [1.05 * p.power_lambda(b, np.pi / p.n, 10) for p, b in zip(batch.plans, betas)]
    prm = ct.default_params(graph_block=0)
    best, best_t = None, None
    for pol in policies:
        apply(pol)
        t = _time(lambda: batch.solve(fs, masks, alphas, deltas, iters, params=prm, betas=betas, cs=cs,
                                      want_diag=False), 1)
        if best_t is None or t < best_t:
            best, best_t = pol, t
    apply(best)
    _store(key, best)
    return best


def tune_solve(plan, f, mask, alpha: float, delta: float, iters: int = 30, reps: int = 2, params=None,
               groups: Iterable[int] = (1, 2, 3, 4, 5, 6, 8), shapes=None, use_cache: bool = True):
    """Pick the backprojection split and the forward projector's launch shape by timing
    `iters` iterations of Alg. 4 on the given data (beta and c from params, or from short
    power iterations): inside the solve the split also decides how many partial images the
    preconditioner's first pass folds, which a standalone operator timing does not see.
    The split is chosen first (default shape), then the shape.  Sets both; returns
    {"bp_groups": G, "fwd_shape": [jobs_per_cta, segments]} (no shape off the symmetric path)."""
    import numpy as np
    from . import ctrecon as ct
    key = f"solve/{_device_key()}/{plan.dtype}/n{plan.n}/N{plan.n_angles}/M{plan.n_bins}"
    if use_cache:
        hit = _load_cache().get(key)
        if isinstance(hit, dict):
            try:
                plan.set_bp_groups(int(hit["bp_groups"]))
                if hit.get("fwd_shape") and plan.fwd_shape[0]:
                    plan.set_fwd_shape(*hit["fwd_shape"])
                return hit
            except Exception:
                pass
    if params is None or not (params.beta > 0 and params.c > 0):
        beta = plan.power_beta(10)
        params = ct.default_params(beta=beta, c=1.05 * plan.power_lambda(beta, np.pi / plan.n, 10))
    run = lambda: plan.tv_pd_solve(f, mask, alpha, delta, iters, params=params)

    best_g, best_t = plan.bp_groups, None
    for G in groups:
        try:
            plan.set_bp_groups(G)
        except Exception:
            continue
        t = _time(run, reps)
        if best_t is None or t < best_t:
            best_g, best_t = G, t
    plan.set_bp_groups(best_g)
    choice = {"bp_groups": best_g}
    if plan.fwd_shape[0]:
        best_s, best_st = plan.fwd_shape, None
        for shp in (shapes or plan.FWD_SHAPES):
            if not _try_shape(plan, shp):
                continue
            t = _time(run, reps)
            if best_st is None or t < best_st:
                best_s, best_st = tuple(shp), t
        plan.set_fwd_shape(*best_s)
        choice["fwd_shape"] = list(best_s)
    _store(key, choice)
    return choice
