#!/usr/bin/env python
"""Benchmark: preconditioned primal-dual (Alg. 4, PDRQS1) iterations per second on
the 512 x 512, 720-view, 729-bin metal-artifact-reduction workload (FP32), one full
solve per step (power iterations for beta and c, 500 iterations, diagnostics).

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle on the
same workload instead (a bounded sample per step).  Multi-GPU (torchrun): every
rank solves its own copy of the workload (independent slices, no collective on the
data path); value = all ranks' iterations / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "preconditioned PD iters/sec and Gray-samples/s (R_h+R_h^T) at 512²×720 views; %HBM peak"
UNIT = "PD iters/s"
WORKLOAD = "mar_fp32_512x512_720views_729bins_500iters"
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
FMA_PER_SAMPLE = 2   # algorithmic work of R_h / R_h^*: interpolate (FMA) and accumulate (FMA) per (pixel, angle)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_init():
    from paper_1810_03275_gb300 import dist
    return dist.init()


def barrier(ws):
    from paper_1810_03275_gb300 import dist
    dist.barrier()


def max_over_ranks(x, ws):
    from paper_1810_03275_gb300 import dist
    return dist.max_over_ranks(x)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def src_sha(*rel):
    h = hashlib.sha256()
    for r in rel:
        with open(os.path.join(ROOT, r), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_record(call: str):
    """DRAM bytes per operator call (summed over the kernels it launches) from the
    committed ncu summary, if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        rec = d.get(call)
        if rec and rec.get("src_sha") == src_sha("paper_1810_03275_gb300/csrc/radon.cu"):
            return rec.get("dram_bytes_per_call")
    except Exception:
        pass
    return None


def cpu_oracle_rate(problem, budget_s: float = 12.0, max_iters: int = 40):
    """The FP64 oracle's Alg. 4 on the same problem: iterations/s on the host cores.
    beta and c are fixed constants (the per-iteration cost does not depend on them)."""
    import oracle
    geo = oracle.Geometry(problem.n, problem.n_angles, problem.n_bins, theta=problem.theta)
    desc = oracle.make_descriptors(problem.f, problem.mask, problem.delta)
    kw = dict(sigma=1.0, tau=1 / np.sqrt(8), eps=np.pi / problem.n, beta=100.0, c=1.0)
    st = oracle.pdrq_solve(geo, desc, problem.alpha, 1, **kw)      # warm-up (page-in, OpenMP pool)
    t0 = time.perf_counter()
    k = 0
    while k < max_iters and (time.perf_counter() - t0) < budget_s:
        st = oracle.pdrq_solve(geo, desc, problem.alpha, 1, state=st, **kw)
        k += 1
    dt = time.perf_counter() - t0
    return k / dt, k, dt, oracle.num_threads()


def measure_algorithms(plan, f, mask, pr, iters: int = 200):
    """Every solver and preconditioner kind on the benchmark plan and data: iterations/s
    at fixed (beta, c), CUDA events on the torch stream.  Alg. 4 with each preconditioner
    kind (0 inverse norm, 1 impulse response, 2 circulant, 3 Richardson), Alg. 5 (u >= 0,
    with its most negative pixel), Alg. 3 and ADMM (2 CG steps) on the unconstrained
    problem, Alg. 1 (Chambolle-Pock) on (C_h)."""
    import numpy as np
    import torch
    from paper_1810_03275_gb300 import ctrecon as ct
    beta = plan.power_beta(20)
    c = 1.05 * plan.power_lambda(beta, np.pi / pr.n, 20)

    def timed(fn):
        fn(5)
        best = 0.0
        for _ in range(2):                      # the better of two timings
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            u = fn(iters)
            b.record()
            torch.cuda.synchronize()
            best = max(best, iters / (a.elapsed_time(b) / 1e3))
        return {"iters_per_s": best, "min_u": float(u.min())}

    out = {}
    for kind in (0, 1, 2, 3):
        ck = c if kind == 0 else plan.tv_pd_solve(f, mask, pr.alpha, pr.delta, 1, params=ct.default_params(
            beta=beta, precond=kind, power_iters=20))[1]["c"]          # c of this kind's own power iteration
        prm = ct.default_params(beta=beta, c=ck, precond=kind)
        out[f"alg4_precond{kind}"] = timed(lambda k: plan.tv_pd_solve(f, mask, pr.alpha, pr.delta, k, params=prm)[0])
    prm = ct.default_params(beta=beta, c=c)
    # Alg. 4 (kind 0) with each launch option switched back: plain stream order instead of
    # programmatic dependent launch, and the CTA-level preconditioner passes (form 1)
    run4 = lambda k: plan.tv_pd_solve(f, mask, pr.alpha, pr.delta, k, params=prm)[0]
    plan.set_launch_overlap(0)
    out["alg4_launch_overlap_off"] = timed(run4)
    plan.set_launch_overlap(1)
    form0 = plan.fft_form
    plan.set_fft_form(1)
    out["alg4_fft_form1"] = timed(run4)
    plan.set_fft_form(form0)
    out["alg5_nonneg"] = timed(lambda k: plan.tv_pd_solve(f, mask, pr.alpha, pr.delta, k,
                                                          params=ct.default_params(beta=beta, c=c, nonneg=1))[0])
    out["alg3_unconstrained"] = timed(lambda k: plan.tv_pdrq2_solve(f, pr.alpha, k, params=prm)[0])
    out["admm_cg2_unconstrained"] = timed(lambda k: plan.tv_admm_solve(f, pr.alpha, k, mu=1.0, cg_iters=2,
                                                                       params=prm)[0])
    out["alg1_cp"] = timed(lambda k: plan.tv_cp_solve(f, mask, pr.alpha, pr.delta, k, params=prm)[0])
    out["workload"] = f"512x512/720/729 MAR data, {iters} iterations per timing (beta, c fixed)"
    return out


def measure_autograd(slices: int = 16, K: int = 20, ckpt: int = 5):
    """The differentiable form: `slices` phantoms of 256 x 256 (360 views, 363 bins, FP32),
    K unrolled iterations of Alg. 4 with checkpoints every `ckpt`, gradient of
    ||u_K - u_true||^2 w.r.t. f and alpha per slice; CUDA events on the torch stream around
    all slices' forward + backward (beta and c fixed once per plan)."""
    import torch
    from paper_1810_03275_gb300 import autograd as ag
    from paper_1810_03275_gb300 import ctrecon as ct
    from paper_1810_03275_gb300 import phantom
    n, N, M = 256, 360, 363
    probs = [phantom.make_problem(f"ad{i}", n, N, M, seed=40 + i, n_ellipses=4, n_metal=1, noise="poisson",
                                  alpha=0.3) for i in range(slices)]
    plan = ct.Plan(n, N, M, angles=probs[0].theta)
    prm = ag.fixed_scaling(plan)
    data = [(torch.as_tensor(p.f, dtype=torch.float32, device="cuda"), torch.as_tensor(p.mask, device="cuda"),
             torch.as_tensor(p.truth, dtype=torch.float32, device="cuda"), p.alpha, p.delta) for p in probs]

    def run(ds):
        for f0, mask, truth, alpha0, delta in ds:
            f = f0.clone().requires_grad_(True)
            alpha = torch.tensor(alpha0, dtype=torch.float64, requires_grad=True)
            u = ag.unrolled_pdrq(f, alpha, plan, mask, delta, iters=K, ckpt=ckpt, params=prm)
            ((u - truth) ** 2).sum().backward()

    run(data[:2])
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    run(data)
    b.record()
    torch.cuda.synchronize()
    secs = a.elapsed_time(b) / 1e3
    fwd_only = 0.0
    a.record()
    for f0, mask, truth, alpha0, delta in data:
        ag.unrolled_pdrq(f0, torch.tensor(alpha0, dtype=torch.float64), plan, mask, delta, iters=K, ckpt=ckpt,
                         params=prm)
    b.record()
    torch.cuda.synchronize()
    fwd_only = a.elapsed_time(b) / 1e3
    return {"slices": slices, "K": K, "ckpt": ckpt,
            "unrolled_iters_per_s_fwd_bwd": slices * K / secs, "ms_per_slice_fwd_bwd": 1e3 * secs / slices,
            "ms_per_slice_fwd": 1e3 * fwd_only / slices,
            "workload": "16 x 256^2 phantoms, 360 views, 363 bins, FP32, gradient w.r.t. f and alpha"}


def operator_roofline(plan, pr, fma_peak, reps: int = 10):
    """R_h (rh_forward_t) and R_h^* (rh_adjoint) of `plan` timed alone (CUDA events on the
    launching stream, inputs larger than L2 at 2048^2): ms per call, GFMA/s against the
    measured FMA ceiling, and algorithmic HBM GB/s (operands read once, result written
    once, in the plan's storage type) against the measured copy peak."""
    import torch
    n, N, M = pr.n, pr.n_angles, pr.n_bins
    opd = plan.op_dtype
    u = torch.rand((n, n), device="cuda").to(opd)
    uT = u.t().contiguous()
    g_in = torch.rand((N, M), device="cuda").to(opd)
    g_out = torch.empty((N, M), dtype=torch.float32, device="cuda")
    u_out = torch.empty((n, n), dtype=torch.float32, device="cuda")
    esz = 2 if opd == torch.bfloat16 else 4
    hbm_peak, _ = peaks()
    res = {}
    for name, fn, nbytes in (("rh_forward_t", lambda: plan.rh_forward_t(u, uT, g_out), 2 * esz * n * n + 4 * N * M),
                             ("rh_adjoint", lambda: plan.rh_adjoint(g_in, u_out), esz * N * M + 4 * n * n)):
        for _ in range(2):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        t = a.elapsed_time(b) / reps / 1e3
        fma = FMA_PER_SAMPLE * n * n * N
        res[name] = {"ms": 1e3 * t, "gfma_s": fma / t / 1e9, "fma_frac": fma / t / fma_peak,
                     "hbm_gbs": nbytes / t / 1e9, "hbm_frac": nbytes / t / 1e9 / hbm_peak, "alg_bytes": nbytes}
    return res


def measure_forms(iters: int = 30, fma_peak: float = 4.03e13):
    """The BF16 form against the plain FP32 path on the 2048 x 2048 / 2048 views /
    2897 bins geometry: iterations/s of Alg. 4 (fixed beta and c, so only the
    iteration is timed), CUDA events on the torch stream; and each projector timed alone
    (the HBM-sized roofline: the image and sinogram exceed L2 there)."""
    import torch
    from paper_1810_03275_gb300 import ctrecon as ct
    from paper_1810_03275_gb300 import phantom
    pr = phantom.make_problem("forms_2048", 2048, 2048, 2897, seed=5, n_ellipses=2, n_metal=1, noise="poisson",
                              alpha=0.3, iters=iters)
    f = torch.as_tensor(pr.f, dtype=torch.float32, device="cuda")
    mask = torch.as_tensor(pr.mask, device="cuda")
    out = {}
    beta = c = None
    for dt in ("f32", "bf16"):
        plan = ct.Plan(pr.n, pr.n_angles, pr.n_bins, angles=pr.theta, dtype=dt)
        from paper_1810_03275_gb300 import autotune
        if beta is None:
            beta = plan.power_beta(20)
            c = 1.05 * plan.power_lambda(beta, np.pi / pr.n, 20)
        prm = ct.default_params(beta=beta, c=c)
        autotune.tune_solve(plan, f, mask, pr.alpha, pr.delta, iters=4, reps=1, params=prm, use_cache=False)  # untimed
        plan.tv_pd_solve(f, mask, pr.alpha, pr.delta, 5, params=prm)      # warm-up
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        plan.tv_pd_solve(f, mask, pr.alpha, pr.delta, iters, params=prm)
        b.record()
        torch.cuda.synchronize()
        t = a.elapsed_time(b) / 1e3
        out[dt] = {"iters_per_s": iters / t, "gsamples_per_s": 2.0 * pr.n * pr.n * pr.n_angles * iters / t / 1e9,
                   "operators": operator_roofline(plan, pr, fma_peak),
                   "tuned": {"bp_groups": plan.bp_groups, "fwd_shape_jobs_segments": list(plan.fwd_shape)}}
        del plan
        torch.cuda.empty_cache()
    out["bf16_speedup"] = out["bf16"]["iters_per_s"] / out["f32"]["iters_per_s"]
    out["workload"] = f"2048x2048, 2048 views, 2897 bins, {iters} iterations per timing (beta, c fixed)"
    return out


def measure_batched(iters: int = 30, count: int = 64):
    """The batched form on 64 slices of uneven size (n in {256..1024}, 180-1440 views,
    ceil(sqrt(2) n) bins): slice-iterations/s of one batched solve (one launch per
    stage over all slices, graph-captured, autotuned angle split) against solving the
    same slices one after another with tv_pd_solve.  beta and c fixed per slice."""
    import torch
    from paper_1810_03275_gb300 import autotune
    from paper_1810_03275_gb300 import ctrecon as ct
    from paper_1810_03275_gb300 import phantom
    probs = phantom.config_batched(count, iters=iters, n_ellipses=2, n_metal=1)
    batch = ct.Batch([dict(n=p.n, n_angles=p.n_angles, n_bins=p.n_bins, angles=p.theta) for p in probs])
    fs = [torch.as_tensor(p.f, dtype=torch.float32, device="cuda") for p in probs]
    ms = [torch.as_tensor(p.mask, device="cuda") for p in probs]
    al = [p.alpha for p in probs]
    de = [p.delta for p in probs]
    betas = [pl.power_beta(10) for pl in batch.plans]
    cs = [1.05 * pl.power_lambda(b, np.pi / pl.n, 10) for pl, b in zip(batch.plans, betas)]
    policy = autotune.tune_batch(batch, fs, ms, al, de, iters=3, betas=betas, cs=cs, use_cache=False)
    prm = ct.default_params()
    batch.solve(fs, ms, al, de, 5, params=prm, betas=betas, cs=cs, want_diag=False)      # warm-up
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    l0 = batch.launch_count
    a.record()
    batch.solve(fs, ms, al, de, iters, params=prm, betas=betas, cs=cs, want_diag=False)
    b.record()
    torch.cuda.synchronize()
    t_batch = a.elapsed_time(b) / 1e3
    launches = batch.launch_count - l0
    persistent = None
    if batch.persistent_ctas > 0:                   # the same solve as one persistent launch per iteration
        batch.set_mode(1)
        batch.solve(fs, ms, al, de, 3, params=prm, betas=betas, cs=cs, want_diag=False)
        torch.cuda.synchronize()
        l1 = batch.launch_count
        a.record()
        batch.solve(fs, ms, al, de, iters, params=prm, betas=betas, cs=cs, want_diag=False)
        b.record()
        torch.cuda.synchronize()
        t_p = a.elapsed_time(b) / 1e3
        persistent = {"slice_iters_per_s": count * iters / t_p, "ctas": batch.persistent_ctas,
                      "kernel_launches": batch.launch_count - l1, "vs_staged": t_batch / t_p}
        batch.set_mode(0)
    us = [torch.empty((p.n, p.n), dtype=torch.float32, device="cuda") for p in probs]
    plans = [ct.Plan(p.n, p.n_angles, p.n_bins, angles=p.theta) for p in probs]
    for pl, bp in zip(plans, batch.plans):
        pl.set_bp_groups(bp.bp_groups)
    for pl, f, m, p, bb, cc, u in zip(plans, fs, ms, probs, betas, cs, us):
        pl.tv_pd_solve(f, m, p.alpha, p.delta, 2, params=ct.default_params(beta=bb, c=cc), u_out=u)
    torch.cuda.synchronize()
    a.record()
    for pl, f, m, p, bb, cc, u in zip(plans, fs, ms, probs, betas, cs, us):
        pl.tv_pd_solve(f, m, p.alpha, p.delta, iters, params=ct.default_params(beta=bb, c=cc), u_out=u)
    b.record()
    torch.cuda.synchronize()
    t_seq = a.elapsed_time(b) / 1e3
    samples = sum(2.0 * p.n * p.n * p.n_angles for p in probs) * iters
    return {"slices": count, "iters": iters, "policy": policy,
            "batched": {"slice_iters_per_s": count * iters / t_batch, "gsamples_per_s": samples / t_batch / 1e9,
                        "kernel_launches": launches},
            "sequential": {"slice_iters_per_s": count * iters / t_seq, "gsamples_per_s": samples / t_seq / 1e9},
            "speedup": t_seq / t_batch, "persistent": persistent,
            "workload": "64 slices, n in {256,384,512,768,1024}, 180-1440 views, ceil(sqrt(2) n) bins, FP32"}


def run_ops(args):
    """The operator calls of one plan (R_h, R_h^* and the preconditioner), `--steps` times
    each after `--warmup` (a profiler's target: seeded uniform inputs, uniform angles over
    [0, pi))."""
    import torch
    from paper_1810_03275_gb300 import ctrecon as ct
    fields = args.ops.split(",")
    n, N, M, dt = int(fields[0]), int(fields[1]), int(fields[2]), fields[3]
    plan = ct.Plan(n, N, M, dtype=dt)
    if len(fields) > 4:                             # forward shape "JxS" (jobs per CTA x row segments)
        plan.set_fwd_shape(*(int(x) for x in fields[4].split("x")))
    gen = torch.Generator(device="cuda").manual_seed(0)
    u = torch.rand((n, n), device="cuda", generator=gen).to(plan.op_dtype)
    uT = u.t().contiguous()
    g = torch.rand((N, M), device="cuda", generator=gen).to(plan.op_dtype)
    go = torch.empty((N, M), device="cuda", dtype=plan.torch_dtype)
    uo = torch.empty((n, n), device="cuda", dtype=plan.torch_dtype)
    uf = u.to(plan.torch_dtype)
    xo = torch.empty_like(uo)
    prm = ct.default_params(c=1.0)
    for k in range(args.warmup + args.steps):
        torch.cuda.nvtx.range_push("ops_step" if k >= args.warmup else "ops_warmup")
        plan.rh_forward_t(u, uT, go)
        plan.rh_adjoint(g, uo)
        plan.precond_apply(uf, prm, xo)
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    return 0


def run_batch_step(args):
    """The 64-slice batch of `forms.batched` (a profiler's target): per-slice set-up and a
    warm-up solve outside, then one batched solve of `--batch-step` iterations inside the NVTX
    range `batch_step`."""
    import torch
    from paper_1810_03275_gb300 import ctrecon as ct
    from paper_1810_03275_gb300 import phantom
    probs = phantom.config_batched(64, iters=30, n_ellipses=2, n_metal=1)
    batch = ct.Batch([dict(n=p.n, n_angles=p.n_angles, n_bins=p.n_bins, angles=p.theta) for p in probs])
    fs = [torch.as_tensor(p.f, dtype=torch.float32, device="cuda") for p in probs]
    ms = [torch.as_tensor(p.mask, device="cuda") for p in probs]
    al, de = [p.alpha for p in probs], [p.delta for p in probs]
    betas = [pl.power_beta(10) for pl in batch.plans]
    cs = [1.05 * pl.power_lambda(b, np.pi / pl.n, 10) for pl, b in zip(batch.plans, betas)]
    prm = ct.default_params()
    batch.solve(fs, ms, al, de, 3, params=prm, betas=betas, cs=cs, want_diag=False)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("batch_step")
    batch.solve(fs, ms, al, de, args.batch_step, params=prm, betas=betas, cs=cs, want_diag=False)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    return 0


def run_reference(args, rank, ws):
    if rank != 0:
        return 0
    from paper_1810_03275_gb300 import phantom
    pr = phantom.config_mar_fp32()
    import oracle
    geo = oracle.Geometry(pr.n, pr.n_angles, pr.n_bins, theta=pr.theta)
    desc = oracle.make_descriptors(pr.f, pr.mask, pr.delta)
    kw = dict(sigma=1.0, tau=1 / np.sqrt(8), eps=np.pi / pr.n, beta=100.0, c=1.0)
    per_step = 2
    st = None
    for _ in range(args.warmup):
        st = oracle.pdrq_solve(geo, desc, pr.alpha, 1, state=st, **kw)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        st = oracle.pdrq_solve(geo, desc, pr.alpha, per_step, state=st, **kw)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = per_step * args.steps / total
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": pr.n, "views": pr.n_angles, "bins": pr.n_bins,
                   "iters_per_solve": pr.iters, "step": f"{per_step} oracle iterations (bounded sample)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} PDRQS1 iterations per step of the 512x512/720/729 problem, FP64 C+numpy"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--iters", type=int, default=None, help="override iterations per solve (profiling only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the BF16-vs-FP32 2048^2 timing")
    ap.add_argument("--batch-step", type=int, default=0, help="K: only run the 64-slice batched solve of K "
                                                                 "iterations in an NVTX range (profiling)")
    ap.add_argument("--shape", default=None, help="G,J,S: backprojection groups and forward shape instead of the "
                                                  "tuner (for runs under a profiler)")
    ap.add_argument("--ops", default=None, help="n,views,bins,dtype[,JxS]: only run R_h, R_h^* and the "
                    "preconditioner of that plan --steps times (for a profiler; JxS a forward shape), print nothing")
    args = ap.parse_args()
    if args.ops:
        return run_ops(args)
    if args.batch_step > 0:
        return run_batch_step(args)
    if args.warmup < 3 and args.impl == "ours" and args.iters is None:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    rank, ws, local = dist_init()
    if args.impl == "reference":
        return run_reference(args, rank, ws)

    import torch
    from paper_1810_03275_gb300 import ctrecon as ct
    from paper_1810_03275_gb300 import phantom

    torch.cuda.set_device(local)
    fma_peak = ct.fp32_fma_rate()                   # measured FP32 FMA ceiling (roofline denominator)
    pr = phantom.config_mar_fp32(seed=2 + rank)     # each rank: its own slice
    iters = args.iters or pr.iters
    n, N, M = pr.n, pr.n_angles, pr.n_bins
    plan = ct.Plan(n, N, M, angles=pr.theta, dtype="f32")
    f = torch.as_tensor(pr.f, dtype=torch.float32, device="cuda")
    mask = torch.as_tensor(pr.mask, device="cuda")
    u = torch.empty((n, n), dtype=torch.float32, device="cuda")
    from paper_1810_03275_gb300 import autotune
    if args.shape:                                  # a fixed launch setting (profiling: no timing under a profiler)
        g, j, sg = (int(x) for x in args.shape.split(","))
        plan.set_bp_groups(g)
        plan.set_fwd_shape(j, sg)
        tuned = {"bp_groups": g, "fwd_shape": [j, sg], "fixed": True}
    else:
        tuned = autotune.tune_solve(plan, f, mask, pr.alpha, pr.delta, iters=40, use_cache=False)   # untimed
    prm = ct.default_params()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        plan.tv_pd_solve(f, mask, pr.alpha, pr.delta, iters, params=prm, u_out=u)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    if not args.no_clocks:
        clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    launches0 = plan.launch_count
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    diag = None
    for k in range(args.steps):
        flush.fill_(float(k))                       # evict L2 between steps
        torch.cuda.nvtx.range_push("bench_step")
        ev[k][0].record(stream)
        _, diag = plan.tv_pd_solve(f, mask, pr.alpha, pr.delta, iters, params=prm, u_out=u)
        ev[k][1].record(stream)
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier(ws)
    launches = (plan.launch_count - launches0) / args.steps
    step_ms = [a.elapsed_time(b) for a, b in ev]
    clk = clocks.stop() if not args.no_clocks else None
    t_step = max_over_ranks(sum(step_ms) / args.steps / 1e3, ws)
    value = ws * iters / t_step
    samples = 2.0 * n * n * N * iters

    # --- dominant kernels, timed alone on the launching stream -------------------------
    uT = u.t().contiguous()
    g = torch.empty((N, M), dtype=torch.float32, device="cuda")
    reps = 20
    kt = {}
    sym = plan.symmetric_jobs > 0
    call_kernels = {"rh_adjoint": ["k_backproject_orbit", "k_bp_fold"] if sym else
                    (["k_backproject", "k_bp_reduce"] if plan.bp_groups > 1 else ["k_backproject"]),
                    "rh_forward_t": ["k_orbit_image", "k_forward_orbit"] if sym else ["k_forward"]}
    for name, fn in (("rh_adjoint", lambda: plan.rh_adjoint(f, u)), ("rh_forward_t", lambda: plan.rh_forward_t(u, uT, g))):
        for _ in range(3):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        kt[name] = a.elapsed_time(b) / reps / 1e3
    dom = max(kt, key=kt.get)
    # the preconditioner passes alone (M^{-1} y, symbols cached), in both kernel forms
    prm_pc = ct.default_params(c=1.0, eps=np.pi / n)
    xo = torch.empty_like(u)
    form0, pc_ms = plan.fft_form, {}
    for form in (0, 1):
        plan.set_fft_form(form)
        if plan.fft_form != form:
            continue
        for _ in range(3):
            plan.precond_apply(u, prm_pc, xo)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            plan.precond_apply(u, prm_pc, xo)
        b.record(stream)
        torch.cuda.synchronize()
        pc_ms[f"form{form}"] = a.elapsed_time(b) / reps
        # the same calls replayed from a CUDA graph: the GPU time without the host's launch cost
        gs = torch.cuda.Stream()
        gs.wait_stream(stream)
        with torch.cuda.stream(gs):
            plan.precond_apply(u, prm_pc, xo)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gs):
            for _ in range(reps):
                plan.precond_apply(u, prm_pc, xo)
        graph.replay()
        torch.cuda.synchronize()
        a.record(stream)
        graph.replay()
        b.record(stream)
        torch.cuda.synchronize()
        pc_ms[f"form{form}_graph"] = a.elapsed_time(b) / reps
        del graph
    plan.set_fft_form(form0)
    hbm_peak, peak_kind = peaks()
    nominal = SM_COUNT * FP32_LANES * SM_MAX_MHZ * 1e6                # FMA/s, FP32 lanes x max clock
    fmas = FMA_PER_SAMPLE * n * n * N                                  # algorithmic FMAs per operator call
    bytes_alg = 4.0 * (n * n + N * M)
    kernels = {k: {"ms": 1e3 * v, "kernels": call_kernels[k], "gsamples_per_s": n * n * N / v / 1e9,
                   "gfma_s": fmas / v / 1e9, "fma_frac": fmas / v / fma_peak, "hbm_gbs": bytes_alg / v / 1e9,
                   "hbm_frac": bytes_alg / v / 1e9 / hbm_peak} for k, v in kt.items()}
    kernels["precond_apply"] = {"ms": pc_ms.get(f"form{plan.fft_form}"),
                                "graph_ms": pc_ms.get(f"form{plan.fft_form}_graph"), "form": plan.fft_form,
                                "forms_ms": pc_ms,
                                "note": "form 0: warp-level passes, form 1: CTA-level Stockham passes; ms: calls "
                                        "launched from the host one by one, graph_ms: the same calls replayed from a "
                                        "CUDA graph (GPU time without the host launch cost)"}
    roof = {"bound": "alu", "kernel": f"{dom} ({' + '.join(call_kernels[dom])})", "path":
            f"symmetric, {plan.symmetric_jobs} jobs for {N} angles" if sym else "per angle",
            "achieved": fmas / kt[dom] / 1e9, "peak": fma_peak / 1e9, "unit": "GFMA/s",
            "frac": fmas / kt[dom] / fma_peak, "traffic": traffic_record(dom),
            "work_per_launch": f"{FMA_PER_SAMPLE} FMA x n^2 N = {fmas:.4g} FMA",
            "peak_source": "measured: ctr_fp32_fma_rate (FMA chains, 8 x 256 threads per SM)",
            "nominal_fma_s": nominal, "frac_of_nominal": fmas / kt[dom] / nominal,
            "hbm": {"achieved_gbs": bytes_alg / kt[dom] / 1e9, "peak_gbs": hbm_peak, "peak_source": peak_kind,
                    "frac": bytes_alg / kt[dom] / 1e9 / hbm_peak}}

    # --- end to end through the C ABI with host buffers ---------------------------------
    f_h = torch.as_tensor(pr.f, dtype=torch.float32).pin_memory()
    m_h = torch.as_tensor(pr.mask).pin_memory()
    u_h = torch.empty((n, n), dtype=torch.float32).pin_memory()
    e2e_steps = max(2, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        f.copy_(f_h, non_blocking=True)
        mask.copy_(m_h, non_blocking=True)
        plan.tv_pd_solve(f, mask, pr.alpha, pr.delta, iters, params=prm, u_out=u)
        u_h.copy_(u, non_blocking=True)
        torch.cuda.synchronize()
    e2e_t = max_over_ranks((time.perf_counter() - t0) / e2e_steps, ws)

    forms = None
    if rank == 0 and not args.no_forms:
        forms = {"bf16": measure_forms(fma_peak=fma_peak), "batched": measure_batched(),
                 "algorithms": measure_algorithms(plan, f, mask, pr), "autograd": measure_autograd()}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, k, dt, cores = cpu_oracle_rate(pr)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{k} PDRQS1 iterations ({dt:.1f} s) of the same 512x512/720/729 problem, FP64 C+numpy, "
                         f"beta and c fixed"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "views": N, "bins": M, "iters_per_solve": iters,
                       "step": "one tv_pd_solve: power iterations (50+50) + iterations + diagnostics",
                       "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{ws}",
                       "tuned": tuned},
            "gsamples_per_s": ws * samples / t_step / 1e9,
            "roofline": roof,
            "kernels": kernels,
            "forms": forms,
            "cpu_baseline": cpu,
            "e2e": {"value": ws * iters / e2e_t, "unit": UNIT, "h2d_bytes_per_step": int(f_h.numel() * 4 + m_h.numel()),
                    "d2h_bytes_per_step": int(u_h.numel() * 4)},
            "gpu_launches": int(launches),
            "clocks": clk,
            "diag": dict({k: diag[k] for k in ("objective", "violation", "gap", "dual_residual", "rel_change")},
                         violation_over_delta=diag["violation"] / pr.delta,
                         note="gap leaves the box indicators out: a certificate only once violation = 0"),
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
