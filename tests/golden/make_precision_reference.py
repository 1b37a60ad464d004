"""Write the FP64 reference of the 2048 x 2048 precision workload (2048 views on
[0, pi), 2897 bins, 10 ellipses and 6 metal disks, 1e5-photon Poisson data,
alpha = 0.3, delta = 3 x the off-trace noise RMS, metal-trace inequality): 300
iterations of Alg. 4 by the FP64 oracle, with beta and c from the oracle's own
power iterations (Sec. 5.1 scaling, Sec. 4.3.1 constant).

Only the oracle and the seeded input generator are called.  The stored file
``precision_2048_reference.npz`` holds the central 512 x 512 crop of u (rows and
columns 768..1279, rounded to float32: 6e-8 relative, far below the errors it
judges), beta, c, the seed, the iteration count, the oracle's diagnostics of
the full image, and a fingerprint of the inputs (sums, extrema, sampled values)
so that a test can check that it regenerated the same data before comparing.

Usage: python tests/golden/make_precision_reference.py [--checkpoint PATH]
(about 2-3 hours on 8 host cores; a checkpoint file lets an interrupted run resume).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1810_03275_gb300 import phantom  # noqa: E402

OUT = os.path.join(HERE, "precision_2048_reference.npz")
SEED = 5
ITERS = 300
POWER_ITERS = 30
CROP = (768, 1280)


def input_fingerprint(pr) -> dict:
    """Statistics of the regenerated inputs that differ if any sample of the noise
    stream moved (and agree to ~1e-12 across platforms otherwise)."""
    f = np.asarray(pr.f, dtype=np.float64)
    return {
        "f_sum": float(f.sum()),
        "f_sumsq": float((f * f).sum()),
        "f_max": float(f.max()),
        "f_min": float(f.min()),
        "f_samples": [float(x) for x in f[::211, ::173].ravel()],
        "mask_sum": int(np.asarray(pr.mask).sum()),
        "delta": float(pr.delta),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--checkpoint", default=None, help="npz file to save/resume the oracle state")
    ap.add_argument("--every", type=int, default=25)
    args = ap.parse_args()

    pr = phantom.config_bf16_2048(seed=SEED)
    geo = oracle.Geometry(pr.n, pr.n_angles, pr.n_bins, theta=pr.theta)
    eps, tau, sigma = np.pi / pr.n, 1.0 / np.sqrt(8.0), 1.0
    desc = oracle.make_descriptors(pr.f, pr.mask, pr.delta)
    print(f"oracle threads: {oracle.num_threads()}", flush=True)

    st = None
    beta = c = None
    if args.checkpoint and os.path.exists(args.checkpoint):
        z = np.load(args.checkpoint)
        beta, c = float(z["beta"]), float(z["c"])
        st = oracle.PDRQState(z["u"], z["Ru"], z["v1b"], z["v2bx"], z["v2by"], z["t1"], z["t2x"], z["t2y"],
                              int(z["k"]))
        print(f"resumed at k = {st.k}", flush=True)
    if beta is None:
        t0 = time.time()
        beta = oracle.power_beta(geo, POWER_ITERS)
        print(f"beta = {beta!r} ({time.time() - t0:.0f} s)", flush=True)
        t0 = time.time()
        c = oracle.power_c(geo, beta, eps, POWER_ITERS)
        print(f"c = {c!r} ({time.time() - t0:.0f} s)", flush=True)

    t0 = time.time()
    while st is None or st.k < ITERS:
        k0 = 0 if st is None else st.k
        step = min(args.every, ITERS - k0)
        st = oracle.pdrq_solve(geo, desc, pr.alpha, step, sigma=sigma, tau=tau, eps=eps, beta=beta, c=c, state=st)
        rate = (time.time() - t0) / max(st.k - k0, 1)
        print(f"k = {st.k}  ({rate:.1f} s per iteration)", flush=True)
        t0 = time.time()
        if args.checkpoint:
            tmp = args.checkpoint + ".tmp.npz"
            np.savez(tmp, u=st.u, Ru=st.Ru, v1b=st.v1b, v2bx=st.v2bx, v2by=st.v2by, t1=st.t1, t2x=st.t2x,
                     t2y=st.t2y, k=st.k, beta=beta, c=c)
            os.replace(tmp, args.checkpoint)

    d = oracle.diagnostics(geo, desc, pr.alpha, st.u, beta=beta, tau=tau, t1=st.t1, t2x=st.t2x, t2y=st.t2y)
    a, b = CROP
    meta = {
        "workload": "2048x2048, 2048 views on [0, pi), 2897 bins, 10 ellipses + 6 metal disks, Poisson 1e5",
        "generator": "phantom.config_bf16_2048", "seed": SEED, "iters": ITERS, "power_iters": POWER_ITERS,
        "sigma": sigma, "tau": tau, "eps": eps, "beta": beta, "c": c, "crop": [a, b],
        "alpha": pr.alpha, "delta": pr.delta, "u_max_full": float(np.abs(st.u).max()),
        "diagnostics": d, "inputs": input_fingerprint(pr),
    }
    np.savez_compressed(OUT, u_crop=st.u[a:b, a:b].astype(np.float32), meta=json.dumps(meta))
    print(f"wrote {OUT}: beta {beta:.9g}, c {c:.9g}, objective {d['objective']:.9g}", flush=True)


if __name__ == "__main__":
    main()
