"""Parity at the sizes the benchmark and the batched form run: the 512 x 512, 720-view,
729-bin metal-artifact workload (the one bench.py times, same graph blocks and projector
path) compared with the FP64 oracle's Alg. 4 after 1, 10 and 200 iterations, and a batch
with one slice each of 256, 512 and 1024 pixels (1440, 361 and 180 views, bins
ceil(sqrt(2) n)) compared with single-slice solves and with the oracle."""
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


def _oracle_constants(geo, eps, steps=20):
    beta = oracle.power_beta(geo, steps)
    return beta, oracle.power_c(geo, beta, eps, steps)


def test_headline_workload_iterates_match_oracle(ct):
    """u, R u, bar v1 and bar v2 after 1, 10 and 200 iterations within 1e-5 (relative l2)
    of the oracle on the 512^2/720/729 workload with its metal trace and data box; the
    GPU runs on the symmetric projector path in graph blocks of 10, as in the benchmark."""
    pr = phantom.config_mar_fp32()
    geo = oracle.Geometry(pr.n, pr.n_angles, pr.n_bins, theta=pr.theta)
    eps, tau = np.pi / pr.n, 1 / np.sqrt(8)
    beta, c = _oracle_constants(geo, eps)
    desc = oracle.make_descriptors(pr.f, pr.mask, pr.delta)
    plan = ct.Plan(pr.n, pr.n_angles, pr.n_bins, angles=pr.theta)
    assert plan.symmetric_jobs > 0
    prm = ct.default_params(beta=beta, c=c, eps=eps, tau=tau)
    assert prm.graph_block == 10
    dev = [to_dev(x, plan.torch_dtype) for x in desc]
    state = plan.new_state()
    st, done = None, 0
    for k in (1, 10, 200):
        st = oracle.pdrq_solve(geo, desc, pr.alpha, k - done, sigma=1.0, tau=tau, eps=eps, beta=beta, c=c, state=st)
        plan.tv_pd_run(*dev, pr.alpha, k - done, params=prm, state=state)
        done = k
        got = {kk: to_np(v) for kk, v in state.items() if v is not None}
        errs = {"u": rel_l2(got["u"], st.u), "Ru": rel_l2(got["Ru"], st.Ru), "v1b": rel_l2(got["v1b"], st.v1b),
                "v2b": rel_l2(got["v2b"], np.stack([st.v2bx, st.v2by]))}
        print(f"512^2/720/729, k = {k}: " + ", ".join(f"{a} {e:.2e}" for a, e in errs.items()))
        for name, e in errs.items():
            assert e < 1e-5, (k, name, e)


def _config3_slices():
    spec = [(256, 1440), (512, 361), (1024, 180), (384, 241)]
    probs = [phantom.make_problem(f"c3_{n}", n, N, int(np.ceil(np.sqrt(2.0) * n)), seed=31 + i, n_ellipses=4,
                                  n_metal=2, noise="poisson", alpha=0.3) for i, (n, N) in enumerate(spec)]
    probs[3].theta = probs[3].theta + 0.013      # off the uniform grid: the per-angle path
    return probs


def test_batched_form_at_config3_sizes(ct):
    """One batch of 256^2/1440, 512^2/361 (odd: pair jobs), 1024^2/180 and 384^2/241 with
    angles off the uniform grid (per-angle path): 30 iterations equal the same slices solved
    alone (<= 2e-6) and the oracle (<= 1e-5)."""
    import torch
    probs = _config3_slices()
    batch = ct.Batch([dict(n=p.n, n_angles=p.n_angles, n_bins=p.n_bins, angles=p.theta) for p in probs])
    assert [pl.symmetric_jobs > 0 for pl in batch.plans] == [True, True, True, False]
    fs = [to_dev(p.f, torch.float32) for p in probs]
    ms = [torch.as_tensor(p.mask, device="cuda") for p in probs]
    consts = [_oracle_constants(oracle.Geometry(p.n, p.n_angles, p.n_bins, theta=p.theta), np.pi / p.n, 15)
              for p in probs]
    betas, cs = [b for b, _ in consts], [c for _, c in consts]
    iters = 30
    us, diags = batch.solve(fs, ms, [p.alpha for p in probs], [p.delta for p in probs], iters,
                            params=ct.default_params(), betas=betas, cs=cs)
    for i, p in enumerate(probs):
        plan = ct.Plan(p.n, p.n_angles, p.n_bins, angles=p.theta)
        plan.set_bp_groups(batch.plans[i].bp_groups)
        u1, d1 = plan.tv_pd_solve(fs[i], ms[i], p.alpha, p.delta, iters,
                                  params=ct.default_params(beta=betas[i], c=cs[i]))
        e1 = rel_l2(to_np(us[i]), to_np(u1))
        geo = oracle.Geometry(p.n, p.n_angles, p.n_bins, theta=p.theta)
        ref = oracle.pdrq_solve(geo, oracle.make_descriptors(p.f, p.mask, p.delta), p.alpha, iters, sigma=1.0,
                                tau=1 / np.sqrt(8), eps=np.pi / p.n, beta=betas[i], c=cs[i])
        e0 = rel_l2(to_np(us[i]), ref.u)
        print(f"slice {p.n}^2/{p.n_angles}: batch vs single {e1:.2e}, vs oracle {e0:.2e}")
        assert e1 < 2e-6, (i, e1)
        assert e0 < 1e-5, (i, e0)
        assert diags[i]["objective"] == pytest.approx(d1["objective"], rel=1e-5)
