"""Pin of the oracle's reverse mode (pdrq_grad) by FP64 central finite differences
of its own forward iteration: the derivative along random directions of the data and
of alpha must match (f(x + h d) - f(x - h d)) / (2h) with h = 1e-6."""
import numpy as np
import pytest

import oracle
from oracle import Geometry
from paper_1810_03275_gb300 import phantom


def _loss(geo, f, mask, delta, alpha, iters, truth, kw):
    desc = oracle.make_descriptors(f, mask, delta)
    u = oracle.pdrq_solve(geo, desc, alpha, iters, **kw).u
    return float(np.sum((u - truth) ** 2))


@pytest.mark.parametrize("metal,delta_scale", [(False, -1.0), (True, 3.0), (True, 0.5)])
def test_reverse_mode_matches_finite_differences(metal, delta_scale):
    n, N, M, K = 16, 20, 25, 10
    pr = phantom.make_problem("g", n, N, M, seed=3, n_ellipses=3, n_metal=1 if metal else 0,
                              noise="gaussian", alpha=0.2)
    geo = Geometry(n, N, M, theta=pr.theta)
    delta = delta_scale * pr.delta if delta_scale > 0 else -1.0
    mask = pr.mask if metal else None
    beta = oracle.power_beta(geo, 30)
    kw = dict(sigma=1.0, tau=1 / np.sqrt(8), eps=np.pi / n, beta=beta, c=oracle.power_c(geo, beta, np.pi / n, 30))
    desc = oracle.make_descriptors(pr.f, mask, delta)
    uK = oracle.pdrq_solve(geo, desc, pr.alpha, K, **kw).u
    df, dalpha = oracle.pdrq_grad(geo, pr.f, mask, delta, pr.alpha, K, 2.0 * (uK - pr.truth), **kw)
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(3):
        d = rng.standard_normal(pr.f.shape)
        fd = (_loss(geo, pr.f + h * d, mask, delta, pr.alpha, K, pr.truth, kw)
              - _loss(geo, pr.f - h * d, mask, delta, pr.alpha, K, pr.truth, kw)) / (2 * h)
        assert np.sum(df * d) == pytest.approx(fd, rel=1e-5, abs=1e-8)
    fd = (_loss(geo, pr.f, mask, delta, pr.alpha + h, K, pr.truth, kw)
          - _loss(geo, pr.f, mask, delta, pr.alpha - h, K, pr.truth, kw)) / (2 * h)
    assert dalpha == pytest.approx(fd, rel=1e-5, abs=1e-8)
