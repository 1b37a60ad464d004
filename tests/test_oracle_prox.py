"""Pins of the oracle's unified dual resolvent and TV projection: every resolvent
printed in Sec. 3.3-3.5 and 4.4 is a special case, plus Moreau's identity and brute
force minimisation."""
import numpy as np
import pytest

import oracle

inf = np.inf
V = np.linspace(-5, 5, 41)


@pytest.mark.parametrize("sigma", [0.3, 1.0, 2.5])
def test_thesis_resolvents_are_special_cases(sigma):
    f, C, om = 1.7, 0.9, 3.0
    # Lemma lem_f_ast_resolv1 (data fit): (v - sigma f)/(1 + sigma)
    np.testing.assert_allclose(oracle.prox_dual(V, sigma, 1.0, f, -inf, inf), (V - sigma * f) / (1 + sigma), atol=1e-12)
    # Lemma lem_f_ast_resolv1 (metal trace): min(v - sigma C, 0)
    np.testing.assert_allclose(oracle.prox_dual(V, sigma, 0.0, 0.0, C, inf), np.minimum(V - sigma * C, 0.0), atol=1e-12)
    # Lemma lem_f_ast_resolv_ignore: 0
    np.testing.assert_allclose(oracle.prox_dual(V, sigma, 0.0, 0.0, -inf, inf), 0.0, atol=1e-15)
    # Sec. 3.5 hard constraints: v - sigma f
    np.testing.assert_allclose(oracle.prox_dual(V, sigma, 0.0, 0.0, f, f), V - sigma * f, atol=1e-12)
    # Lemma lem_f_ast1_w (weighted): (v - sigma f)/(1 + sigma/omega)
    np.testing.assert_allclose(oracle.prox_dual(V, sigma, om, f, -inf, inf), (V - sigma * f) / (1 + sigma / om), atol=1e-12)
    # Lemma lem_f_ast_resolv_other (fit everywhere with z >= C)
    exp = np.where(V >= C * (1 + sigma) - f, (V - sigma * f) / (1 + sigma), V - sigma * C)
    np.testing.assert_allclose(oracle.prox_dual(V, sigma, 1.0, f, C, inf), exp, atol=1e-12)


def _g(z, w, a, lo, hi):
    return np.where((z >= lo) & (z <= hi), 0.5 * w * (z - a) ** 2, inf)


CASES = [(1.0, 0.5, -0.3, 1.2), (0.0, 0.0, 0.4, inf), (2.0, -1.0, -inf, inf),
         (1.0, 2.0, 1.5, 2.5), (0.0, 0.0, -1.0, -1.0), (0.5, 0.0, 0.2, inf)]


@pytest.mark.parametrize("w,a,lo,hi", CASES)
def test_conjugate_brute_force(w, a, lo, hi):
    """g^*(t) = sup_z t z - g(z) by a dense grid over z, where finite."""
    zs = np.linspace(-30, 30, 600001)
    gz = _g(zs, w, a, lo, hi)
    for t in np.linspace(-3, 3, 13):
        bf = np.max(t * zs - gz)
        got = oracle.conj_data_term(np.array([t]), w, a, lo, hi)[0]
        if np.isfinite(got):
            assert got == pytest.approx(bf, abs=1e-3)
        else:
            assert bf > 0.8 * 30 * abs(t)  # unbounded: grows with the grid extent


@pytest.mark.parametrize("w,a,lo,hi", CASES)
@pytest.mark.parametrize("sigma", [0.5, 1.0, 3.0])
def test_moreau_and_brute_force_prox(w, a, lo, hi, sigma):
    """(i) Moreau: prox_{sigma g*}(v) + sigma prox_{g/sigma}(v/sigma) = v with the
    primal prox found by grid search; (ii) prox_{sigma g*}(v) minimises
    1/2 (t - v)^2 + sigma g*(t) over a grid of t."""
    zs = np.linspace(-12, 12, 240001)
    ts = np.linspace(-12, 12, 24001)
    gts = oracle.conj_data_term(ts, w, a, lo, hi)
    for v in np.linspace(-4, 4, 9):
        got = oracle.prox_dual(np.array([v]), sigma, w, a, lo, hi)[0]
        zp = zs[np.argmin(_g(zs, w, a, lo, hi) / sigma + 0.5 * (zs - v / sigma) ** 2)]
        assert got + sigma * zp == pytest.approx(v, abs=2e-4 * (1 + sigma))
        tp = ts[np.argmin(0.5 * (ts - v) ** 2 + sigma * gts)]
        assert got == pytest.approx(tp, abs=2e-3)


def test_tv_projection():
    """P onto {|z| <= lam/tau} pointwise: identity inside, radial scaling outside,
    and it is the closest point (checked against random feasible points)."""
    rng = np.random.default_rng(0)
    zx, zy = rng.standard_normal((2, 50)) * 3
    lam, tau = 0.7, 0.5
    px, py = oracle.tv_project(zx, zy, lam, tau)
    r = np.hypot(px, py)
    assert np.all(r <= lam / tau + 1e-12)
    inside = np.hypot(zx, zy) <= lam / tau
    np.testing.assert_allclose(px[inside], zx[inside])
    np.testing.assert_allclose(px * zy - py * zx, 0, atol=1e-12)   # same direction
    d = np.hypot(px - zx, py - zy)
    for _ in range(200):
        ang = rng.uniform(0, 2 * np.pi, 50)
        rad = lam / tau * np.sqrt(rng.uniform(size=50))
        qx, qy = rad * np.cos(ang), rad * np.sin(ang)
        assert np.all(d <= np.hypot(qx - zx, qy - zy) + 1e-12)
    ox, oy = oracle.tv_project(zx, zy, 0.0, tau)
    assert np.all(ox == 0) and np.all(oy == 0)


def test_descriptors():
    f = np.array([[1.0, 2.0], [3.0, 4.0]])
    mask = np.array([[0, 1], [0, 0]], np.uint8)
    w, a, lo, hi = oracle.make_descriptors(f, mask, 0.5)
    np.testing.assert_array_equal(w, [[1, 0], [1, 1]])
    np.testing.assert_allclose(lo, [[0.5, 1.6], [2.5, 3.5]])
    assert hi[0, 1] == inf and hi[1, 1] == 4.5
    w, a, lo, hi = oracle.make_descriptors(f, mask, -1.0)
    assert lo[0, 0] == -inf and hi[0, 0] == inf and lo[0, 1] == pytest.approx(1.6)
