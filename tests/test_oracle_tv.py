"""Pins of the oracle's isotropic total variation ||grad_h u||_1 (Sec. 3.1, the one-norm
on V) and of the objective of (C_h) (Sec. 3.2) that diagnostics() reports, by cases
worked out by hand and by closed forms: a slip to the anisotropic norm |q1| + |q2|, a
missing 1/h, a wrong factor on alpha or on the data term, or a data term that counts
trace bins would each fail one of them."""
import numpy as np
import pytest

import oracle
from oracle import Geometry


def test_tv_hand_3x3_isotropic_not_anisotropic():
    """u = [[0,4,4],[3,4,4],[3,4,4]]: forward differences (Neumann) give (3, 4) at (0,0),
    (0, 1) at (1,0) and (2,0), zero elsewhere, so ||grad u||_1 = 5 + 1 + 1 = 7; the
    anisotropic sum would be 9.  With h = 0.5 every difference doubles: 14."""
    u = np.array([[0.0, 4.0, 4.0], [3.0, 4.0, 4.0], [3.0, 4.0, 4.0]])
    assert oracle.tv_norm(u) == pytest.approx(7.0, abs=1e-14)
    assert oracle.tv_norm(u, h=0.5) == pytest.approx(14.0, abs=1e-14)


@pytest.mark.parametrize("n,h,a,b", [(5, 1.0, 2.0, -1.0), (8, 0.5, 0.3, 0.4), (1, 1.0, 3.0, 3.0)])
def test_tv_of_a_ramp_closed_form(n, h, a, b):
    """u_ij = a i + b j: the (n-1)^2 interior pixels have |grad u| = sqrt(a^2 + b^2)/h, the
    last row (no x difference) |b|/h on its first n-1 pixels, the last column |a|/h on
    its first n-1, and the corner 0."""
    I, J = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    want = ((n - 1) ** 2 * np.hypot(a, b) + (n - 1) * (abs(a) + abs(b))) / h
    assert oracle.tv_norm(a * I + b * J, h) == pytest.approx(want, rel=1e-13)


def test_tv_constant_zero_and_one_homogeneous():
    rng = np.random.default_rng(0)
    u = rng.standard_normal((9, 9))
    assert oracle.tv_norm(np.full((9, 9), 2.5)) == 0.0
    assert oracle.tv_norm(-3.0 * u) == pytest.approx(3.0 * oracle.tv_norm(u), rel=1e-13)


def test_objective_hand_case():
    """n = 2, one angle theta = 0, M = 3 bins, h = ds = 1: pixel rows sit at x = -1/2 and
    +1/2, i.e. detector coordinates p = 1/2 and 3/2, so each pixel splits half and half
    between two bins and R u = (r0/2, (r0 + r1)/2, r1/2) with r_i the row sums.
    u = [[1, 3], [2, 6]]: r = (4, 8), R u = (2, 6, 4).  Gradient: (1, 2) at (0,0),
    (3, 0) at (0,1), (0, 4) at (1,0): TV = sqrt(5) + 7.
    Data f = (1, 6, 0), bin 2 on the metal trace, delta = 0.5: the data term counts bins
    0 and 1 only, 1/2 ((2-1)^2 + 0^2) = 1/2; bin 0 leaves its box [0.5, 1.5] by 0.5; the
    trace bin needs R u >= 0.8 * 0 and holds.  alpha = 0.1."""
    geo = Geometry(2, 1, 3, theta=np.array([0.0]))
    u = np.array([[1.0, 3.0], [2.0, 6.0]])
    np.testing.assert_allclose(oracle.rh_forward(u, geo), [[2.0, 6.0, 4.0]], atol=1e-14)
    f = np.array([[1.0, 6.0, 0.0]])
    mask = np.array([[0, 0, 1]], np.uint8)
    desc = oracle.make_descriptors(f, mask, 0.5)
    d = oracle.diagnostics(geo, desc, 0.1, u)
    tv = np.sqrt(5.0) + 7.0
    assert d["tv"] == pytest.approx(tv, abs=1e-13)
    assert d["data_fit"] == pytest.approx(0.5, abs=1e-13)
    assert d["objective"] == pytest.approx(0.5 + 0.1 * tv, abs=1e-13)
    assert d["violation"] == pytest.approx(0.5, abs=1e-13)


def test_gap_tv_part_vanishes_on_the_aligned_certificate():
    """The TV part of the Fenchel-Young gap, lambda |grad u|_1 - tau <grad u, t2>, is zero
    for t2 = (lambda/tau) grad u / |grad u| (the support point of the ball of radius
    lambda/tau) and equals lambda TV(u) for t2 = 0.  The data part is made zero by a
    consistent sinogram without boxes (w = 1, a = f = R_h u, so z = a and t1 = 0)."""
    n, N, M = 6, 5, 11
    geo = Geometry(n, N, M)
    rng = np.random.default_rng(3)
    u = rng.uniform(0, 1, (n, n))
    beta, tau, alpha = 2.0, 0.4, 0.3
    lam = alpha / beta ** 2
    f = oracle.rh_forward(u, geo)
    desc = oracle.make_descriptors(f, None, -1.0)
    gx, gy = oracle.grad(u)
    mag = np.sqrt(gx * gx + gy * gy)
    safe = np.where(mag > 0, mag, 1.0)
    t2x = np.where(mag > 0, (lam / tau) * gx / safe, 0.0)
    t2y = np.where(mag > 0, (lam / tau) * gy / safe, 0.0)
    t1 = np.zeros((N, M))
    d = oracle.diagnostics(geo, desc, alpha, u, beta=beta, tau=tau, t1=t1, t2x=t2x, t2y=t2y)
    assert abs(d["gap"]) < 1e-12
    d0 = oracle.diagnostics(geo, desc, alpha, u, beta=beta, tau=tau, t1=t1, t2x=0 * t2x, t2y=0 * t2y)
    assert d0["gap"] == pytest.approx(lam * oracle.tv_norm(u), rel=1e-12)
