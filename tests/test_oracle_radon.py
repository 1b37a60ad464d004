"""Pins of the oracle's R_h / R_h^* (Sec. 3.1) against facts that do not come from
the oracle itself: closed forms, textbook special cases, exact invariants."""
import numpy as np
import pytest

import oracle
from oracle import Geometry

GEOMS = [
    dict(n=8, n_angles=12, n_bins=13),
    dict(n=8, n_angles=7, n_bins=12),
    dict(n=9, n_angles=10, n_bins=15, h=0.7, ds=1.3),
    dict(n=16, n_angles=24, n_bins=25),
    dict(n=5, n_angles=3, n_bins=4, h=1.5, ds=0.8),
]


def _geo(d, random_angles=False, seed=0):
    g = Geometry(**d)
    if random_angles:
        g = Geometry(**d, theta=np.random.default_rng(seed).uniform(0, np.pi, d["n_angles"]))
    return g


@pytest.mark.parametrize("d", GEOMS)
@pytest.mark.parametrize("random_angles", [False, True])
def test_adjoint_identity(d, random_angles):
    """<R u, g> = <u, R^* g>: the splat (forward) and gather (adjoint) loops are
    written independently, so agreement pins that they are transposes."""
    geo = _geo(d, random_angles)
    rng = np.random.default_rng(1)
    u = rng.standard_normal(geo.image_shape)
    g = rng.standard_normal(geo.sino_shape)
    lhs = np.sum(oracle.rh_forward(u, geo) * g)
    rhs = np.sum(u * oracle.rh_adjoint(g, geo))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.linalg.norm(u) * np.linalg.norm(g))


@pytest.mark.parametrize("d", GEOMS[:4])
def test_hat_brute_force_matches_floor_frac(d):
    """Every entry by brute force with Lambda(p - k) = max(0, 1 - |p - k|) equals
    the floor/frac loops (a third formulation of the same weights)."""
    geo = _geo(d, True, 3)
    rng = np.random.default_rng(2)
    u = rng.standard_normal(geo.image_shape)
    g = rng.standard_normal(geo.sino_shape)
    L, K = np.meshgrid(np.arange(geo.n_angles), np.arange(geo.n_bins), indexing="ij")
    fw = oracle.rh_forward_entries(u, geo, L.ravel(), K.ravel()).reshape(geo.sino_shape)
    np.testing.assert_allclose(fw, oracle.rh_forward(u, geo), rtol=0, atol=1e-12)
    I, J = np.meshgrid(np.arange(geo.n), np.arange(geo.n), indexing="ij")
    bw = oracle.rh_adjoint_entries(g, geo, I.ravel(), J.ravel()).reshape(geo.image_shape)
    np.testing.assert_allclose(bw, oracle.rh_adjoint(g, geo), rtol=0, atol=1e-12)


def test_point_projection_hand_values():
    """Pixel (i=7, j=2) of an 8x8 image sits at x = 3.5, y = -1.5 (grid centred at
    3.5).  With M = 13 bins (centre bin 6): at theta = 0, s = 3.5 -> p = 9.5, split
    0.5/0.5 into bins 9, 10; at theta = pi/2, s = y = -1.5 -> p = 4.5, bins 4, 5;
    at theta = pi/4, s = 2/sqrt(2) = 1.41421 -> p = 7.41421: bin 7 gets 0.58579,
    bin 8 gets 0.41421 (linear interpolation, reading P2: the nearer bin gets the
    larger weight)."""
    geo = Geometry(8, 3, 13, theta=np.array([0.0, np.pi / 2, np.pi / 4]))
    u = np.zeros((8, 8))
    u[7, 2] = 1.0
    g = oracle.rh_forward(u, geo)
    exp = np.zeros((3, 13))
    exp[0, 9] = exp[0, 10] = 0.5
    exp[1, 4] = exp[1, 5] = 0.5
    exp[2, 7] = 1 - (np.sqrt(2) - 1)
    exp[2, 8] = np.sqrt(2) - 1
    np.testing.assert_allclose(g, exp, atol=1e-12)


@pytest.mark.parametrize("d", GEOMS)
def test_point_centroid_and_mass(d):
    """For a single pixel whose footprint is inside the detector, each projection
    has unit mass and its centroid is the pixel's detector coordinate
    x cos + y sin (in bin units, centred) -- the first moment of linear
    interpolation.  Pins the interpolation direction and the centring."""
    geo = _geo(d, True, 5)
    n, M = geo.n, geo.n_bins
    rng = np.random.default_rng(4)
    for _ in range(6):
        i, j = rng.integers(0, n, 2)
        u = np.zeros((n, n))
        u[i, j] = 1.0
        g = oracle.rh_forward(u, geo)
        x = geo.h * (i - (n - 1) / 2)
        y = geo.h * (j - (n - 1) / 2)
        s = x * np.cos(geo.theta) + y * np.sin(geo.theta)
        pos = s / geo.ds + (M - 1) / 2
        inside = (pos >= 0) & (pos <= M - 1)
        k = np.arange(M)
        np.testing.assert_allclose(g.sum(1)[inside], 1.0, atol=1e-12)
        np.testing.assert_allclose((g * k).sum(1)[inside], pos[inside], atol=1e-12)


def test_theta0_column_sums_textbook():
    """theta = 0 with n even, M odd: every column-sum S_i = sum_j u[i, j] lies
    half-way between two bin centres, so bin k = (S_{k-c-1} + S_{k-c})/2 with
    c = (M - n - 1)/2; at theta = pi/2 the same with row sums (j <-> y)."""
    n, M = 10, 15
    geo = Geometry(n, 2, M, theta=np.array([0.0, np.pi / 2]))
    u = np.random.default_rng(7).uniform(size=(n, n))
    g = oracle.rh_forward(u, geo)
    c = (M - n - 1) // 2
    for row, S in ((0, u.sum(1)), (1, u.sum(0))):
        Sp = np.concatenate([np.zeros(M), S, np.zeros(M)])
        exp = np.array([0.5 * (Sp[M + k - c - 1] + Sp[M + k - c]) for k in range(M)])
        np.testing.assert_allclose(g[row], exp, atol=1e-12)


def test_rotation_by_quarter_turn():
    """Rotating the image by 90 degrees (u'[i, j] = u[n-1-j, i]) shifts the
    sinogram by pi/2; past pi the detector flips (k -> M-1-k)."""
    n, N, M = 12, 16, 19
    geo = Geometry(n, N, M)
    u = np.random.default_rng(8).uniform(size=(n, n))
    ur = np.empty_like(u)
    for i in range(n):
        for j in range(n):
            ur[i, j] = u[n - 1 - j, i]
    g = oracle.rh_forward(u, geo)
    gr = oracle.rh_forward(ur, geo)
    q = N // 2
    np.testing.assert_allclose(gr[:N - q], g[q:], atol=1e-11)
    np.testing.assert_allclose(gr[N - q:], g[:q, ::-1], atol=1e-11)


def test_disk_chord_length():
    """R of the indicator of a disk is the chord 2 sqrt(r^2 - s^2) (Sec. 2.2).  A
    pixelised disk of radius 20 px must match it to within the pixelisation error
    in the interior, and its total mass per angle is its pixel count."""
    n, M, r = 64, 95, 20.0
    xs = np.arange(n) - (n - 1) / 2
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    u = ((X ** 2 + Y ** 2) <= r * r).astype(float)
    geo = Geometry(n, 30, M)
    g = oracle.rh_forward(u, geo)
    s = np.arange(M) - (M - 1) / 2
    chord = 2 * np.sqrt(np.maximum(r * r - s * s, 0.0))
    inner = np.abs(s) < r - 3
    err = np.abs(g[:, inner] - chord[inner]) / chord[inner]
    assert err.max() < 0.06, err.max()
    assert np.abs(g.mean(0)[inner] - chord[inner]).max() < 0.5
    np.testing.assert_allclose(g.sum(1), u.sum(), rtol=1e-12)


def test_rh_norm_bound():
    """||R_h|| <= sqrt(2 N (sqrt(2) n + 1)) (Lemma lem_Rh_bound)."""
    for d in GEOMS[:4]:
        geo = _geo(d)
        n = geo.n
        A = np.stack([oracle.rh_forward(e.reshape(n, n), geo).ravel() for e in np.eye(n * n)], 1)
        assert np.linalg.norm(A, 2) <= np.sqrt(2 * geo.n_angles * (np.sqrt(2) * n + 1))
