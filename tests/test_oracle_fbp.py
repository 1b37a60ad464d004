"""Pins of the oracle's detector-axis ramp filter and filtered backprojection (Sec. 2):
the Ram-Lak kernel's frequency response against |nu| / ds, the linear convolution
against a zero-padded FFT convolution, and the FBP of exact disk line integrals
(chord lengths 2 sqrt(r^2 - s^2)) reconstructing the disk."""
import numpy as np
import pytest

import oracle
from paper_1810_03275_gb300 import phantom


@pytest.mark.parametrize("ds", [1.0, 0.7])
def test_ramlak_frequency_response_is_the_ramp(ds):
    """sum_m ds k(m) e^{-2 pi i nu m} -> |nu| / ds on |nu| <= 1/2 as the kernel grows
    (the band-limited ramp in cycles per sample over the bin width)."""
    M = 200001
    k = oracle.ramlak_kernel(M, ds)
    m = np.arange(-(M - 1), M)
    for nu in (0.0, 0.05, 0.13, 0.31, 0.5):
        H = float(np.sum(ds * k * np.cos(2 * np.pi * nu * m)))
        assert H == pytest.approx(abs(nu) / ds, abs=2e-5 / ds)


@pytest.mark.parametrize("M", [1, 2, 17, 95])
def test_linear_convolution_equals_padded_fft(M):
    rng = np.random.default_rng(M)
    g = rng.standard_normal((5, M))
    L = 2 * M + 3
    ker = oracle.ramlak_kernel(M, 0.8)
    wrapped = np.zeros(L)
    for j, v in enumerate(ker):
        wrapped[(j - (M - 1)) % L] += v
    ref = np.real(np.fft.ifft(np.fft.fft(np.pad(g, ((0, 0), (0, L - M))), axis=1) * np.fft.fft(wrapped), axis=1))
    np.testing.assert_allclose(oracle.ramp_filter(g, 0.8), 0.8 * ref[:, :M], atol=1e-12)


def test_fbp_of_a_disk():
    n, N, M, r = 96, 360, 137, 30.0
    theta = np.arange(N) * np.pi / N
    s = phantom.bin_centres(M)
    chord = 2.0 * np.sqrt(np.maximum(r * r - s * s, 0.0))
    g = np.tile(chord, (N, 1))
    u = oracle.fbp(g, oracle.Geometry(n, N, M, theta=theta))
    x = phantom.pixel_centres(n)
    R = np.hypot(*np.meshgrid(x, x, indexing="ij"))
    assert abs(u[R < r - 3].mean() - 1.0) < 0.01
    assert np.abs(u[R < r - 3] - 1.0).max() < 0.06
    assert abs(u[(R > r + 3) & (R < 0.7 * n)].mean()) < 0.01
