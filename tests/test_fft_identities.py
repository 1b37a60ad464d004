"""The identities the preconditioner's FFT kernels are built on, checked in numpy (host
logic, no GPU): the four-step split of the length-n^2 DFT of the column-major flattened
image used by the circulant kind's twisted column pass, and the real-input form that
transforms two real rows with one complex FFT and keeps n/2 + 1 columns."""
import numpy as np
import pytest


@pytest.mark.parametrize("n", [4, 6, 9, 12])
def test_four_step_split_of_the_flattened_dft(n):
    """Row FFTs over j, times e^{-2 pi i i kB / n^2}, column FFTs over i: position
    (kA, kB) then holds F_1(x)_k at k = kB + n kA, i.e. at flat position kA n + kB; the
    inverse runs the same steps backwards with the conjugate twiddle."""
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n, n))
    N = n * n
    y = np.fft.fft(x, axis=1)                                   # rows: over j -> kB
    i = np.arange(n)[:, None]
    kB = np.arange(n)[None, :]
    y = y * np.exp(-2j * np.pi * i * kB / N)                   # twiddle
    z = np.fft.fft(y, axis=0)                                   # columns: over i -> kA
    ref = np.fft.fft(x.reshape(-1, order="F"))                  # t = i + n j
    np.testing.assert_allclose(z.reshape(-1), ref, atol=1e-9 * np.abs(ref).max())
    # inverse: columns, conjugate twiddle, rows (and 1/N)
    w = np.fft.ifft(z, axis=0) * np.exp(2j * np.pi * i * kB / N)
    back = np.fft.ifft(w, axis=1)
    np.testing.assert_allclose(back.real, x, atol=1e-12)


@pytest.mark.parametrize("n", [1, 2, 5, 8, 9])
def test_real_input_form(n):
    """Rows a, b of a real image through one complex FFT of z = a + i b:
    X_a(k) = (Z(k) + conj Z(n-k)) / 2, X_b(k) = (Z(k) - conj Z(n-k)) / (2i), kept for
    k <= n/2; the inverse rebuilds X(k) = conj X(n-k) beyond n/2 and returns a and b as
    the real and imaginary parts of one inverse FFT."""
    rng = np.random.default_rng(10 + n)
    a, b = rng.standard_normal(n), rng.standard_normal(n)
    Z = np.fft.fft(a + 1j * b)
    k = np.arange(n // 2 + 1)
    Zm = Z[(-k) % n]
    Xa = 0.5 * (Z[k] + np.conj(Zm))
    Xb = (Z[k] - np.conj(Zm)) / 2j
    np.testing.assert_allclose(Xa, np.fft.fft(a)[k], atol=1e-12)
    np.testing.assert_allclose(Xb, np.fft.fft(b)[k], atol=1e-12)
    full = lambda X: np.array([X[m] if m <= n // 2 else np.conj(X[n - m]) for m in range(n)])
    zz = np.fft.ifft(full(Xa) + 1j * full(Xb))
    np.testing.assert_allclose(zz.real, a, atol=1e-12)
    np.testing.assert_allclose(zz.imag, b, atol=1e-12)


def test_real_even_symbol_keeps_the_form():
    """A real symbol with m(-k) = m(k) (every kind but the circulant one) maps the kept
    half to the kept half, so multiplying only n/2 + 1 columns gives the full product."""
    n = 8
    rng = np.random.default_rng(3)
    x = rng.standard_normal((n, n))
    ks = np.fft.fftfreq(n)
    m = 1.0 / (1.0 + ks[:, None] ** 2 + 3.0 * ks[None, :] ** 2)      # real, even in (kA, kB)
    ref = np.real(np.fft.ifft2(np.fft.fft2(x) * m))
    half = np.fft.rfft2(x) * m[:, : n // 2 + 1]
    np.testing.assert_allclose(np.fft.irfft2(half, s=(n, n)), ref, atol=1e-12)
