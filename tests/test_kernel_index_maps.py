"""Host checks of the index arithmetic the CUDA kernels rely on (no GPU, no library call):

* the warp-level preconditioner passes compute a length n = 32 V DFT (V = 8, 16, 32) as a
  four-step factorisation n = V x 32 over a warp's 32 lanes x V registers: a V-point DFT per
  lane, twiddles W_n^{l k1}, a transpose through a buffer padded to 32 + G complex per row
  (G = 32 / V lanes per k1), a second V-point DFT, twiddles W_32^{la k2'} and a G-point DFT
  across each lane group, leaving lane lam, register i with X[k1 + V brev(i) + V^2 brev(la)];
  the inverse runs the adjoint steps in reverse order.  Restated here in numpy in the kernels'
  lane/register layout and compared with numpy's FFT; the transpose buffer's padding is checked
  conflict-free (distinct 8-byte banks in every half warp);
* the staging loops divide element indices by a row width as the high word of x m with
  m = floor((2^32 - 1) / d) + 1, exact whenever x d < 2^32."""
import numpy as np
import pytest


def _brev(i, bits):
    r = 0
    for b in range(bits):
        r = (r << 1) | ((i >> b) & 1)
    return r


def _w32(t, s):
    return np.exp(s * 2j * np.pi * t / 32)


def _dif(v, s):                      # natural order in, bit-reversed order out
    v = v.copy()
    V = len(v)
    for st in range(V.bit_length() - 1):
        span = V >> (st + 1)
        for b in range(0, V, 2 * span):
            for j in range(span):
                a, c = v[b + j], v[b + j + span]
                v[b + j] = a + c
                v[b + j + span] = (a - c) * _w32(j * (16 // span), s)
    return v


def _dit(v, s):                      # bit-reversed order in, natural order out
    v = v.copy()
    V = len(v)
    for st in range(V.bit_length() - 2, -1, -1):
        span = V >> (st + 1)
        for b in range(0, V, 2 * span):
            for j in range(span):
                a, c = v[b + j], v[b + j + span] * _w32(j * (16 // span), s)
                v[b + j] = a + c
                v[b + j + span] = a - c
    return v


def _xlane_dif(regs, G, s):
    d = G // 2
    while d >= 1:
        out = []
        for lam in range(32):
            la, p, v = lam % G, regs[lam ^ d], regs[lam]
            o = (p - v) if la & d else (v + p)
            if (la & d) and (la & (d - 1)):
                o = o * np.exp(s * 2j * np.pi * (la & (d - 1)) / (2 * d))
            out.append(o)
        regs, d = out, d // 2
    return regs


def _xlane_dit(regs, G, s):
    d = 1
    while d < G:
        tw = []
        for lam in range(32):
            la, v = lam % G, regs[lam]
            if (la & d) and (la & (d - 1)):
                v = v * np.exp(s * 2j * np.pi * (la & (d - 1)) / (2 * d))
            tw.append(v)
        regs = [(tw[lam ^ d] - tw[lam]) if (lam % G) & d else (tw[lam] + tw[lam ^ d]) for lam in range(32)]
        d *= 2
    return regs


def _kmap(V, lam, i):
    G = 32 // V
    return lam // G + V * _brev(i, V.bit_length() - 1) + V * V * _brev(lam % G, G.bit_length() - 1)


def _wfft_fwd(x, s):
    n = len(x)
    V, G = n // 32, 32 // (n // 32)
    bits, P = V.bit_length() - 1, 32 + G
    wn = lambda t: np.exp(s * 2j * np.pi * t / n)
    buf = np.zeros(V * P, complex)
    for l in range(32):
        v = _dif(np.array([x[l + 32 * m] for m in range(V)]), s)
        for i in range(V):
            k1 = _brev(i, bits)
            buf[k1 * P + l] = v[i] * wn(l * k1)
    regs = []
    for lam in range(32):
        k1, la = lam // G, lam % G
        w = _dif(np.array([buf[k1 * P + la + G * lb] for lb in range(V)]), s)
        regs.append(np.array([w[i] * wn(la * _brev(i, bits) * V) for i in range(V)]))
    return _xlane_dif(regs, G, s)


def _wfft_adj(regs, n, s):
    V, G = n // 32, 32 // (n // 32)
    bits, P = V.bit_length() - 1, 32 + G
    wn = lambda t: np.exp(s * 2j * np.pi * t / n)
    regs = _xlane_dit(regs, G, s)
    buf = np.zeros(V * P, complex)
    for lam in range(32):
        k1, la = lam // G, lam % G
        w = _dit(np.array([regs[lam][i] * wn(la * _brev(i, bits) * V) for i in range(V)]), s)
        for lb in range(V):
            buf[k1 * P + la + G * lb] = w[lb]
    y = np.zeros(n, complex)
    for l in range(32):
        v = _dit(np.array([buf[_brev(i, bits) * P + l] * wn(l * _brev(i, bits)) for i in range(V)]), s)
        for m in range(V):
            y[l + 32 * m] = v[m]
    return y


@pytest.mark.parametrize("n", [256, 512, 1024])
def test_warp_four_step_dft_layout(n):
    V = n // 32
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    regs = _wfft_fwd(x, -1)
    got = np.zeros(n, complex)
    for lam in range(32):
        for i in range(V):
            got[_kmap(V, lam, i)] = regs[lam][i]
    np.testing.assert_allclose(got, np.fft.fft(x), rtol=0, atol=1e-9 * np.sqrt(n))
    # the inverse straight from the scrambled layout (the column pass multiplies the symbol there)
    Y = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    y = _wfft_adj([np.array([Y[_kmap(V, lam, i)] for i in range(V)]) for lam in range(32)], n, +1)
    np.testing.assert_allclose(y, n * np.fft.ifft(Y), rtol=0, atol=1e-9 * n)
    # every frequency is held by exactly one (lane, register)
    assert sorted(_kmap(V, lam, i) for lam in range(32) for i in range(V)) == list(range(n))


@pytest.mark.parametrize("V", [8, 16, 32])
def test_warp_transpose_buffer_conflict_free(V):
    G = 32 // V
    P = 32 + G
    for lb in range(V):                      # the group read of the transpose, per half warp
        for h in (0, 16):
            banks = [((lam // G) * P + lam % G + G * lb) % 16 for lam in range(h, h + 16)]
            assert len(set(banks)) == 16
    for k1 in range(V):                      # the lane-major write
        for h in (0, 16):
            assert len({(k1 * P + l) % 16 for l in range(h, h + 16)}) == 16


def test_multiply_high_division_exact():
    rng = np.random.default_rng(0)
    for d in list(range(1, 300)) + [1024, 2049, 4097]:
        m = 0 if d <= 1 else (0xFFFFFFFF // d) + 1
        xmax = (2 ** 32 - 1) // d
        xs = np.unique(np.concatenate([np.arange(0, min(xmax, 5000) + 1),
                                       rng.integers(0, xmax + 1, 2000), [xmax]]))
        q = xs if d <= 1 else (xs.astype(object) * m) >> 32
        assert all(int(a) == int(b) // d for a, b in zip(q, xs)), d
