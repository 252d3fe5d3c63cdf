"""Pins of the oracle's own FFT (radix-2 + Bluestein) against numpy.fft (a
library special case) and against the oracle's plain O(n^2) DFT, which is in
turn pinned to numpy.fft.  Both signs, power-of-two, odd and prime lengths."""
import numpy as np
import pytest


def rand_complex(n, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(n) + 1j * r.standard_normal(n)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 64, 1024, 3, 5, 7, 12, 17, 100, 243, 1000, 4886])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_matches_numpy(orc, n, sign):
    x = rand_complex(n, n)
    ref = np.fft.fft(x) if sign == -1 else np.fft.ifft(x) * n
    got = orc.fft(x, sign)
    assert np.linalg.norm(got - ref) <= 1e-13 * max(1.0, np.linalg.norm(ref))


@pytest.mark.parametrize("n", [1, 6, 31, 64])
@pytest.mark.parametrize("sign", [-1, 1])
def test_naive_dft_matches_numpy(orc, n, sign):
    x = rand_complex(n, 7 * n)
    ref = np.fft.fft(x) if sign == -1 else np.fft.ifft(x) * n
    assert np.linalg.norm(orc.dft(x, sign) - ref) <= 1e-13 * max(1.0, np.linalg.norm(ref))


def test_fft_of_unit_impulse_and_tone(orc):
    n = 48
    e = np.zeros(n, complex)
    e[5] = 1.0
    k = np.arange(n)
    assert np.allclose(orc.fft(e, +1), np.exp(2j * np.pi * 5 * k / n), atol=1e-14)
    tone = np.exp(-2j * np.pi * 3 * k / n)
    out = orc.fft(tone, +1)
    expect = np.zeros(n, complex)
    expect[3] = n
    assert np.allclose(out, expect, atol=1e-12)
