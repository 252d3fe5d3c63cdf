"""Seeded synthetic inputs shared by the tests, the oracle checks and bench.py.

This module only draws inputs: signals with the shapes and statistics of the
paper's workloads and log-spaced scale lists.  It holds none of the wavelet
transform's arithmetic, so both the CUDA path and the CPU oracle can consume
its arrays without sharing any code of the method.

Workloads (seed = 20230209 + workload index unless given):

* ``multitone``: three sines plus Gaussian noise, the shape of the paper's
  periodic test signal f1 (Sec. 4, Eq. for f1) at sample counts 1e3..1e7.
* ``lognormal_field``: a 1D lognormal density contrast
  delta = exp(g - sigma^2/2) - 1 with g a Gaussian random field of power
  spectrum P(k) ~ k^-1.5 exp(-k/k_c), k_c = 0.5 k_Nyquist, rescaled to unit
  sample standard deviation.  It stands in for the paper's 1D Zel'dovich
  density fields (Sec. 5), whose realisation is not published.
* ``gaussian_f2``: the paper's non-periodic test signal f2 = exp(-x^2/2)
  sampled on [-6, 6) (Sec. 4).
* ``paper_f1``: the paper's periodic test signal
  f1 = 2 cos x + cos(8x)/2 + sin(32x)/4 sampled on [0, 2 pi) (Sec. 4).
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20230209


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def log_scales(s_min: float, s_max: float, n: int) -> np.ndarray:
    """n dilations (in samples) evenly spaced in log between s_min and s_max."""
    if n == 1:
        return np.array([float(s_min)])
    i = np.arange(n, dtype=np.float64)
    return s_min * (s_max / s_min) ** (i / (n - 1))


def multitone(n: int, periods=(16.0, 128.0, 700.0), amps=(1.0, 0.5, 0.3),
              sigma: float = 0.1, seed: int = BASE_SEED) -> np.ndarray:
    """sum_j a_j sin(2 pi t / T_j) + N(0, sigma^2), t = 0..n-1, float64."""
    t = np.arange(n, dtype=np.float64)
    f = np.zeros(n, dtype=np.float64)
    for a, p in zip(amps, periods):
        f += a * np.sin(2.0 * np.pi * t / p)
    f += sigma * rng(seed).standard_normal(n)
    return f


def lognormal_field(n: int, slope: float = -1.5, cutoff_frac: float = 0.5,
                    sigma_g: float = 1.0, seed: int = BASE_SEED + 1) -> np.ndarray:
    """Lognormal density contrast of length n (float64).

    g has Hermitian Gaussian Fourier modes with variance P(k) = k^slope *
    exp(-k / k_c), k in units of the fundamental, k_c = cutoff_frac * n/2,
    P(0) = 0; g is rescaled to sample std sigma_g; delta = exp(g - sigma_g^2/2) - 1.
    """
    r = rng(seed)
    nk = n // 2 + 1
    k = np.arange(nk, dtype=np.float64)
    kc = cutoff_frac * (n / 2.0)
    pk = np.zeros(nk)
    pk[1:] = k[1:] ** slope * np.exp(-k[1:] / kc)
    modes = (r.standard_normal(nk) + 1j * r.standard_normal(nk)) * np.sqrt(pk / 2.0)
    if n % 2 == 0:
        modes[-1] = modes[-1].real * np.sqrt(2.0)
    g = np.fft.irfft(modes, n=n)
    g = g - g.mean()
    g *= sigma_g / g.std()
    return np.exp(g - 0.5 * sigma_g ** 2) - 1.0


def paper_f1(n: int = 512):
    """Paper's periodic test signal f1 on [0, 2 pi): returns (x, f, dx)."""
    dx = 2.0 * np.pi / n
    x = np.arange(n) * dx
    f = 2.0 * np.cos(x) + 0.5 * np.cos(8.0 * x) + 0.25 * np.sin(32.0 * x)
    return x, f, dx


def gaussian_f2(n: int = 512):
    """Paper's non-periodic test signal f2 = exp(-x^2/2) on [-6, 6): (x, f, dx)."""
    dx = 12.0 / n
    x = -6.0 + np.arange(n) * dx
    return x, np.exp(-0.5 * x * x), dx


def sample_points(n_scales: int, n: int, count: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """count random (scale index, position) pairs, always including the corners."""
    r = rng(seed)
    s = r.integers(0, n_scales, size=count).astype(np.int32)
    p = r.integers(0, n, size=count).astype(np.int64)
    s[:4] = [0, 0, n_scales - 1, n_scales - 1]
    p[:4] = [0, n - 1, 0, n - 1]
    return s, p


# Named workloads with the sizes of the paper-shaped configurations.
WORKLOADS = {
    # one float64 multitone signal, periodic, Mexican-hat-type GDW, 32 scales
    "multitone_n4096_gdw_s32": dict(n=4096, n_scales=32, s_min=2.0, s_max=1024.0,
                                    wavelet="gdw", boundaries=("periodic",)),
    # float32 lognormal field, Morlet omega0=6, 64 scales, both boundaries
    "lognormal_n1m_morlet_s64": dict(n=1 << 20, n_scales=64, s_min=4.0, s_max=float(1 << 18),
                                     wavelet="morlet", boundaries=("periodic", "zero")),
    # float32 lognormal field, 128 scales, both wavelets and boundaries
    "lognormal_n4m_gdw_s128": dict(n=1 << 22, n_scales=128, s_min=2.0, s_max=float(1 << 20),
                                   wavelet="gdw", boundaries=("periodic", "zero")),
    "lognormal_n4m_morlet_s128": dict(n=1 << 22, n_scales=128, s_min=4.0, s_max=float(1 << 20),
                                      wavelet="morlet", boundaries=("periodic", "zero")),
}


def workload_signal(name: str) -> np.ndarray:
    w = WORKLOADS[name]
    if name.startswith("multitone"):
        return multitone(w["n"], seed=BASE_SEED)
    seed = BASE_SEED + (1 if "n1m" in name else 2)
    return lognormal_field(w["n"], seed=seed)


def workload_scales(name: str) -> np.ndarray:
    w = WORKLOADS[name]
    return log_scales(w["s_min"], w["s_max"], w["n_scales"])
