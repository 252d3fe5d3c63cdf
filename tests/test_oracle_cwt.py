"""Pins of the oracle's CWT tiers against the paper and the mathematics.

T0 = direct sum of Eq. 4; T1 = FFTCWT (Eqs. 8-10) with O(M^2) DFTs;
T2 = FFTCWT with the oracle's FFT.  None of these checks re-types the FFTCWT
formula: each compares against the definition (Eq. 1 / Eq. 4), a closed form
derived from it, a value the paper prints, or an exact invariant.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def rel_l2(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def es_percent(num, ana):
    """Error spectrum of Eq. 39 per scale (rows), in percent."""
    return np.sum(np.abs(num - ana), axis=1) / np.sum(np.abs(ana), axis=1) * 100.0


def accuracy_bands():
    out = {}
    with open(os.path.join(HERE, "golden", "fftcwt_accuracy.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            sig, bnd, lo, hi = line.split()
            out[sig] = (float(lo), float(hi))
    return out


def paper_grid(N, cw, n_subs):
    """Sec. 3.1 scale grid: w~ = w~_min 2^{i + j/N_subs}, w~_min = c_w pi / N,
    N_levs = Nint(log2(c_w k_Nyq / (w~_min/dx))) = Nint(log2 N)."""
    wmin = cw * math.pi / N
    n_levs = int(round(math.log2(N)))
    return np.array([wmin * 2.0 ** (i + j / n_subs) for i in range(n_levs) for j in range(n_subs)])


CW = {"cbsw": 0.466094761079290, "gdw": 2 / math.sqrt(5), "cwgdw": 0.428218886729052,
      "morlet": 0.242640671273266}
CHI = {"cbsw": 3.0, "gdw": 12.0, "cwgdw": 8.0, "morlet": 7.5}


# --------------------------------------------------------- T0 vs T1 vs T2

@pytest.mark.parametrize("N", [8, 13, 31, 64])
@pytest.mark.parametrize("w,omega0,smin", [("gdw", 6.0, 2.0), ("morlet", 6.0, 5.0),
                                           ("cwgdw", 6.0, 4.0)])
def test_direct_equals_dft_periodic(orc, N, w, omega0, smin):
    f = synth.multitone(N, seed=N)
    sc = synth.log_scales(smin, 4.0 * N, 7)
    t0 = orc.cwt_direct(f, sc, w, "periodic", omega0=omega0)
    t1 = orc.cwt_fft(f, sc, w, omega0=omega0, naive=True)
    assert rel_l2(t1, t0) < 1e-12


@pytest.mark.parametrize("N", [8, 13, 31, 64])
@pytest.mark.parametrize("w,omega0,smin", [("gdw", 6.0, 2.0), ("morlet", 6.0, 5.0)])
def test_direct_equals_dft_zero_boundary(orc, N, w, omega0, smin):
    # zero boundary: T1 equals the linear sum when M - N covers the dilated support
    f = synth.multitone(N, seed=N + 1)
    smax = N / (CHI[w] + 4.0)
    sc = synth.log_scales(smin, max(smin, smax), 5)
    M = 2 * N + int(math.ceil((CHI[w] + 4.0) * sc.max()))
    t0 = orc.cwt_direct(f, sc, w, "zero", omega0=omega0)
    t1 = orc.cwt_fft(f, sc, w, M=M, omega0=omega0, naive=True)
    assert rel_l2(t1, t0) < 1e-12


@pytest.mark.parametrize("N,M", [(64, 64), (100, 100), (97, 97), (256, 512), (300, 640), (37, 101)])
@pytest.mark.parametrize("w", ["gdw", "morlet"])
def test_fft_tier_equals_dft_tier(orc, N, M, w):
    f = synth.lognormal_field(N, seed=N)
    sc = synth.log_scales(2.0, N / 2.0, 6)
    t1 = orc.cwt_fft(f, sc, w, M=M, naive=True)
    t2 = orc.cwt_fft(f, sc, w, M=M)
    assert rel_l2(t2, t1) < 1e-13


def test_points_match_full_arrays(orc):
    N = 200
    f = synth.lognormal_field(N, seed=3)
    sc = synth.log_scales(2.0, 50.0, 5)
    ps, pn = synth.sample_points(5, N, 40, seed=9)
    for bnd, M in [("periodic", N), ("zero", 512)]:
        full = orc.cwt_fft(f, sc, "morlet", M=M)
        pts = orc.cwt_fft_points(f, sc, "morlet", ps, pn, M=M)
        assert np.max(np.abs(pts - full[ps, pn])) < 1e-13 * np.max(np.abs(full))
        d_full = orc.cwt_direct(f, sc, "gdw", bnd)
        d_pts = orc.cwt_direct_points(f, sc, "gdw", ps, pn, bnd)
        assert np.max(np.abs(d_pts - d_full[ps, pn])) < 1e-13 * np.max(np.abs(d_full))


# ------------------------------------------------------ closed forms

def tone_cwt(orc, w, omega0, amps, k0s, phases, x, wscale):
    """Analytic CWT (Eq. 1) of sum_j A_j cos(k_j x + phi_j):
    W(w,x) = sum_j A_j/(2 sqrt w) [e^{-i(k x + phi)} psi_hat(k/w) + e^{+i(k x + phi)} psi_hat(-k/w)]."""
    out = np.zeros((len(wscale), len(x)), complex)
    for i, ws in enumerate(wscale):
        for a, k, ph in zip(amps, k0s, phases):
            p = orc.psi_hat(w, k / ws, omega0)[0]
            m = orc.psi_hat(w, -k / ws, omega0)[0]
            out[i] += a / (2 * math.sqrt(ws)) * (np.exp(-1j * (k * x + ph)) * p
                                                  + np.exp(1j * (k * x + ph)) * m)
    return out


def test_tone_closed_form_by_quadrature(orc):
    # the tone formula itself, checked against direct quadrature of Eq. 1
    w, ws, k, x = "morlet", 3.0, 5.0, 0.4
    ana = tone_cwt(orc, w, 4.0, [1.0], [k], [0.3], np.array([x]), [ws])[0, 0]
    f = lambda u: np.cos(k * u + 0.3) * math.sqrt(ws) * orc.psi(w, ws * (x - u), 4.0)[0]
    re = integrate.quad(lambda u: f(u).real, x - 5, x + 5, limit=400, epsabs=1e-14)[0]
    im = integrate.quad(lambda u: f(u).imag, x - 5, x + 5, limit=400, epsabs=1e-14)[0]
    assert abs(ana - (re + 1j * im)) < 1e-11


@pytest.mark.parametrize("w", ["cbsw", "gdw", "cwgdw", "morlet"])
def test_paper_f1_periodic_accuracy(orc, w):
    """Sec. 4.1: FFTCWT of f1 on [0, 2pi), N = 512, periodic: ES < 1e-10 %."""
    x, f, dx = synth.paper_f1(512)
    wt = paper_grid(512, CW[w], 4)
    num = orc.cwt_fft(f, wt, w, omega0=4.0, dx=dx, w_tilde=True)
    ana = tone_cwt(orc, w, 4.0, [2.0, 0.5, 0.25], [1.0, 8.0, 32.0], [0.0, 0.0, -math.pi / 2],
                   x, wt / dx)
    es = es_percent(num, ana)
    # the top scales sit where f1 has no power, so fp64 FFT rounding sets the
    # floor; the paper's range (1e-14 % .. 1e-10 %) is a decade read off Fig. 10
    assert es.max() < 2.0 * accuracy_bands()["f1"][1]
    assert es.min() < 1e-13


def gaussian_cwt(w, omega0, x, ws, cn):
    """Analytic CWT of f2 = exp(-x^2/2) by the Fourier route of App. A:
    W = (1/2pi) int f_hat(k) psi_hat(k/w) / sqrt(w) e^{-ikx} dk, Gaussian integrals."""
    if w == "gdw":
        a = 0.5 + 1.0 / ws ** 2
        pre = 8 * math.sqrt(math.pi) * cn * math.sqrt(2 * math.pi) / (2 * math.pi * ws ** 2.5)
        return pre * np.sqrt(math.pi / a) / (2 * a) * (1 - x ** 2 / (2 * a)) * np.exp(-x ** 2 / (4 * a))
    if w == "morlet":
        al = 0.5 * (1.0 + 1.0 / ws ** 2)
        b1 = omega0 / ws - 1j * x
        t1 = np.exp(b1 ** 2 / (4 * al) - omega0 ** 2 / 2)
        t2 = np.exp(-x ** 2 / (4 * al) - omega0 ** 2 / 2)
        return cn / math.sqrt(ws) * math.sqrt(math.pi / al) * (t1 - t2)
    raise ValueError(w)


@pytest.mark.parametrize("w", ["gdw", "morlet"])
def test_gaussian_closed_form_by_quadrature(orc, w):
    cn = orc.cn(w, 4.0)
    for ws, x in [(0.7, 0.3), (2.5, -1.1), (6.0, 0.05)]:
        g = lambda u: math.exp(-u * u / 2) * math.sqrt(ws) * orc.psi(w, ws * (x - u), 4.0)[0]
        re = integrate.quad(lambda u: g(u).real, -30, 30, limit=800, epsabs=1e-15)[0]
        im = integrate.quad(lambda u: g(u).imag, -30, 30, limit=800, epsabs=1e-15)[0]
        assert abs(gaussian_cwt(w, 4.0, np.array([x]), ws, cn)[0] - (re + 1j * im)) < 1e-12


@pytest.mark.parametrize("w", ["gdw", "morlet"])
def test_paper_f2_zero_boundary_accuracy(orc, w):
    """Sec. 4.1 with Eq. 40 padding: FFTCWT error of f2 within the paper's 1e-8 % .. 0.1 %."""
    N = 512
    x, f, dx = synth.gaussian_f2(N)
    wt = paper_grid(N, CW[w], 4)
    n_zeros = int(round(CHI[w] / wt.min()))
    M = N + 2 * n_zeros
    num = orc.cwt_fft(f, wt, w, M=M, omega0=4.0, dx=dx, w_tilde=True)
    cn = orc.cn(w, 4.0)
    ana = np.array([gaussian_cwt(w, 4.0, x, s, cn) for s in wt / dx])
    es = es_percent(num, ana)
    lo, hi = accuracy_bands()["f2"]
    assert es.max() <= 2.0 * hi
    assert es.max() >= 0.5 * lo   # padding error is visible, unlike the periodic case


@pytest.mark.parametrize("w,omega0", [("gdw", 4.0), ("morlet", 6.0), ("cwgdw", 4.0)])
def test_modulus_peak_at_cw_times_k(orc, w, omega0):
    """|W| of a pure tone k0 peaks at the scale w* = c_w k0 (Table 2 c_w;
    Morlet omega0=6: u* = (omega0 + sqrt(omega0^2 + 2)) / 2)."""
    N, q = 4096, 64
    f = np.cos(2 * np.pi * q * np.arange(N) / N)
    k0 = 2 * np.pi * q / N
    if w == "morlet" and omega0 == 6.0:
        cw = 2.0 / (omega0 + math.sqrt(omega0 ** 2 + 2.0))
    else:
        cw = CW[w]
    wt = cw * k0 * np.exp(np.linspace(-0.05, 0.05, 41))
    W = orc.cwt_fft(f, wt, w, omega0=omega0, w_tilde=True)
    amp = np.abs(W[:, 100])
    i = int(np.argmax(amp))
    assert 0 < i < len(wt) - 1
    la = np.log(wt)
    y0, y1, y2 = amp[i - 1], amp[i], amp[i + 1]
    h = la[1] - la[0]
    peak = la[i] + 0.5 * h * (y0 - y2) / (y0 - 2 * y1 + y2)
    assert math.exp(peak) == pytest.approx(cw * k0, rel=2e-5)


def test_morlet_phase_follows_paper_sign(orc):
    """Paper's convention (forward e^{+ikx}): for f = cos(k0 x) the Morlet CWT
    turns as e^{-i k0 x} (reading of Eq. 8 and Table 2)."""
    N, q = 1024, 40
    n = np.arange(N)
    f = np.cos(2 * np.pi * q * n / N)
    k0 = 2 * np.pi * q / N
    W = orc.cwt_fft(f, [k0 / 6.0], "morlet", omega0=6.0, w_tilde=True)[0]
    ratio = W * np.exp(1j * k0 * n)
    assert np.std(ratio) < 1e-6 * np.abs(ratio).mean()
    assert ratio.real.mean() > 0


# ------------------------------------------------------------ invariants

def test_invariants_periodic(orc):
    N = 512
    f = synth.lognormal_field(N, seed=5)
    sc = synth.log_scales(2.0, 128.0, 9)
    W = orc.cwt_fft(f, sc, "gdw")
    assert np.max(np.abs(W.sum(axis=1))) < 1e-11 * np.max(np.abs(W))      # zero mean
    assert np.max(np.abs(W.imag)) < 1e-14 * np.max(np.abs(W.real))          # real wavelet
    Ws = orc.cwt_fft(np.roll(f, 37), sc, "gdw")                              # shift equivariance
    assert rel_l2(Ws, np.roll(W, 37, axis=1)) < 1e-13
    Wr = orc.cwt_fft(f[(-np.arange(N)) % N], sc, "gdw")                      # even wavelet
    assert rel_l2(Wr, W[:, (-np.arange(N)) % N]) < 1e-13
    g = synth.multitone(N, seed=6)
    Wl = orc.cwt_fft(2.0 * f - 3.0 * g, sc, "morlet")                         # linearity
    assert rel_l2(Wl, 2.0 * orc.cwt_fft(f, sc, "morlet") - 3.0 * orc.cwt_fft(g, sc, "morlet")) < 1e-13


def test_tone_power_closed_form(orc):
    """Eq. 42 for f = A cos(k0 x) and a real even wavelet: P(w) = A^2 psi_hat(k0/w)^2 / (2w)."""
    N, q, A = 2048, 50, 1.7
    f = A * np.cos(2 * np.pi * q * np.arange(N) / N)
    k0 = 2 * np.pi * q / N
    wt = k0 * np.array([0.3, 0.9, 2.0])
    P = orc.wavelet_power(orc.cwt_fft(f, wt, "gdw", w_tilde=True))
    expect = np.array([A * A * orc.psi_hat("gdw", k0 / w)[0] ** 2 / (2 * w) for w in wt])
    assert np.allclose(P, expect, rtol=1e-12)


def test_env_power_recovers_global(orc):
    """Eq. 43: P(w) = f_+ P(w, delta>0) + f_- P(w, delta<0) when no delta is exactly 0."""
    N = 1024
    d = synth.lognormal_field(N, seed=11)
    assert np.all(d != 0)
    W = orc.cwt_fft(d, synth.log_scales(2.0, 200.0, 6), "morlet")
    pp, pn, fp, fn = orc.env_power(W, d)
    assert fp + fn == pytest.approx(1.0)
    assert np.allclose(fp * pp + fn * pn, orc.wavelet_power(W), rtol=1e-13)


ICWT_TOL = {"cbsw": 1e-7, "gdw": 1e-8, "cwgdw": 1e-12}


@pytest.mark.parametrize("w,omega0", [("cbsw", 6.0), ("gdw", 6.0), ("cwgdw", 6.0),
                                      ("morlet", 4.0), ("morlet", 6.0)])
def test_inverse_cwt_reconstructs(orc, w, omega0):
    """Eq. 6 (real even wavelets) and Eq. 5 (Morlet): oracle.icwt of the oracle's
    W over a fine log grid of scales gives back the signal minus its mean.
    Odd N: an even-length real signal's Nyquist bin is its own mirror image, so
    the analytic-wavelet formula (Eq. 5) would count it twice.  The Morlet's
    floor is its psi_hat at k < 0 (about e^{-omega0^2/2}), which Eq. 5 assumes
    zero."""
    N = 1023
    f = synth.multitone(N, periods=(16.0, 128.0, 341.0), seed=2)
    wt = np.exp(np.arange(math.log(2e-4), math.log(3e4), 0.04))
    W = orc.cwt_fft(f, wt, w, omega0=omega0, w_tilde=True)
    rec = orc.icwt(W, wt, w, omega0=omega0, w_tilde=True)
    tol = ICWT_TOL[w] if w != "morlet" else 10.0 * math.exp(-0.5 * omega0 ** 2)
    assert rel_l2(rec, f - f.mean()) < tol


def test_inverse_cwt_irregular_grid_and_dx(orc):
    """Scales in any order, unevenly spaced in ln w, and dx != 1: the trapezoid
    rule over the sorted grid still reconstructs the signal (GDW, Eq. 6), to the
    second-order accuracy of the trapezoid rule on an uneven grid."""
    N = 1023
    f = synth.multitone(N, periods=(16.0, 128.0, 341.0), seed=4)
    rng = np.random.default_rng(7)
    h = 0.03
    lw = np.arange(math.log(2e-4), math.log(3e4), h)
    lw += rng.uniform(-0.4, 0.4, len(lw)) * h                     # uneven gaps in (0.2h, 1.8h)
    wt = np.exp(lw)[rng.permutation(len(lw))]
    W = orc.cwt_fft(f, wt, "gdw", dx=0.5, w_tilde=True)
    rec = orc.icwt(W, wt, "gdw", dx=0.5, w_tilde=True)
    assert rel_l2(rec, f - f.mean()) < 2e-5      # second-order trapezoid on an uneven grid
    # dilations (w~ = 1 / s) give the same numbers as the equivalent w~ grid
    rec2 = orc.icwt(W, 1.0 / wt, "gdw", dx=0.5)
    assert np.allclose(rec2, rec, rtol=0, atol=1e-13 * np.abs(rec).max())


def test_env_power_labels_and_fractions(orc):
    """Eq. 41 on a W built by hand, so that the answer is known without the
    oracle: |W|^2 = (s+1)^2 on the positions with delta > 0 (the overdense
    environment), 1e-4 on those with delta < 0, and delta = 0 at a few
    positions that belong to neither environment.  Swapping the environments,
    or counting the delta = 0 positions in either, fails this; Eq. 43 alone
    does not see a swap."""
    N, S = 1000, 4
    rng = np.random.default_rng(3)
    delta = np.where(rng.random(N) < 0.3, 1.5, -0.4)
    delta[[5, 500, 999]] = 0.0
    pos, neg = delta > 0, delta < 0
    phase = np.exp(1j * rng.uniform(0, 2 * np.pi, (S, N)))
    amp = np.where(pos[None, :], np.arange(1, S + 1)[:, None], 0.01)
    W = amp * phase
    pp, pn, fp, fn = orc.env_power(W, delta)
    assert fp == pos.sum() / N and fn == neg.sum() / N
    assert fp + fn == pytest.approx(1.0 - 3.0 / N)
    assert np.allclose(pp, np.arange(1, S + 1) ** 2.0, rtol=1e-13)
    assert np.allclose(pn, 1e-4, rtol=1e-12)
    # an environment with no position gets 0 (Eq. 41 over an empty set)
    pp0, pn0, fp0, fn0 = orc.env_power(W, -np.abs(delta) - 1.0)
    assert np.all(pp0 == 0.0) and fp0 == 0.0 and fn0 == 1.0
