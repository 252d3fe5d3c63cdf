"""The identities behind the GPU path's own ways of evaluating the FFTCWT,
checked with the oracle alone (every transform below is the oracle's Eqs. 8-10
at the stated padded length M).

* Zero boundary, short wavelets: the M = 2N transform equals the N-periodic
  one minus the wrapped terms of the dilated wavelet's response h.
* Periodic boundary, any N: the N-periodic transform equals the zero-boundary
  transform of the signal extended periodically by E on each side, padded to
  M >= N + 2E + 1, on the window [E, E + N).
* Zero boundary, any N: any padded length M' >= N + E + 1 gives the first N
  outputs of the M = pow2 >= 2N transform.

* The forward transform of a real signal from the half-length transform of
  its samples packed in pairs (this one needs no condition).

Each of the first three needs the dilated wavelet to be short (negligible beyond E samples) and
its spectrum to be negligible at the Nyquist frequency; the last test shows
an identity failing where the second condition does not hold.
"""
import math

import numpy as np
import pytest

import synth

OMEGA0 = 6.0
CHI = {"gdw": 12.5, "morlet": 8.5}       # |psi(x)| < 1e-13 of its peak beyond |x| = CHI
# the planner's supports: |psi(x)| < 1e-9 of its peak beyond them (GDW
# (x^2 - 2) e^{-x^2/4} / 2 = 6.8e-10 at x = 10, Morlet e^{-x^2/2} = 6.7e-10 at
# x = 6.5); the identities then hold to the 1e-9 level, far below FP32 rounding
CHI_PLAN = {"gdw": 10.0, "morlet": 6.5}
# (support table, tolerance of the identity)
SUPPORTS = pytest.mark.parametrize("chi,tol", [(CHI, 1e-10), (CHI_PLAN, 1e-9)], ids=["exact", "planner"])


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def pow2_at_least(n):
    return 1 << int(math.ceil(math.log2(n)))


def support(w, s, chi=CHI):
    return int(math.ceil(chi[w] * s)) + 1


def nyquist_clear(orc, w, s):
    k = np.linspace(0.0, 40.0, 4001)
    peak = np.max(np.abs(orc.psi_hat(w, k, OMEGA0)))
    return abs(orc.psi_hat(w, [math.pi * s], OMEGA0)[0]) < 1e-7 * peak


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@SUPPORTS
@pytest.mark.parametrize("w,s", [("gdw", 2.0), ("gdw", 9.0), ("morlet", 4.0), ("morlet", 7.0)])
def test_zero_boundary_is_periodic_minus_wrapped_terms(orc, w, s, chi, tol):
    N = 1024
    E = support(w, s, chi)
    assert nyquist_clear(orc, w, s) and E < N // 4
    f = synth.lognormal_field(N, seed=31)
    W_N = orc.cwt_fft(f, [s], w, M=N, omega0=OMEGA0)[0]
    W_0 = orc.cwt_fft(f, [s], w, M=2 * N, omega0=OMEGA0)[0]
    # h(j), |j| <= E: the zero-boundary response to a unit impulse at m0
    m0 = N // 2
    imp = np.zeros(N)
    imp[m0] = 1.0
    resp = orc.cwt_fft(imp, [s], w, M=2 * N, omega0=OMEGA0)[0]
    h = {j: resp[m0 + j] for j in range(-E, E + 1)}
    fix = np.zeros(N, dtype=complex)
    for n in range(E):                    # left edge: m = N + n - j, j in [n + 1, E]
        fix[n] = sum(h[j] * f[N + n - j] for j in range(n + 1, E + 1))
    for n in range(N - E, N):             # right edge: m = n - N - j, j in [-E, n - N]
        fix[n] = sum(h[j] * f[n - N - j] for j in range(-E, n - N + 1))
    assert rel(W_N - fix, W_0) < tol
    assert np.max(np.abs(W_N[E:N - E] - W_0[E:N - E])) < tol * np.max(np.abs(W_0))
    assert rel(W_N, W_0) > 1e-6           # the wrapped terms are not negligible on their own


@SUPPORTS
@pytest.mark.parametrize("N", [1000, 997, 1500])
@pytest.mark.parametrize("w,s", [("gdw", 2.0), ("gdw", 30.0), ("morlet", 4.0), ("morlet", 60.0), ("gdw", 250.0),
                                 ("morlet", 375.0)])
def test_periodic_any_n_is_zero_boundary_of_the_extended_signal(orc, N, w, s, chi, tol):
    E = support(w, s, chi)
    assert nyquist_clear(orc, w, s)
    f = synth.lognormal_field(N, seed=N)
    W_N = orc.cwt_fft(f, [s], w, M=N, omega0=OMEGA0)[0]            # the oracle's own N-point FFTCWT
    g = f[(np.arange(N + 2 * E) - E) % N]
    # the power of two the planner takes, and the extension's own length (no
    # padding at all): the window's wrapped neighbours still fall outside it
    # (1e-10: the Morlet at s = 4 keeps 4e-10 of its peak spectrum at the
    # Nyquist frequency, so its band-limited wavelet rings at that level)
    for Mg in (pow2_at_least(N + 2 * E + 1), N + 2 * E):
        W_g = orc.cwt_fft(g, [s], w, M=Mg, omega0=OMEGA0)[0][E:E + N]
        assert rel(W_g, W_N) < tol
    # the whole zero-boundary output of the extension is not periodic: outside
    # the window it differs
    if E < N:
        W_all = orc.cwt_fft(g, [s], w, M=N + 2 * E, omega0=OMEGA0)[0]
        assert rel(W_all[:E], W_N[N - E:]) > 1e-4


@SUPPORTS
@pytest.mark.parametrize("N", [1100, 3001])
@pytest.mark.parametrize("w,s", [("gdw", 2.0), ("gdw", 40.0), ("morlet", 4.0), ("morlet", 50.0)])
def test_zero_boundary_needs_only_n_plus_e_padding(orc, N, w, s, chi, tol):
    E = support(w, s, chi)
    assert nyquist_clear(orc, w, s)
    f = synth.lognormal_field(N, seed=N + 1)
    M = pow2_at_least(2 * N)
    Mp = pow2_at_least(N + E + 1)
    assert Mp < M
    W = orc.cwt_fft(f, [s], w, M=M, omega0=OMEGA0)[0]
    Wp = orc.cwt_fft(f, [s], w, M=Mp, omega0=OMEGA0)[0]
    assert rel(Wp, W) < tol


def test_a_spectrum_cut_at_nyquist_breaks_the_identities(orc):
    """The Morlet at s = 2 has a large spectrum at the Nyquist frequency; its
    band-limited wavelet rings, so shorter padding changes the result."""
    N, s = 1000, 2.0
    assert not nyquist_clear(orc, "morlet", s)
    f = synth.lognormal_field(N, seed=5)
    W = orc.cwt_fft(f, [s], "morlet", M=pow2_at_least(2 * N), omega0=OMEGA0)[0]
    Wp = orc.cwt_fft(f, [s], "morlet", M=pow2_at_least(N + support("morlet", s) + 1), omega0=OMEGA0)[0]
    assert rel(Wp, W) > 1e-5


@pytest.mark.parametrize("M,N", [(16, 16), (64, 40), (1024, 1000), (4096, 1537), (1 << 14, 1 << 13)])
def test_real_forward_from_the_half_length_packed_transform(orc, M, N):
    """The GPU path forms the forward transform of a real signal (Eq. 8, the
    e^{+} sign) from the M/2-point transform Z of z(q) = f(2q) + i f(2q + 1):
    F(k) = conj(E(k) + e^{-2 pi i k/M} O(k)), E(k) = (Z(k) + conj Z(-k)) / 2,
    O(k) = (Z(k) - conj Z(-k)) / (2i), k <= M/2, indices of Z mod M/2.
    Checked here with the oracle's own FFT, and the in-place pairing
    (k, M/2 - k) the kernel uses."""
    f = np.zeros(M)
    f[:N] = synth.lognormal_field(N, seed=M + N)
    h = M // 2
    F_ref = orc.fft(f.astype(complex), sign=+1)[:h + 1]          # sum_n f(n) e^{+2 pi i k n / M}
    Z = orc.fft(f[0::2] + 1j * f[1::2], sign=-1)
    buf = np.zeros(h + 1, complex)
    buf[:h] = Z

    def one(a, za, zb):
        E = (za + np.conj(zb)) / 2
        O = (za - np.conj(zb)) / 2j
        return np.conj(E + np.exp(-2j * np.pi * a / M) * O)
    for k in range(h // 2 + 1):
        kp = h - k
        zk, zkp = buf[k], buf[kp % h]
        buf[k], buf[kp] = one(k, zk, zkp), one(kp, zkp, zk)
    assert np.max(np.abs(buf - F_ref)) < 1e-12 * np.max(np.abs(F_ref))
    # a mistake in the pairing (Z(-k) taken as Z(k)) fails
    bad = np.conj((Z[:h] + np.conj(Z[:h])) / 2 + np.exp(-2j * np.pi * np.arange(h) / M) * (Z[:h] - np.conj(Z[:h])) / 2j)
    assert np.max(np.abs(bad - F_ref[:h])) > 1e-3 * np.max(np.abs(F_ref))
