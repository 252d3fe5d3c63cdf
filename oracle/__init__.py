"""Python access to the FP64 CPU oracle of the FFTCWT (cwt_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark load this module; the CUDA library never does, and this
module imports nothing from it.  The oracle is a plain C restatement of the
paper's definitions (Eq. 4 direct sum; Eqs. 8-10 FFTCWT; Eq. 42 power;
Eqs. 41 and 43 environment power) and is built with gcc on first use (or by
``build()``); the inverse CWT (Eqs. 5 and 6) and its constant K_psi are
written here in numpy.

Scales are passed as dilations ``s`` in samples and converted to the paper's
dimensionless scale w~ = 1/s here, unless ``w_tilde=True``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cwt_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libcwt_oracle.so")
_lock = threading.Lock()
_lib = None

WAVELETS = {"cbsw": 0, "gdw": 1, "cwgdw": 2, "morlet": 3}
BOUNDARIES = {"periodic": 0, "zero": 1}


def build(force: bool = False) -> str:
    """Compile cwt_oracle.c into a shared library with gcc (OpenMP if available)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        d, i64, i32, ci = ctypes.c_double, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
        pd, pi32, pi64 = (ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32),
                          ctypes.POINTER(ctypes.c_int64))
        lib.orc_cn.restype = d
        lib.orc_cn.argtypes = [ci, d]
        lib.orc_psi_hat.restype = d
        lib.orc_psi_hat.argtypes = [ci, d, d]
        lib.orc_psi.restype = None
        lib.orc_psi.argtypes = [ci, d, d, pd, pd]
        lib.orc_fft.restype = ci
        lib.orc_fft.argtypes = [i64, pd, pd, ci]
        lib.orc_dft.restype = ci
        lib.orc_dft.argtypes = [i64, pd, pd, ci, pd, pd]
        lib.orc_cwt_fft.restype = ci
        lib.orc_cwt_fft.argtypes = [pd, i64, i64, pd, i32, ci, d, d, ci, ci, pd, pd]
        lib.orc_cwt_fft_points.restype = ci
        lib.orc_cwt_fft_points.argtypes = [pd, i64, i64, pd, i32, ci, d, d, pi32, pi64, i64,
                                           ci, pd, pd]
        lib.orc_cwt_direct.restype = ci
        lib.orc_cwt_direct.argtypes = [pd, i64, pd, i32, ci, d, d, ci, ci, pd, pd]
        lib.orc_cwt_direct_points.restype = ci
        lib.orc_cwt_direct_points.argtypes = [pd, i64, pd, i32, ci, d, d, ci, pi32, pi64, i64,
                                              ci, pd, pd]
        lib.orc_wavelet_power.restype = ci
        lib.orc_wavelet_power.argtypes = [pd, pd, i64, i32, pd]
        lib.orc_env_power.restype = ci
        lib.orc_env_power.argtypes = [pd, pd, pd, i64, i32, pd, pd, pd, pd]
        _lib = lib
        return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _wt(scales, w_tilde):
    s = _f64(scales)
    return s.copy() if w_tilde else 1.0 / s


def cn(wavelet: str, omega0: float = 4.0) -> float:
    return _load().orc_cn(WAVELETS[wavelet], omega0)


def psi_hat(wavelet: str, k, omega0: float = 4.0) -> np.ndarray:
    lib = _load()
    k = np.atleast_1d(_f64(k))
    return np.array([lib.orc_psi_hat(WAVELETS[wavelet], omega0, float(x)) for x in k])


def psi(wavelet: str, x, omega0: float = 4.0) -> np.ndarray:
    lib = _load()
    x = np.atleast_1d(_f64(x))
    out = np.empty(x.shape, dtype=np.complex128)
    re, im = ctypes.c_double(), ctypes.c_double()
    for i, v in enumerate(x):
        lib.orc_psi(WAVELETS[wavelet], omega0, float(v), ctypes.byref(re), ctypes.byref(im))
        out[i] = complex(re.value, im.value)
    return out


def fft(x, sign: int = -1) -> np.ndarray:
    """Unnormalised DFT X(k) = sum_j x(j) e^{sign 2 pi i jk/n} (radix-2 / Bluestein)."""
    x = np.asarray(x, dtype=np.complex128)
    re, im = _f64(x.real).copy(), _f64(x.imag).copy()
    if _load().orc_fft(len(x), _dp(re), _dp(im), sign) != 0:
        raise RuntimeError("orc_fft failed")
    return re + 1j * im


def dft(x, sign: int = -1) -> np.ndarray:
    x = np.asarray(x, dtype=np.complex128)
    re, im = _f64(x.real), _f64(x.imag)
    o_re, o_im = np.empty(len(x)), np.empty(len(x))
    if _load().orc_dft(len(x), _dp(re), _dp(im), sign, _dp(o_re), _dp(o_im)) != 0:
        raise RuntimeError("orc_dft failed")
    return o_re + 1j * o_im


def cwt_fft(f, scales, wavelet: str, M: int | None = None, omega0: float = 6.0,
            dx: float = 1.0, naive: bool = False, w_tilde: bool = False,
            nthreads: int = 0) -> np.ndarray:
    """FFTCWT (Eqs. 8-10): complex128 array [S, N].  M defaults to N (periodic);
    M > N is the zero boundary (signal at offset 0, zeros after, first N kept)."""
    f = _f64(f)
    N = len(f)
    M = N if M is None else int(M)
    wt = _wt(scales, w_tilde)
    S = len(wt)
    re, im = np.empty((S, N)), np.empty((S, N))
    rc = _load().orc_cwt_fft(_dp(f), N, M, _dp(wt), S, WAVELETS[wavelet], omega0, dx,
                             int(naive), nthreads, _dp(re), _dp(im))
    if rc != 0:
        raise RuntimeError("orc_cwt_fft failed")
    return re + 1j * im


def cwt_fft_points(f, scales, wavelet: str, ps, pn, M: int | None = None,
                   omega0: float = 6.0, dx: float = 1.0, w_tilde: bool = False,
                   nthreads: int = 0) -> np.ndarray:
    f = _f64(f)
    N = len(f)
    M = N if M is None else int(M)
    wt = _wt(scales, w_tilde)
    ps = np.ascontiguousarray(ps, dtype=np.int32)
    pn = np.ascontiguousarray(pn, dtype=np.int64)
    re, im = np.empty(len(ps)), np.empty(len(ps))
    rc = _load().orc_cwt_fft_points(
        _dp(f), N, M, _dp(wt), len(wt), WAVELETS[wavelet], omega0, dx,
        ps.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
        pn.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(ps), nthreads, _dp(re), _dp(im))
    if rc != 0:
        raise RuntimeError("orc_cwt_fft_points failed")
    return re + 1j * im


def cwt_direct(f, scales, wavelet: str, boundary: str = "periodic", omega0: float = 6.0,
               dx: float = 1.0, w_tilde: bool = False, nthreads: int = 0) -> np.ndarray:
    """Direct sum of Eq. 4: complex128 array [S, N]."""
    f = _f64(f)
    N = len(f)
    wt = _wt(scales, w_tilde)
    S = len(wt)
    re, im = np.empty((S, N)), np.empty((S, N))
    rc = _load().orc_cwt_direct(_dp(f), N, _dp(wt), S, WAVELETS[wavelet], omega0, dx,
                                BOUNDARIES[boundary], nthreads, _dp(re), _dp(im))
    if rc != 0:
        raise RuntimeError("orc_cwt_direct failed")
    return re + 1j * im


def cwt_direct_points(f, scales, wavelet: str, ps, pn, boundary: str = "periodic",
                      omega0: float = 6.0, dx: float = 1.0, w_tilde: bool = False,
                      nthreads: int = 0) -> np.ndarray:
    f = _f64(f)
    N = len(f)
    wt = _wt(scales, w_tilde)
    ps = np.ascontiguousarray(ps, dtype=np.int32)
    pn = np.ascontiguousarray(pn, dtype=np.int64)
    re, im = np.empty(len(ps)), np.empty(len(ps))
    rc = _load().orc_cwt_direct_points(
        _dp(f), N, _dp(wt), len(wt), WAVELETS[wavelet], omega0, dx, BOUNDARIES[boundary],
        ps.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
        pn.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(ps), nthreads, _dp(re), _dp(im))
    if rc != 0:
        raise RuntimeError("orc_cwt_direct_points failed")
    return re + 1j * im


def wavelet_power(W) -> np.ndarray:
    """Eq. 42: P(w_s) = mean_n |W(w_s, n)|^2 over the rows of W [S, N]."""
    W = np.asarray(W)
    re, im = _f64(W.real), _f64(np.imag(W))
    S, N = W.shape
    P = np.empty(S)
    if _load().orc_wavelet_power(_dp(re), _dp(im), N, S, _dp(P)) != 0:
        raise RuntimeError("orc_wavelet_power failed")
    return P


def env_power(W, delta):
    """Eqs. 41 and 43 for the environments delta > 0 and delta < 0:
    returns (P_pos[S], P_neg[S], f_pos, f_neg)."""
    W = np.asarray(W)
    re, im = _f64(W.real), _f64(np.imag(W))
    delta = _f64(delta)
    S, N = W.shape
    pp, pn = np.empty(S), np.empty(S)
    fp, fn = ctypes.c_double(), ctypes.c_double()
    if _load().orc_env_power(_dp(re), _dp(im), _dp(delta), N, S, _dp(pp), _dp(pn),
                             ctypes.byref(fp), ctypes.byref(fn)) != 0:
        raise RuntimeError("orc_env_power failed")
    return pp, pn, fp.value, fn.value


# Table 2 closed forms of K_psi = int_0^inf psi_hat(k) / k dk
_K_CLOSED = {
    "cbsw": lambda: 0.5 * np.sqrt(15.0 / 62.0) * (27.0 * np.log(3.0) - 32.0 * np.log(2.0)),
    "gdw": lambda: 2.0 * (8.0 * np.pi / 9.0) ** 0.25,
    "cwgdw": lambda: 4.0 * np.pi ** 0.25 / np.sqrt(1.0 + 5.0 * np.e),
}


def admissibility(wavelet: str, omega0: float = 6.0) -> float:
    """K_psi = int_0^inf psi_hat(k)/k dk, the constant of Eqs. 5 and 6.
    CBSW, GDW and CW-GDW: the closed forms printed in Table 2.  Morlet (any
    omega0): adaptive quadrature of the oracle's psi_hat."""
    if wavelet in _K_CLOSED:
        return float(_K_CLOSED[wavelet]())
    from scipy import integrate
    lib = _load()
    g = lambda k: lib.orc_psi_hat(WAVELETS[wavelet], omega0, k) / k
    return integrate.quad(g, 0.0, omega0 + 40.0, limit=400, epsabs=1e-15, epsrel=1e-13)[0]


def icwt(W, scales, wavelet: str, omega0: float = 6.0, dx: float = 1.0,
         w_tilde: bool = False) -> np.ndarray:
    """Inverse CWT over a finite set of scales (Sec. 2): Eq. 6 for the real even
    wavelets, Eq. 5 (twice the real part) for the Morlet, without the mean
    term.  The discrete W of Eq. 7 equals W_f(w, x) at w = w~ / dx, and the
    scale integral int_0^inf W / sqrt(w) dw = int W sqrt(w) d(ln w) is taken by
    the trapezoid rule in ln w over the scales sorted by w."""
    W = np.asarray(W)
    w = _wt(scales, w_tilde) / dx
    order = np.argsort(w, kind="stable")
    lnw = np.log(w[order])
    g = W[order] * np.sqrt(w[order])[:, None]
    integral = np.zeros(W.shape[1], dtype=np.complex128)
    for i in range(len(lnw) - 1):
        integral += 0.5 * (lnw[i + 1] - lnw[i]) * (g[i] + g[i + 1])
    rec = integral.real / admissibility(wavelet, omega0)
    return 2.0 * rec if wavelet == "morlet" else rec
