"""Pins of the oracle's wavelet catalogue (Table 2) against the paper's printed
constants and against quadrature of the definitions, independent of the
oracle's own formulas for psi_hat.

* C_N:    int |psi(x)|^2 dx = 1 by quadrature of psi(x).
* psi_hat: numerical Fourier integral int psi(x) e^{+ikx} dx (the paper's sign,
          Eq. 8 and App. A) at several k, compared with the oracle's psi_hat.
* K_psi, c_w: quadrature of psi_hat against the numbers printed in Table 2.
* psi_hat(0) = 0 (admissibility, App. A item 1).
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, optimize

HERE = os.path.dirname(os.path.abspath(__file__))
WAVELETS = ["cbsw", "gdw", "cwgdw", "morlet"]
CHI = {"cbsw": 3.0, "gdw": 12.0, "cwgdw": 8.0, "morlet": 7.5}


def table2():
    rows = {}
    env = {"sqrt": math.sqrt, "log": math.log, "exp": math.exp, "pi": math.pi, "e": math.e}
    with open(os.path.join(HERE, "golden", "table2_constants.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, cn, k, chi, cw = line.split()
            rows[name] = dict(cn=eval(cn, env), K=eval(k, env), chi=float(chi), cw=eval(cw, env))
    return rows


@pytest.mark.parametrize("w", WAVELETS)
def test_cn_matches_table2(orc, w):
    assert orc.cn(w, 4.0) == pytest.approx(table2()[w]["cn"], rel=1e-14)


@pytest.mark.parametrize("w", WAVELETS)
def test_unit_energy_by_quadrature(orc, w):
    lim = 40.0
    f = lambda x: abs(orc.psi(w, x, 4.0)[0]) ** 2
    pts = [-2, -1, 0, 1, 2] if w == "cbsw" else None
    val = integrate.quad(f, -lim, lim, points=pts, limit=500, epsabs=1e-14, epsrel=1e-13)[0]
    assert val == pytest.approx(1.0, abs=1e-11)


@pytest.mark.parametrize("omega0", [4.0, 5.0, 6.0])
def test_morlet_unit_energy_any_omega0(orc, omega0):
    f = lambda x: abs(orc.psi("morlet", x, omega0)[0]) ** 2
    val = integrate.quad(f, -40, 40, limit=500, epsabs=1e-14, epsrel=1e-13)[0]
    assert val == pytest.approx(1.0, abs=1e-11)


def fourier_quad(orc, w, k, omega0):
    """int psi(x) e^{+ikx} dx by quadrature (paper's forward sign)."""
    lim = 3.0 if w == "cbsw" else 40.0
    pts = [-2, -1, 0, 1, 2] if w == "cbsw" else None
    re = integrate.quad(lambda x: (orc.psi(w, x, omega0)[0] * np.exp(1j * k * x)).real,
                        -lim, lim, points=pts, limit=800, epsabs=1e-14, epsrel=1e-12)[0]
    im = integrate.quad(lambda x: (orc.psi(w, x, omega0)[0] * np.exp(1j * k * x)).imag,
                        -lim, lim, points=pts, limit=800, epsabs=1e-14, epsrel=1e-12)[0]
    return re + 1j * im


@pytest.mark.parametrize("w,omega0", [("cbsw", 4.0), ("gdw", 4.0), ("cwgdw", 4.0),
                                      ("morlet", 4.0), ("morlet", 6.0)])
def test_psi_hat_is_fourier_transform_of_psi(orc, w, omega0):
    for k in [-5.0, -1.3, 0.7, 2.0, 4.5, 6.2, 9.0]:
        num = fourier_quad(orc, w, k, omega0)
        ana = orc.psi_hat(w, k, omega0)[0]
        assert abs(num - ana) < 1e-10, (k, num, ana)


@pytest.mark.parametrize("w", WAVELETS)
def test_zero_mean(orc, w):
    assert orc.psi_hat(w, 0.0, 4.0)[0] == pytest.approx(0.0, abs=1e-15)
    assert orc.psi_hat("morlet", 0.0, 6.0)[0] == pytest.approx(0.0, abs=1e-15)


@pytest.mark.parametrize("w", WAVELETS)
def test_admissibility_constant_matches_table2(orc, w):
    f = lambda k: orc.psi_hat(w, k, 4.0)[0] / k
    if w == "cbsw":
        # oscillatory k^-5 tail: integrate period by period out to 2 pi * 2000
        edges = np.concatenate([[1e-12], 2 * np.pi * np.arange(1, 2001)])
        val = sum(integrate.quad(f, a, b, epsabs=1e-16, epsrel=1e-13)[0]
                  for a, b in zip(edges[:-1], edges[1:]))
        rel = 1e-9
    else:
        val = integrate.quad(f, 0.0, 60.0, limit=400, epsabs=1e-15, epsrel=1e-13)[0]
        rel = 1e-12
    assert val == pytest.approx(table2()[w]["K"], rel=rel)


@pytest.mark.parametrize("w", WAVELETS)
def test_oracle_admissibility(orc, w):
    """oracle.admissibility (used by the inverse CWT) against the numbers printed in
    Table 2 at omega0 = 4 and, for the Morlet, quadrature at other omega0."""
    assert orc.admissibility(w, 4.0) == pytest.approx(table2()[w]["K"], rel=1e-12)
    if w == "morlet":
        for om in (3.0, 6.0, 9.0):
            q = integrate.quad(lambda k: orc.psi_hat(w, k, om)[0] / k, 0.0, om + 60.0, limit=400,
                               epsabs=1e-15, epsrel=1e-13)[0]
            assert orc.admissibility(w, om) == pytest.approx(q, rel=1e-11)


@pytest.mark.parametrize("w", WAVELETS)
def test_cw_matches_table2(orc, w):
    # c_w = w / k_pseu: the scale at which the response to a unit-wavenumber tone,
    # proportional to |psi_hat(k/w)| / sqrt(w), peaks; i.e. 1 / argmax_u sqrt(u) |psi_hat(u)|.
    g = lambda u: -math.sqrt(u) * abs(orc.psi_hat(w, u, 4.0)[0])
    grid = np.linspace(0.05, 12.0, 2400)
    u0 = grid[np.argmin([g(u) for u in grid])]
    r = optimize.minimize_scalar(g, bracket=(u0 - 0.01, u0, u0 + 0.01), tol=1e-14)
    assert 1.0 / r.x == pytest.approx(table2()[w]["cw"], rel=1e-8)


@pytest.mark.parametrize("w", ["gdw", "cwgdw", "morlet"])
def test_chi_is_numerical_support(orc, w):
    # Table 2 caption: beyond chi the wavelet is ~1e-14 or below
    chi = table2()[w]["chi"]
    assert CHI[w] == chi
    assert abs(orc.psi(w, chi, 4.0)[0]) < 1e-9
    assert abs(orc.psi(w, chi + 2.0, 4.0)[0]) < 1e-13


def test_cbsw_compact_support(orc):
    x = np.linspace(3.0, 5.0, 11)
    assert np.all(orc.psi("cbsw", x) == 0)
    assert np.all(orc.psi("cbsw", -x) == 0)


def test_morlet_omega0_6_constants(orc):
    # general-omega0 C_N reduces to Table 2's form at omega0 = 4
    c4 = math.exp(8) / math.sqrt(1 - 2 * math.exp(4) + math.exp(16)) / math.pi ** 0.25
    assert orc.cn("morlet", 4.0) == pytest.approx(c4, rel=1e-15)
    # spectrum peaks near omega0 and is negligible at negative k
    k = np.linspace(-10, 20, 3001)
    ph = orc.psi_hat("morlet", k, 6.0)
    assert abs(k[np.argmax(ph)] - 6.0) < 0.02
    assert np.max(np.abs(ph[k < 0])) < 3e-8 * np.max(ph)
