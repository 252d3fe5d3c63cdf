"""Parity of the statistics of W computed on the GPU (through the C ABI) with
the FP64 oracle: the environment-dependent power spectrum (Eqs. 41 and 43) and
the inverse CWT (Eqs. 5 and 6).  Both sides read the same W (the GPU's), so the
comparison isolates the reduction / integration kernels.
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    import paper_2302_03909_gb300 as cwt
    cwt.load_library()
    oracle.build()
    return torch, cwt, oracle


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("N,wavelet,boundary,dtype", [
    (1 << 15, "morlet", "periodic", "f32"),
    ((1 << 16) + 77, "gdw", "zero", "f32"),
    (100000, "cwgdw", "zero", "f64"),
    (1 << 14, "cbsw", "periodic", "f64"),
    (5, "morlet", "zero", "f32"),
])
def test_env_power(env, N, wavelet, boundary, dtype):
    """P_pos, P_neg and the environment fractions of Eqs. 41 and 43 against the
    oracle on the GPU's W, with delta the transformed density contrast and a few
    positions set to exactly zero (in neither environment)."""
    torch, cwt, orc = env
    f = synth.lognormal_field(N, seed=N % 1000 + 3)
    f[::97] = 0.0
    sc = synth.log_scales(2.0, max(2.5, N / 8), 9)
    plan = cwt.cwt_plan_create(N, sc, wavelet, boundary, input_dtype=dtype)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    sig = torch.tensor(f, dtype=tdt, device="cuda")
    W, spec = cwt.cwt_exec_with_power(plan, sig)
    pp, pn, fr = cwt.cwt_env_power(plan, W, sig)
    pp2, pn2, fr2 = cwt.cwt_env_power(plan, W, sig)
    torch.cuda.synchronize()
    Wc = W.cpu().numpy().astype(np.complex128)
    delta = sig.cpu().numpy().astype(np.float64)
    rp, rn, fp, fn = orc.env_power(Wc, delta)
    frac = fr.cpu().numpy()
    assert frac[0] == fp and frac[1] == fn                     # integer counts: exact
    for got, ref in ((pp.cpu().numpy(), rp), (pn.cpu().numpy(), rn)):
        nz = ref > 0
        assert np.all(got[~nz] == 0.0)
        assert np.max(np.abs(got[nz] - ref[nz]) / ref[nz]) < 1e-5
    # Eq. 43 with the zero positions added back
    zero = np.abs(Wc[:, delta == 0]) ** 2
    tot = fp * pp.cpu().numpy() + fn * pn.cpu().numpy() + zero.sum(axis=1) / N
    assert np.allclose(tot, spec.cpu().numpy(), rtol=1e-5, atol=0)
    assert torch.equal(pp, pp2) and torch.equal(pn, pn2)        # fixed-order reductions
    plan.close()


@pytest.mark.parametrize("wavelet,omega0", [("gdw", 6.0), ("morlet", 6.0), ("cbsw", 6.0),
                                            ("cwgdw", 6.0), ("morlet", 4.0)])
def test_icwt_reconstructs(env, wavelet, omega0):
    """GPU inverse over a fine log grid of scales: equal to the oracle's Eq. 5/6
    trapezoid on the same W, and back to the signal minus its mean (periodic
    multitone with whole periods, so there is no Nyquist content)."""
    torch, cwt, orc = env
    N = 1024
    f = synth.multitone(N, periods=(16.0, 128.0, 256.0), sigma=0.0)
    wt = np.exp(np.arange(math.log(2e-4), math.log(3e4), 0.04))
    plan = cwt.cwt_plan_create(N, wt, wavelet, "periodic", scale_unit="w_tilde", omega0=omega0)
    sig = torch.tensor(f, dtype=torch.float32, device="cuda")
    W = cwt.cwt_exec(plan, sig)
    rec = cwt.cwt_icwt(plan, W)
    torch.cuda.synchronize()
    ref = orc.icwt(W.cpu().numpy().astype(np.complex128), wt, wavelet, omega0=omega0, w_tilde=True)
    got = rec.cpu().numpy().astype(np.float64)
    assert rel_l2(got, ref) < 1e-5
    f32 = sig.cpu().numpy().astype(np.float64)
    floor = 10.0 * math.exp(-0.5 * omega0 ** 2) if wavelet == "morlet" else 0.0
    assert rel_l2(got, f32 - f32.mean()) < 1e-5 + floor
    plan.close()


def test_icwt_uneven_unsorted_scales_dx(env):
    """Dilations in random order, dx != 1, zero boundary: parity of the trapezoid
    weights with the oracle."""
    torch, cwt, orc = env
    N = 3000
    f = synth.lognormal_field(N, seed=11)
    rng = np.random.default_rng(5)
    sc = np.exp(rng.uniform(0.0, math.log(4000.0), 40))
    plan = cwt.cwt_plan_create(N, sc, "cwgdw", "zero", dx=0.5)
    sig = torch.tensor(f, dtype=torch.float32, device="cuda")
    W = cwt.cwt_exec(plan, sig)
    rec = cwt.cwt_icwt(plan, W)
    torch.cuda.synchronize()
    ref = orc.icwt(W.cpu().numpy().astype(np.float64), sc, "cwgdw", dx=0.5)
    assert rel_l2(rec.cpu().numpy().astype(np.float64), ref) < 1e-5
    plan.close()


def test_stats_argument_checks(env):
    torch, cwt, _ = env
    plan = cwt.cwt_plan_create(64, [4.0], "gdw", "periodic")
    W = plan.empty_output()
    with pytest.raises(cwt.CwtError):
        cwt.cwt_icwt(plan, W)                                   # one scale: no integral
    with pytest.raises(ValueError):
        cwt.cwt_env_power(plan, W, torch.zeros(63, device="cuda"))
    plan.close()
