"""The tensor-core forms of the 1024-point DFT stages (cwt_precision: the
second pass of the wide-band scales as 32-point DFT-matrix products with FP32
accumulation) against the FP64 oracle, per wavelet and boundary.

Gates (relative L2 over the whole W array): the FP16 hi + lo form keeps about
22 bits per product and is held to the FP32 gate, 1e-5; the single-product
FP16 and BF16 forms to the reduced-precision gate, 3e-3 before any
refinement; the BF16 hi + lo form (about 16 bits) to 1e-4.  Rows that do not
go through the wide path are computed by the FP32 kernels and must equal the
FP32 plan's rows bit for bit.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
GATE = {"fp16x3": 1e-5, "bf16x3": 1e-4, "fp16": 3e-3, "bf16": 3e-3}


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


def f32(f):
    return np.asarray(f, dtype=np.float32).astype(np.float64)


def run(env, f, sc, wavelet, boundary, precision):
    torch, cwt, _ = env
    plan = cwt.cwt_plan_create(len(f), sc, wavelet, boundary, precision=precision)
    sig = torch.tensor(f, dtype=torch.float32, device="cuda")
    W, spec = cwt.cwt_exec_with_power(plan, sig)
    torch.cuda.synchronize()
    M = plan.M
    plan.close()
    return W.cpu().numpy(), spec.cpu().numpy(), M


@pytest.mark.parametrize("wavelet", ["gdw", "morlet"])
@pytest.mark.parametrize("boundary", ["periodic", "zero"])
def test_precision_forms_against_oracle(env, wavelet, boundary):
    """N = 2^16, 24 scales: the smallest dilations have bands of more than 4096
    bins and take the two-pass path whose second pass runs on the tensor cores
    (the zero boundary's padded plan with the crop, its periodic child plan
    without)."""
    _, _, orc = env
    N = 1 << 16
    f = synth.lognormal_field(N, seed=77)
    sc = synth.log_scales(2.0 if wavelet == "gdw" else 4.0, N / 4, 24)
    W32, sp32, M = run(env, f, sc, wavelet, boundary, "fp32")
    ref = orc.cwt_fft(f32(f), sc, wavelet, M=M if boundary == "zero" else N)
    assert rel_l2(W32.astype(np.complex128), ref) <= 1e-5
    rows_tc = None
    for form, gate in GATE.items():
        W, sp, _ = run(env, f, sc, wavelet, boundary, form)
        err = rel_l2(W.astype(np.complex128), ref)
        worst = max(np.linalg.norm(W[s] - ref[s]) / np.linalg.norm(ref[s]) for s in range(len(sc)))
        print(f"{wavelet}/{boundary} {form}: rel-L2 {err:.2e}, worst row {worst:.2e}")
        assert err <= gate, (form, err)
        same = [s for s in range(len(sc)) if np.array_equal(W[s], W32[s])]
        rows_tc = [s for s in range(len(sc)) if s not in same] if rows_tc is None else rows_tc
        # only the wide rows differ from the FP32 plan, and the same rows for every form
        assert [s for s in range(len(sc)) if not np.array_equal(W[s], W32[s])] == rows_tc
        P = orc.wavelet_power(ref)
        assert np.max(np.abs(sp - P) / P) <= 10 * gate
    assert len(rows_tc) >= 2, "no row went through the tensor-core pass"


@pytest.mark.parametrize("form", sorted(GATE))
def test_precision_forms_bench_workload_1m(env, form):
    """N = 2^20 lognormal field, Morlet omega0 = 6, 64 scales, both boundaries:
    the whole array against the oracle."""
    _, _, orc = env
    name = "lognormal_n1m_morlet_s64"
    f = synth.workload_signal(name)
    sc = synth.workload_scales(name)
    for boundary in ("periodic", "zero"):
        W, sp, M = run(env, f, sc, "morlet", boundary, form)
        ref = orc.cwt_fft(f32(f), sc, "morlet", M=M if boundary == "zero" else len(f))
        err = rel_l2(W.astype(np.complex128), ref)
        print(f"{name}/{boundary} {form}: rel-L2 {err:.2e}")
        assert err <= GATE[form]


def test_precision_forms_repeat_bitwise_and_batch(env):
    """A tensor-core plan gives the same W on every call, and the same W as
    one plan of a grouped batch."""
    torch, cwt, _ = env
    N = 1 << 15
    f = synth.lognormal_field(N, seed=5)
    sc = synth.log_scales(4.0, N / 4, 12)
    sig = torch.tensor(f, dtype=torch.float32, device="cuda")
    for form in ("fp16", "fp16x3"):
        plan = cwt.cwt_plan_create(N, sc, "morlet", "zero", precision=form)
        W0, s0 = cwt.cwt_exec_with_power(plan, sig)
        W1, s1 = cwt.cwt_exec_with_power(plan, sig)
        items = [(plan, sig, torch.empty_like(W0), torch.empty_like(s0))]
        b = cwt.cwt_batch_create(items, n_streams=1)
        b.exec()
        torch.cuda.synchronize()
        assert torch.equal(W0, W1) and torch.equal(s0, s1)
        assert torch.equal(W0, items[0][2]) and torch.equal(s0, items[0][3])
        b.close()
        plan.close()


def test_precision_option_is_checked(env):
    _, cwt, _ = env
    with pytest.raises(KeyError):
        cwt.cwt_plan_create(1024, [4.0], "gdw", "periodic", precision="fp8")
