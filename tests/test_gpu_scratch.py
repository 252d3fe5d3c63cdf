"""Plans with caller-supplied scratch (cwt_plan_opts.scratch = CWT_SCRATCH_CALLER,
cwt_exec_scratch): the same FFTCWT (Sec. 3.1, Eqs. 8-10) and power spectrum
(Eq. 42) as a plan with its own buffers, bit for bit, whatever scratch a call
brings; the argument checks of the caller-scratch entry points."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

CASES = [
    # (N, scales, wavelet, boundary, extra options): every plan structure
    (1 << 16, np.geomspace(2.0, 2.0 ** 14, 24), "morlet", "periodic", {}),          # band + wide
    (1 << 16, np.geomspace(2.0, 2.0 ** 14, 24), "gdw", "zero", {}),                 # child plan + edges
    (50001, np.geomspace(2.0, 12500.0, 20), "gdw", "zero", {}),                     # sub-plans by length
    (30001, np.geomspace(4.0, 7500.0, 20), "morlet", "periodic", {}),               # extended signal
    (3001, np.geomspace(1.0, 750.0, 12), "cbsw", "periodic", {}),                   # Bluestein rows
    (3001, np.geomspace(0.7, 750.0, 12), "gdw", "periodic", {}),                    # Bluestein + extended
    (1 << 21, np.geomspace(2.0, 64.0, 6), "morlet", "periodic", {"wide2_kernel": 1}),    # tile pipeline (TMA map of Y)
    (1 << 20, np.geomspace(2.0, 64.0, 6), "gdw", "zero", {"precision": "fp16x3"}),       # tensor-core pass 2
]


@pytest.fixture(scope="module")
def cwt():
    import paper_2302_03909_gb300 as m
    return m


@pytest.mark.parametrize("case", range(len(CASES)))
def test_caller_scratch_equals_own_scratch(cwt, case):
    import torch
    N, sc, wav, bnd, extra = CASES[case]
    f = torch.tensor(synth.lognormal_field(N, seed=700 + case), dtype=torch.float32, device="cuda")
    own = cwt.cwt_plan_create(N, sc, wav, bnd, **extra)
    W0, P0 = cwt.cwt_exec_with_power(own, f)
    cal = cwt.cwt_plan_create(N, sc, wav, bnd, scratch="caller", **extra)
    nbytes = cwt.cwt_plan_scratch_bytes(cal)
    assert nbytes > 0 and cwt.cwt_plan_scratch_bytes(own) == 0
    # the caller plan holds its tables only
    assert cwt.cwt_plan_info(cal)[1] < cwt.cwt_plan_info(own)[1]
    s = torch.cuda.current_stream()
    for k in range(2):
        # a fresh scratch each call, filled with NaN: nothing may be read before it is written
        scratch = torch.full(((nbytes + 7) // 8 + 32 * k,), float("nan"), dtype=torch.float64, device="cuda")
        W = cal.empty_output("cuda")
        P = torch.empty(cal.n_scales, dtype=torch.float64, device="cuda")
        cwt.cwt_exec_scratch(cal, f, W, P, scratch, s)
        torch.cuda.synchronize()
        assert torch.equal(W, W0), k
        assert torch.equal(P, P0), k
    # no power spectrum
    W = cal.empty_output("cuda")
    cwt.cwt_exec_scratch(cal, f, W, None, scratch, s)
    torch.cuda.synchronize()
    assert torch.equal(W, W0)
    own.close()
    cal.close()


def test_caller_scratch_argument_checks(cwt):
    import torch
    N = 1 << 14
    sc = np.geomspace(2.0, 2.0 ** 12, 8)
    f = torch.randn(N, device="cuda")
    cal = cwt.cwt_plan_create(N, sc, "morlet", "periodic", scratch="caller")
    own = cwt.cwt_plan_create(N, sc, "morlet", "periodic")
    nbytes = cwt.cwt_plan_scratch_bytes(cal)
    W = cal.empty_output("cuda")
    scratch = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    for bad in (lambda: cwt.cwt_exec_with_power(cal, f, W),              # needs its scratch
                lambda: cwt.cwt_exec(cal, f, W),
                lambda: cwt.cwt_exec_scratch(own, f, W, None, scratch),   # has its own
                lambda: cwt.cwt_exec_scratch(cal, f, W, None, scratch[: nbytes - 256]),   # too small
                lambda: cwt.cwt_exec_scratch(cal, f, W, None, scratch[8:]),               # misaligned
                lambda: cwt.cwt_batch_create([(cal, f, W, None)])):
        with pytest.raises(cwt.CwtError) as e:
            bad()
        assert e.value.status == 1
    cwt.cwt_exec_scratch(cal, f, W, None, scratch)
    torch.cuda.synchronize()
    W0 = cwt.cwt_exec(own, f)
    torch.cuda.synchronize()
    assert torch.equal(W, W0)
    cal.close()
    own.close()
