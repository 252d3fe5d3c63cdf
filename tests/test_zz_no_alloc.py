"""The allocation-free power spectrum (cwt_wavelet_power_noalloc) against the
plan-based cwt_wavelet_power on the same W arrays.

Some callers cannot allocate device memory when they need the spectrum (their
device memory is all owned by another allocator, or the loop must not pay for
cudaMalloc's synchronisation); this entry point serves them from a fixed array
inside the library.  Two calls in a row with different shapes check that the
shared scratch carries nothing over from one call to the next.  Both entry
points run the same row and finalise kernels in the same fixed order, so the
spectra must be equal bit for bit.  The device's free memory is the same
before and after repeated calls (after a first call has loaded the kernels).
This file is collected last on purpose, and it also passes when run on its
own.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_power_matches_plan_power():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_03909_gb300 as cwt

    cases = [(1 << 16, "morlet", "zero", 10), (100_003, "gdw", "zero", 7)]
    results = []
    for N, wavelet, boundary, S in cases:
        f = synth.lognormal_field(N, seed=N)
        plan = cwt.cwt_plan_create(N, synth.log_scales(2.0, N / 8.0, S), wavelet, boundary)
        sig = torch.tensor(f, dtype=torch.float32, device="cuda")
        W = cwt.cwt_exec(plan, sig)
        ref = cwt.cwt_wavelet_power(plan, W)
        got = torch.full((S,), float("nan"), dtype=torch.float64, device="cuda")
        cwt.cwt_wavelet_power_noalloc(W, got)
        torch.cuda.synchronize()
        results.append((ref.cpu().numpy(), got.cpu().numpy(), W))
        plan.close()
    for ref, got, _ in results:
        assert np.all(np.isfinite(got))
        assert np.array_equal(got, ref)
    # no allocation: repeated calls leave the device's free memory unchanged
    W = results[1][2]
    sp = torch.empty(W.shape[0], dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(20):
        cwt.cwt_wavelet_power_noalloc(W, sp)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert np.array_equal(sp.cpu().numpy(), results[1][1])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_03909_gb300 as cwt
    lib = cwt.load_library()
    W = torch.zeros(4, dtype=torch.float32, device="cuda")
    sp = torch.zeros(129, dtype=torch.float64, device="cuda")
    # 129 rows x 512 chunks of 2^24 samples exceed the 65536 partial sums; rejected before any launch
    st = lib.cwt_wavelet_power_noalloc(ctypes.c_void_p(W.data_ptr()), 1 << 24, 129, 0,
                                       ctypes.c_void_p(sp.data_ptr()), None)
    assert st == 2
    assert lib.cwt_wavelet_power_noalloc(None, 10, 1, 0, ctypes.c_void_p(sp.data_ptr()), None) == 1


def test_noalloc_rejects_memory_that_is_not_on_the_current_device():
    """Host memory (pinned or not) is refused before any launch: the kernels
    would address memory the device cannot reach."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_03909_gb300 as cwt
    lib = cwt.load_library()
    W = torch.zeros(2, 64, dtype=torch.float32, device="cuda")
    sp = torch.zeros(2, dtype=torch.float64, device="cuda")
    Wh = torch.zeros(2, 64, dtype=torch.float32).pin_memory()
    sh = np.zeros(2, dtype=np.float64)
    assert lib.cwt_wavelet_power_noalloc(ctypes.c_void_p(Wh.data_ptr()), 64, 2, 0,
                                         ctypes.c_void_p(sp.data_ptr()), None) == 1
    assert lib.cwt_wavelet_power_noalloc(ctypes.c_void_p(W.data_ptr()), 64, 2, 0,
                                         ctypes.c_void_p(sh.ctypes.data), None) == 1
    with pytest.raises(ValueError):
        cwt.cwt_wavelet_power_noalloc(W, sp.cpu())
