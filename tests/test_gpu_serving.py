"""The request server on the GPU: every request served in a mixed,
concurrent trace gives the same W and spectrum, bit for bit, as the same
transform run alone."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_served_results_equal_standalone():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_03909_gb300 as cwt
    from paper_2302_03909_gb300 import serving
    trace = serving.poisson_trace(2000.0, 0.02, seed=11, log2n=(10, 15), n_scales=(8, 24))
    assert len(trace) >= 20
    sig = {}
    for r in trace:
        if r.N not in sig:
            sig[r.N] = torch.tensor(synth.lognormal_field(r.N, seed=r.N), dtype=torch.float32).pin_memory()
        r.signal = sig[r.N]
    srv = serving.Server(budget_bytes=4 << 30, slots=4, keep_results=True)
    stats = serving.run_trace(srv, trace, max_seconds=120.0)
    assert stats["requests"] == len(trace)
    for r in srv.completed:
        plan = cwt.cwt_plan_create(r.N, np.asarray(r.scales), r.wavelet, r.boundary)
        W, sp = cwt.cwt_exec_with_power(plan, r.signal.cuda())
        torch.cuda.synchronize()
        assert torch.equal(W, r.W) and torch.equal(sp, r.spectrum), r.rid
        plan.close()
    srv.close()


def test_served_with_caller_scratch_equals_standalone():
    """Integer lengths (most not powers of two) and no buffers owned by plan
    instances: every request runs its plan with caller scratch
    (cwt_exec_scratch, a scratch per request) and still equals, bit for bit,
    a plan with its own scratch run alone."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_03909_gb300 as cwt
    from paper_2302_03909_gb300 import serving
    trace = serving.poisson_trace(2000.0, 0.02, seed=12, log2n=(10, 16), n_scales=(8, 24), integer_lengths=2)
    assert len(trace) >= 20 and any(r.N & (r.N - 1) for r in trace)
    sig = {}
    for r in trace:
        if r.N not in sig:
            sig[r.N] = torch.tensor(synth.lognormal_field(r.N, seed=r.N), dtype=torch.float32).pin_memory()
        r.signal = sig[r.N]
    srv = serving.Server(budget_bytes=4 << 30, slots=4, keep_results=True, reuse_max_bytes=0)
    stats = serving.run_trace(srv, trace, max_seconds=120.0)
    assert stats["requests"] == len(trace)
    assert all(v > 0 for v in srv.scratch_known.values())
    for r in srv.completed:
        plan = cwt.cwt_plan_create(r.N, np.asarray(r.scales), r.wavelet, r.boundary)
        W, sp = cwt.cwt_exec_with_power(plan, r.signal.cuda())
        torch.cuda.synchronize()
        assert torch.equal(W, r.W) and torch.equal(sp, r.spectrum), r.rid
        plan.close()
    srv.close()


def test_batch_graph_equals_direct_calls():
    """A batch of uneven lengths (periodic lengths that are not powers of two
    included) captured as one CUDA graph and replayed gives the same W and
    spectra, bit for bit, as one direct call per signal."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_03909_gb300 as cwt
    from paper_2302_03909_gb300 import serving
    rng = np.random.default_rng(4)
    items, ref = [], []
    for i in range(12):
        N = int(rng.integers(1000, 20000))
        wav = "gdw" if i % 2 else "morlet"
        bnd = "periodic" if (i // 2) % 2 else "zero"
        sc = np.exp(np.linspace(np.log(2.0 if wav == "gdw" else 4.0), np.log(N / 4), int(rng.integers(6, 20))))
        p = cwt.cwt_plan_create(N, sc, wav, bnd)
        sig = torch.tensor(synth.multitone(N, seed=i), dtype=torch.float32, device="cuda")
        W0, s0 = cwt.cwt_exec_with_power(p, sig)
        ref.append((W0, s0))
        items.append((p, sig, p.empty_output("cuda"), torch.empty(len(sc), dtype=torch.float64, device="cuda")))
    torch.cuda.synchronize()
    g = serving.capture_batch(items, n_streams=3)
    for _ in range(2):
        for _, _, W, sp in items:
            W.zero_()
            sp.zero_()
        g.replay()
        torch.cuda.synchronize()
        for (W0, s0), (_, _, W, sp) in zip(ref, items):
            assert torch.equal(W, W0) and torch.equal(sp, s0)
    del g
    for p, *_ in items:
        p.close()


@pytest.mark.parametrize("N,wavelet,boundary,smin,smax,S", [
    (1 << 10, "gdw", "periodic", 2.0, 256.0, 16),
    (1 << 16, "morlet", "zero", 4.0, 1 << 14, 64),
    (5000, "gdw", "periodic", 2.0, 1250.0, 40),
    (70001, "morlet", "periodic", 4.0, 17500.0, 96),
    (70001, "gdw", "zero", 2.0, 17500.0, 96),
    (1 << 22, "morlet", "zero", 4.0, 1 << 20, 128),
    (1 << 24, "gdw", "periodic", 2.0, 1 << 22, 16),
])
def test_workspace_bound_covers_the_plans(N, wavelet, boundary, smin, smax, S):
    """The admission charges a never-seen shape serving.workspace_bound until
    its plan exists: the bound must cover the plan's real workspace."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_03909_gb300 as cwt
    from paper_2302_03909_gb300 import serving
    sc = tuple(float(x) for x in np.geomspace(smin, smax, S))
    p = cwt.cwt_plan_create(N, np.asarray(sc), wavelet, boundary)
    ws = p.workspace_bytes
    p.close()
    assert 0 < ws <= serving.workspace_bound(N, sc, wavelet, boundary)
