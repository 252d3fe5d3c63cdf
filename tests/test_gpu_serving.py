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
