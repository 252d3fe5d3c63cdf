"""Host-side pieces of bench.py that need no GPU."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def test_traffic_scales_with_the_launch_size():
    """The profiled DRAM bytes per pass-2 launch apply to launches of the same
    algorithmic size; a launch with half the jobs is charged half."""
    full = bench.load_traffic("wide2", "lognormal_n4m_s128", 134217728.0)
    half = bench.load_traffic("wide2", "lognormal_n4m_s128", 67108864.0)
    assert full is not None and abs(full - 216036096.0) < 1.0
    assert abs(half - full / 2) < 1.0
    assert bench.load_traffic("forward", "lognormal_n4m_s128", 1.0) is None
    # no capture of the current pass-2 kernel on this workload: no traffic figure
    assert bench.load_traffic("wide2", "lognormal_n1m_morlet_s64", 26.0e6) is None
    assert bench.load_traffic("wide2", "no_such_workload", 1.0) is None


def test_weak_scaling_value_counts_all_ranks():
    # 4 steps of 1000 units on each of 2 ranks in 8 ms (max over ranks)
    assert abs(bench.weak_scaling_value(1000.0, 4, 2, 8.0) - 1.0e6) < 1e-6


def test_batch_cpu_baseline_times_a_bounded_sample():
    import numpy as np
    from paper_2302_03909_gb300 import serving
    reqs = []
    for i, (N, wav, bnd) in enumerate([(300, "gdw", "periodic"), (257, "morlet", "zero"), (512, "gdw", "zero")]):
        r = serving.Request(i, N, tuple(np.geomspace(2.0, N / 4, 5)), wav, bnd, 0.0)
        r.signal = np.random.default_rng(i).standard_normal(N).astype(np.float32)
        reqs.append(r)
    cb = bench.batch_cpu_baseline(reqs, 0.0)          # stops after the first signal
    assert cb["value"] > 0 and cb["kind"] == "oracle" and cb["cores"] >= 1
    assert cb["sample"].startswith("the first 1 of 3 signals (1500 scale-samples)")
    cb = bench.batch_cpu_baseline(reqs, 60.0)
    assert cb["sample"].startswith("the first 3 of 3 signals")


def test_default_workload_runs_both_wavelets_and_boundaries_at_n4m_s128():
    """The default step is the N = 2^22, 128-scale field under the GDW and the
    Morlet, each with the periodic and the zero boundary."""
    import synth
    parts = bench.workload_parts(bench.DEFAULT_WORKLOAD)
    assert sorted(synth.WORKLOADS[q]["wavelet"] for q in parts) == ["gdw", "morlet"]
    for q in parts:
        w = synth.WORKLOADS[q]
        assert w["n"] == 1 << 22 and w["n_scales"] == 128
        assert tuple(w["boundaries"]) == ("periodic", "zero")
    sigs = [synth.workload_signal(q) for q in parts]
    assert all((s == sigs[0]).all() for s in sigs)       # one field, transformed four ways
    assert bench.workload_parts("lognormal_n1m_morlet_s64") == ("lognormal_n1m_morlet_s64",)
