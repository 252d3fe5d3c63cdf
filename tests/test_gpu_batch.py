"""Grouped batches (cwt_batch_*): the launches of many plans merged by kernel
and dependency level give, bit for bit, the W and spectra of one direct call
per plan, on every code path a plan can take (band and two-pass wide scales,
the zero boundary with its short-wavelet child plan, periodic lengths that are
not powers of two, all four wavelets, f64 input, no power spectrum)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_03909_gb300 as cwt
    cwt.load_library()
    return torch, cwt


def _items(torch, cwt, seed, n):
    rng = np.random.default_rng(seed)
    cases = [
        # N, wavelet, boundary, dtype, power
        (3000, "morlet", "zero", "f32", True),
        (4096, "gdw", "periodic", "f32", True),
        (1 << 15, "morlet", "periodic", "f32", True),      # wide two-pass scales
        (1 << 15, "gdw", "zero", "f64", True),             # M = 2^16, child plan for short rows
        (5000, "gdw", "periodic", "f32", True),            # periodic extension sub-plans
        (20011, "morlet", "periodic", "f32", False),       # prime N, no spectrum
        (4096, "cbsw", "periodic", "f32", True),
        (2000, "cwgdw", "zero", "f32", True),
        (1 << 17, "gdw", "periodic", "f32", True),
        (64, "morlet", "zero", "f32", True),
    ]
    while len(cases) < n:
        N = int(round(np.exp(rng.uniform(np.log(1024), np.log(65536)))))
        cases.append((N, "gdw" if rng.random() < 0.5 else "morlet",
                      "periodic" if rng.random() < 0.5 else "zero", "f32", True))
    items = []
    for i, (N, wav, bnd, dt, power) in enumerate(cases[:n]):
        smin = 2.0 if wav in ("gdw", "cbsw", "cwgdw") else 4.0
        S = int(rng.integers(6, 24))
        sc = np.exp(np.linspace(np.log(smin), np.log(max(N / 4, 2 * smin)), S))
        p = cwt.cwt_plan_create(N, sc, wav, bnd, input_dtype=dt)
        tdt = torch.float64 if dt == "f64" else torch.float32
        sig = torch.tensor(synth.multitone(N, seed=seed * 1000 + i), dtype=tdt, device="cuda")
        sp = torch.empty(S, dtype=torch.float64, device="cuda") if power else None
        items.append((p, sig, p.empty_output("cuda"), sp))
    return items


def _reference(torch, cwt, items):
    ref = []
    for p, sig, _, sp in items:
        if sp is not None:
            ref.append(cwt.cwt_exec_with_power(p, sig))
        else:
            ref.append((cwt.cwt_exec(p, sig), None))
    torch.cuda.synchronize()
    return ref


@pytest.mark.parametrize("n_streams", [1, 4])
def test_batch_equals_direct_calls(env, n_streams):
    torch, cwt = env
    items = _items(torch, cwt, 5, 24)
    ref = _reference(torch, cwt, items)
    b = cwt.cwt_batch_create(items, n_streams=n_streams)
    info = b.info()
    assert info["launches"] < info["plan_launches"]
    assert info["levels"] >= 2 and info["ctas"] > 0
    st = torch.cuda.Stream()
    for _ in range(2):                       # a second run rewrites the same results
        for _, _, W, sp in items:
            W.fill_(float("nan"))
            if sp is not None:
                sp.fill_(float("nan"))
        torch.cuda.synchronize()
        with torch.cuda.stream(st):
            b.exec(st)
        torch.cuda.synchronize()
        for (W0, s0), (p, _, W, sp) in zip(ref, items):
            assert torch.equal(W, W0), (p.N, p.n_scales)
            if sp is not None:
                assert torch.equal(sp, s0), (p.N, p.n_scales)
    b.close()
    for p, *_ in items:
        p.close()


def test_batch_of_one_and_against_the_oracle(env):
    """A single-plan batch against the FP64 oracle directly (N = 3000, zero
    boundary, M = 8192)."""
    torch, cwt = env
    import oracle
    oracle.build()
    N = 3000
    f = synth.lognormal_field(N, seed=17)
    sc = synth.log_scales(4.0, 700.0, 9)
    p = cwt.cwt_plan_create(N, sc, "morlet", "zero")
    sig = torch.tensor(f, dtype=torch.float32, device="cuda")
    W = p.empty_output("cuda")
    sp = torch.empty(len(sc), dtype=torch.float64, device="cuda")
    b = cwt.cwt_batch_create([(p, sig, W, sp)], n_streams=2)
    b.exec()
    torch.cuda.synchronize()
    ref = oracle.cwt_fft(np.asarray(f, dtype=np.float32).astype(np.float64), sc, "morlet", M=p.M)
    got = W.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    P = oracle.wavelet_power(ref)
    assert np.max(np.abs(sp.cpu().numpy() - P) / P) < 1e-4
    b.close()
    p.close()


def test_batch_argument_checks(env):
    torch, cwt = env
    items = _items(torch, cwt, 9, 2)
    with pytest.raises(cwt.CwtError) as e:
        cwt.cwt_batch_create([items[0], items[0]])              # a plan twice
    assert e.value.status == 1
    with pytest.raises(cwt.CwtError) as e:
        cwt.cwt_batch_create(items, n_streams=0)
    assert e.value.status == 1
    with pytest.raises(cwt.CwtError) as e:
        cwt.cwt_batch_create(items, n_streams=9)
    assert e.value.status == 1
    cwt.cwt_plan_set_timing(items[1][0], True)
    with pytest.raises(cwt.CwtError) as e:
        cwt.cwt_batch_create(items)
    assert e.value.status == 1
    cwt.cwt_plan_set_timing(items[1][0], False)
    lib = cwt.load_library()
    assert lib.cwt_batch_exec(None, None) == 1
    assert lib.cwt_batch_info(None, None, None, None, None) == 1
    assert lib.cwt_batch_destroy(None) == 0
    for p, *_ in items:
        p.close()


def test_batch_with_bluestein_plans(env):
    """Periodic plans of lengths that are not powers of two, with rows of the
    Bluestein form (CBSW, CW-GDW, a scale whose spectrum reaches the Nyquist
    frequency) beside extended-signal rows, in one batch: bit-equal to direct
    calls."""
    torch, cwt = env
    specs = [(1000, "cbsw", 1.0, 250.0, 7), (3001, "cwgdw", 1.0, 700.0, 6), (1023, "morlet", 0.6, 300.0, 6),
             (5000, "gdw", 0.5, 1200.0, 8)]
    items = []
    for i, (N, wav, lo, hi, S) in enumerate(specs):
        p = cwt.cwt_plan_create(N, synth.log_scales(lo, hi, S), wav, "periodic")
        sig = torch.tensor(synth.multitone(N, seed=40 + i), dtype=torch.float32, device="cuda")
        items.append((p, sig, p.empty_output("cuda"), torch.empty(S, dtype=torch.float64, device="cuda")))
    ref = _reference(torch, cwt, items)
    b = cwt.cwt_batch_create(items, n_streams=3)
    st = torch.cuda.Stream()
    for _, _, W, sp in items:
        W.fill_(float("nan"))
        sp.fill_(float("nan"))
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        b.exec(st)
    torch.cuda.synchronize()
    for (W0, s0), (p, _, W, sp) in zip(ref, items):
        assert torch.equal(W, W0), p.N
        assert torch.equal(sp, s0), p.N
    b.close()
    for p, *_ in items:
        p.close()
