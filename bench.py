#!/usr/bin/env python
"""Throughput of the GB300 FFTCWT in scale-samples/s.

Default workload: one N = 2^22 float32 lognormal density field at 128
log-spaced scales, transformed with the Mexican-hat-type GDW (dilations 2 ..
2^20) and with the Morlet wavelet (omega0 = 6, dilations 4 .. 2^20), each with
the periodic AND the zero boundary (zero padding to M = 2^23), each with the
fused wavelet power spectrum.  One step = these four transforms.  Inputs are
resident in HBM when the timed region starts; the L2 is flushed (a 512 MiB
write) between timed steps, outside the timed events.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on the
host cores instead (a bounded sample of the same workload per step).
Multi-GPU (torchrun): every rank transforms its own signal; no collective is
on the data path (weak scaling); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "CWT scale-samples/s"
UNIT = "scale-samples/s"

# Bench workloads: a named workload of synth, or several run in one step.
COMPOSITE = {
    # N = 2^22, 128 scales: GDW and Morlet, both boundaries (four transforms per step)
    "lognormal_n4m_s128": ("lognormal_n4m_gdw_s128", "lognormal_n4m_morlet_s128"),
}
DEFAULT_WORKLOAD = "lognormal_n4m_s128"


def workload_parts(name: str) -> tuple:
    """The synth workloads a bench workload runs in one step."""
    return COMPOSITE.get(name, (name,))


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(synth.WORKLOADS) + sorted(COMPOSITE))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="default launch shape instead of the plan-time tuning (cwt_plan_opts.tune)")
    ap.add_argument("--no-fft-baseline", action="store_true",
                    help="skip the comparison with the library FFT (torch.fft / cuFFT) written the usual way")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-batch", action="store_true",
                    help="default run: skip the embedded batch measurement (--batch-signals signals)")
    ap.add_argument("--no-serving", action="store_true",
                    help="default run: skip the embedded serving measurement (a short trace)")
    ap.add_argument("--precisions", default="fp16x3,bf16x3,fp16,bf16",
                    help="tensor-core forms of the 1024-point DFT stages timed beside FP32 (comma list; "
                         "empty: none)")
    # narrower cases of a workload for profiler captures (not a bench line)
    ap.add_argument("--wide2-kernel", type=int, default=0, choices=[0, 1, 2],
                    help="FP32 pass 2 of the wide scales: 1 tile pipeline, 2 CTA Stockham kernel, 0 library default")
    ap.add_argument("--boundary", default="both", choices=["both", "periodic", "zero"],
                    help="run one boundary of the workload only")
    ap.add_argument("--scale-range", type=int, nargs=2, metavar=("I", "J"),
                    help="keep the workload's scales I..J-1 only (ascending dilation)")
    # serving: a Poisson trace of requests through paper_2302_03909_gb300.serving
    ap.add_argument("--serving", action="store_true", help="measure request latency instead of throughput")
    ap.add_argument("--rate", type=float, default=500.0, help="serving: requests per second")
    ap.add_argument("--max-wait", type=float, default=0.1,
                    help="serving, smallest-first policy: a request older than this (s) goes first")
    ap.add_argument("--serving-lengths", default="integer", choices=["integer", "pow2"],
                    help="serving: signal lengths log-uniform integers (2 per octave) or powers of two")
    ap.add_argument("--seconds", type=float, default=5.0, help="serving: length of the arrival trace")
    ap.add_argument("--slots", type=int, default=4, help="serving: requests in flight at once")
    ap.add_argument("--budget-gb", type=float, default=120.0, help="serving: device-memory budget")
    ap.add_argument("--policy", default="smallest", choices=["fifo", "smallest"],
                    help="serving: admission order of the concurrent run (smallest first, 0.1 s maximum wait by default)")
    ap.add_argument("--fresh-buffers", action="store_true",
                    help="serving: new device buffers per request (direct launches) instead of per-instance buffers")
    # batching: many signals of uneven lengths, each with its own plan
    ap.add_argument("--batch", action="store_true", help="measure a batch of uneven-length signals")
    ap.add_argument("--batch-signals", type=int, default=512, help="batch: number of signals")
    ap.add_argument("--batch-streams", type=int, default=16, help="batch: streams the graph spreads the signals over")
    ap.add_argument("--batch-min-ctas", type=int, default=1,
                    help="batch: the plans' min_ctas option (1: up to 8 tiles per CTA)")
    ap.add_argument("--batch-streams-grouped", type=int, default=4,
                    help="batch: streams a level of the batch API's grouped launches is spread over")
    return ap.parse_args()


def workload_subset(args, part=None):
    """(boundaries, scales) of one part of the workload after --boundary /
    --scale-range, and a description of the subset (None for the whole
    workload)."""
    part = part or workload_parts(args.workload)[0]
    w = synth.WORKLOADS[part]
    bounds = tuple(w["boundaries"]) if args.boundary == "both" else (args.boundary,)
    sc = synth.workload_scales(part)
    note = []
    if args.boundary != "both":
        note.append(f"{args.boundary} boundary only")
    if args.scale_range:
        i, j = args.scale_range
        sc = sc[i:j]
        note.append(f"scales {i}..{j - 1} of {w['n_scales']}")
    if not len(sc) or not bounds:
        raise SystemExit("empty workload subset")
    return bounds, sc, ("; ".join(note) if note else None)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def load_traffic(kernel: str, workload: str, alg_bytes_per_launch: float):
    """DRAM bytes per launch from the committed ncu summary, if one exists for
    this kernel class and workload (profiles/traffic.txt: kernel, workload, DRAM
    bytes per launch and algorithmic bytes per launch of the profiled launches),
    scaled to this run's launches by their algorithmic bytes (the launch size
    depends on the plan's launch shape; the traffic grows with the jobs a launch
    takes)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        for line in fh:
            parts = line.split()
            if len(parts) >= 4 and not line.startswith("#") and parts[0] == kernel and parts[1] == workload:
                return float(parts[2]) * alg_bytes_per_launch / float(parts[3])
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def rank_signal(name: str, rank: int, world: int) -> np.ndarray:
    """The workload signal of one replica: rank 0 (and single-GPU runs) use the
    workload's own seed, other ranks an independent seed of the same recipe."""
    if world <= 1 or rank == 0:
        return synth.workload_signal(name)
    w = synth.WORKLOADS[name]
    seed = synth.BASE_SEED + 100 + rank
    return synth.lognormal_field(w["n"], seed=seed) if "lognormal" in name else synth.multitone(w["n"], seed=seed)


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank time over all ranks (a no-op without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_step: float, steps: int, world: int, total_ms: float) -> float:
    """Whole-job throughput: every rank processes units_per_step per step."""
    return world * units_per_step * steps / (total_ms * 1e-3)


def cpu_baseline(name, budget_s, steps=1, warmup=0):
    """The FP64 oracle (FFT tier) on the host cores over a bounded sample of the
    workload: evenly spread scales of every transform of the step (each wavelet
    and boundary), sized to about budget_s per sample."""
    import oracle
    oracle.build()
    parts = workload_parts(name)
    cores = os.cpu_count() or 1
    runs = []                            # (wavelet, M, scales) of every transform of the step
    for part in parts:
        w = synth.WORKLOADS[part]
        N = w["n"]
        for b in w["boundaries"]:
            M = N if b == "periodic" else 1 << int(np.ceil(np.log2(2 * N)))
            runs.append((w["wavelet"], M, synth.workload_scales(part)))
    f = synth.workload_signal(parts[0]).astype(np.float32).astype(np.float64)
    N = len(f)
    # calibrate on one scale per transform
    t0 = time.perf_counter()
    for wav, M, sc in runs:
        oracle.cwt_fft(f, sc[:1], wav, M=M, nthreads=cores)
    per_scale = time.perf_counter() - t0
    # OpenMP runs the scales in parallel: a batch of `cores` scales costs about one scale
    n_batches = max(1, int(budget_s / max(per_scale, 1e-3)))
    n_sc = len(runs[0][2])
    n_sub = int(min(n_sc, n_batches * cores))
    idx = np.linspace(0, n_sc - 1, n_sub).astype(int)
    times = []
    for it in range(warmup + steps):
        t0 = time.perf_counter()
        for wav, M, sc in runs:
            oracle.cwt_fft(f, sc[idx], wav, M=M, nthreads=cores)
        if it >= warmup:
            times.append(time.perf_counter() - t0)
    units = n_sub * N * len(runs)
    t = float(np.mean(times))
    return {"value": units / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_sub} of {n_sc} scales (evenly spread) x {len(runs)} transforms "
                      f"({', '.join(sorted({r[0] for r in runs}))}; periodic and zero boundary), "
                      f"N={N}, FP64 FFT tier, OpenMP over scales; {t:.1f} s per sample",
            "seconds": t}


def fft_library_baseline(f, sc, wavelet, plans, outs, flush, stream, steps, warmup=2):
    """The same transforms written the usual way on the GPU with the library FFT
    (torch.fft, i.e. cuFFT).  Set-up, untimed: the wavelet spectra
    sqrt(s) psi_hat(2 pi m~ s / M) of Eq. 10 for every scale, kept in HBM.
    Step: one forward FFT per boundary; per chunk of scales the product with the
    spectrum and a batched inverse FFT (C2R for the real GDW, C2C for the
    Morlet), written straight into W when M = N and cropped to the first N
    outputs otherwise; the power spectrum as row norms of W.  Timed like the
    library's steps (CUDA events on the stream, the L2 flushed between steps).
    A comparison baseline only: the library itself never calls it."""
    import torch
    dev = outs[0][0].device
    N, S = len(f), len(sc)
    real = wavelet == "gdw"
    if wavelet not in ("gdw", "morlet"):
        raise ValueError(wavelet)
    omega0 = 6.0     # the Morlet's centre wavenumber of every bench workload
    if real:   # Table 2: GDW, C_N = (18 pi)^(-1/4)
        cn = (18.0 * math.pi) ** -0.25
    else:      # Morlet with the correction term, unit energy
        cn = math.pi ** -0.25 / math.sqrt(1.0 - 2.0 * math.exp(-0.75 * omega0 ** 2) + math.exp(-omega0 ** 2))

    def psi_hat(k):
        if real:
            return (8.0 * math.sqrt(math.pi) * cn) * k * k * torch.exp(-k * k)
        return (math.sqrt(2.0 * math.pi) * cn) * (torch.exp(-0.5 * (k - omega0) ** 2)
                                                   - torch.exp(-0.5 * (k * k + omega0 ** 2)))

    sig = torch.tensor(f, dtype=torch.float32, device=dev)
    sd = torch.tensor(np.asarray(sc, dtype=np.float64), dtype=torch.float64, device=dev)
    res = []
    for p in plans:
        M = p.M
        nb = M // 2 + 1 if real else M
        mi = torch.arange(nb, device=dev, dtype=torch.float64)
        mt = mi if real else torch.where(2 * mi <= M, mi, mi - M)     # signed frequency
        chunk = max(1, min(S, (256 << 20) // (nb * 8)))
        Psi = torch.empty(S, nb, dtype=torch.float32, device=dev)
        for c0 in range(0, S, chunk):
            s_ = sd[c0:c0 + chunk, None]
            Psi[c0:c0 + chunk] = (torch.sqrt(s_) * psi_hat(mt[None, :] * (2.0 * math.pi / M) * s_)).float()
        res.append((M, chunk, Psi, p.empty_output(dev), torch.empty(S, dtype=torch.float64, device=dev)))

    def step():
        for M, chunk, Psi, W, sp in res:
            # rfft: the conjugate of the paper's e^{+} spectrum on [0, M/2]; ifft: that spectrum / M
            F = torch.fft.rfft(sig, n=M) if real else torch.fft.ifft(sig, n=M)
            for c0 in range(0, S, chunk):
                X = F[None, :] * Psi[c0:c0 + chunk]
                inv = (lambda x, **kw: torch.fft.irfft(x, n=M, **kw)) if real else torch.fft.fft
                if M == N:
                    inv(X, out=W[c0:c0 + chunk])
                else:
                    W[c0:c0 + chunk] = inv(X)[:, :N]
            torch.square(torch.linalg.vector_norm(W, dim=1).double(), out=sp)
            sp.div_(N)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    # the same outputs as the library's (its last step): like is timed against like
    err = 0.0
    err_p = 0.0
    for (M, chunk, Psi, W, sp), (Wo, spo) in zip(res, outs):
        d = torch.linalg.vector_norm((W - Wo).reshape(-1)) / torch.linalg.vector_norm(Wo.reshape(-1))
        err = max(err, float(d))
        err_p = max(err_p, float(((sp - spo).abs() / spo).max()))
    units = S * N * len(plans)
    out = {"value": units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
           "rel_l2_vs_library": err, "power_max_rel_dev_vs_library": err_p,
           "what": "torch.fft (cuFFT), FP32: wavelet spectra precomputed in HBM (untimed); per step a "
                   "forward FFT per boundary, per chunk of scales one product and a batched C2R (GDW) or "
                   "C2C (Morlet) inverse into W (cropped copy for the zero boundary), power as row norms"}
    del res
    torch.cuda.empty_cache()
    return out


def batch_cpu_baseline(reqs, budget_s: float):
    """The FP64 oracle (FFT tier, all host cores) over the batch's first
    signals, one after another, until about budget_s has passed: a bounded
    sample of the batch, reported per scale-sample."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    units, n = 0, 0
    t0 = time.perf_counter()
    for r in reqs:
        f = np.asarray(r.signal, dtype=np.float32).astype(np.float64)
        M = r.N if r.boundary == "periodic" else 1 << int(math.ceil(math.log2(2 * r.N)))
        oracle.cwt_fft(f, np.asarray(r.scales), r.wavelet, M=M, nthreads=cores)
        units += len(r.scales) * r.N
        n += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    t = time.perf_counter() - t0
    return {"value": units / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"the first {n} of {len(reqs)} signals ({units} scale-samples), FP64 FFT tier, "
                      f"OpenMP over scales; {t:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    parts = workload_parts(args.workload)
    w = synth.WORKLOADS[parts[0]]
    cb = cpu_baseline(args.workload, args.cpu_seconds / 3.0, steps=args.steps, warmup=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": cb["seconds"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "N": w["n"], "n_scales": w["n_scales"],
                   "wavelets": [synth.WORKLOADS[q]["wavelet"] for q in parts],
                   "boundaries": list(w["boundaries"]), "sample": cb["sample"]},
        "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_serving(args, embedded=False):
    """Poisson arrivals (N in 2^10..2^24: log-uniform integers from a pool of two
    per octave, or powers of two; 16..128 scales, GDW or Morlet, periodic or
    zero boundary) served with ``--slots`` streams, then the same trace with one
    slot (serial execution); plans of every request shape are created first
    (a resident plan cache).  Prints one JSON line of latency percentiles."""
    import torch

    from paper_2302_03909_gb300 import serving

    torch.cuda.set_device(0)
    per_octave = 2 if args.serving_lengths == "integer" else 0
    trace = serving.poisson_trace(args.rate, args.seconds, integer_lengths=per_octave)
    pool = {}
    for r in trace:
        if r.N not in pool:
            pool[r.N] = torch.tensor(synth.lognormal_field(r.N, seed=synth.BASE_SEED + 50 + r.N % 100003),
                                     dtype=torch.float32).pin_memory()
        r.signal = pool[r.N]
    budget = int(args.budget_gb * (1 << 30))
    out = {}
    for label, slots, policy in (("concurrent", args.slots, args.policy), ("concurrent_fifo", args.slots, "fifo"),
                                 ("serial", 1, "fifo")):
        for r in trace:
            r.t_admit = r.t_done = float("nan")
        srv = serving.Server(budget, slots=slots, plan_cache_bytes=budget // 2, max_wait_s=args.max_wait,
                             reuse_buffers=not args.fresh_buffers, policy=policy)
        keys = sorted({r.key for r in trace})
        for k in keys:                                       # resident plans
            srv.cache.release(k, srv.cache.acquire(k))
        srv.cache.hits = srv.cache.misses = 0
        # two untimed passes over the shapes (first-use costs; the second captures each
        # instance's graph), then the timed trace
        for _ in range(2):
            warm = [serving.Request(i, *k, 0.0, signal=pool[k[0]]) for i, k in enumerate(keys)]
            serving.run_trace(srv, warm)
        srv.completed.clear()
        torch.cuda.synchronize()
        out[label] = serving.run_trace(srv, [dataclasses_replace(r) for r in trace])
        srv.close()
        del srv
        torch.cuda.empty_cache()
    mean_units = float(np.mean([len(r.scales) * r.N for r in trace]))
    line = {"impl": "ours", "metric": "CWT serving latency", "unit": "ms", "higher_is_better": False,
            "p50_ms": out["concurrent"]["p50_ms"], "p99_ms": out["concurrent"]["p99_ms"],
            "serial_p50_ms": out["serial"]["p50_ms"], "serial_p99_ms": out["serial"]["p99_ms"],
            "offered_scale_samples_per_s": mean_units * len(trace) / args.seconds,
            "concurrent": out["concurrent"], "concurrent_fifo": out["concurrent_fifo"], "serial": out["serial"],
            "config": {"rate_per_s": args.rate, "seconds": args.seconds, "requests": len(trace),
                       "slots": args.slots, "policy": args.policy, "max_wait_s": args.max_wait,
                       "budget_gb": args.budget_gb,
                       "N": ("log-uniform integers in 2^10..2^24 (a pool of 2 per octave, mostly not powers "
                             "of two)" if per_octave else "2^10..2^24 (powers of two)"),
                       "distinct_shapes": len({r.key for r in trace}),
                       "n_scales": "16..128", "wavelets": ["gdw", "morlet"], "boundaries": ["periodic", "zero"],
                       "plans": "resident, created before the trace",
                       "buffers": "new per request" if args.fresh_buffers
                       else "per plan instance up to 64 MiB (graph replay), new per request above"},
            "data": "synthetic"}
    if embedded:
        return line
    print(json.dumps(line), flush=True)


def run_batch(args, embedded=False):
    """A batch of signals of uneven lengths: N log-uniform in [1024, 65536]
    (integers, mostly not powers of two), 16..96 log-spaced dilations from 2
    (GDW) or 4 (Morlet) to N/4, the wavelet and the boundary 50/50, multi-tone
    plus noise with periods scaled to N.  Each signal has its own plan, created
    first and timed apart; the inputs are resident in HBM.  Timed three ways:
    the batch API (all plans' launches merged by kernel and dependency level),
    one CUDA graph over the per-signal launch sequences on --batch-streams
    streams, and one launch sequence per signal on one stream.  Prints one
    JSON line."""
    import torch

    from paper_2302_03909_gb300 import serving

    torch.cuda.set_device(0)
    rng = np.random.default_rng(synth.BASE_SEED + 3)
    reqs = []
    for i in range(args.batch_signals):
        N = int(round(math.exp(rng.uniform(math.log(1024), math.log(65536)))))
        S = int(rng.integers(16, 97))
        wav = "gdw" if rng.random() < 0.5 else "morlet"
        bnd = "periodic" if rng.random() < 0.5 else "zero"
        smin = 2.0 if wav == "gdw" else 4.0
        sc = tuple(float(x) for x in np.exp(np.linspace(math.log(smin), math.log(N / 4), S)))
        f = synth.multitone(N, periods=tuple(p * N / 4096 for p in (16.0, 128.0, 700.0)), seed=synth.BASE_SEED + i)
        r = serving.Request(i, N, sc, wav, bnd, 0.0)
        r.signal = torch.tensor(f, dtype=torch.float32).pin_memory()
        reqs.append(r)
    units = sum(len(r.scales) * r.N for r in reqs)
    import paper_2302_03909_gb300 as cwt
    # plans (one per signal) and resident device buffers, before any timing
    t0 = time.perf_counter()
    # plans for a batch take the fewest, largest CTAs: the batch supplies the parallelism
    plans = [cwt.cwt_plan_create(r.N, np.asarray(r.scales), r.wavelet, r.boundary, min_ctas=args.batch_min_ctas)
             for r in reqs]
    torch.cuda.synchronize()
    t_plan = time.perf_counter() - t0
    items = []
    for r, p in zip(reqs, plans):
        items.append((p, r.signal.cuda(), p.empty_output("cuda"),
                      torch.empty(p.n_scales, dtype=torch.float64, device="cuda")))
    free_b, total_b = torch.cuda.mem_get_info()
    out = {"plans_s": t_plan, "device_bytes_in_use": total_b - free_b}

    def timed(fn, k=5):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(k):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b) * 1e-3)
        return float(np.median(ts))

    # one graph launch over the whole batch (captured once, replayed)
    t0 = time.perf_counter()
    graph = serving.capture_batch(items, n_streams=args.batch_streams)
    torch.cuda.synchronize()
    out["capture_s"] = time.perf_counter() - t0
    t_graph = timed(graph.replay)
    # the batch API: every plan's launches merged by kernel and dependency level
    t0 = time.perf_counter()
    batch = cwt.cwt_batch_create(items, n_streams=args.batch_streams_grouped)
    torch.cuda.synchronize()
    out["grouped_create_s"] = time.perf_counter() - t0
    out["grouped_info"] = batch.info()
    t_grouped = timed(batch.exec)
    out["grouped_s"] = t_grouped
    batch.close()
    # one launch sequence per signal, the signals one after another on one stream
    st = torch.cuda.current_stream()

    def one_by_one():
        for p, sig, W, sp in items:
            cwt.cwt_exec_with_power(p, sig, W, sp, st)
    t_seq = timed(one_by_one)
    out["graph_s"], out["one_by_one_s"] = t_graph, t_seq
    del graph
    for p in plans:
        p.close()
    cpu = None if (args.no_cpu_baseline or embedded) else batch_cpu_baseline(reqs, args.cpu_seconds)
    line = {"impl": "ours", "metric": "CWT scale-samples/s, batch of uneven lengths", "unit": "scale-samples/s",
            "higher_is_better": True, "value": units / out["grouped_s"], "graph": units / out["graph_s"],
            "one_by_one": units / out["one_by_one_s"], "cpu_baseline": cpu,
            "detail": out,
            "config": {"signals": len(reqs), "N": "log-uniform integers in [1024, 65536]", "n_scales": "16..96",
                       "scale_samples": units, "wavelets": ["gdw", "morlet"], "boundaries": ["periodic", "zero"],
                       "streams": args.batch_streams, "inputs": "resident in HBM",
                       "plans": "one per signal, created before the timed runs",
                       "grouped_streams": args.batch_streams_grouped, "plan_min_ctas": args.batch_min_ctas,
                       "timed": "value: the batch API (cwt_batch_exec, launches merged by kernel and level); "
                                "graph: one CUDA graph over the per-signal launch sequences; one_by_one: one "
                                "launch sequence per signal on one stream"},
            "data": "synthetic"}
    if embedded:
        return line
    print(json.dumps(line), flush=True)


def dataclasses_replace(r):
    import dataclasses
    return dataclasses.replace(r)


def run_ours(args):
    import torch

    import paper_2302_03909_gb300 as cwt

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # a dedicated stream: the library replays each plan's launches as a CUDA graph
    # captured on it (the legacy default stream cannot be captured)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)

    parts = workload_parts(args.workload)
    f = rank_signal(parts[0], rank, world)
    N = len(f)
    sig = torch.tensor(f, dtype=torch.float32, device=dev)
    def make_runs(precision="fp32"):
        """Every transform of the step: (part, wavelet, boundary, scales, plan, W, spectrum)."""
        out, sub = [], None
        for part in parts:
            w = synth.WORKLOADS[part]
            bounds, sc, sub = workload_subset(args, part)
            for b in bounds:
                p = cwt.cwt_plan_create(N, sc, w["wavelet"], b, tune=not args.no_tune, precision=precision,
                                        wide2_kernel=args.wide2_kernel)
                out.append((part, w["wavelet"], b, sc, p, p.empty_output(dev),
                            torch.empty(len(sc), dtype=torch.float64, device=dev)))
        return out, sub

    t_plan0 = time.perf_counter()
    runs, subset = make_runs()
    t_plan = time.perf_counter() - t_plan0
    plans = [r[4] for r in runs]
    fft_lens = [p.M for p in plans]
    transforms = [f"{r[1]}/{r[2]}" for r in runs]
    boundaries_used = sorted({r[2] for r in runs})
    shapes = [{k: cwt.cwt_plan_get_opts(p)[k] for k in ("tune", "min_ctas", "wide_batch_bytes", "band_depth", "wide2_kernel")}
              for p in plans]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def step(rs=None):
        for _, _, _, _, p, W, sp in (rs or runs):
            cwt.cwt_exec_with_power(p, sig, W, sp, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def timed(K: int, timing, rs=None):
        """K steps bracketed by a barrier and a synchronize; each step timed with
        CUDA events on the step's stream.  timing: the plans' timing hook (0: the
        library's own path, graph replay; "serial": an event pair around every
        launch, all launches on the step's stream one after another)."""
        rs = rs or runs
        for r in rs:
            cwt.cwt_plan_set_timing(r[4], timing)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(local)
        clk.start()
        for k in range(K):
            flush.zero_()
            evs[k][0].record(stream)
            step(rs)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clocks_ = clk.stop()
        ms = max_over_ranks(float(sum(a.elapsed_time(b) for a, b in evs)), dev)
        return ms, clocks_

    # the timed steps: graph replays (the library's path on a non-default stream)
    t_wall0 = time.perf_counter()
    total_ms, clocks = timed(args.steps, 0)
    t_wall = time.perf_counter() - t_wall0
    # the same steps again with every launch serialised and timed alone: the
    # kernel-class breakdown and the roofline kernel's own duration
    k_serial = max(1, min(args.steps, 5))
    total_ms_serial, _ = timed(k_serial, "serial")
    cls_tot = {}
    for p in plans:
        for name, (ms, n, b) in cwt.cwt_plan_get_timing(p).items():
            a = cls_tot.setdefault(name, [0.0, 0, 0.0])
            a[0] += ms
            a[1] += n
            a[2] += b
        cwt.cwt_plan_set_timing(p, False)
    # launches of this library's kernels per step, and in the K timed steps
    launches_per_step = int(round(sum(v[1] for v in cls_tot.values()) / k_serial))
    # the roofline kernel: of the classes that write W (the algorithmic output),
    # the one with the most device time
    dom = max([k for k in ("wide2", "band") if k in cls_tot] or list(cls_tot), key=lambda k: cls_tot[k][0])
    peak, peak_src = load_peaks()
    achieved = cls_tot[dom][2] / (cls_tot[dom][0] * 1e-3) / 1e9 if cls_tot[dom][0] > 0 else 0.0
    traffic = (load_traffic(dom, args.workload, cls_tot[dom][2] / max(1, cls_tot[dom][1]))
               if not subset else None)
    units_per_step = sum(len(r[3]) * N for r in runs)
    w_bytes_per_step = sum(r[5].numel() * r[5].element_size() for r in runs)
    alg_bytes_per_step = sum(v[2] for v in cls_tot.values()) / k_serial
    value = weak_scaling_value(units_per_step, args.steps, world, total_ms)
    ms_step = total_ms / args.steps

    # end to end through the host-buffer entry point: H2D of the signal, D2H of W and spectrum
    e2e = None
    if not args.no_e2e:
        sig_h = torch.tensor(f, dtype=torch.float32).pin_memory()
        Wh = [torch.empty(r[4].out_shape, dtype=(torch.complex64 if r[4].is_complex else torch.float32)).pin_memory()
              for r in runs]
        sh = [torch.empty(len(r[3]), dtype=torch.float64).pin_memory() for r in runs]
        for r, W_, s_ in zip(runs, Wh, sh):
            cwt.cwt_exec_host(r[4], sig_h, W_, s_, stream)
        e2e_steps = max(1, min(args.steps, 5))
        torch.cuda.synchronize()
        step_ms = []
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            ts = time.perf_counter()
            for r, W_, s_ in zip(runs, Wh, sh):
                cwt.cwt_exec_host(r[4], sig_h, W_, s_, stream)
            step_ms.append((time.perf_counter() - ts) * 1e3)
        te = time.perf_counter() - t0
        h2d = N * 4 * len(runs)
        d2h = sum(W_.numel() * W_.element_size() + s_.numel() * 8 for W_, s_ in zip(Wh, sh))
        # the host link alone: the same bytes copied from device memory into the same pinned buffers
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for r, W_ in zip(runs, Wh):
            W_.copy_(r[5], non_blocking=True)
        torch.cuda.synchronize()
        tc = time.perf_counter() - t0
        e2e = {"value": world * units_per_step * e2e_steps / te, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": te * 1e3 / e2e_steps,
               "ms_per_step_each": [round(x, 2) for x in step_ms],
               "ms_per_step_median": float(np.median(step_ms)),
               "d2h_copy_only_ms": tc * 1e3, "d2h_copy_only_GBps": d2h / tc / 1e9}
        del Wh, sh

    # the tensor-core forms of the 1024-point DFT stages, timed the same way on the same
    # signal, with their W against this FP32 run's W (the oracle gates are the tests')
    prec = {}
    forms = [x for x in args.precisions.split(",") if x] if rank == 0 and world == 1 else []
    for form in forms:
        rs, _ = make_runs(form)
        for _ in range(args.warmup):
            step(rs)
        ms_f, _ = timed(args.steps, 0, rs)
        ms_fs, _ = timed(k_serial, "serial", rs)
        w2 = sum(cwt.cwt_plan_get_timing(r[4])["wide2"][0] for r in rs) / k_serial
        for r in rs:
            cwt.cwt_plan_set_timing(r[4], False)
        err = 0.0
        for r, r32 in zip(rs, runs):
            d = torch.linalg.vector_norm((r[5] - r32[5]).reshape(-1)) / torch.linalg.vector_norm(r32[5].reshape(-1))
            err = max(err, float(d))
        prec[form] = {"ms_per_step": ms_f / args.steps, "value": units_per_step * args.steps / (ms_f * 1e-3),
                      "speedup_vs_fp32": total_ms / ms_f,
                      "wide2_ms_per_step_serialised": w2,
                      "wide2_speedup_vs_fp32": (cls_tot["wide2"][0] / k_serial) / w2 if w2 > 0 and "wide2" in cls_tot
                      else None,
                      "rel_l2_vs_fp32_max_over_transforms": err}
        for r in rs:
            r[4].close()
        del rs
        torch.cuda.empty_cache()

    fftb = None
    if rank == 0 and world == 1 and not args.no_fft_baseline:
        per = []
        for part in parts:
            sub = [r for r in runs if r[0] == part]
            per.append(fft_library_baseline(f, sub[0][3], sub[0][1], [r[4] for r in sub],
                                            [(r[5], r[6]) for r in sub], flush, stream, min(args.steps, 10)))
        ms_f = sum(q["ms_per_step"] for q in per)
        fftb = {"value": units_per_step / (ms_f * 1e-3), "unit": UNIT, "ms_per_step": ms_f,
                "steps": per[0]["steps"],
                "rel_l2_vs_library": max(q["rel_l2_vs_library"] for q in per),
                "power_max_rel_dev_vs_library": max(q["power_max_rel_dev_vs_library"] for q in per),
                "what": per[0]["what"]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(args.workload, args.cpu_seconds)
        cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}

    # the batched and served forms on the same GPU in the same run (summaries; --batch and
    # --serving print the full lines)
    for p in plans:
        p.close()
    plans = []
    del runs
    torch.cuda.empty_cache()
    batch = serving_line = None
    if rank == 0 and world == 1 and not args.no_batch:
        b = run_batch(args, embedded=True)
        batch = {"value": b["value"], "unit": UNIT, "graph": b["graph"], "one_by_one": b["one_by_one"],
                 "signals": b["config"]["signals"], "scale_samples": b["config"]["scale_samples"],
                 "grouped_info": b["detail"]["grouped_info"], "what": b["config"]["timed"]}
    if rank == 0 and world == 1 and not args.no_serving:
        torch.cuda.empty_cache()
        sv = run_serving(args, embedded=True)
        serving_line = {k: sv[k] for k in ("p50_ms", "p99_ms", "serial_p50_ms", "serial_p99_ms",
                                           "offered_scale_samples_per_s")}
        serving_line["served_scale_samples_per_s"] = sv["concurrent"]["scale_samples_per_s"]
        serving_line["serial_scale_samples_per_s"] = sv["serial"]["scale_samples_per_s"]
        serving_line["config"] = sv["config"]

    if rank == 0:
        w0 = synth.WORKLOADS[parts[0]]
        wavs = [synth.WORKLOADS[q]["wavelet"] for q in parts]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step,
            "ms_per_step_serialised": total_ms_serial / k_serial, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "N": N, "n_scales": w0["n_scales"], "wavelets": wavs,
                       **({"omega0": 6.0} if "morlet" in wavs else {}),
                       "boundaries": boundaries_used,
                       "transforms": transforms,
                       "fft_len": fft_lens, "power_spectrum": True,
                       "l2": "flushed between timed steps (512 MiB write outside the events)",
                       "inputs": "resident in HBM", "parallelism": f"replicas x{world}",
                       "launch_shape": shapes, "plan_s": round(t_plan, 3),
                       **({"subset": subset} if subset else {})},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": dom,
                         "peak_source": peak_src,
                         "algorithmic_bytes_per_launch": cls_tot[dom][2] / max(1, cls_tot[dom][1]),
                         "ms_per_launch": cls_tot[dom][0] / max(1, cls_tot[dom][1]),
                         "timing": "CUDA events around every launch of the dominant class, each launch "
                                   "alone on the step's stream (a second pass of the same steps with every "
                                   "launch serialised); dominant = the W-writing class with the most "
                                   "device time; achieved = its algorithmic bytes / its summed durations"},
            "kernel_classes": {k: {"ms": v[0] / k_serial, "launches": int(round(v[1] / k_serial)),
                                   "GBps": (v[2] / (v[0] * 1e-3) / 1e9) if v[0] > 0 else 0.0}
                               for k, v in cls_tot.items() if v[1] > 0},
            # whole step against the roofline: W written (the spec measure), and all
            # algorithmic bytes (W, the spectrum bands read, the forward transform)
            "hbm_frac_output": w_bytes_per_step / (ms_step * 1e-3) / 1e9 / peak,
            "hbm_frac_whole_step": alg_bytes_per_step / (ms_step * 1e-3) / 1e9 / peak,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "fft_library_baseline": fftb,
            "precision_forms": prec or None,
            "batch": batch,
            "serving": serving_line,
            "wall_s_timed": t_wall,
        }
        print(json.dumps(line), flush=True)
    for p in plans:
        p.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse_args()
    if args.serving and args.impl == "ours":
        run_serving(args)
        return
    if args.batch and args.impl == "ours":
        run_batch(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
