"""Serving loop for CWT requests on one GPU.

Requests (a signal, its scales, a wavelet and a boundary) arrive over time.
The loop has three parts:

* ``Admission``: a queue admitted against a device-memory budget
  (``Ledger``).  A request needs its signal, its W and its spectrum, plus the
  workspace of its plan instance; idle cached instances count against the
  same budget and are evicted to make room.  An instance of a never-seen
  shape is charged an upper bound of its workspace (``workspace_bound``)
  until it exists.  With the "fifo" policy requests are
  admitted in arrival order: the head of the queue waits for memory and for a
  free slot, and nothing overtakes it.  With "smallest" the smallest queued
  request (by scale-samples) goes first, except that a request waiting longer
  than ``max_wait_s`` goes before any other (oldest first), so large requests
  are delayed but not starved.  A request larger than the whole budget is
  rejected at submission.
* ``PlanCache``: plans resident on the device, keyed by request shape.  A
  plan instance runs on one stream at a time (its workspace is shared), so a
  key can have several instances.  Idle instances are evicted
  least-recently-used once the cache exceeds its byte budget.
* ``Server``: ``slots`` CUDA streams.  An admitted request takes a free slot
  and a plan instance, copies its signal to the device, runs
  ``cwt_exec_with_power`` and records an event; completions are found by
  polling the events, and free their memory and slot.  By default a plan
  instance of a small shape (signal + W + spectrum up to ``reuse_max_bytes``)
  owns its buffers, so its calls repeat the same pointers and the library
  replays the instance's captured CUDA graph: one graph launch per request
  instead of a launch sequence, which is what small requests are dominated
  by.  Larger shapes get new buffers per request: their launch cost is small
  against their run time, and instances holding their W would crowd the plan
  cache.  Their plans are made with caller scratch (``scratch="caller"``):
  the cached instance keeps its constant tables only, and each request takes
  the plan's per-call buffers from torch's allocator for its own lifetime
  (``cwt_exec_scratch``), charged to the request.  Many shapes then stay
  resident at once.  A result the server keeps is copied out of the
  instance's W on the request's stream.

``run_trace`` replays a timed arrival trace (open loop) and reports latency
percentiles; ``poisson_trace`` draws the arrivals, with power-of-two lengths
or log-uniform integer lengths from ``length_pool``.  Both the admission and
the cache are plain host logic, tested on CPU with fakes.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time
from typing import Callable, Dict, List, Optional, Tuple

import numpy as np

_WBYTES = {"morlet": 8, "gdw": 4, "mexhat": 4, "cbsw": 4, "cwgdw": 4}


@dataclasses.dataclass
class Request:
    rid: int
    N: int
    scales: Tuple[float, ...]
    wavelet: str
    boundary: str
    t_arrival: float
    signal: object = None           # host float32 array / pinned CPU tensor of N samples
    t_admit: float = math.nan
    t_done: float = math.nan
    W: object = None                # device result, kept when the server is asked to
    spectrum: object = None

    @property
    def key(self):
        return (self.N, self.scales, self.wavelet, self.boundary)

    @property
    def io_bytes(self) -> int:
        """Device bytes of the request's own buffers: signal, W and spectrum."""
        S = len(self.scales)
        return self.N * 4 + S * self.N * _WBYTES[self.wavelet] + S * 8


class PlanCache:
    """Plan instances by key.  ``acquire`` lends an idle instance (or makes
    one with ``factory``); ``release`` returns it.  Idle instances are
    evicted least-recently-used while the cache holds more than
    ``max_bytes`` of plan workspace."""

    def __init__(self, factory: Callable, max_bytes: int, size_of: Callable = lambda p: p.workspace_bytes,
                 close: Callable = lambda p: p.close()):
        self.factory, self.max_bytes, self.size_of, self.close = factory, max_bytes, size_of, close
        self.idle: "collections.OrderedDict[tuple, List]" = collections.OrderedDict()
        self.busy = 0
        self.bytes = 0          # all live instances, busy or idle
        self.idle_bytes = 0     # idle instances only
        self.hits = self.misses = self.evictions = 0

    def has_idle(self, key) -> bool:
        return bool(self.idle.get(key))

    def acquire(self, key):
        lst = self.idle.get(key)
        if lst:
            self.hits += 1
            p = lst.pop()
            if not lst:
                del self.idle[key]
            self.idle_bytes -= self.size_of(p)
        else:
            self.misses += 1
            p = self.factory(key)
            self.bytes += self.size_of(p)
            self.trim()
        self.busy += 1
        return p

    def release(self, key, p):
        self.busy -= 1
        self.idle.setdefault(key, []).append(p)
        self.idle.move_to_end(key)
        self.idle_bytes += self.size_of(p)
        self.trim()

    def _evict_one(self, avoid=None) -> bool:
        for key, lst in self.idle.items():
            if avoid is not None and key == avoid:
                continue
            p = lst.pop(0)
            if not lst:
                del self.idle[key]
            n = self.size_of(p)
            self.bytes -= n
            self.idle_bytes -= n
            self.close(p)
            self.evictions += 1
            return True
        return False

    def trim(self):
        while self.bytes > self.max_bytes and self.idle:
            self._evict_one()

    def evict_idle(self, nbytes: int, avoid=None) -> int:
        """Evicts idle instances, least recently used first and never of the
        key ``avoid``, until ``nbytes`` are freed or none is left to evict;
        returns the bytes freed."""
        freed = 0
        while freed < nbytes:
            before = self.idle_bytes
            if not self._evict_one(avoid):
                break
            freed += before - self.idle_bytes
        return freed

    def clear(self):
        for lst in self.idle.values():
            for p in lst:
                self.close(p)
                self.bytes -= self.size_of(p)
        self.idle.clear()
        self.idle_bytes = 0


class Admission:
    """Admission against a byte budget and a number of slots ("fifo" or
    "smallest" first with a maximum wait)."""

    def __init__(self, budget_bytes: int, slots: int, policy: str = "fifo", max_wait_s: float = 0.1):
        if policy not in ("fifo", "smallest"):
            raise ValueError(policy)
        self.budget, self.slots = budget_bytes, slots
        self.policy, self.max_wait = policy, max_wait_s
        self.queue: "collections.deque[Request]" = collections.deque()
        self.in_flight_bytes = 0
        self.free_slots = list(range(slots))[::-1]

    def submit(self, req: Request, extra_bytes: int = 0):
        if req.io_bytes + extra_bytes > self.budget:
            raise ValueError(f"request {req.rid} needs {req.io_bytes + extra_bytes} bytes, "
                             f"over the {self.budget}-byte budget")
        self.queue.append(req)

    def next_admissible(self, need: Callable[[Request], int], now: float = 0.0,
                        room: Optional[Callable[[Request, int], bool]] = None) -> Optional[Tuple[Request, int, int]]:
        """Pops the next request by the policy if a slot is free and its bytes
        fit: (request, slot, bytes).  ``room(req, b)`` decides whether b more
        bytes fit (it may free memory to make them fit); by default they fit
        while the bytes in flight stay within the budget.  The chosen request
        waits for memory; nothing else overtakes it meanwhile."""
        if not self.queue or not self.free_slots:
            return None
        req = self.queue[0]
        if self.policy == "smallest" and now - req.t_arrival <= self.max_wait:
            req = min(self.queue, key=lambda q: (len(q.scales) * q.N, q.t_arrival))
        b = need(req)
        if not (room(req, b) if room is not None else self.in_flight_bytes + b <= self.budget):
            return None
        self.queue.remove(req)
        self.in_flight_bytes += b
        return req, self.free_slots.pop(), b

    def done(self, slot: int, nbytes: int):
        self.in_flight_bytes -= nbytes
        self.free_slots.append(slot)


def _pow2(x: int) -> int:
    return 1 << max(0, int(x - 1).bit_length())


def _plan_bound(M: int, S: int) -> int:
    """Upper bound on the device workspace of one plan of transform length M
    with S rows: the spectrum (M/2 + 1 complex64) and its transposed copy (M),
    the wide-scale intermediate (three streams, each max(M, 16 Mi) complex64,
    the default 128 MiB batch of wide scales per launch),
    the band values (at most 4096 complex64 per row), the power partial sums
    (fewer than M / 256 per row), the edge tables of a zero-boundary plan
    (2 x 4096 + 1 complex64 per row) and 2 MiB of small tables."""
    return 16 * M + 3 * max(8 * M, 128 << 20) + S * (96 << 10) + S * (M // 32) + (2 << 20)


def workspace_bound(N: int, scales, wavelet: str, boundary: str) -> int:
    """Upper bound on the device workspace of the library's plan for one
    request shape, from the same structure the planner uses: the zero
    boundary pads to M = pow2 >= 2N, with a periodic N-point child plan when N
    is a power of two and shorter sub-plans (M/2 and M) otherwise; the
    periodic boundary uses M = N for a power of two, else sub-plans of length
    pow2 >= N + 2E + 1 per row (E = ceil(chi s) + 1 the dilated wavelet's
    support, chi = 10 for the GDW and 6.5 for the Morlet) over a buffer of
    N + 2 max E samples."""
    S = len(scales)
    if boundary == "zero":
        M = _pow2(2 * N)
        return _plan_bound(M, S) + (_plan_bound(N, S) if N == _pow2(N) else _plan_bound(M // 2, S))
    if N == _pow2(N):
        return _plan_bound(N, S)
    chi = 10.0 if wavelet == "gdw" else 6.5
    E = [int(math.ceil(chi * float(sv))) + 1 for sv in scales]
    Ms = sorted({_pow2(N + 2 * e + 1) for e in E})
    return sum(_plan_bound(M, S) for M in Ms) + 8 * (N + 2 * max(E))


class Ledger:
    """Device memory of a server, kept within one budget: the requests in
    flight (their own buffers, unless they run in their plan instance's, and
    their plan instance) plus the idle plan instances of the cache.  A request
    is admitted when the bytes it adds fit, after evicting idle instances of
    other shapes if needed; an instance of a never-seen shape is charged
    ``bound(request)`` until it exists and its size is known."""

    def __init__(self, budget_bytes: int, slots: int, cache: "PlanCache", own_bytes: Callable[[Request], int],
                 policy: str = "fifo", max_wait_s: float = 0.1,
                 bound: Callable[[Request], int] = lambda r: workspace_bound(r.N, r.scales, r.wavelet, r.boundary)):
        self.adm = Admission(budget_bytes, slots, policy, max_wait_s)
        self.cache, self.own_bytes, self.bound = cache, own_bytes, bound
        self.known: Dict[tuple, int] = {}      # workspace of an instance, by key
        self.peak_bytes = 0

    @property
    def device_bytes(self) -> int:
        return self.adm.in_flight_bytes + self.cache.idle_bytes

    def submit(self, req: Request):
        # a request whose own bytes plus a new instance exceed the budget could never run
        self.adm.submit(req, extra_bytes=self.own_bytes(req) - req.io_bytes
                        + self.known.get(req.key, self.bound(req)))

    def need(self, req: Request) -> int:
        """Bytes admitting req adds to the device: its own buffers, and a new
        instance unless an idle one (already counted) is there."""
        own = self.own_bytes(req)
        if self.cache.has_idle(req.key):
            return own
        return own + self.known.get(req.key, self.bound(req))

    def room(self, req: Request, b: int) -> bool:
        over = self.device_bytes + b - self.adm.budget
        if over > 0:
            self.cache.evict_idle(over, avoid=req.key)
        return self.device_bytes + b <= self.adm.budget

    def admit(self, now: float = 0.0):
        """(request, slot, plan instance, bytes reserved) of the next admitted
        request, or None."""
        nxt = self.adm.next_admissible(self.need, now, self.room)
        if nxt is None:
            return None
        req, slot, b = nxt
        inst = self.cache.acquire(req.key)
        size = self.cache.size_of(inst)
        self.known[req.key] = size
        reserved = self.own_bytes(req) + size
        # the instance is now in flight: an idle one's bytes move out of the
        # cache's count, a new one's size replaces the bound it was charged
        self.adm.in_flight_bytes += reserved - b
        self.peak_bytes = max(self.peak_bytes, self.device_bytes)
        return req, slot, inst, reserved

    def finish(self, req: Request, slot: int, inst, reserved: int):
        self.cache.release(req.key, inst)
        self.adm.done(slot, reserved)


class Server:
    """Runs admitted requests on ``slots`` CUDA streams of one device."""

    def __init__(self, budget_bytes: int, slots: int = 4, plan_cache_bytes: Optional[int] = None,
                 keep_results: bool = False, device: int = 0, reuse_buffers: bool = True,
                 reuse_max_bytes: int = 64 << 20, policy: str = "fifo", max_wait_s: float = 0.1,
                 plan_opts: Optional[dict] = None, caller_scratch: bool = True):
        import torch

        import paper_2302_03909_gb300 as cwt
        self.torch, self.cwt = torch, cwt
        # plan options of every request shape.  The default keeps the wide
        # scales' pass 2 on the CTA Stockham kernel: the tile pipeline holds one
        # CTA per SM for the whole launch and, with several requests in flight,
        # delays the others' kernels (measured p99 286 ms against 170 ms at
        # 500 requests/s, same served rate)
        self.plan_opts = {"wide2_kernel": 2} if plan_opts is None else dict(plan_opts)
        self.dev = torch.device("cuda", device)
        # shapes whose requests get new buffers also get their plan's per-call
        # scratch per request (cwt_exec_scratch): the cached instance then holds
        # its tables only, so many such shapes stay resident
        self.caller_scratch = caller_scratch
        self.scratch_known: Dict[tuple, int] = {}
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(slots)]
        self.reuse = reuse_buffers
        self.reuse_max = reuse_max_bytes
        self.keep = keep_results
        self.cache = PlanCache(self._make_plan, plan_cache_bytes if plan_cache_bytes is not None
                               else budget_bytes // 4, size_of=self._size_of)
        self.ledger = Ledger(budget_bytes, slots, self.cache, self._own_bytes, policy, max_wait_s)
        self.adm = self.ledger.adm
        self.in_flight: List[tuple] = []      # (req, slot, bytes, plan, event, tensors)
        self.completed: List[Request] = []

    def _uses_caller_scratch(self, key) -> bool:
        return self.caller_scratch and not self._owns_buffers(Request(-1, *key, 0.0))

    def _make_plan(self, key):
        torch = self.torch
        N, scales, wavelet, boundary = key
        opts = dict(self.plan_opts)
        if self._uses_caller_scratch(key):
            opts["scratch"] = "caller"
        try:
            p = self.cwt.cwt_plan_create(N, np.asarray(scales), wavelet, boundary, **opts)
        except self.cwt.CwtError as e:
            # device memory that torch's caching allocator holds (freed request
            # buffers) is not visible to the library's allocations: release it
            # and try once more
            if e.status != 3:
                raise
            torch.cuda.synchronize(self.dev)
            torch.cuda.empty_cache()
            p = self.cwt.cwt_plan_create(N, np.asarray(scales), wavelet, boundary, **opts)
        p._scratch = self.cwt.cwt_plan_scratch_bytes(p) if opts.get("scratch") == "caller" else 0
        self.scratch_known[key] = p._scratch
        p._io, p._io_bytes = None, 0
        if self._owns_buffers(Request(-1, *key, 0.0)):
            p._io = (torch.empty(N, dtype=torch.float32, device=self.dev), p.empty_output(self.dev),
                     torch.empty(p.n_scales, dtype=torch.float64, device=self.dev))
            p._io_bytes = sum(t.numel() * t.element_size() for t in p._io)
        return p

    def _owns_buffers(self, req: Request) -> bool:
        return self.reuse and req.io_bytes <= self.reuse_max

    @staticmethod
    def _size_of(p) -> int:
        return p.workspace_bytes + getattr(p, "_io_bytes", 0)

    def _own_bytes(self, req: Request) -> int:
        # requests that run in their instance's buffers need nothing of their
        # own, unless their result is kept (a copy); the instance (workspace
        # and buffers) is charged by the ledger.  A request with caller scratch
        # also holds its plan's scratch (bounded until the plan exists).
        own = req.io_bytes if (not self._owns_buffers(req) or self.keep) else 0
        if self._uses_caller_scratch(req.key):
            own += self.scratch_known.get(req.key, workspace_bound(req.N, req.scales, req.wavelet, req.boundary))
        return own

    def submit(self, req: Request):
        self.ledger.submit(req)

    def _launch(self, req: Request, slot: int, plan, nbytes: int, now: float):
        torch = self.torch
        st = self.streams[slot]
        with torch.cuda.stream(st):
            if plan._io is not None:
                sig, W, sp = plan._io
            else:
                sig = torch.empty(req.N, dtype=torch.float32, device=self.dev)
                W = plan.empty_output(self.dev)
                sp = torch.empty(plan.n_scales, dtype=torch.float64, device=self.dev)
            sig.copy_(req.signal, non_blocking=True)
            scratch = None
            if getattr(plan, "_scratch", 0):
                scratch = torch.empty(plan._scratch, dtype=torch.uint8, device=self.dev)
                self.cwt.cwt_exec_scratch(plan, sig, W, sp, scratch, st)
            else:
                self.cwt.cwt_exec_with_power(plan, sig, W, sp, st)
            if self.keep and plan._io is not None:
                W, sp = W.clone(), sp.clone()
            ev = torch.cuda.Event()
            ev.record(st)
        req.t_admit = now
        # the scratch stays referenced until the request completes
        self.in_flight.append((req, slot, nbytes, plan, ev, (sig, W, sp, scratch)))

    def poll(self, now: float) -> int:
        """Retires finished requests and admits queued ones; returns the number retired."""
        n = 0
        still = []
        for item in self.in_flight:
            req, slot, nbytes, plan, ev, (sig, W, sp, _) = item
            if ev.query():
                req.t_done = now
                if self.keep:
                    req.W, req.spectrum = W, sp
                self.ledger.finish(req, slot, plan, nbytes)
                self.completed.append(req)
                n += 1
            else:
                still.append(item)
        self.in_flight = still
        while True:
            nxt = self.ledger.admit(now)
            if nxt is None:
                break
            self._launch(*nxt, now)
        return n

    def idle(self) -> bool:
        return not self.in_flight and not self.adm.queue

    def close(self):
        self.torch.cuda.synchronize(self.dev)
        self.cache.clear()


def run_trace(server: Server, trace: List[Request], max_seconds: float = 600.0) -> dict:
    """Replays the arrivals of ``trace`` (t_arrival in seconds from the start)
    in real time and returns latency statistics (milliseconds)."""
    trace = sorted(trace, key=lambda r: r.t_arrival)
    t0 = time.perf_counter()
    i = 0
    while i < len(trace) or not server.idle():
        now = time.perf_counter() - t0
        if now > max_seconds:
            raise TimeoutError("trace did not drain in time")
        while i < len(trace) and trace[i].t_arrival <= now:
            server.submit(trace[i])
            i += 1
        server.poll(now)
        if i < len(trace) and server.idle():
            time.sleep(max(0.0, min(trace[i].t_arrival - now, 1e-3)))
    wall = time.perf_counter() - t0
    lat = np.array([(r.t_done - r.t_arrival) * 1e3 for r in server.completed])
    units = sum(len(r.scales) * r.N for r in server.completed)
    return {"requests": len(lat), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "wall_s": wall, "scale_samples_per_s": units / wall,
            "plan_hits": server.cache.hits, "plan_misses": server.cache.misses,
            "plan_evictions": server.cache.evictions}


def length_pool(log2n=(10, 24), per_octave: int = 2, seed: int = 20230214) -> List[int]:
    """``per_octave`` integer lengths drawn log-uniformly in each octave
    [2^u, 2^(u+1)) for u in [log2n[0], log2n[1]), plus 2^log2n[1]: a
    service's set of signal lengths, mostly not powers of two."""
    rng = np.random.default_rng(seed)
    out = set()
    for u in range(log2n[0], log2n[1]):
        for _ in range(per_octave):
            out.add(int(min(2 ** (u + 1) - 1, round(2.0 ** (u + rng.uniform(0.0, 1.0))))))
    out.add(1 << log2n[1])
    return sorted(out)


def poisson_trace(rate: float, seconds: float, seed: int = 20230213, log2n=(10, 24), n_scales=(16, 128),
                  shapes_per_log2n: int = 4, integer_lengths: int = 0) -> List[Request]:
    """Poisson arrivals at ``rate`` per second for ``seconds``.  Each request:
    N = 2^u with u uniform over log2n (power-of-two lengths), or, with
    ``integer_lengths`` > 0, N drawn log-uniformly from ``length_pool`` with
    that many integer lengths per octave; a scale count drawn from
    ``shapes_per_log2n`` values spread over n_scales (requests of one service
    repeat shapes, which the plan cache exploits), log-spaced dilations from 4
    to N/4, the GDW or the Morlet and the periodic or zero boundary with equal
    odds."""
    rng = np.random.default_rng(seed)
    t, out, rid = 0.0, [], 0
    counts = np.unique(np.linspace(n_scales[0], n_scales[1], shapes_per_log2n).astype(int))
    pool = np.array(length_pool(log2n, integer_lengths)) if integer_lengths > 0 else None
    while True:
        t += rng.exponential(1.0 / rate)
        if t > seconds:
            break
        if pool is not None:
            # log-uniform over the pool's range: the pool entry nearest (in log) to 2^u
            x = rng.uniform(log2n[0], log2n[1])
            N = int(pool[np.argmin(np.abs(np.log2(pool) - x))])
        else:
            u = int(rng.integers(log2n[0], log2n[1] + 1))
            N = 1 << u
        S = int(rng.choice(counts))
        sc = tuple(float(x) for x in np.exp(np.linspace(np.log(4.0), np.log(max(8.0, N / 4)), S)))
        out.append(Request(rid, N, sc, "gdw" if rng.random() < 0.5 else "morlet",
                           "periodic" if rng.random() < 0.5 else "zero", t))
        rid += 1
    return out


def capture_batch(items, n_streams: int = 4):
    """One CUDA graph over a batch of transforms.  ``items`` are (plan,
    signal, W, spectrum) with device tensors allocated beforehand; the
    transforms are dealt round-robin over ``n_streams`` streams (each plan
    still forks its own side streams) and joined at the end.  Returns the
    graph; ``graph.replay()`` runs the whole batch with one launch from the
    host.  The plans see a capturing stream and record their kernels directly."""
    import torch

    import paper_2302_03909_gb300 as cwt
    s0 = torch.cuda.Stream()
    streams = [torch.cuda.Stream() for _ in range(n_streams)]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s0):
        start = torch.cuda.Event()
        start.record(s0)
        for st in streams:
            st.wait_event(start)
        for i, (plan, sig, W, sp) in enumerate(items):
            st = streams[i % n_streams]
            cwt.cwt_exec_with_power(plan, sig, W, sp, st)
        for st in streams:
            e = torch.cuda.Event()
            e.record(st)
            s0.wait_event(e)
    return g
