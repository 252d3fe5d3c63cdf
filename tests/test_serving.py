"""Host logic of the request server (paper_2302_03909_gb300.serving): the plan
cache and the FIFO admission, with fakes in place of the GPU; the arrival
trace generator."""
import numpy as np
import pytest

from paper_2302_03909_gb300 import serving


class FakePlan:
    def __init__(self, key, nbytes):
        self.key, self.workspace_bytes, self.closed = key, nbytes, False

    def close(self):
        self.closed = True


def test_plan_cache_reuses_idle_instances_and_evicts_lru():
    made = []

    def factory(key):
        p = FakePlan(key, 100)
        made.append(p)
        return p

    c = serving.PlanCache(factory, max_bytes=250)
    a = c.acquire("a")
    a2 = c.acquire("a")                    # busy instance: a second one is made
    assert a is not a2 and c.misses == 2 and c.busy == 2
    c.release("a", a)
    assert c.acquire("a") is a and c.hits == 1
    c.release("a", a)
    c.release("a", a2)
    b = c.acquire("b")                     # 300 bytes > 250: an idle "a" goes
    assert c.evictions == 1 and c.bytes == 200 and sum(p.closed for p in made) == 1
    assert not b.closed                    # busy instances are never evicted
    c.release("b", b)
    c.clear()
    assert all(p.closed for p in made) and c.bytes == 0


def req(rid, N=1024, S=4, wavelet="morlet", t=0.0):
    return serving.Request(rid, N, tuple(np.linspace(2, 10, S)), wavelet, "periodic", t)


def test_admission_fifo_budget_and_slots():
    r = [req(i) for i in range(5)]
    nb = r[0].io_bytes
    adm = serving.Admission(budget_bytes=3 * nb, slots=2)
    for x in r:
        adm.submit(x)
    got = []
    while True:
        nxt = adm.next_admissible(lambda q: q.io_bytes)
        if nxt is None:
            break
        got.append(nxt)
    assert [g[0].rid for g in got] == [0, 1]          # two slots
    adm.done(got[0][1], got[0][2])
    nxt = adm.next_admissible(lambda q: q.io_bytes)
    assert nxt[0].rid == 2                             # arrival order
    big = req(9, N=1 << 20, S=128)
    with pytest.raises(ValueError):
        serving.Admission(budget_bytes=nb, slots=1).submit(big)


def test_admission_head_of_line_waits_for_memory():
    small, large = req(0), req(1, N=1 << 14, S=16)
    adm = serving.Admission(budget_bytes=large.io_bytes + small.io_bytes // 2, slots=4)
    adm.submit(small)
    adm.submit(large)
    adm.submit(req(2))
    a = adm.next_admissible(lambda q: q.io_bytes)
    assert a[0].rid == 0
    assert adm.next_admissible(lambda q: q.io_bytes) is None     # large waits, small behind it too
    adm.done(a[1], a[2])
    assert adm.next_admissible(lambda q: q.io_bytes)[0].rid == 1
    assert adm.in_flight_bytes == large.io_bytes


def test_poisson_trace_shape():
    tr = serving.poisson_trace(400.0, 2.0, seed=3)
    assert 650 < len(tr) < 950                          # ~800 arrivals
    t = np.array([r.t_arrival for r in tr])
    assert np.all(np.diff(t) > 0) and t[-1] <= 2.0
    assert {r.N for r in tr} <= {1 << u for u in range(10, 25)}
    assert all(16 <= len(r.scales) <= 128 for r in tr)
    assert {r.wavelet for r in tr} == {"gdw", "morlet"} and {r.boundary for r in tr} == {"periodic", "zero"}
    tr2 = serving.poisson_trace(400.0, 2.0, seed=3)
    assert [(r.N, r.key) for r in tr] == [(r.N, r.key) for r in tr2]


def test_admission_smallest_first_with_a_maximum_wait():
    big = req(0, N=1 << 14, S=16, t=0.0)
    small = [req(i, t=0.01 * i) for i in range(1, 4)]
    adm = serving.Admission(budget_bytes=1 << 30, slots=1, policy="smallest", max_wait_s=0.5)
    for x in [big] + small:
        adm.submit(x)
    order = []
    now = 0.1
    while adm.queue:
        nxt = adm.next_admissible(lambda q: q.io_bytes, now)
        order.append(nxt[0].rid)
        adm.done(nxt[1], nxt[2])
    assert order == [1, 2, 3, 0]                       # smaller requests overtake the large head
    # once the head has waited longer than max_wait it goes first
    adm = serving.Admission(budget_bytes=1 << 30, slots=1, policy="smallest", max_wait_s=0.5)
    for x in [big] + small:
        adm.submit(x)
    assert adm.next_admissible(lambda q: q.io_bytes, 0.6)[0].rid == 0
    with pytest.raises(ValueError):
        serving.Admission(1, 1, policy="lifo")


def test_ledger_keeps_device_bytes_within_the_budget_under_a_burst_of_new_shapes():
    """Every request of a burst has a shape never seen before, so each needs a
    new plan instance whose size is unknown until it exists.  The ledger
    charges the bound for it, counts idle cached instances against the same
    budget and evicts them to make room: the bytes actually live on the
    device (instances alive + the buffers of requests in flight) never exceed
    the budget, and neither does the ledger's own count."""
    rng = np.random.default_rng(5)
    alive = {}

    def factory(key):
        p = FakePlan(key, int(key[0]) * 37 + 1000)      # the real size, known only once made
        alive[id(p)] = p
        return p

    def close(p):
        p.close()
        alive.pop(id(p))

    cache = serving.PlanCache(factory, max_bytes=10 ** 9, close=close)   # no cap of its own
    budget = 400_000
    led = serving.Ledger(budget, slots=3, cache=cache, own_bytes=lambda r: r.io_bytes,
                         bound=lambda r: int(r.N) * 37 + 5000)         # above every real size
    reqs = []
    for i in range(60):
        N = int(rng.integers(256, 2048))
        reqs.append(req(i, N=N, S=int(rng.integers(2, 6)), t=0.0))
        if i % 3 == 0:                                   # some shapes repeat
            reqs.append(req(1000 + i, N=N, S=len(reqs[-1].scales), t=0.0))
    for r in reqs:
        led.submit(r)
    in_flight, done = [], 0

    def live_bytes():
        return sum(p.workspace_bytes for p in alive.values()) + sum(x[0].io_bytes for x in in_flight)

    while done < len(reqs):
        while True:
            nxt = led.admit()
            if nxt is None:
                break
            in_flight.append(nxt)
            assert led.device_bytes <= budget
            assert live_bytes() <= budget
        assert in_flight, "nothing admitted with an empty device"
        x = in_flight.pop(int(rng.integers(len(in_flight))))
        led.finish(*x)
        done += 1
        assert led.device_bytes <= budget and live_bytes() <= budget
    assert led.adm.in_flight_bytes == 0
    assert led.device_bytes == cache.idle_bytes == sum(p.workspace_bytes for p in alive.values())
    assert cache.evictions > 0 and led.peak_bytes <= budget


def test_workspace_bound_grows_with_the_transform():
    b = serving.workspace_bound
    sc = tuple(np.geomspace(4.0, 256.0, 16))
    assert b(1 << 12, sc, "morlet", "zero") > b(1 << 12, sc, "morlet", "periodic")
    assert b(5000, sc, "gdw", "periodic") > b(4096, sc, "gdw", "periodic")
    assert b(1 << 20, sc * 2, "gdw", "zero") > b(1 << 20, sc, "gdw", "zero")


def test_plan_creation_retries_once_after_releasing_the_torch_cache():
    """A plan that fails with CWT_ERR_OOM is created again after the torch
    caching allocator has released its free blocks; any other error, or a
    second OOM, propagates."""
    import paper_2302_03909_gb300 as cwt

    calls = {"create": 0, "empty": 0}

    class FakeCuda:
        @staticmethod
        def synchronize(dev=None):
            pass

        @staticmethod
        def empty_cache():
            calls["empty"] += 1

    class FakeTorch:
        cuda = FakeCuda

    def make_cwt(fail_times, status=3):
        class FakeCwt:
            CwtError = cwt.CwtError

            @staticmethod
            def cwt_plan_create(N, scales, wavelet, boundary, **opts):
                assert opts == {"wide2_kernel": 2}
                calls["create"] += 1
                if calls["create"] <= fail_times:
                    raise cwt.CwtError(status, "out of memory")
                return FakePlan((N, tuple(scales), wavelet, boundary), 1000)
        return FakeCwt

    srv = serving.Server.__new__(serving.Server)
    srv.torch, srv.dev, srv.reuse, srv.plan_opts = FakeTorch, None, False, {"wide2_kernel": 2}
    srv.caller_scratch, srv.scratch_known = False, {}
    key = (1024, (2.0, 4.0), "gdw", "periodic")
    srv.cwt = make_cwt(1)
    p = srv._make_plan(key)
    assert p.workspace_bytes == 1000 and calls == {"create": 2, "empty": 1}
    calls.update(create=0, empty=0)
    srv.cwt = make_cwt(2)
    with pytest.raises(cwt.CwtError):
        srv._make_plan(key)
    assert calls == {"create": 2, "empty": 1}
    calls.update(create=0, empty=0)
    srv.cwt = make_cwt(1, status=1)
    with pytest.raises(cwt.CwtError):
        srv._make_plan(key)
    assert calls == {"create": 1, "empty": 0}


def test_integer_length_pool_and_trace():
    """Two integer lengths per octave, log-uniform in each, the top power of two
    included; a trace drawn from the pool is reproducible and spans it."""
    pool = serving.length_pool((10, 24), per_octave=2, seed=5)
    assert pool == sorted(set(pool)) and pool[-1] == 1 << 24
    for u in range(10, 24):
        assert 1 <= sum((1 << u) <= n < (1 << (u + 1)) for n in pool) <= 2
    assert sum(n & (n - 1) == 0 for n in pool) <= 2          # mostly not powers of two
    t1 = serving.poisson_trace(500.0, 2.0, seed=3, integer_lengths=2)
    t2 = serving.poisson_trace(500.0, 2.0, seed=3, integer_lengths=2)
    assert [(r.N, r.scales, r.wavelet, r.boundary, r.t_arrival) for r in t1] == \
           [(r.N, r.scales, r.wavelet, r.boundary, r.t_arrival) for r in t2]
    full = set(serving.length_pool((10, 24), per_octave=2))
    assert {r.N for r in t1} <= full and len({r.N for r in t1}) > len(full) // 2
    assert all(r.scales[0] == 4.0 and abs(r.scales[-1] - max(8.0, r.N / 4)) < 1e-6 * r.N for r in t1)


def test_caller_scratch_is_charged_to_the_request():
    """A shape whose requests bring new buffers gets a caller-scratch plan: the
    ledger charges the request its scratch (a bound until the plan exists, then
    the plan's own figure) and the cached instance its tables only, so the
    bytes counted never exceed the budget."""
    import paper_2302_03909_gb300 as cwt

    class ScratchPlan(FakePlan):
        pass

    made = []

    class FakeCwt:
        CwtError = cwt.CwtError

        @staticmethod
        def cwt_plan_create(N, scales, wavelet, boundary, **opts):
            p = ScratchPlan((N, tuple(scales), wavelet, boundary), 1000 if opts.get("scratch") == "caller" else 10**6)
            p.opts = opts
            made.append(p)
            return p

        @staticmethod
        def cwt_plan_scratch_bytes(p):
            return 5000

    srv = serving.Server.__new__(serving.Server)
    srv.torch, srv.dev, srv.cwt = None, None, FakeCwt
    srv.reuse, srv.reuse_max, srv.keep, srv.plan_opts = True, 64 << 20, False, {"wide2_kernel": 2}
    srv.caller_scratch, srv.scratch_known = True, {}
    big = serving.Request(0, 1 << 22, tuple(np.geomspace(4.0, 1 << 20, 32)), "morlet", "zero", 0.0)
    small = serving.Request(1, 1 << 10, (4.0, 8.0), "gdw", "periodic", 0.0)
    assert srv._uses_caller_scratch(big.key) and not srv._uses_caller_scratch(small.key)
    bound = serving.workspace_bound(big.N, big.scales, big.wavelet, big.boundary)
    assert srv._own_bytes(big) == big.io_bytes + bound         # before the plan exists
    p = srv._make_plan(big.key)
    assert p.opts == {"wide2_kernel": 2, "scratch": "caller"} and p._scratch == 5000
    assert srv._own_bytes(big) == big.io_bytes + 5000           # the plan's own figure
    assert srv._size_of(p) == 1000                              # tables only in the cache
    srv.caller_scratch = False
    assert srv._own_bytes(big) == big.io_bytes
