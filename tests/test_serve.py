"""Service logic of paper_1906_10944_gb300.serve on the host (no GPU): a
stand-in solve function that sleeps, so queueing, dispatch and the latency
bookkeeping can be checked exactly."""
import threading
import time

from paper_1906_10944_gb300 import serve as S


def test_poisson_trace_is_seeded_and_ordered():
    a = S.poisson_trace(200, 50.0, seed=3, choices=4)
    b = S.poisson_trace(200, 50.0, seed=3, choices=4)
    assert a == b
    t = [x[0] for x in a]
    assert all(t2 > t1 for t1, t2 in zip(t, t[1:]))
    assert {x[1] for x in a} <= set(range(4)) and {x[2] for x in a} <= set(range(1, 9))
    # mean gap of an exponential with rate 50 is 20 ms (loose bound for 200 draws)
    assert 0.014 < t[-1] / len(t) < 0.028


def test_percentile_nearest_rank():
    v = list(range(1, 101))
    assert S.percentile(v, 50) == 50 and S.percentile(v, 99) == 99 and S.percentile(v, 100) == 100
    assert S.percentile([7.0], 99) == 7.0


def test_server_fifo_latency_and_concurrency():
    def solve(req, stream):
        time.sleep(0.05)
        return req.rid

    # four requests at once on two workers: two finish after ~1 service time,
    # two after ~2; first come, first served
    reqs = [S.Request(i, None, arrival=0.0) for i in range(4)]
    S.Server(solve, workers=2).run(reqs)
    assert [r.result for r in reqs] == [0, 1, 2, 3]
    lat = sorted(r.latency for r in reqs)
    assert 0.045 < lat[0] < 0.09 and 0.095 < lat[-1] < 0.16
    assert all(r.latency >= r.service - 1e-9 for r in reqs)
    assert max(r.start for r in reqs[:2]) < min(r.start for r in reqs[2:])
    s = S.summarize(reqs)
    assert s["requests"] == 4 and s["errors"] == 0 and s["p50_ms"] <= s["p99_ms"]


def test_server_records_errors_and_continues():
    def solve(req, stream):
        if req.rid == 1:
            raise RuntimeError("boom")
        return req.rid

    reqs = [S.Request(i, None, arrival=0.01 * i) for i in range(3)]
    S.Server(solve, workers=1).run(reqs)
    assert reqs[1].error and reqs[0].result == 0 and reqs[2].result == 2
    assert S.summarize(reqs)["errors"] == 1


def test_admission_keeps_footprint_under_budget_and_order():
    # six requests arrive together; footprints 4, 4, 4, 2, 2, 2 under a budget
    # of 8 with three workers: at most two of the large ones run together
    fps = [4.0, 4.0, 4.0, 2.0, 2.0, 2.0]
    live = {"bytes": 0.0, "peak": 0.0}
    import threading
    lock = threading.Lock()

    def solve(req, stream):
        with lock:
            live["bytes"] += fps[req.rid]
            live["peak"] = max(live["peak"], live["bytes"])
        time.sleep(0.04)
        with lock:
            live["bytes"] -= fps[req.rid]
        return req.rid

    reqs = [S.Request(i, None, arrival=0.0) for i in range(6)]
    srv = S.Server(solve, workers=3, hbm_budget=8.0, footprint=lambda r: fps[r.rid])
    srv.run(reqs)
    assert [r.result for r in reqs] == list(range(6))
    assert live["peak"] <= 8.0 and srv.peak_bytes <= 8.0
    # first come, first served: starts are in arrival (id) order
    starts = [r.start for r in reqs]
    assert starts == sorted(starts)
    # request 2 had to wait for one of the first two to finish
    assert reqs[2].start >= min(reqs[0].finish, reqs[1].finish) - 1e-3


def test_admission_lets_an_oversized_request_run_alone():
    def solve(req, stream):
        time.sleep(0.02)
        return req.rid

    reqs = [S.Request(i, None, arrival=0.0) for i in range(3)]
    fps = [1.0, 100.0, 1.0]
    srv = S.Server(solve, workers=2, hbm_budget=10.0, footprint=lambda r: fps[r.rid])
    srv.run(reqs)
    assert [r.result for r in reqs] == [0, 1, 2]
    # the oversized request starts after request 0 finished, and request 2 after it
    assert reqs[1].start >= reqs[0].finish - 1e-3
    assert reqs[2].start >= reqs[1].finish - 1e-3


def test_footprint_by_dofs():
    problems = [(None, None, 1000), (None, None, 8000)]
    fp = S.footprint_by_dofs(problems, 2800.0)
    assert fp(S.Request(0, 1, nrhs=2)) == 2800.0 * 8000 + 16.0 * 8000 * 2
    assert fp(S.Request(1, 0, nrhs=1)) == 2800.0 * 1000 + 16.0 * 1000


class _FakeLib:
    """Host stand-in for the library calls of a ResidentPool."""

    def __init__(self, sizes):
        self.sizes = sizes
        self.live = {}
        self.setups = 0
        self.lock = threading.Lock()

    def setup(self, key, stream):
        with self.lock:
            self.setups += 1
            h = object()
            self.live[id(h)] = (h, key)
        time.sleep(0.002)
        return h

    def destroy(self, h):
        with self.lock:
            del self.live[id(h)]

    def bytes_of(self, h):
        return self.sizes[self.live[id(h)][1]]


def test_resident_pool_reuses_and_evicts_lru():
    lib = _FakeLib({0: 40.0, 1: 40.0, 2: 40.0})
    pool = S.ResidentPool(lib.setup, lib.destroy, lib.bytes_of, estimate=lambda k: 40.0, budget=100.0)
    for k in (0, 1, 0, 0, 1):
        pool.release(pool.acquire(k))
    assert lib.setups == 2 and pool.hits == 3
    e0 = pool.acquire(0)
    pool.release(e0)            # 0 used last: 1 is the least recently used
    pool.release(pool.acquire(2))
    assert pool.evictions == 1 and set(k for _, k in lib.live.values()) == {0, 2}
    assert pool.peak <= 100.0
    pool.close()
    assert not lib.live


def test_resident_pool_waits_for_busy_memory():
    """A setup that does not fit next to busy handles waits until they are
    released (nothing is evicted from under a solve)."""
    lib = _FakeLib({0: 60.0, 1: 60.0})
    pool = S.ResidentPool(lib.setup, lib.destroy, lib.bytes_of, estimate=lambda k: 60.0, budget=100.0)
    e0 = pool.acquire(0)
    got = []

    def other():
        e = pool.acquire(1)
        got.append(time.perf_counter())
        pool.release(e)

    th = threading.Thread(target=other)
    th.start()
    time.sleep(0.05)
    assert not got                     # waiting: 0 is busy
    t_rel = time.perf_counter()
    pool.release(e0)
    th.join(5)
    assert got and got[0] >= t_rel and pool.evictions == 1
    pool.close()


def test_resident_pool_oversized_request_alone():
    lib = _FakeLib({0: 30.0, 1: 500.0})
    pool = S.ResidentPool(lib.setup, lib.destroy, lib.bytes_of, estimate=lambda k: lib.sizes[k], budget=100.0)
    pool.release(pool.acquire(0))
    pool.release(pool.acquire(1))   # evicts 0, then runs alone
    assert pool.evictions == 1 and [k for _, k in lib.live.values()] == [1]
    pool.close()
