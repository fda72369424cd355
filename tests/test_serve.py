"""Service logic of paper_1906_10944_gb300.serve on the host (no GPU): a
stand-in solve function that sleeps, so queueing, dispatch and the latency
bookkeeping can be checked exactly."""
import time

from paper_1906_10944_gb300 import serve as S


def test_poisson_trace_is_seeded_and_ordered():
    a = S.poisson_trace(200, 50.0, seed=3, choices=4)
    b = S.poisson_trace(200, 50.0, seed=3, choices=4)
    assert a == b
    t = [x[0] for x in a]
    assert all(t2 > t1 for t1, t2 in zip(t, t[1:]))
    assert {x[1] for x in a} <= set(range(4)) and {x[2] for x in a} <= {1, 2, 3, 4}
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
