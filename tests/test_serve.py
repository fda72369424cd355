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
