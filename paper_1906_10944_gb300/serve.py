"""Concurrent solve service over the C ABI.

A request is one linear system family A x_i = b_i (i < nrhs): PCG for each
right-hand side (Section 5) with the GenEO preconditioner of A (Sections 3
and 4).  Worker threads take requests first come, first served, each on its
own CUDA stream, so the setups and solves of different requests overlap on
the GPU (the library allocates from the stream-ordered pool, so no call
synchronises the device).  With a ResidentPool the set-up handle of each
problem stays on the device between requests (admitted by device-memory
footprint, released least recently used first), so a request for a
resident problem only solves; `library_solve_fn` instead sets up and
releases per request.  Latency is measured from a request's arrival to its
last solution.

The arithmetic lives in the library; this module only queues, dispatches and
records times.  `solve_fn` may be replaced (tests use a host stand-in).
"""
import math
import queue
import random
import threading
import time
from dataclasses import dataclass, field
from typing import Any, Callable, List, Optional


@dataclass
class Request:
    """One request: `payload` is handed to the solve function."""
    rid: int
    payload: Any
    nrhs: int = 1
    arrival: float = 0.0          # seconds after the start of the trace
    start: float = math.nan       # service start (same clock)
    finish: float = math.nan      # last solution ready (same clock)
    result: Any = None
    error: Optional[str] = None

    @property
    def latency(self) -> float:
        return self.finish - self.arrival

    @property
    def service(self) -> float:
        return self.finish - self.start


def poisson_trace(n: int, rate: float, seed: int, choices: int, max_nrhs: int = 8):
    """Seeded arrival offsets (exponential gaps of mean 1 / rate), the index of
    the problem each request uses and its number of right-hand sides."""
    rng = random.Random(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.expovariate(rate)
        out.append((t, rng.randrange(choices), 1 + rng.randrange(max_nrhs)))
    return out


def library_solve_fn(problems, rhs, tol=1e-8, maxit=2000):
    """Solve function over the library: problems[k] = (geneo_problem_t,
    geneo_options_t, n); rhs[k] = device tensor (n * max_nrhs) of right-hand
    sides; the payload of a request is the index k.  Returns the list of
    solve infos.  One output buffer per worker thread."""
    import torch
    from . import geneo as G
    local = threading.local()

    def solve(req: Request, stream):
        k = req.payload
        problem, opts, n = problems[k]
        x = getattr(local, "x", None)
        if x is None or x.numel() < n * req.nrhs:
            with torch.cuda.stream(stream):
                x = torch.empty(max(n * req.nrhs, 1), dtype=torch.float64, device="cuda")
            local.x = x
        h = G.geneo_setup(problem, opts, stream)
        try:
            infos = [G.geneo_pcg_solve(h, rhs[k][i * n:(i + 1) * n], x[i * n:(i + 1) * n], 1, tol, maxit,
                                       G.GENEO_MEM_DEVICE, stream=stream) for i in range(req.nrhs)]
        finally:
            G.geneo_destroy(h)
        return infos

    return solve


class ResidentPool:
    """Set-up handles kept on the device between requests, one per problem
    key, so a request for a problem already set up only solves.

    Admission by device-memory footprint: a new setup is admitted when the
    bytes of the resident handles plus its estimate (`estimate(key)`) fit in
    `budget`; idle handles are released least recently used first to make
    room; while busy handles hold the memory the setup waits; a setup larger
    than the whole budget is admitted once nothing else is resident.  After a
    setup the estimate is replaced by the handle's measured bytes
    (`bytes_of(handle)`).  Solves on one handle are serialised (a handle owns
    one set of work vectors); different handles run concurrently.
    `setup(key, stream)` and `destroy(handle)` do the library calls."""

    class Entry:
        def __init__(self, key):
            self.key = key
            self.handle = None
            self.bytes = 0.0
            self.ready = False
            self.busy = 0
            self.last = 0.0
            self.lock = threading.Lock()

    def __init__(self, setup: Callable, destroy: Callable, bytes_of: Callable, estimate: Callable,
                 budget: float):
        self.setup, self.destroy, self.bytes_of, self.estimate = setup, destroy, bytes_of, estimate
        self.budget = float(budget)
        self.entries = {}
        self.used = 0.0
        self.peak = 0.0
        self.hits = self.misses = self.evictions = 0
        self.cond = threading.Condition()

    def _evict_one(self):
        idle = [e for e in self.entries.values() if e.ready and e.busy == 0]
        if not idle:
            return False
        e = min(idle, key=lambda x: x.last)
        del self.entries[e.key]
        self.used -= e.bytes
        self.evictions += 1
        self.cond.release()
        try:
            self.destroy(e.handle)
        finally:
            self.cond.acquire()
        return True

    def acquire(self, key, stream=None):
        """The entry of `key`, set up if needed, marked busy; call release()."""
        with self.cond:
            while True:
                e = self.entries.get(key)
                if e is not None:
                    if e.ready:
                        e.busy += 1
                        self.hits += 1
                        return e
                    self.cond.wait()
                    continue
                need = float(self.estimate(key))
                while self.used + need > self.budget and self._evict_one():
                    pass
                if self.used + need > self.budget and self.entries:
                    self.cond.wait()
                    continue
                e = self.Entry(key)
                e.bytes = need
                e.busy = 1
                self.entries[key] = e
                self.used += need
                self.peak = max(self.peak, self.used)
                self.misses += 1
                break
        try:
            h = self.setup(key, stream)
        except Exception:
            with self.cond:
                del self.entries[key]
                self.used -= e.bytes
                self.cond.notify_all()
            raise
        with self.cond:
            e.handle = h
            b = float(self.bytes_of(h))
            self.used += b - e.bytes
            self.peak = max(self.peak, self.used)
            e.bytes = b
            e.ready = True
            self.cond.notify_all()
        return e

    def release(self, e):
        with self.cond:
            e.busy -= 1
            e.last = time.perf_counter()
            self.cond.notify_all()

    def close(self):
        with self.cond:
            for e in list(self.entries.values()):
                if e.handle is not None:
                    self.destroy(e.handle)
            self.entries.clear()
            self.used = 0.0

    def stats(self):
        n = self.hits + self.misses
        return {"resident_hits": self.hits, "setups": self.misses, "evictions": self.evictions,
                "hit_rate": self.hits / n if n else float("nan"), "peak_resident_gb": self.peak / 1e9,
                "budget_gb": self.budget / 1e9}


def resident_solve_fn(problems, rhs, pool: ResidentPool, tol=1e-8, maxit=2000):
    """Solve function over resident handles: the payload of a request is a
    problem key; rhs[key] = device tensor (n * max_nrhs) of right-hand sides.
    The request's right-hand sides go to the library in one geneo_pcg_solve
    call (nrhs columns).  One output buffer per worker thread."""
    import torch
    from . import geneo as G
    local = threading.local()

    def solve(req: Request, stream):
        k = req.payload
        n = problems[k][2]
        x = getattr(local, "x", None)
        if x is None or x.numel() < n * req.nrhs:
            with torch.cuda.stream(stream):
                x = torch.empty(max(n * req.nrhs, 1), dtype=torch.float64, device="cuda")
            local.x = x
        e = pool.acquire(k, stream)
        try:
            with e.lock:
                info = G.geneo_pcg_solve(e.handle, rhs[k], x, req.nrhs, tol, maxit, G.GENEO_MEM_DEVICE,
                                         stream=stream)
        finally:
            pool.release(e)
        return [info]

    return solve


def library_pool(problems, budget, bytes_per_dof=2.8e3):
    """A ResidentPool over problems[k] = (geneo_problem_t, geneo_options_t, n)."""
    from . import geneo as G
    return ResidentPool(setup=lambda k, stream: G.geneo_setup(problems[k][0], problems[k][1], stream),
                        destroy=G.geneo_destroy,
                        bytes_of=lambda h: G.geneo_query(h)["device_bytes"],
                        estimate=lambda k: bytes_per_dof * problems[k][2], budget=budget)


def footprint_by_dofs(problems, bytes_per_dof: float, bytes_per_rhs_dof: float = 16.0):
    """Device-memory estimate of a library request: problems[k] = (problem,
    options, n); a handle holds about bytes_per_dof per dof (measured on the
    128^3 Darcy workload with FP32 factors: 2.8 KB per dof, setup
    temporaries included), and each right-hand side adds its solution and
    right-hand-side vectors."""
    def fp(req: Request) -> float:
        n = problems[req.payload][2]
        return bytes_per_dof * n + bytes_per_rhs_dof * n * req.nrhs
    return fp


class Server:
    """`workers` threads, each with its own stream (`make_stream()`), serving
    requests first come, first served.

    Admission control (optional): with `hbm_budget` bytes and `footprint(req)`
    an estimate of a request's device memory, a request is admitted, in
    arrival order, only when its footprint fits next to the footprints of the
    admitted requests that have not finished; the head of the queue waits for
    memory (no overtaking), and a request larger than the whole budget is
    admitted alone.  `peak_bytes` records the largest admitted total."""

    def __init__(self, solve_fn: Callable, workers: int = 3, make_stream: Optional[Callable] = None,
                 hbm_budget: Optional[float] = None, footprint: Optional[Callable] = None):
        self.solve_fn = solve_fn
        self.workers = workers
        self.make_stream = make_stream
        self.hbm_budget = hbm_budget
        self.footprint = footprint
        self.peak_bytes = 0.0

    def run(self, requests: List[Request]) -> List[Request]:
        """Release each request at its arrival offset (and, with a budget,
        once it fits) and return them all with start, finish and result
        filled in."""
        q: "queue.Queue[Optional[Request]]" = queue.Queue()
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        cond = threading.Condition()
        state = {"bytes": 0.0, "inflight": 0}
        fp = (lambda r: float(self.footprint(r))) if self.footprint else (lambda r: 0.0)

        def worker():
            stream = self.make_stream() if self.make_stream else None
            while True:
                req = q.get()
                if req is None:
                    return
                req.start = now()
                try:
                    req.result = self.solve_fn(req, stream)
                except Exception as e:  # recorded, the service continues
                    req.error = repr(e)
                req.finish = now()
                if self.hbm_budget is not None:
                    with cond:
                        state["bytes"] -= fp(req)
                        state["inflight"] -= 1
                        cond.notify_all()

        threads = [threading.Thread(target=worker, daemon=True) for _ in range(self.workers)]
        for th in threads:
            th.start()
        for req in sorted(requests, key=lambda r: r.arrival):
            delay = req.arrival - now()
            if delay > 0:
                time.sleep(delay)
            if self.hbm_budget is not None:
                need = fp(req)
                with cond:
                    while state["inflight"] > 0 and state["bytes"] + need > self.hbm_budget:
                        cond.wait()
                    state["bytes"] += need
                    state["inflight"] += 1
                    self.peak_bytes = max(self.peak_bytes, state["bytes"])
            q.put(req)
        for _ in threads:
            q.put(None)
        for th in threads:
            th.join()
        return requests


def percentile(values, p):
    """Nearest-rank percentile (p in [0, 100])."""
    v = sorted(values)
    if not v:
        return math.nan
    k = max(0, min(len(v) - 1, int(math.ceil(p / 100.0 * len(v))) - 1))
    return v[k]


def summarize(requests: List[Request], warmup: int = 0):
    """Latency percentiles, throughput and solves per second over the
    requests after the first `warmup` arrivals."""
    done = sorted(requests, key=lambda r: r.arrival)[warmup:]
    ok = [r for r in done if r.error is None]
    lat = [r.latency for r in ok]
    span = max(r.finish for r in ok) - min(r.arrival for r in ok) if ok else math.nan
    return {
        "requests": len(done), "errors": len(done) - len(ok),
        "p50_ms": 1e3 * percentile(lat, 50), "p99_ms": 1e3 * percentile(lat, 99),
        "mean_service_ms": 1e3 * sum(r.service for r in ok) / max(len(ok), 1),
        "achieved_rps": len(ok) / span if ok else math.nan,
        "solves_per_s": sum(r.nrhs for r in ok) / span if ok else math.nan,
    }
