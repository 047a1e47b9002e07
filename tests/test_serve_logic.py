"""Scheduler of the continuous-batching server, on the CPU with a fake
executor: FIFO admission, batching of waiting requests, the memory budget
over all batches in flight, lane concurrency, routing of results, and
rejection of requests that can never fit."""
import numpy as np
import pytest

from paper_2009_13349_gb300.serve import QUERY_BYTES, RejectedRequest, Request, Server


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeExecutor:
    """Completes a batch `dur` fake seconds after launch; results encode
    (request id, position) so routing can be checked."""

    def __init__(self, clock, ws_per_query=100, dur=1.0):
        self.clock, self.ws_per_query, self.dur = clock, ws_per_query, dur
        self.launches = []

    def workspace_bytes(self, n):
        return 1000 + self.ws_per_query * n

    def launch(self, lane, reqs):
        h = {"lane": lane, "reqs": [r.id for r in reqs], "t_end": self.clock() + self.dur}
        self.launches.append(h)
        return h

    def ready(self, h):
        return self.clock() >= h["t_end"]

    def harvest(self, h, reqs):
        for r in reqs:
            r.collides = np.full(r.n, r.id % 2, np.uint8)
            r.toi = r.id + np.arange(r.n) / 1e6
            r.out_tol = np.zeros(r.n)


def req(i, n, kind=0, ms=0.0, delta=1e-6):
    return Request(i, kind, np.zeros((n, 24)), ms=ms, delta=delta)


def test_fifo_batching_and_routing():
    clk = FakeClock()
    ex = FakeExecutor(clk)
    s = Server(ex, lanes=2, budget=10**9, max_batch=100, clock=clk)
    for i, n in enumerate([30, 30, 30, 30, 80, 20]):
        s.submit(req(i, n))
    s.poll()
    # lane 0 takes the first three (90 <= 100; +30 would exceed), lane 1 the
    # next one (30 + 80 > 100 stops there); the rest waits for a free lane
    assert [h["reqs"] for h in ex.launches] == [[0, 1, 2], [3]]
    clk.t = 1.0
    done = s.poll()
    assert sorted(r.id for r in done) == [0, 1, 2, 3]
    assert [h["reqs"] for h in ex.launches][-1] == [4, 5]
    clk.t = 2.0
    s.poll()
    assert s.idle() and len(s.completed) == 6
    for r in s.completed:
        assert r.toi[0] == r.id and r.collides[0] == r.id % 2


def test_budget_caps_memory_in_flight():
    clk = FakeClock()
    ex = FakeExecutor(clk, ws_per_query=10)
    per = lambda n: n * QUERY_BYTES + 1000 + 10 * n
    budget = per(40) + per(40) // 2          # room for one 40-query batch, not two
    s = Server(ex, lanes=4, budget=budget, max_batch=40, clock=clk)
    for i in range(6):
        s.submit(req(i, 40))
    steps = 0
    while not s.idle():
        s.poll()
        assert s.in_flight_bytes <= budget
        assert len(s.busy) <= 1
        clk.t += 0.5
        steps += 1
        assert steps < 100
    assert len(s.completed) == 6 and s.peak_bytes <= budget


def test_lanes_bound_concurrency_and_late_arrivals_join():
    clk = FakeClock()
    ex = FakeExecutor(clk, dur=2.0)
    s = Server(ex, lanes=3, budget=10**12, max_batch=10, clock=clk)
    for i in range(5):
        s.submit(req(i, 10))
    s.poll()
    assert len(s.busy) == 3
    clk.t = 1.0
    s.submit(req(5, 5))
    s.submit(req(6, 5))
    s.poll()
    assert len(s.busy) == 3            # still running; newcomers wait
    clk.t = 2.0
    s.poll()                           # first three done; waiting ones admitted together
    assert [h["reqs"] for h in ex.launches[3:]] == [[3], [4], [5, 6]]
    clk.t = 4.0
    s.poll()
    assert s.idle() and len(s.completed) == 7


def test_oversized_requests_are_rejected():
    clk = FakeClock()
    ex = FakeExecutor(clk)
    s = Server(ex, lanes=1, budget=10**6, max_batch=50, clock=clk)
    with pytest.raises(RejectedRequest):
        s.submit(req(0, 51))
    with pytest.raises(RejectedRequest):
        s.submit(req(1, 49 * 100))     # within max_batch? no: also over budget
    s2 = Server(ex, lanes=1, budget=2000, max_batch=10**6, clock=clk)
    with pytest.raises(RejectedRequest):
        s2.submit(req(2, 10))


def test_batches_keep_cost_classes_apart():
    clk = FakeClock()
    ex = FakeExecutor(clk)
    s = Server(ex, lanes=3, budget=10**12, max_batch=1000, clock=clk)
    s.submit(req(0, 10))
    s.submit(req(1, 10))
    s.submit(req(2, 10, ms=1e-4, delta=1e-6))     # separation above tolerance
    s.submit(req(3, 10, ms=1e-4, delta=1e-6))
    s.submit(req(4, 10, ms=1e-4, delta=1e-3))     # separation below tolerance: cheap
    s.poll()
    assert [h["reqs"] for h in ex.launches] == [[0, 1], [2, 3], [4]]
    s2 = Server(FakeExecutor(clk), lanes=1, budget=10**12, max_batch=1000, clock=clk,
                classify=None)
    for i in range(5):
        s2.submit(req(i, 10, ms=1e-4 * (i % 2)))
    s2.poll()
    assert [h["reqs"] for h in s2.ex.launches] == [[0, 1, 2, 3, 4]]
