"""Driver of the served form (the C server behind ccd_batch_begin / submit /
poll / cancel / end in include/ccd.h): requests in, finished requests out.

Admission against the device budget, the device-resident request queue,
batch formation, lanes, time-sliced deep rounds and result delivery all run
in the library; this module keeps each request's host arrays alive until the
server reports it, and offers the measurement helpers of the benchmark
(real-time arrival replay, one call per request, latency statistics).
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

VF, EE = 0, 1


@dataclass
class Request:
    id: int
    kind: int
    aos: np.ndarray            # host (n, 24) float64, one query per row
    delta: float = 1e-6
    ms: float = 0.0
    max_itr: int = 10**6
    arrival: float = 0.0
    # filled when the request finishes
    collides: np.ndarray = None
    toi: np.ndarray = None
    out_tol: np.ndarray = None
    checks: np.ndarray = None
    status: int = None
    done: float = None

    @property
    def n(self) -> int:
        return int(self.aos.shape[0])


class Server:
    """One C server (see include/ccd.h, "The served form")."""

    def __init__(self, budget: int = 40 << 30, lanes: int = 4, max_batch: int = 1 << 20,
                 max_itr_bound: int = 10**6, deep_slice_us: int = 0, clock=time.perf_counter,
                 **config):
        from . import ccd
        self.native = ccd.NativeServer(budget_bytes=int(budget), lanes=int(lanes),
                                       max_batch=int(max_batch), max_itr_bound=int(max_itr_bound),
                                       deep_slice_us=int(deep_slice_us), **config)
        self.clock = clock
        self.pending = {}          # ticket -> Request
        self.completed = []

    def submit(self, req: Request) -> bool:
        """Queues the request; False when the server has no room for it now."""
        req.aos = np.ascontiguousarray(req.aos, dtype=np.float64)
        req.collides = np.empty(req.n, dtype=np.uint8)
        req.toi = np.empty(req.n, dtype=np.float64)
        req.out_tol = np.empty(req.n, dtype=np.float64)
        req.checks = np.empty(req.n, dtype=np.int64)
        t = self.native.submit(req.kind, req.aos, req.ms, req.delta, req.max_itr, req.collides,
                               req.toi, req.out_tol, req.checks)
        if t is None:
            return False
        if req.arrival == 0.0:
            req.arrival = self.clock()
        self.pending[t] = req
        return True

    def poll(self, wait_us: int = 0) -> list:
        out = []
        for t, status in self.native.poll(wait_us=wait_us):
            r = self.pending.pop(t)
            r.status = status
            r.done = self.clock()
            out.append(r)
        self.completed.extend(out)
        return out

    def cancel(self, req_ticket: int) -> int:
        return self.native.cancel(req_ticket)

    def idle(self) -> bool:
        return not self.pending

    def drain(self, wait_us: int = 1000) -> None:
        while self.pending:
            self.poll(wait_us)

    def stats(self) -> dict:
        return self.native.stats()

    def close(self):
        self.native.close()


def run_stream(server: Server, requests: list, clock=time.perf_counter, t0=None):
    """Replays ``requests`` (``arrival`` = offset in seconds) in real time:
    each is submitted once its arrival time has passed (and again after a
    poll if the server had no room).  Returns the wall time from the first
    arrival to the last completion."""
    t0 = clock() if t0 is None else t0
    pending = sorted(requests, key=lambda r: r.arrival)
    offsets = {r.id: r.arrival for r in pending}
    i = 0
    while i < len(pending) or not server.idle():
        now = clock() - t0
        while i < len(pending) and offsets[pending[i].id] <= now:
            r = pending[i]
            r.arrival = t0 + offsets[r.id]
            if not server.submit(r):
                break
            i += 1
        server.poll(wait_us=200)
    return clock() - t0


def serial_baseline(run_one, requests: list, clock=time.perf_counter, t0=None):
    """One call per request, in arrival order, each after the previous
    finished (the one-launch-per-request form), under the same real-time
    arrivals; run_one(request) fills the request's outputs."""
    t0 = clock() if t0 is None else t0
    for r in sorted(requests, key=lambda r: r.arrival):
        start = t0 + r.arrival
        while clock() < start:
            time.sleep(0.0002)
        r.arrival = start
        run_one(r)
        r.done = clock()
    return clock() - t0


def latency_stats(requests: list) -> dict:
    lat = np.array([(r.done - r.arrival) * 1e3 for r in requests if r.done is not None])
    q = sum(r.n for r in requests if r.done is not None)
    span = max(r.done for r in requests) - min(r.arrival for r in requests)
    return {"requests": int(lat.size), "queries": int(q),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "queries_per_s": q / span}
