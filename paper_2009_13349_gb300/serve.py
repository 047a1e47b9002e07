"""Continuous-batching CCD request server.

Clients submit requests -- a set of queries of one kind with their own
delta, ms and m_I, as when many simulations' line searches call CCD with
per-step tolerances.  The server keeps several CUDA streams ("lanes").
Whenever a lane is free it forms a batch from the requests waiting at that
moment (FIFO, up to ``max_batch`` queries) admitted against a device-memory
budget that covers every batch in flight (inputs, outputs and workspace),
uploads them into one device array, and runs one multi-instance call (one
segment per request: per-request eps from the request's own bounds, Sec. 6).
Batches on different lanes overlap on the device; requests that arrive
while others run join the next free lane.  Results are identical to solving
each request alone (the solvers are deterministic and independent of how
queries are batched).

The scheduling logic (admission, budget accounting, completion) is plain
host code driving an executor; ``GpuExecutor`` runs batches through the C
ABI.  A request larger than what one batch may hold, or whose memory alone
exceeds the budget, is rejected at submission.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

VF, EE = 0, 1
QUERY_BYTES = 24 * 8 + 1 + 8 + 8   # inputs + collides + toi + out_tol


@dataclass
class Request:
    id: int
    kind: int
    aos: object            # host (n, 24) float64 array or tensor, one query per row
    delta: float = 1e-6
    ms: float = 0.0
    max_itr: int = 10**6
    arrival: float = 0.0
    # filled by the server
    collides: np.ndarray = None
    toi: np.ndarray = None
    out_tol: np.ndarray = None
    done: float = None
    batch: int = None

    @property
    def n(self) -> int:
        return int(self.aos.shape[0])


class RejectedRequest(ValueError):
    pass


@dataclass
class _Batch:
    id: int
    lane: int
    requests: list
    nbytes: int
    handle: object = None


def cost_class(r: Request) -> int:
    """Requests whose minimum separation exceeds their tolerance subdivide a
    whole |F| <= d region down to w(B) < delta (often to the check limit);
    they are batched only with each other so that cheap requests do not wait
    for them."""
    return int(r.ms > 0.0 and r.delta < r.ms)


class Server:
    """Continuous batching over ``lanes`` executor lanes within ``budget`` bytes.
    A batch takes requests from the FIFO head while they share the head's
    cost class (``classify``; None puts every request in one class)."""

    def __init__(self, executor, lanes: int = 4, budget: int = 40 << 30,
                 max_batch: int = 1 << 20, clock=time.perf_counter, classify=cost_class):
        self.ex = executor
        self.lanes = lanes
        self.budget = int(budget)
        self.max_batch = int(max_batch)
        self.clock = clock
        self.waiting = collections.deque()
        self.busy = {}                  # lane -> _Batch
        self.in_flight_bytes = 0
        self.completed = []
        self._next_batch = 0
        self.peak_bytes = 0
        self.classify = classify

    def batch_bytes(self, n: int) -> int:
        return int(n) * QUERY_BYTES + self.ex.workspace_bytes(int(n))

    def submit(self, req: Request) -> None:
        if req.n > self.max_batch or self.batch_bytes(req.n) > self.budget:
            raise RejectedRequest(f"request {req.id}: {req.n} queries exceed the batch or "
                                  f"memory budget")
        if req.arrival == 0.0:
            req.arrival = self.clock()
        self.waiting.append(req)

    def _admit(self, lane: int) -> bool:
        """Form one batch for a free lane from the FIFO head, within budget."""
        take, n = [], 0
        room = self.budget - self.in_flight_bytes
        cls = self.classify(self.waiting[0]) if (self.classify and self.waiting) else None
        while self.waiting:
            r = self.waiting[0]
            if n + r.n > self.max_batch or self.batch_bytes(n + r.n) > room:
                break
            if cls is not None and self.classify(r) != cls:
                break
            take.append(self.waiting.popleft())
            n += r.n
        if not take:
            return False
        b = _Batch(self._next_batch, lane, take, self.batch_bytes(n))
        self._next_batch += 1
        self.in_flight_bytes += b.nbytes
        self.peak_bytes = max(self.peak_bytes, self.in_flight_bytes)
        for r in take:
            r.batch = b.id
        b.handle = self.ex.launch(lane, take)
        self.busy[lane] = b
        return True

    def poll(self) -> list:
        """Harvest finished batches, then give free lanes new work."""
        done = []
        for lane, b in list(self.busy.items()):
            if self.ex.ready(b.handle):
                now = self.clock()
                self.ex.harvest(b.handle, b.requests)
                for r in b.requests:
                    r.done = now
                done.extend(b.requests)
                self.in_flight_bytes -= b.nbytes
                del self.busy[lane]
        for lane in range(self.lanes):
            if lane not in self.busy and self.waiting:
                if not self._admit(lane):
                    break
        self.completed.extend(done)
        return done

    def idle(self) -> bool:
        return not self.waiting and not self.busy

    def drain(self, sleep: float = 0.0) -> None:
        while not self.idle():
            self.poll()
            if sleep:
                time.sleep(sleep)


class GpuExecutor:
    """Runs a batch of requests on one CUDA stream per lane through the C ABI:
    per-request uploads into one (24, n) device array, per-segment eps from
    bounds, ccd_multi_batch, and result copies into pinned host memory."""

    def __init__(self, lanes: int, max_itr_bound: int = 10**6, tuning=None, device=None):
        import torch
        from . import ccd
        self.torch, self.ccd = torch, ccd
        self.dev = torch.device(device or "cuda")
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(lanes)]
        self.max_itr_bound = int(max_itr_bound)
        self.tuning = tuning

    def workspace_bytes(self, n: int) -> int:
        return self.ccd.multi_workspace_bytes(max(n, 1), self.max_itr_bound, self.tuning)

    def launch(self, lane: int, reqs: list):
        torch, ccd = self.torch, self.ccd
        s = self.streams[lane]
        n = sum(r.n for r in reqs)
        seg = ccd.make_segments([r.n for r in reqs], [r.kind for r in reqs],
                                [r.ms for r in reqs], [r.delta for r in reqs],
                                [r.max_itr for r in reqs])
        with torch.cuda.stream(s):
            aos = torch.empty((n, 24), dtype=torch.float64, device=self.dev)
            verts = torch.empty((24, n), dtype=torch.float64, device=self.dev)
            off = 0
            for r in reqs:
                src = r.aos if isinstance(r.aos, torch.Tensor) else torch.from_numpy(r.aos)
                aos[off:off + r.n].copy_(src, non_blocking=True)
                off += r.n
            ccd.aos_to_soa(aos, verts, 0, stream=s)
            seg_host = torch.from_numpy(seg.view(np.uint8).copy()).pin_memory()
            seg_dev = seg_host.to(self.dev, non_blocking=True)
            ws = torch.empty(self.workspace_bytes(n), dtype=torch.uint8, device=self.dev)
            ccd.segments_err_from_bounds(verts, seg_dev, stream=s)
            res = ccd.multi_batch(verts, seg_dev, self.max_itr_bound, ws=ws, tuning=self.tuning,
                                  with_checks=False, stream=s)
            host = (torch.empty(n, dtype=torch.uint8).pin_memory(),
                    torch.empty(n, dtype=torch.float64).pin_memory(),
                    torch.empty(n, dtype=torch.float64).pin_memory())
            host[0].copy_(res.collides, non_blocking=True)
            host[1].copy_(res.toi, non_blocking=True)
            host[2].copy_(res.out_tol, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        # keep device tensors alive until the stream is past them
        return {"event": ev, "host": host, "keep": (aos, verts, seg_host, seg_dev, ws, res)}

    def ready(self, handle) -> bool:
        return handle["event"].query()

    def harvest(self, handle, reqs: list) -> None:
        handle["event"].synchronize()
        col, toi, tol = (h.numpy() for h in handle["host"])
        off = 0
        for r in reqs:
            r.collides = col[off:off + r.n].copy()
            r.toi = toi[off:off + r.n].copy()
            r.out_tol = tol[off:off + r.n].copy()
            off += r.n
        handle["keep"] = None


def run_stream(server: Server, requests: list, clock=time.perf_counter, t0=None):
    """Replays ``requests`` (sorted by their ``arrival`` offsets in seconds)
    in real time: each is submitted once its arrival time has passed.
    Returns the wall time from the first arrival to the last completion."""
    t0 = clock() if t0 is None else t0
    pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
    offsets = {r.id: r.arrival for r in pending}
    while pending or not server.idle():
        now = clock() - t0
        while pending and offsets[pending[0].id] <= now:
            r = pending.popleft()
            r.arrival = t0 + offsets[r.id]
            server.submit(r)
        server.poll()
    return clock() - t0


def serial_baseline(executor, requests: list, clock=time.perf_counter, t0=None):
    """One call per request, in arrival order, each waiting for the previous
    (the one-launch-per-request form).  Same real-time arrival replay."""
    t0 = clock() if t0 is None else t0
    for r in sorted(requests, key=lambda r: r.arrival):
        start = t0 + r.arrival
        while clock() < start:
            pass
        r.arrival = start
        h = executor.launch(0, [r])
        executor.harvest(h, [r])
        r.done = clock()
    return clock() - t0


def latency_stats(requests: list) -> dict:
    lat = np.array([(r.done - r.arrival) * 1e3 for r in requests if r.done is not None])
    q = sum(r.n for r in requests if r.done is not None)
    span = max(r.done for r in requests) - min(r.arrival for r in requests)
    return {"requests": int(lat.size), "queries": int(q),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "queries_per_s": q / span}
