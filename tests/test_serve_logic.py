"""Host-side scheduling of the request server (csrc/serve_queue.h), on the
CPU: where a request goes in the inbox ring, which waiting requests form a
lane's batch, and which finished requests give their space back.  A
randomized run of the server's host flow (submissions, batches on lanes of
both priorities, completions out of order, reports, releases) checks that
live requests never overlap in the inbox, every batch is a contiguous run of
waiting requests of one class within the limits, high-priority lanes take
only cheap requests, and space comes back in inbox order."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WAITING, RUNNING, DONE, CANCELLED = range(4)


@pytest.fixture(scope="module")
def Q():
    tmp = tempfile.mkdtemp()
    so = os.path.join(tmp, "serve_queue_harness.so")
    subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-I",
                    os.path.join(ROOT, "paper_2009_13349_gb300", "csrc"), "-o", so,
                    os.path.join(ROOT, "tests", "serve_queue_harness.cpp")], check=True)
    L = ctypes.CDLL(so)
    pl, pi, pu = (ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int),
                  ctypes.POINTER(ctypes.c_ubyte))
    L.h_alloc.argtypes = [pl, pl, ctypes.c_int, ctypes.c_longlong, ctypes.c_longlong]
    L.h_alloc.restype = ctypes.c_longlong
    L.h_select.argtypes = [pl, pl, pi, pi, ctypes.c_int, ctypes.c_int, ctypes.c_longlong,
                           ctypes.c_int, pl, pl]
    L.h_select.restype = ctypes.c_int
    L.h_releasable.argtypes = [pi, pu, ctypes.c_int]
    L.h_releasable.restype = ctypes.c_longlong
    return L


def _arr(x, t):
    return (t * max(1, len(x)))(*x)


def alloc(Q, reqs, cap, want):
    return Q.h_alloc(_arr([r["off"] for r in reqs], ctypes.c_longlong),
                     _arr([r["n"] for r in reqs], ctypes.c_longlong), len(reqs), cap, want)


def select(Q, reqs, high, max_batch, max_segs):
    f, k = ctypes.c_longlong(), ctypes.c_longlong()
    ok = Q.h_select(_arr([r["off"] for r in reqs], ctypes.c_longlong),
                    _arr([r["n"] for r in reqs], ctypes.c_longlong),
                    _arr([r["state"] for r in reqs], ctypes.c_int),
                    _arr([r["cls"] for r in reqs], ctypes.c_int), len(reqs), int(high), max_batch,
                    max_segs, ctypes.byref(f), ctypes.byref(k))
    return (f.value, k.value) if ok else None


def releasable(Q, reqs):
    return Q.h_releasable(_arr([r["state"] for r in reqs], ctypes.c_int),
                          _arr([int(r["reported"]) for r in reqs], ctypes.c_ubyte), len(reqs))


def test_inbox_ring_cases(Q):
    cap = 100
    assert alloc(Q, [], cap, 100) == 0 and alloc(Q, [], cap, 101) == -1
    a = [{"off": 10, "n": 30}]
    assert alloc(Q, a, cap, 60) == 40          # after the last one
    assert alloc(Q, a, cap, 61) == -1          # neither after it nor before the first
    assert alloc(Q, a, cap, 10) == 40
    b = [{"off": 40, "n": 50}]
    assert alloc(Q, b, cap, 20) == 0           # wraps to the start, before the first
    assert alloc(Q, b, cap, 41) == -1
    w = [{"off": 40, "n": 50}, {"off": 0, "n": 20}]   # wrapped
    assert alloc(Q, w, cap, 20) == 20 and alloc(Q, w, cap, 21) == -1


def test_batch_selection_cases(Q):
    R = lambda off, n, st, c: {"off": off, "n": n, "state": st, "cls": c}
    reqs = [R(0, 10, DONE, 0), R(10, 10, RUNNING, 0), R(20, 10, WAITING, 1),
            R(30, 10, WAITING, 1), R(40, 10, WAITING, 0), R(50, 10, WAITING, 0)]
    assert select(Q, reqs, False, 1000, 100) == (2, 2)    # oldest waiting run, one class
    assert select(Q, reqs, True, 1000, 100) == (4, 2)     # a high lane skips class 1
    assert select(Q, reqs, False, 15, 100) == (2, 1)      # the batch limit
    assert select(Q, reqs, True, 1000, 1) == (4, 1)       # the request limit
    wrap = [R(90, 10, WAITING, 0), R(0, 10, WAITING, 0)]
    assert select(Q, wrap, False, 1000, 100) == (0, 1)    # not contiguous across the ring end
    assert select(Q, [R(0, 5, RUNNING, 0)], False, 10, 10) is None


def test_release_in_order(Q):
    reqs = [{"state": DONE, "reported": True}, {"state": CANCELLED, "reported": True},
            {"state": DONE, "reported": False}, {"state": DONE, "reported": True}]
    assert releasable(Q, reqs) == 2
    reqs[2]["reported"] = True
    assert releasable(Q, reqs) == 4
    assert releasable(Q, [{"state": RUNNING, "reported": False}] + reqs) == 0


def test_randomized_host_flow(Q):
    rng = np.random.default_rng(5)
    cap, max_batch, max_segs = 5000, 1200, 6
    lanes = [{"high": i < 2, "batch": None} for i in range(4)]
    order, live_done = [], 0
    next_id = 0
    for step in range(3000):
        op = rng.random()
        if op < 0.45:                                       # a submission
            n = int(rng.integers(1, 900))
            off = alloc(Q, order, cap, n)
            if off >= 0:
                new = {"id": next_id, "off": off, "n": n, "state": WAITING,
                       "cls": int(rng.random() < 0.3), "reported": False}
                # never overlaps a live request
                for r in order:
                    assert off + n <= r["off"] or r["off"] + r["n"] <= off
                order.append(new)
                next_id += 1
        elif op < 0.75:                                     # an idle lane takes a batch
            L = lanes[int(rng.integers(0, 4))]
            if L["batch"] is None:
                got = select(Q, order, L["high"], max_batch, max_segs)
                if got is not None:
                    f, k = got
                    run = order[f:f + k]
                    assert 1 <= k <= max_segs and sum(r["n"] for r in run) <= max_batch
                    assert all(r["state"] == WAITING for r in run)
                    assert len({r["cls"] for r in run}) == 1
                    if L["high"]:
                        assert run[0]["cls"] == 0
                    first_wait = [r for r in order if r["state"] == WAITING and
                                  (not L["high"] or r["cls"] == 0)][0]
                    assert run[0] is first_wait
                    for a, b in zip(run, run[1:]):
                        assert b["off"] == a["off"] + a["n"]
                    for r in run:
                        r["state"] = RUNNING
                    L["batch"] = run
        elif op < 0.9:                                      # a lane's batch finishes
            busy = [L for L in lanes if L["batch"] is not None]
            if busy:
                L = busy[int(rng.integers(0, len(busy)))]
                for r in L["batch"]:
                    r["state"] = DONE
                L["batch"] = None
        else:                                               # reports, then releases
            for r in order:
                if r["state"] in (DONE, CANCELLED):
                    r["reported"] = True
            k = releasable(Q, order)
            assert all(r["state"] in (DONE, CANCELLED) for r in order[:k])
            live_done += k
            order = order[k:]
    assert live_done > 100 and next_id > 500
