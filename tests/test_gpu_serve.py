"""The served form on the GPU (the C server: ccd_batch_begin / submit / poll /
cancel / end), with requests shaped like the served workload: the uniform
unit-cube generator, sizes log-uniform, per-request delta in {1e-4, 1e-6},
ms in {0, 1e-4}, m_I = 1e6.

Every request's answer must equal the oracle's (on a sample of its queries;
eps from the request's own bounds, Sec. 6) and the answer of a call of its
own, while several batches are in flight at once and the deep stage runs in
rounds (ended by a fixed slice, or when a cheap batch needs the SMs).
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2009_13349_gb300 import workloads as W

pytestmark = pytest.mark.gpu
NT = os.cpu_count() or 1


def test_aos_to_soa_layout_kernel():
    from paper_2009_13349_gb300 import ccd
    a = torch.randn(1000, 24, dtype=torch.float64, device="cuda")
    out = torch.zeros(24, 1300, dtype=torch.float64, device="cuda")
    ccd.aos_to_soa(a, out, 123)
    torch.cuda.synchronize()
    assert torch.equal(out[:, 123:1123], a.t())
    assert torch.count_nonzero(out[:, :123]) == 0 and torch.count_nonzero(out[:, 1123:]) == 0


def _requests(count, lo, hi, seed):
    from paper_2009_13349_gb300.serve import Request
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        kind = int(rng.integers(0, 2))
        n = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        b = W.unit_cube(kind, n, seed=seed * 1000 + i)
        reqs.append(Request(i, kind, b.verts, delta=float(rng.choice([1e-4, 1e-6])),
                            ms=float(rng.choice([0.0, 1e-4])), max_itr=10**6))
    return reqs


def test_served_requests_equal_oracle_and_their_own_calls():
    from paper_2009_13349_gb300 import ccd
    from paper_2009_13349_gb300.serve import Server
    reqs = _requests(28, 100, 20_000, seed=51)
    srv = Server(budget=12 << 30, lanes=4, max_batch=40_000, deep_slice_us=5_000)
    # deep rounds of at most 5 ms, besides the rounds cheap batches end
    for r in reqs:
        assert srv.submit(r)
    srv.drain()
    st = srv.stats()
    srv.close()
    assert len(srv.completed) == len(reqs)
    assert all(r.status == 0 for r in reqs)
    assert st["batches"] > 1 and st["batches"] < len(reqs)      # requests shared batches
    assert st["lanes_busy_peak"] >= 2                           # batches overlapped
    assert st["deep_rounds"] > st["batches"]                    # deep stages were sliced
    assert 0 < st["pages_peak"] <= st["pages"]
    rng = np.random.default_rng(52)
    for r in reqs:
        v = ccd.to_soa(r.aos)
        e = ccd.err_from_bounds(r.kind, v, ms_nonzero=r.ms > 0)
        alone = ccd.batch(r.kind, v, e, ms=r.ms, delta=r.delta, max_itr=r.max_itr)
        torch.cuda.synchronize()
        got = (r.collides, r.toi, r.out_tol, r.checks)
        ref = (alone.collides.cpu().numpy(), alone.toi.cpu().numpy(),
               alone.out_tol.cpu().numpy(), alone.checks.cpu().numpy())
        for x, y in zip(got, ref):
            assert np.array_equal(x, y), f"request {r.id}: served differs from its own call"
        eo = oracle.err_from_bounds(r.kind, r.aos, ms_nonzero=r.ms > 0)
        assert np.array_equal(e.cpu().numpy(), eo)
        idx = np.sort(rng.choice(r.n, min(r.n, 40), replace=False))
        o = oracle.ccd_batch(r.kind, r.aos[idx], eo, ms=r.ms, delta=r.delta, max_itr=r.max_itr,
                             nthreads=NT)
        for x, y in zip(got, o):
            assert np.array_equal(x[idx], y), f"request {r.id}: served differs from the oracle"


def test_cheap_batches_end_expensive_deep_rounds():
    """Expensive requests (ms > delta) run on the low-priority lane; cheap
    ones submitted while its deep stage runs make its rounds end (no fixed
    slice here), and every answer still equals the request's own call."""
    from paper_2009_13349_gb300 import ccd
    from paper_2009_13349_gb300.serve import Request, Server
    rng = np.random.default_rng(71)
    heavy = [Request(i, i % 2, W.unit_cube(i % 2, 6000, seed=700 + i).verts, delta=1e-6,
                     ms=1e-4) for i in range(2)]
    light = [Request(10 + i, i % 2, W.unit_cube(i % 2, int(rng.integers(200, 3000)),
                                                 seed=710 + i).verts, delta=1e-6, ms=0.0)
             for i in range(12)]
    srv = Server(budget=8 << 30, lanes=3, max_batch=20_000)
    for r in heavy:
        assert srv.submit(r)
    for r in light:                      # arrive while the heavy batch runs
        srv.poll(wait_us=2000)
        assert srv.submit(r)
    srv.drain()
    st = srv.stats()
    srv.close()
    assert st["yields"] > 0 and st["deep_rounds"] > st["batches"]
    assert max(r.done for r in light) < max(r.done for r in heavy)
    for r in heavy + light:
        assert r.status == 0
        v = ccd.to_soa(r.aos)
        e = ccd.err_from_bounds(r.kind, v, ms_nonzero=r.ms > 0)
        alone = ccd.batch(r.kind, v, e, ms=r.ms, delta=r.delta, max_itr=r.max_itr)
        torch.cuda.synchronize()
        for x, y in zip((r.collides, r.toi, r.out_tol, r.checks),
                        (alone.collides, alone.toi, alone.out_tol, alone.checks)):
            assert np.array_equal(x, y.cpu().numpy()), f"request {r.id}"


def test_served_backpressure_cancel_and_refusals():
    from paper_2009_13349_gb300 import ccd
    from paper_2009_13349_gb300.serve import Request, Server
    reqs = _requests(12, 200, 900, seed=61)
    # an inbox of 1,000 records: most requests wait for room
    srv = Server(budget=4 << 30, lanes=2, max_batch=1000, inbox_queries=1000,
                 max_itr_bound=10**6)
    taken, refused = [], 0
    for r in reqs:
        if srv.submit(r):
            taken.append(r)
        else:
            refused += 1
    assert refused > 0
    # a request larger than a batch, or with m_I above the bound, can never run
    big = Request(99, 0, np.zeros((1001, 24)))
    with pytest.raises(ccd.CCDError):
        srv.submit(big)
    with pytest.raises(ccd.CCDError):
        srv.submit(Request(98, 0, np.zeros((10, 24)), max_itr=10**7))
    srv.drain()
    # the rest go in as room frees up; cancel the last one while it waits
    taken_ids = {r.id for r in taken}
    rest = [r for r in reqs if r.id not in taken_ids]
    tickets = {}
    for r in rest:
        while not srv.submit(r):
            srv.poll(wait_us=1000)
        tickets[r.id] = max(srv.pending)
    last = rest[-1]
    code = srv.cancel(tickets[last.id])
    srv.drain()
    srv.close()
    done = {r.id: r for r in srv.completed}
    if code == 0:
        assert done[last.id].status == -7
    else:
        assert code == -6 and done[last.id].status == 0     # it was already running
    for r in reqs:
        if r.status != 0:
            continue
        eo = oracle.err_from_bounds(r.kind, r.aos, ms_nonzero=r.ms > 0)
        o = oracle.ccd_batch(r.kind, r.aos, eo, ms=r.ms, delta=r.delta, max_itr=r.max_itr,
                             nthreads=NT)
        for x, y in zip((r.collides, r.toi, r.out_tol, r.checks), o):
            assert np.array_equal(x, y), f"request {r.id}"
