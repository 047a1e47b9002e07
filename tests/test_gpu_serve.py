"""Served mode on the GPU: every request's answer is the same in the mix as
when solved alone (and as from the single-batch entry points)."""
import numpy as np
import pytest
import torch

from paper_2009_13349_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_aos_to_soa_layout_kernel():
    from paper_2009_13349_gb300 import ccd
    a = torch.randn(1000, 24, dtype=torch.float64, device="cuda")
    out = torch.zeros(24, 1300, dtype=torch.float64, device="cuda")
    ccd.aos_to_soa(a, out, 123)
    torch.cuda.synchronize()
    assert torch.equal(out[:, 123:1123], a.t())
    assert torch.count_nonzero(out[:, :123]) == 0 and torch.count_nonzero(out[:, 1123:]) == 0


def test_each_result_same_alone_and_in_the_mix():
    from paper_2009_13349_gb300 import ccd
    from paper_2009_13349_gb300.serve import GpuExecutor, Request, Server
    rng = np.random.default_rng(17)
    reqs = []
    for i in range(24):
        kind = int(rng.integers(0, 2))
        n = int(np.exp(rng.uniform(np.log(50), np.log(20_000))))
        b = W.unit_cube(kind, n, seed=1000 + i) if i % 3 else W.simulation_mixed(
            n=2 * n, seed=2000 + i).batches[kind]
        reqs.append(Request(i, kind, np.ascontiguousarray(b.verts),
                            delta=float(rng.choice([1e-4, 1e-6])),
                            ms=float(rng.choice([0.0, 1e-4])),
                            max_itr=int(rng.choice([1000, 10**6]))))
    ex = GpuExecutor(lanes=3, max_itr_bound=10**6,
                     tuning={"deep_threads": 512, "deep_slots": 16, "small_blocks_per_sm": 8,
                             "small_cap": 1024})
    srv = Server(ex, lanes=3, budget=12 << 30, max_batch=60_000)
    for r in reqs:
        srv.submit(r)
    srv.drain()
    assert len(srv.completed) == len(reqs)
    assert len({r.batch for r in reqs}) > 1          # several batches, some shared
    assert any(sum(q.batch == r.batch for q in reqs) > 1 for r in reqs)
    for r in reqs:
        v = ccd.to_soa(r.aos)
        e = ccd.err_from_bounds(r.kind, v, ms_nonzero=r.ms > 0)
        alone = ccd.batch(r.kind, v, e, ms=r.ms, delta=r.delta, max_itr=r.max_itr)
        torch.cuda.synchronize()
        assert np.array_equal(r.collides, alone.collides.cpu().numpy())
        assert np.array_equal(r.toi, alone.toi.cpu().numpy())
        assert np.array_equal(r.out_tol, alone.out_tol.cpu().numpy())
