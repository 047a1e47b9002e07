"""GPU: the four solver stages account for every query and every check.

A query is answered by the level-0 kernel (one check) or by exactly one of
the pooled, one-warp and deep solvers; the per-stage sums of check counts
the kernels tally must add up to the per-query counts they write.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_13349_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ccd():
    from paper_2009_13349_gb300 import ccd as m
    assert torch.cuda.is_available()
    return m


@pytest.mark.parametrize("wl", ["simulation", "degenerate"])
def test_stage_accounting(ccd, wl):
    batches = (W.simulation_mixed(n=20_000, seed=5).batches if wl == "simulation"
               else W.degenerate_heavy(n=2_000, seed=6).batches)
    for b in batches:
        v = ccd.to_soa(b.verts)
        eo = oracle.err_from_bounds(b.kind, b.verts)
        e = torch.as_tensor(eo, device="cuda")
        ws = ccd.workspace(b.n, 10**6)
        r = ccd.batch(b.kind, v, e, delta=1e-6, max_itr=10**6, ws=ws)
        torch.cuda.synchronize()
        c = ccd.workspace_counters(ws)
        chk = r.checks.cpu().numpy()
        assert c["status"] == 0
        assert int(chk.sum()) == (b.n - c["survivors"]) + c["checks_pool"] + \
            c["checks_small"] + c["checks_deep"]
        assert c["mid_queries"] <= c["survivors"]
        assert c["deep_queries"] <= c["mid_queries"]
        assert c["evals_pool"] >= c["checks_pool"]
        if wl == "degenerate":
            # long frontiers: some queries leave the pooled solver
            assert c["mid_queries"] > 0
        o = oracle.ccd_batch(b.kind, b.verts, eo, delta=1e-6, max_itr=10**6,
                             nthreads=8)
        assert np.array_equal(chk, o[3])


def test_deep_chunks_beyond_the_run_table(ccd):
    """Deep queries whose 256-box chunks hold more than 128 runs of equal t_L
    (nearly every box with its own t_L) are evaluated as sub-chunks of 128
    boxes; outputs equal the oracle's.  By a level-synchronous model of
    Algorithm 2's frontiers, queries 2893 (VF: levels up to 20,170 boxes, up
    to 162 runs in a chunk) and 1577 (EE: 8,010 boxes, 173 runs) of this
    seeded workload reach the deep solver with such chunks; 246 and 902 (VF)
    are deep queries with up to 140 and 114 runs."""
    wl = W.simulation_mixed(n=20_000, seed=1)
    picks = {0: [246, 902, 2893], 1: [1577]}
    for b in wl.batches:
        idx = picks[b.kind]
        eo = oracle.err_from_bounds(b.kind, b.verts)      # the scene's eps
        rows = b.verts[idx]
        ws = ccd.workspace(len(idx), 10**6)
        r = ccd.batch(b.kind, ccd.to_soa(rows), torch.as_tensor(eo, device="cuda"), delta=1e-6,
                      max_itr=10**6, ws=ws)
        torch.cuda.synchronize()
        c = ccd.workspace_counters(ws)
        assert c["status"] == 0 and c["deep_queries"] >= 1
        assert c["split_chunks_deep"] > 0
        assert c["evals_shared_deep"] == c["evals_deep"]
        o = oracle.ccd_batch(b.kind, rows, eo, delta=1e-6, max_itr=10**6, nthreads=4)
        got = (r.collides.cpu().numpy(), r.toi.cpu().numpy(), r.out_tol.cpu().numpy(),
               r.checks.cpu().numpy())
        for x, y in zip(got, o):
            assert np.array_equal(x, y)
