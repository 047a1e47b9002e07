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
        e = ccd.err_from_bounds(b.kind, v)
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
        o = oracle.ccd_batch(b.kind, b.verts, e.cpu().numpy(), delta=1e-6, max_itr=10**6,
                             nthreads=8)
        assert np.array_equal(chk, o[3])
