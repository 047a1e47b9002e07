"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

The GPU evaluates the same fixed F expression with the same rounding and
reproduces Algorithm 2's sequential order exactly, so the bar is equality:
collision flags bit-exact, toi and out_tol equal (the stated tolerance
|dtoi| <= 1e-6 is implied), check counts equal.  Constructed collisions must
never be missed (zero false negatives) and toi must not exceed t*.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2009_13349_gb300 import workloads as W

pytestmark = pytest.mark.gpu
NT = os.cpu_count() or 1
TOI_TOL = 1e-6


@pytest.fixture(scope="module")
def ccd():
    from paper_2009_13349_gb300 import ccd as m
    assert torch.cuda.is_available()
    return m


def gpu_run(ccd, kind, verts, ms=0.0, delta=1e-6, max_itr=10**6, per_query=False, ws=None,
            err=None):
    """The CUDA batch on the oracle's eps (the GPU's own eps is checked bit
    for bit in test_err_from_bounds_bit_exact); returns its outputs and that
    eps, for the oracle run."""
    v = ccd.to_soa(verts)
    if err is None:
        err = oracle.err_from_bounds(kind, verts, ms_nonzero=ms > 0, per_query=per_query)
    e = torch.as_tensor(err, dtype=torch.float64, device="cuda").contiguous()
    r = ccd.batch(kind, v, e, ms=ms, delta=delta, max_itr=max_itr, ws=ws)
    torch.cuda.synchronize()
    out = (r.collides.cpu().numpy(), r.toi.cpu().numpy(), r.out_tol.cpu().numpy(),
           r.checks.cpu().numpy())
    return out, np.asarray(err, dtype=np.float64)


def oracle_run(kind, verts, err, ms=0.0, delta=1e-6, max_itr=10**6):
    return oracle.ccd_batch(kind, verts, err, ms=ms, delta=delta, max_itr=max_itr, nthreads=NT)


def assert_parity(g, o, label):
    gc, gt, gw, gk = g
    oc, ot, ow, ok = o
    bad = np.nonzero(gc != oc)[0]
    assert bad.size == 0, f"{label}: {bad.size} flag mismatches, e.g. {bad[:8]}"
    hit = oc == 1
    assert np.all(np.abs(gt[hit] - ot[hit]) <= TOI_TOL), f"{label}: toi beyond 1e-6"
    assert np.all(np.isinf(gt[~hit]))
    bad = np.nonzero(gt != ot)[0]
    assert bad.size == 0, f"{label}: {bad.size} toi differ, e.g. {bad[:8]}"
    bad = np.nonzero(gw != ow)[0]
    assert bad.size == 0, f"{label}: {bad.size} out_tol differ, e.g. {bad[:8]}"
    bad = np.nonzero(gk != ok)[0]
    assert bad.size == 0, f"{label}: {bad.size} check counts differ, e.g. {bad[:8]}"


def assert_truth(g, b, label):
    gc, gt = g[0], g[1]
    hit = b.truth == 1
    assert np.all(gc[hit] == 1), f"{label}: false negative on a constructed collision"
    assert np.all(gt[hit] <= b.t_star[hit]), f"{label}: toi after the constructed contact"
    assert np.all(gc[b.truth == 0] == 0)


def test_err_from_bounds_bit_exact(ccd):
    b = W.simulation_mixed(n=5000, seed=9).batches
    for bb in b:
        for ms in (False, True):
            for pq in (False, True):
                g = ccd.err_from_bounds(bb.kind, ccd.to_soa(bb.verts), ms_nonzero=ms,
                                        per_query=pq).cpu().numpy()
                o = oracle.err_from_bounds(bb.kind, bb.verts, ms_nonzero=ms, per_query=pq)
                assert np.array_equal(g, o)


@pytest.mark.parametrize("kind", [0, 1])
def test_uniform_10k(ccd, kind):
    """10,000 queries, seed 0 (VF: the uniform unit-cube workload; EE: its
    edge-edge analogue): half constructed collisions, half disjoint."""
    b = W.uniform_vf_10k().batches[0] if kind == 0 else W.unit_cube(1, 10_000, seed=0)
    g, e = gpu_run(ccd, kind, b.verts)
    o = oracle_run(kind, b.verts, e)
    assert_parity(g, o, f"uniform kind={kind}")
    assert_truth(g, b, f"uniform kind={kind}")


def test_simulation_mixed_sample(ccd):
    wl = W.simulation_mixed(n=40_000, seed=1)
    for b in wl.batches:
        g, e = gpu_run(ccd, b.kind, b.verts)
        o = oracle_run(b.kind, b.verts, e)
        assert_parity(g, o, f"simulation kind={b.kind}")
        assert_truth(g, b, f"simulation kind={b.kind}")


@pytest.mark.parametrize("ms", [0.0, 1e-4])
def test_degenerate_heavy_sample(ccd, ms):
    wl = W.degenerate_heavy(n=300, seed=2)
    for b in wl.batches:
        g, e = gpu_run(ccd, b.kind, b.verts, ms=ms)
        o = oracle_run(b.kind, b.verts, e, ms=ms)
        assert_parity(g, o, f"degenerate kind={b.kind} ms={ms}")


@pytest.mark.parametrize("kind", [0, 1])
def test_edge_cases(ccd, kind):
    base = W.simulation_mixed(n=2000, seed=12).batches[kind].verts
    # empty batch: a valid no-op
    v = ccd.to_soa(np.zeros((0, 24)))
    e = torch.ones(3, dtype=torch.float64, device="cuda")
    r = ccd.batch(kind, v, e)
    torch.cuda.synchronize()
    assert r.collides.numel() == 0
    # ragged sizes around the warp / block widths
    for n in (1, 2, 31, 33, 255, 257):
        g, e = gpu_run(ccd, kind, base[:n])
        assert_parity(g, oracle_run(kind, base[:n], e), f"n={n}")
    # check limits that cut levels at every position, tolerances, per-query eps
    for max_itr in (1, 2, 3, 7, 50, 1000):
        g, e = gpu_run(ccd, kind, base, max_itr=max_itr)
        assert_parity(g, oracle_run(kind, base, e, max_itr=max_itr), f"max_itr={max_itr}")
    for delta in (1e-1, 1e-3, 1e-9):
        g, e = gpu_run(ccd, kind, base, delta=delta)
        assert_parity(g, oracle_run(kind, base, e, delta=delta), f"delta={delta}")
    g, e = gpu_run(ccd, kind, base, per_query=True)
    assert e.shape == (base.shape[0], 3)
    assert_parity(g, oracle_run(kind, base, e), "per-query eps")
    g, e = gpu_run(ccd, kind, base, ms=1e-3)
    assert_parity(g, oracle_run(kind, base, e, ms=1e-3), "ms=1e-3")
    # a large tolerance terminates at level 0
    g, e = gpu_run(ccd, kind, base, delta=10.0)
    assert np.all(g[3] == 1)


def test_termination_branches(ccd):
    """The inputs that pin the inside-C_eps termination (plain and under
    minimum separation) and the depth guard in the oracle's tests: a tiny
    static triangle with a point 2^-52 inside it, and a point resting on a
    unit triangle with eps = 0 and delta = 1e-300."""
    a, p = 2.0**-50, 2.0**-52
    V = [0.0, 0.0, 0.0, a, 0.0, 0.0, 0.0, a, 0.0]
    tiny = np.array([[p, p, 0.0, *V, p, p, 2.0**-51, *V]])
    for ms in (0.0, 16 * 2.0**-52, 32 * 2.0**-52):
        g, e = gpu_run(ccd, 0, tiny, ms=ms, delta=2.0**-52)
        assert_parity(g, oracle_run(0, tiny, e, ms=ms, delta=2.0**-52), f"inside ms={ms}")
    g, e = gpu_run(ccd, 0, tiny, delta=2.0**-52, err=np.full(3, 2.0**-52))
    assert_parity(g, oracle_run(0, tiny, e, delta=2.0**-52), "not inside")
    U1 = [0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0, 0.0]
    rest = np.array([[0.25, 0.25, 0.0, *U1, 0.25, 0.25, 0.0, *U1]])
    g, e = gpu_run(ccd, 0, rest, delta=1e-300, err=np.zeros(3))
    assert_parity(g, oracle_run(0, rest, e, delta=1e-300), "depth guard")
    assert g[2][0] in (2.0**-53, 2.0**-52)


def test_paper_examples(ccd, golden):
    for name in ("hourglass_vf.txt", "inflection_vf.txt", "bsc_false_negative_vf.txt"):
        q, meta = golden(name)
        verts = q.reshape(1, 24)
        g, e = gpu_run(ccd, meta["kind"], verts, max_itr=10**6)
        o = oracle_run(meta["kind"], verts, e, max_itr=10**6)
        assert_parity(g, o, name)
        assert g[0][0] == meta["truth"]


def test_determinism_and_workspace_reuse(ccd):
    wl = W.simulation_mixed(n=20_000, seed=13)
    vf, ee = wl.batches
    ws = ccd.workspace(max(vf.n, ee.n), 10**6)
    outs = []
    for _ in range(2):
        for b in (vf, ee):
            g, _ = gpu_run(ccd, b.kind, b.verts, ws=ws)
            outs.append(g)
    for a, b in zip(outs[:2], outs[2:]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    assert ccd.workspace_status(ws) == (0, 0)


def test_capacity_fallback_is_conservative(ccd):
    """A workspace too small for a full-size slot: its deep tier is one
    contiguous slot of 1024 boxes, so queries whose frontier needs more
    return as at the check limit, flagged CCD_ERR_CAPACITY, and the answer
    stays conservative (never a missed collision, toi never later than the
    oracle's)."""
    b = W.degenerate_heavy(n=200, seed=21).batches[0]
    n, max_itr = b.n, 10**6
    full = ccd.workspace_bytes(n, max_itr)
    fixed = ccd.workspace_layout(n, max_itr, full)["fixed_bytes"]
    ws = torch.empty(fixed + 2 * 1024 * 24, dtype=torch.uint8, device="cuda")
    lay = ccd.workspace_layout(n, max_itr, ws.numel())
    assert lay["paged"] == 0 and lay["slot_boxes"] == 1024
    g, e = gpu_run(ccd, b.kind, b.verts, ws=ws)
    st, fb = ccd.workspace_status(ws)
    assert st == -5 and fb > 0
    o = oracle_run(b.kind, b.verts, e)
    assert np.all(g[0] >= o[0])
    both = (g[0] == 1) & (o[0] == 1)
    assert np.all(g[1][both] <= o[1][both])


@pytest.mark.parametrize("kind", [0, 1])
def test_frontier_pool_size_changes_nothing(ccd, kind):
    """The deep tier's page pool at two pages: nearly every deep query finds
    it empty and restarts in a full-size slot.  Outputs equal the oracle's
    and those of a default workspace, with no capacity fallback."""
    b = W.degenerate_heavy(n=400, seed=23).batches[kind]
    full = ccd.workspace(b.n, 10**6)
    lay = ccd.workspace_layout(b.n, 10**6, full.numel())
    assert lay["paged"] == 1 and lay["full_slots"] == 2
    tiny = ccd.workspace(b.n, 10**6, pages=2)
    assert ccd.workspace_layout(b.n, 10**6, tiny.numel())["pages"] == 2
    g_full, e = gpu_run(ccd, kind, b.verts, ws=full)
    c_full = ccd.workspace_counters(full)
    g_tiny, _ = gpu_run(ccd, kind, b.verts, ws=tiny)
    c_tiny = ccd.workspace_counters(tiny)
    assert c_full["status"] == 0 and c_tiny["status"] == 0
    assert c_tiny["deferred_queries"] > 0 and c_tiny["pages_peak"] <= 2
    assert c_full["pages_peak"] <= lay["pages"]
    for x, y in zip(g_full, g_tiny):
        assert np.array_equal(x, y)
    assert_parity(g_tiny, oracle_run(kind, b.verts, e), f"two-page pool kind={kind}")


def test_full_size_simulation_sampled(ccd):
    """The 1,000,000-query simulation-shaped workload in the benchmark's
    launch configuration; every output is checked against the oracle on a
    random sample, and every constructed collision against its truth."""
    wl = W.simulation_mixed(n=1_000_000, seed=1)
    rng = np.random.default_rng(99)
    for b in wl.batches:
        g, e = gpu_run(ccd, b.kind, b.verts)
        assert_truth(g, b, f"full kind={b.kind}")
        idx = np.sort(rng.choice(b.n, 2500, replace=False))
        o = oracle_run(b.kind, b.verts[idx], e)
        assert_parity(tuple(x[idx] for x in g), o, f"full-size sample kind={b.kind}")
