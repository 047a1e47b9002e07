"""Multi-instance batches (segments with their own kind, eps, ms, delta and
m_I in one call): equal to per-instance single calls and to the oracle,
independent of the launch shapes, and replayable from a CUDA graph."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2009_13349_gb300 import workloads as W

pytestmark = pytest.mark.gpu
NT = os.cpu_count() or 1


@pytest.fixture(scope="module")
def ccd():
    from paper_2009_13349_gb300 import ccd as m
    return m


def _instances(count=6, total=24_000, seed=5):
    wl = W.multi_instance(count=count, total=total, seed=seed)
    rng = np.random.default_rng(seed)
    verts = np.concatenate([b.verts for b in wl.batches])
    kinds = [b.kind for b in wl.batches]
    counts = [b.n for b in wl.batches]
    k = len(counts)
    ms = np.where(rng.random(k) < 0.3, 1e-4, 0.0)
    delta = rng.choice([1e-4, 1e-6], k)
    max_itr = rng.choice([100, 10_000, 1_000_000], k)
    return wl, verts, counts, kinds, ms, delta, max_itr


def _out(r):
    return (r.collides.cpu().numpy(), r.toi.cpu().numpy(), r.out_tol.cpu().numpy(),
            r.checks.cpu().numpy())


def _eq(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_segment_eps_bit_exact(ccd):
    wl, verts, counts, kinds, ms, delta, max_itr = _instances()
    seg = ccd.make_segments(counts, kinds, ms, delta, max_itr)
    v = ccd.to_soa(verts)
    sd = ccd.segments_to_device(seg)
    ccd.segments_err_from_bounds(v, sd)
    got = ccd.segments_from_device(sd)["err"]
    for s in range(len(counts)):
        o, c = seg["offset"][s], seg["count"][s]
        ref = oracle.err_from_bounds(kinds[s], verts[o:o + c], ms_nonzero=ms[s] > 0)
        assert np.array_equal(got[s], ref)


def test_multi_equals_single_calls_and_oracle(ccd):
    wl, verts, counts, kinds, ms, delta, max_itr = _instances()
    seg = ccd.make_segments(counts, kinds, ms, delta, max_itr)
    v = ccd.to_soa(verts)
    sd = ccd.segments_to_device(seg)
    ccd.segments_err_from_bounds(v, sd)
    seg = ccd.segments_from_device(sd)
    got = _out(ccd.multi_batch(v, sd, 1_000_000))
    rng = np.random.default_rng(3)
    for s in range(len(counts)):
        o, c = int(seg["offset"][s]), int(seg["count"][s])
        vs = ccd.to_soa(verts[o:o + c])
        e = torch.as_tensor(seg["err"][s], device="cuda")
        ref = _out(ccd.batch(kinds[s], vs, e, ms=ms[s], delta=delta[s], max_itr=int(max_itr[s])))
        _eq([x[o:o + c] for x in got], ref)
        idx = rng.choice(c, min(c, 300), replace=False)
        oe = oracle.err_from_bounds(kinds[s], verts[o:o + c], ms_nonzero=ms[s] > 0)
        assert np.array_equal(seg["err"][s], oe)
        orc = oracle.ccd_batch(kinds[s], verts[o:o + c][idx], oe, ms=ms[s],
                               delta=delta[s], max_itr=int(max_itr[s]), nthreads=NT)
        _eq([x[o:o + c][idx] for x in got], orc)


def test_results_independent_of_tuning(ccd):
    wl, verts, counts, kinds, ms, delta, max_itr = _instances(count=4, total=16_000, seed=8)
    seg = ccd.make_segments(counts, kinds, 0.0, 1e-6, 1_000_000)
    v = ccd.to_soa(verts)
    sd = ccd.segments_to_device(seg)
    ccd.segments_err_from_bounds(v, sd)
    base = _out(ccd.multi_batch(v, sd, 1_000_000))
    for t in ({"deep_threads": 256, "deep_slots": 7, "small_blocks_per_sm": 3, "small_cap": 64},
              {"deep_threads": 512, "deep_slots": 2, "small_blocks_per_sm": 32, "small_cap": 4096},
              {"deep_threads": 256, "deep_slots": 300, "small_blocks_per_sm": 8, "small_cap": 256},
              {"deep_threads": 128, "deep_slots": 900, "small_blocks_per_sm": 8, "small_cap": 64},
              {"pool_cap": 32}, {"pool_cap": 1024, "small_cap": 64}, {"pool_cap": 4096}):
        _eq(_out(ccd.multi_batch(v, sd, 1_000_000, tuning=t)), base)


def test_graph_capture_and_replay_with_new_segments(ccd):
    wl, verts, counts, kinds, ms, delta, max_itr = _instances(count=4, total=12_000, seed=9)
    seg = ccd.make_segments(counts, kinds, 0.0, 1e-6, 100_000)
    v = ccd.to_soa(verts)
    sd = ccd.segments_to_device(seg)
    n = v.shape[1]
    ws = ccd.multi_workspace(n, 100_000)
    out = ccd.Result(torch.empty(n, dtype=torch.uint8, device="cuda"),
                     torch.empty(n, dtype=torch.float64, device="cuda"),
                     torch.empty(n, dtype=torch.float64, device="cuda"),
                     torch.empty(n, dtype=torch.int64, device="cuda"))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):                      # warm-up outside capture
        ccd.segments_err_from_bounds(v, sd, stream=s)
        ccd.multi_batch(v, sd, 100_000, ws=ws, out=out, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ccd.segments_err_from_bounds(v, sd, stream=s)
        ccd.multi_batch(v, sd, 100_000, ws=ws, out=out, stream=s)
    for d in (1e-6, 1e-3):
        seg2 = seg.copy()
        seg2["delta"] = d
        sd.copy_(ccd.segments_to_device(seg2))
        g.replay()
        torch.cuda.synchronize()
        replay = _out(out)
        sd_e = ccd.segments_to_device(seg2)
        ccd.segments_err_from_bounds(v, sd_e)
        eager = _out(ccd.multi_batch(v, sd_e, 100_000))
        _eq(replay, eager)


def test_invalid_segment_table_reports_arg_error(ccd):
    wl, verts, counts, kinds, ms, delta, max_itr = _instances(count=3, total=3_000, seed=11)
    v = ccd.to_soa(verts)
    for broken in ("gap", "kind", "delta", "bound"):
        seg = ccd.make_segments(counts, kinds, 0.0, 1e-6, 1000)
        if broken == "gap":
            seg["offset"][1] += 1
        elif broken == "kind":
            seg["kind"][0] = 7
        elif broken == "delta":
            seg["delta"][2] = 0.0
        else:
            seg["max_itr"][0] = 5000
        sd = ccd.segments_to_device(seg)
        ws = ccd.multi_workspace(v.shape[1], 1000)
        ccd.multi_batch(v, sd, 1000, ws=ws)
        assert ccd.workspace_status(ws)[0] == -1, broken


def test_shortened_interval_matches_oracle(ccd):
    """SolveMSCCD's time interval [0, t_max] (Sec. 6) per segment, including
    non-dyadic t_max, against the oracle; t_max = 1 equals the plain call."""
    wl = W.simulation_mixed(n=12_000, seed=31)
    rng = np.random.default_rng(31)
    parts, counts, kinds, tmaxes, mss = [], [], [], [], []
    for b in wl.batches:
        for t_max in (1.0, 0.5, 0.3, float(np.float64(1) / 3), 0.9876543210123):
            idx = rng.choice(b.n, 800, replace=False)
            parts.append(b.verts[idx])
            counts.append(800)
            kinds.append(b.kind)
            tmaxes.append(t_max)
            mss.append(float(rng.choice([0.0, 1e-4])))
    verts = np.concatenate(parts)
    seg = ccd.make_segments(counts, kinds, mss, 1e-6, 1_000_000, t_max=tmaxes)
    v = ccd.to_soa(verts)
    sd = ccd.segments_to_device(seg)
    ccd.segments_err_from_bounds(v, sd)
    seg = ccd.segments_from_device(sd)
    got = _out(ccd.multi_batch(v, sd, 1_000_000))
    for s in range(len(counts)):
        o, c = int(seg["offset"][s]), int(seg["count"][s])
        oe = oracle.err_from_bounds(kinds[s], verts[o:o + c], ms_nonzero=mss[s] > 0)
        assert np.array_equal(seg["err"][s], oe)
        ref = oracle.ccd_batch(kinds[s], verts[o:o + c], oe, ms=mss[s], delta=1e-6,
                               max_itr=1_000_000, nthreads=NT, t_max=tmaxes[s])
        _eq([x[o:o + c] for x in got], ref)
        hit = ref[0] == 1
        assert np.all(got[1][o:o + c][hit] <= tmaxes[s])


def test_group_reduce_min_toi_max_tol(ccd):
    wl, verts, counts, kinds, ms, delta, max_itr = _instances(count=6, total=30_000, seed=33)
    k = len(counts)
    groups = np.arange(k) % 3
    seg = ccd.make_segments(counts, kinds, 0.0, 1e-6, 1_000_000, group=groups)
    v = ccd.to_soa(verts)
    sd = ccd.segments_to_device(seg)
    ccd.segments_err_from_bounds(v, sd)
    r = ccd.multi_batch(v, sd, 1_000_000)
    alpha, tol = ccd.group_reduce(r, sd, 4)
    torch.cuda.synchronize()
    toi, ot = r.toi.cpu().numpy(), r.out_tol.cpu().numpy()
    owner = np.repeat(groups, counts)
    for g in range(4):
        m = owner == g
        want_a = toi[m].min() if m.any() else np.inf
        want_t = ot[m].max() if m.any() else 0.0
        assert alpha[g].item() == want_a and tol[g].item() == want_t
