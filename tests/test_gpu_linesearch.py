"""GPU: Algorithm 4's line-search step (Sec. 6) and the L-infinity distance
it uses, through the C ABI, against the oracle.

Both sides evaluate the distance with the same fixed operation sequence and
run the same host-side decisions on bit-identical inputs (d_i, eps_i, the
MSCCD outputs), so every output must be equal.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle.linesearch import line_search_ccd
from paper_2009_13349_gb300 import workloads as W

pytestmark = pytest.mark.gpu
NT = 8
KEYS = ("alpha", "p", "d", "d_i", "eps_i", "delta_i", "passes", "validated")


@pytest.fixture(scope="module")
def ccd():
    from paper_2009_13349_gb300 import ccd as m
    assert torch.cuda.is_available()
    return m


def soa_of(ccd, vf, ee):
    return ccd.to_soa(np.concatenate([vf.reshape(-1, 24), ee.reshape(-1, 24)], axis=0))


def segs_of(ccd, n_vf, n_ee, groups=(0, 0)):
    s = ccd.make_segments([n_vf, n_ee], [0, 1], 0.0, 1e-6, 10**6, group=list(groups))
    return ccd.segments_to_device(s)


@pytest.mark.parametrize("wl", ["random", "line-search", "simulation", "degenerate"])
def test_distance_bit_exact(ccd, wl):
    rng = np.random.default_rng(7)
    if wl == "random":
        vf = rng.uniform(-1, 1, (3000, 24)) * 10 ** rng.uniform(-2, 2, (3000, 1))
        ee = rng.uniform(-1, 1, (3000, 24)) * 10 ** rng.uniform(-2, 2, (3000, 1))
    else:
        w = {"line-search": lambda: W.line_search_scene(n=20_000, seed=8),
             "simulation": lambda: W.simulation_mixed(n=20_000, seed=9),
             "degenerate": lambda: W.degenerate_heavy(n=4_000, seed=10)}[wl]()
        vf, ee = w.batches[0].verts, w.batches[1].verts
    gmin, dist = ccd.linf_distance(soa_of(ccd, vf, ee), segs_of(ccd, len(vf), len(ee), (0, 1)),
                                   ngroups=2, per_query=True)
    torch.cuda.synchronize()
    o = np.concatenate([oracle.linf_distance_batch(0, vf, NT), oracle.linf_distance_batch(1, ee, NT)])
    g = dist.cpu().numpy()
    bad = np.nonzero(g != o)[0]
    assert bad.size == 0, f"{bad.size} distances differ, e.g. {bad[:5]}"
    gm = gmin.cpu().numpy()
    assert gm[0] == o[:len(vf)].min() and gm[1] == o[len(vf):].min()


def test_distance_empty_group_is_inf(ccd):
    vf = np.random.default_rng(1).uniform(-1, 1, (100, 24))
    gmin, _ = ccd.linf_distance(soa_of(ccd, vf, np.zeros((0, 24))),
                                segs_of(ccd, 100, 0, (0, 1)), ngroups=2)
    torch.cuda.synchronize()
    assert np.isinf(gmin.cpu().numpy()[1])


def run_both(ccd, vf, ee, **kw):
    g = ccd.line_search(soa_of(ccd, vf, ee), len(vf), len(ee), **kw)
    o = line_search_ccd(vf, ee, nthreads=NT, **kw)
    return g, o


def assert_same(g, o, label):
    for k in KEYS:
        assert g[k] == o[k], f"{label}: {k} gpu {g[k]} oracle {o[k]}"


@pytest.mark.parametrize("n", [2_000, 40_000])
@pytest.mark.parametrize("cap", ["min", "max"])
def test_line_search_matches_oracle(ccd, n, cap):
    wl = W.line_search_scene(n=n, seed=11)
    vf, ee = wl.batches[0].verts, wl.batches[1].verts
    delta = 1e-6 if cap == "min" else 1e-5
    g, o = run_both(ccd, vf, ee, p=0.5, delta=delta, cap=cap)
    assert_same(g, o, f"n={n} cap={cap}")
    assert g["status"] == 0 and g["validated"] and 0.0 < g["alpha"] < 1.0


def test_line_search_edge_cases(ccd):
    rng = np.random.default_rng(12)
    wl = W.line_search_scene(n=400, seed=13)
    vf, ee = wl.batches[0].verts, wl.batches[1].verts
    z = np.zeros((0, 24))
    for a, b, lab in ((vf, z, "vf only"), (z, ee, "ee only"), (vf[:1], ee[:1], "one each")):
        assert_same(*run_both(ccd, a, b, p=0.5, delta=1e-6), lab)
    # p halving, an unvalidated step, a zero step (touching at t = 0), max_passes
    tri = [0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0, 0.0]
    def fall(h0, h1):
        return np.array([[0.25, 0.25, h0, *tri, 0.25, 0.25, h1, *tri]])
    delta = 2.0**-20
    assert_same(*run_both(ccd, fall(1.5 * delta, -1.0), z, p=0.9, delta=delta, rho=0.0), "halving")
    assert_same(*run_both(ccd, fall(0.5e-6, -1e-3), z, p=0.5, delta=1e-6, max_passes=3),
                "unvalidated")
    assert_same(*run_both(ccd, fall(0.0, -1.0), z, p=0.5, delta=1e-6, max_passes=4), "touching")
    # a mixed set with many passes: large delta_i from check-limited queries
    deg = W.degenerate_heavy(n=400, seed=14)
    assert_same(*run_both(ccd, deg.batches[0].verts, deg.batches[1].verts, p=0.5, delta=1e-6,
                          max_itr=1000, max_passes=4), "degenerate")
    # the empty set: the full step, no pass
    g = ccd.line_search(ccd.to_soa(z), 0, 0, p=0.5, delta=1e-6)
    assert g["alpha"] == 1.0 and g["passes"] == 0


def test_line_search_rejects_bad_arguments(ccd):
    v = ccd.to_soa(np.zeros((1, 24)))
    for kw in ({"p": 0.0}, {"p": 1.0}, {"delta": 0.0}, {"rho": -1.0}, {"max_passes": 0}):
        args = dict(p=0.5, delta=1e-6)
        args.update(kw)
        with pytest.raises(ccd.CCDError):
            ccd.line_search(v, 1, 0, **args)
