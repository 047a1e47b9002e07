"""GPU: Algorithm 3's active-set construction (Sec. 6) and its broad phase,
through the C ABI, against the oracle.

Candidate lists are index work and must match exactly; the active set's
times of impact come from the same CCD arithmetic and must be equal.
"""
import numpy as np
import pytest
import torch

from oracle import activeset as A
from paper_2009_13349_gb300 import workloads as W

pytestmark = pytest.mark.gpu
VF, EE = 0, 1


@pytest.fixture(scope="module")
def ccd():
    from paper_2009_13349_gb300 import ccd as m
    assert torch.cuda.is_available()
    return m


def dev_mesh(m):
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    return t(m.x0, torch.float64), t(m.x1, torch.float64), t(m.faces, torch.int32), \
        t(m.edges, torch.int32)


@pytest.mark.parametrize("nx,seed", [(6, 1), (12, 2), (24, 3)])
def test_broad_phase_and_active_set_match_oracle(ccd, nx, seed):
    m = W.cloth_scene(nx=nx, seed=seed)
    o = A.construct_active_set(m.x0, m.x1, m.faces, m.edges, nthreads=8)
    x0, x1, f, e = dev_mesh(m)
    eps = ccd.scene_eps(x0, x1)
    assert np.array_equal(eps[0], o["eps"][0]) and np.array_equal(eps[1], o["eps"][1])
    g = ccd.construct_active_set(x0, x1, f, e)
    assert g["margin"] == o["r"]
    assert np.array_equal(g["vf_candidates"].cpu().numpy(), o["candidates"][0])
    assert np.array_equal(g["ee_candidates"].cpu().numpy(), o["candidates"][1])
    kind = g["kind"].cpu().numpy()
    pairs = g["pairs"].cpu().numpy()
    toi = g["toi"].cpu().numpy()
    assert np.array_equal(pairs[kind == VF], o["vf"]) and np.array_equal(toi[kind == VF], o["vf_toi"])
    assert np.array_equal(pairs[kind == EE], o["ee"]) and np.array_equal(toi[kind == EE], o["ee_toi"])
    assert np.all(kind[:len(o["vf"])] == VF)          # candidate order: VF first
    assert len(kind) > 0


def test_broad_phase_margins_and_capacity_retry(ccd):
    m = W.cloth_scene(nx=10, seed=4)
    x0, x1, f, e = dev_mesh(m)
    for r in (0.0, 1e-3, 2.0**-6):
        ovf, oee = A.broad_phase(m.x0, m.x1, m.faces, m.edges, r)
        vf, ee = ccd.broad_phase(x0, x1, f, e, r, cap=3)      # forces the retry path
        assert np.array_equal(vf.cpu().numpy(), ovf) and np.array_equal(ee.cpu().numpy(), oee)


def test_empty_and_separated_meshes(ccd):
    m = W.cloth_scene(nx=4, seed=5)
    x0, x1, f, e = dev_mesh(m)
    nf0 = torch.zeros((0, 3), dtype=torch.int32, device="cuda")
    ne0 = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
    vf, ee = ccd.broad_phase(x0, x1, nf0, ne0, 1e-3)
    assert vf.shape[0] == 0 and ee.shape[0] == 0
    g = ccd.construct_active_set(x0, x1, nf0, ne0)
    assert g["pairs"].shape[0] == 0
    # a single static sheet: candidates (neighbours), but nothing collides
    nA = 16
    keep_f = (m.faces < nA).all(1)
    keep_e = (m.edges < nA).all(1)
    sx0, sx1 = m.x0[:nA].copy(), m.x0[:nA].copy()
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    g = ccd.construct_active_set(t(sx0, torch.float64), t(sx1, torch.float64),
                                 t(m.faces[keep_f], torch.int32), t(m.edges[keep_e], torch.int32))
    o = A.construct_active_set(sx0, sx1, m.faces[keep_f], m.edges[keep_e])
    assert len(o["candidates"][1]) > 0
    assert g["pairs"].shape[0] == len(o["vf"]) + len(o["ee"]) == 0


def test_large_mesh_candidates_by_local_brute_force(ccd):
    """nx = 128 (32k vertices): every GPU candidate satisfies the definition,
    and for 300 random faces and 300 random edges the GPU candidates that
    involve them are exactly the brute-force overlaps."""
    m = W.cloth_scene(nx=128, seed=6)
    x0, x1, f, e = dev_mesh(m)
    r = float(ccd.scene_eps(x0, x1).max())
    vf, ee = (t.cpu().numpy() for t in ccd.broad_phase(x0, x1, f, e, r))
    vlo, vhi = A.swept_boxes(m.x0, m.x1, np.arange(len(m.x0))[:, None], r)
    flo, fhi = A.swept_boxes(m.x0, m.x1, m.faces, r)
    elo, ehi = A.swept_boxes(m.x0, m.x1, m.edges, r)
    ov = lambda a0, a1, b0, b1: np.all((a0 <= b1) & (b0 <= a1), axis=-1)
    assert ov(vlo[vf[:, 0]], vhi[vf[:, 0]], flo[vf[:, 1]], fhi[vf[:, 1]]).all()
    assert ov(elo[ee[:, 0]], ehi[ee[:, 0]], elo[ee[:, 1]], ehi[ee[:, 1]]).all()
    assert (ee[:, 0] < ee[:, 1]).all()
    rng = np.random.default_rng(0)
    for fi in rng.choice(len(m.faces), 300, replace=False):
        hit = ov(vlo, vhi, flo[fi], fhi[fi])
        hit[m.faces[fi]] = False
        assert np.array_equal(np.sort(vf[vf[:, 1] == fi, 0]), np.nonzero(hit)[0])
    for a in rng.choice(len(m.edges), 300, replace=False):
        hit = ov(elo, ehi, elo[a], ehi[a])
        hit[a] = False
        hit &= ~np.isin(m.edges, m.edges[a]).any(axis=1)
        got = np.concatenate([ee[ee[:, 0] == a, 1], ee[ee[:, 1] == a, 0]])
        assert np.array_equal(np.sort(got), np.nonzero(hit)[0])
