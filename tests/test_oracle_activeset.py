"""CPU pins of the oracle's active-set construction (Sec. 6, Algorithm 3).

The broad phase is pinned by hand-built cases and by its purpose: no pair
that the CCD oracle reports colliding may be missing from the candidate set,
so the active set built through it must equal the active set over all pairs.
"""
import numpy as np
import pytest

import oracle
from oracle import activeset as A
from paper_2009_13349_gb300 import workloads as W

VF, EE = 0, 1


def all_pairs(faces, edges, nv):
    vf = np.array([(v, f) for v in range(nv) for f in range(len(faces))
                   if v not in faces[f]], dtype=np.int64).reshape(-1, 2)
    ee = np.array([(a, b) for a in range(len(edges)) for b in range(a + 1, len(edges))
                   if not set(edges[a]) & set(edges[b])], dtype=np.int64).reshape(-1, 2)
    return vf, ee


def one_triangle_and_point(p0, p1):
    x0 = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], p0])
    x1 = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], p1])
    faces = np.array([[0, 1, 2]])
    edges = np.array([[0, 1], [0, 2], [1, 2]])
    return x0, x1, faces, edges


def test_point_through_triangle_is_active():
    x0, x1, f, e = one_triangle_and_point([0.25, 0.25, 1.0], [0.25, 0.25, -1.0])
    r = A.construct_active_set(x0, x1, f, e)
    assert r["candidates"][0].tolist() == [[3, 0]]
    assert r["vf"].tolist() == [[3, 0]]
    assert 0.0 < r["vf_toi"][0] <= 0.5             # crossing at t = 0.5
    assert r["ee"].shape == (0, 2)                  # a triangle's edges share vertices


def test_far_point_is_no_candidate():
    x0, x1, f, e = one_triangle_and_point([5.0, 5.0, 1.0], [5.0, 5.0, 0.5])
    r = A.construct_active_set(x0, x1, f, e)
    assert r["candidates"][0].shape == (0, 2) and r["vf"].shape == (0, 2)


def test_boxes_apart_by_just_more_than_two_margins():
    """Swept boxes separated by a gap g on one axis overlap after inflation
    by r exactly when g <= 2 r."""
    r = 2.0**-20
    for g, expect in ((2 * r, 1), (2 * r + 2.0**-40, 0)):
        x0, x1, f, e = one_triangle_and_point([0.25, 0.25, g], [0.25, 0.25, g])
        vf, _ = A.broad_phase(x0, x1, f, e, r)
        assert len(vf) == expect


def test_shared_vertices_are_excluded():
    m = W.cloth_scene(nx=5, seed=1)
    vf, ee = A.broad_phase(m.x0, m.x1, m.faces, m.edges, 1e-3)
    for v, f in vf:
        assert v not in m.faces[f]
    for a, b in ee:
        assert a < b and not set(m.edges[a]) & set(m.edges[b])


@pytest.mark.parametrize("seed", [6, 7])
def test_broad_phase_keeps_every_colliding_pair(seed):
    """Brute force over all pairs: every pair the CCD oracle reports
    colliding is a candidate (Algorithm 3 loses nothing to the broad
    phase), and the active set through the broad phase is the active set
    over all pairs, with the same times of impact."""
    m = W.cloth_scene(nx=6, seed=seed)
    via_bp = A.construct_active_set(m.x0, m.x1, m.faces, m.edges, nthreads=8)
    allp = all_pairs(m.faces, m.edges, len(m.x0))
    full = A.construct_active_set(m.x0, m.x1, m.faces, m.edges, nthreads=8, pairs=allp)
    cand_vf = {tuple(p) for p in via_bp["candidates"][0]}
    cand_ee = {tuple(p) for p in via_bp["candidates"][1]}
    assert {tuple(p) for p in full["vf"]} <= cand_vf
    assert {tuple(p) for p in full["ee"]} <= cand_ee
    assert len(full["vf"]) + len(full["ee"]) > 0
    for k in ("vf", "ee"):
        assert via_bp[k].tolist() == full[k].tolist()
        assert np.array_equal(via_bp[k + "_toi"], full[k + "_toi"])


def test_scene_eps_uses_every_vertex_at_both_times():
    x0 = np.array([[0.5, -3.0, 0.0], [0.0, 0.0, 0.25]])
    x1 = np.array([[2.0, 0.0, 0.0], [0.0, 0.0, -1.5]])
    e = A.scene_err(x0, x1, VF)
    K = oracle.filter_constant(VF, False)
    assert e.tolist() == [K * 8.0, K * 27.0, K * ((1.5 * 1.5) * 1.5)]
