"""Algorithm 3 (Sec. 6, "Active Set Construction") on the CPU oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Given a triangle mesh moving linearly from vertex positions x0 to x1 (nv x 3
each), its faces (nf x 3 vertex ids) and edges (ne x 2 vertex ids):

1. BroadPhase (the paper names it only).  The candidate set C is, by plain
   definition, every vertex-face pair (v, f) with v not a vertex of f, and
   every edge-edge pair (a, b), a < b, without a shared vertex, whose swept
   axis-aligned boxes overlap.  A primitive's swept box is the per-axis
   minimum and maximum of its vertices at both times, minus / plus a margin
   r; boxes overlap when lo_1 <= hi_2 and lo_2 <= hi_1 on every axis.
   If two swept boxes are apart by more than 2 r >= eps on an axis, F has no
   value within eps of 0 on that axis, so the CCD filter cannot report the
   pair: with r >= eps / 2 the broad phase never drops a pair that CCD
   would report.
2. eps of the scene (Sec. 6: the bounds of all the vertices of the
   simulation): gamma_c = max(1, max over all vertices and both times of
   |x_c|), eps_c = K ((gamma_c gamma_c) gamma_c) with the kind's constant.
3. For every candidate c: t <- CCD(x0 of c, x1 of c, delta, m_I) (Algorithm
   2, ms = 0); if 0 <= t <= 1 (a reported collision), (c, t) joins the
   active set C_A.

Everything here is brute force: O(nv nf + ne^2) box tests.
"""
from __future__ import annotations

import numpy as np

from . import VF, EE, ccd_batch, filter_constant


def swept_boxes(x0, x1, prims, r: float):
    """(lo, hi), each (m x 3): per-axis min / max over the primitive's
    vertices at t0 and t1, minus / plus r."""
    pts = np.concatenate([x0[prims], x1[prims]], axis=1)       # (m, 2k, 3)
    return pts.min(axis=1) - r, pts.max(axis=1) + r


def _overlap(lo_a, hi_a, lo_b, hi_b):
    return np.all((lo_a <= hi_b) & (lo_b <= hi_a), axis=-1)


def broad_phase(x0, x1, faces, edges, r: float):
    """Candidate pairs: (vf (k x 2) [v, f], ee (m x 2) [a, b]), each sorted
    lexicographically."""
    x0 = np.asarray(x0, dtype=np.float64)
    x1 = np.asarray(x1, dtype=np.float64)
    faces = np.asarray(faces, dtype=np.int64).reshape(-1, 3)
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    nv = x0.shape[0]
    vlo, vhi = swept_boxes(x0, x1, np.arange(nv)[:, None], r)
    flo, fhi = swept_boxes(x0, x1, faces, r)
    elo, ehi = swept_boxes(x0, x1, edges, r)
    vf = []
    for f in range(faces.shape[0]):
        hit = _overlap(vlo, vhi, flo[f], fhi[f])
        hit[faces[f]] = False
        for v in np.nonzero(hit)[0]:
            vf.append((v, f))
    ee = []
    for a in range(edges.shape[0]):
        hit = _overlap(elo[a + 1:], ehi[a + 1:], elo[a], ehi[a])
        b = np.nonzero(hit)[0] + a + 1
        shared = np.isin(edges[b], edges[a]).any(axis=1)
        for bb in b[~shared]:
            ee.append((a, bb))
    vf = np.array(sorted(vf), dtype=np.int64).reshape(-1, 2)
    ee = np.array(sorted(ee), dtype=np.int64).reshape(-1, 2)
    return vf, ee


def scene_err(x0, x1, kind: int) -> np.ndarray:
    """eps per axis from the bounds of every vertex at both times."""
    g = np.maximum(1.0, np.abs(np.concatenate([x0, x1])).max(axis=0))
    return filter_constant(kind, False) * ((g * g) * g)


def vf_queries(x0, x1, faces, pairs):
    """Query rows (p, v1, v2, v3 at t0, then at t1) of vertex-face pairs."""
    ids = np.concatenate([pairs[:, :1], faces[pairs[:, 1]]], axis=1)
    return np.concatenate([x0[ids].reshape(-1, 12), x1[ids].reshape(-1, 12)], axis=1)


def ee_queries(x0, x1, edges, pairs):
    """Query rows (p1, p2, p3, p4 at t0, then at t1) of edge-edge pairs."""
    ids = np.concatenate([edges[pairs[:, 0]], edges[pairs[:, 1]]], axis=1)
    return np.concatenate([x0[ids].reshape(-1, 12), x1[ids].reshape(-1, 12)], axis=1)


def construct_active_set(x0, x1, faces, edges, delta: float = 1e-6, max_itr: int = 10**6,
                         r: float | None = None, nthreads: int = 1, pairs=None):
    """C_A as (vf_pairs, vf_toi, ee_pairs, ee_toi) in candidate order, plus the
    candidate set.  r defaults to the largest eps of the scene."""
    x0 = np.asarray(x0, dtype=np.float64)
    x1 = np.asarray(x1, dtype=np.float64)
    faces = np.asarray(faces, dtype=np.int64).reshape(-1, 3)
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    e_vf, e_ee = scene_err(x0, x1, VF), scene_err(x0, x1, EE)
    if r is None:
        r = float(max(e_vf.max(), e_ee.max()))
    vf, ee = broad_phase(x0, x1, faces, edges, r) if pairs is None else pairs
    out = []
    for kind, pr, q, e in ((VF, vf, vf_queries, e_vf), (EE, ee, ee_queries, e_ee)):
        if pr.shape[0] == 0:
            out += [pr, np.zeros(0)]
            continue
        rows = q(x0, x1, faces if kind == VF else edges, pr)
        col, toi, _, _ = ccd_batch(kind, rows, e, ms=0.0, delta=delta, max_itr=max_itr,
                                   nthreads=nthreads)
        keep = (col == 1) & (toi >= 0.0) & (toi <= 1.0)
        out += [pr[keep], toi[keep]]
    return {"vf": out[0], "vf_toi": out[1], "ee": out[2], "ee_toi": out[3],
            "candidates": (vf, ee), "r": r, "eps": (e_vf, e_ee)}
