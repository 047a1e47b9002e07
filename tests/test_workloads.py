"""The degenerate-heavy generator (100,000 queries, seed 2, coordinates on a
2^-20 grid): each family is what it claims, checked in exact rationals.

Vertex-on-vertex and grazing-tangent queries are constructed contacts: the
two primitives meet at the recorded t* at a point of the closed domain.  A
grazing contact is a touch at that single time with zero normal speed: the
coplanarity function f(t) = <n(t), q(t)> (Sec. 3, Eq. univariate) is a
nonzero multiple of (t - t*)^2.
"""
from fractions import Fraction as Fr

import numpy as np

import oracle.exact as ex
from paper_2009_13349_gb300 import workloads as W


def _contact_params(kind, query, t):
    """Exact (u, v) with F(t, u, v) = 0 (Eq. F-vf / F-ee), or None."""
    qv = ex.to_fr(query)
    F0 = ex.F(kind, qv, t, Fr(0), Fr(0))
    Fu = [a - b for a, b in zip(ex.F(kind, qv, t, Fr(1), Fr(0)), F0)]
    Fv = [a - b for a, b in zip(ex.F(kind, qv, t, Fr(0), Fr(1)), F0)]
    for c1, c2 in ((0, 1), (0, 2), (1, 2)):
        det = Fu[c1] * Fv[c2] - Fv[c1] * Fu[c2]
        if det != 0:
            u = (-F0[c1] * Fv[c2] + Fv[c1] * F0[c2]) / det
            v = (-Fu[c1] * F0[c2] + F0[c1] * Fu[c2]) / det
            if all(F0[c] + u * Fu[c] + v * Fv[c] == 0 for c in range(3)):
                return u, v
            return None
    return None


def _in_domain(kind, u, v):
    if u < 0 or v < 0:
        return False
    return u + v <= 1 if kind == W.VF else (u <= 1 and v <= 1)


def test_degenerate_heavy_grid_and_families():
    wl = W.degenerate_heavy(n=100_000, seed=2)
    assert wl.n == 100_000
    for b in wl.batches:
        g = b.verts * 2.0**20
        assert np.all(g == np.round(g)), "every coordinate on the 2^-20 grid"
        counts = np.bincount(b.family, minlength=10)
        fams = [W.FAM_COPLANAR, W.FAM_COLLINEAR, W.FAM_PARALLEL, W.FAM_VERTEX, W.FAM_GRAZING]
        assert counts[fams].min() >= b.n // 5 and counts.sum() == b.n     # equal parts
        labelled = np.isin(b.family, [W.FAM_VERTEX, W.FAM_GRAZING])
        assert np.array_equal(b.truth == 1, labelled)
        assert np.all(np.isfinite(b.t_star[labelled])) and np.all(np.isnan(b.t_star[~labelled]))
        assert np.all((b.t_star[labelled] > 0) & (b.t_star[labelled] < 1))


def test_constructed_contacts_are_exact():
    wl = W.degenerate_heavy(n=4000, seed=2)
    for b in wl.batches:
        for fam in (W.FAM_VERTEX, W.FAM_GRAZING):
            for i in np.nonzero(b.family == fam)[0][:60]:
                t = Fr(b.t_star[i])
                uv = _contact_params(b.kind, b.verts[i], t)
                if fam == W.FAM_VERTEX:
                    # the meeting vertices are (u, v) = (0, 0) of both kinds
                    assert ex.F(b.kind, ex.to_fr(b.verts[i]), t, Fr(0), Fr(0)) == [0, 0, 0]
                else:
                    assert uv is not None and _in_domain(b.kind, *uv)
                    assert 0 < uv[0] < 1 and 0 < uv[1] < 1
                c0, c1, c2, c3 = ex.coplanarity_cubic(b.kind, b.verts[i])
                if fam == W.FAM_GRAZING:
                    # f(t) = c2 (t - t*)^2 with c2 != 0: one touch, zero normal speed
                    assert c3 == 0 and c2 != 0
                    assert c1 == -2 * c2 * t and c0 == c2 * t * t
                else:
                    assert c0 + c1 * t + c2 * t * t + c3 * t**3 == 0
