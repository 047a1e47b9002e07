"""CPU pins of the oracle's line-search step (Sec. 6, Algorithm 4) and of the
L-infinity distance it uses (Sec. 5.1 norm).

The distance is pinned against an independent LP solver, closed forms and
exact scaling; the step against hand-worked cases of its p-validation rule,
the guarantee the paper states for it (a validated step has a positive
time of impact), and the sequence property that motivates it.
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
from oracle import exact
from oracle.linesearch import line_search_ccd

VF, EE = 0, 1


def vf_query(p0, v1, v2, v3, p1=None, w1=None, w2=None, w3=None):
    """Query row: points at t0 then at t1 (static where t1 is not given)."""
    t0 = [*p0, *v1, *v2, *v3]
    t1 = [*(p1 or p0), *(w1 or v1), *(w2 or v2), *(w3 or v3)]
    return np.array(t0 + t1, dtype=np.float64)


def ee_query(a0, b0, c0, d0, a1=None, b1=None, c1=None, d1=None):
    t0 = [*a0, *b0, *c0, *d0]
    t1 = [*(a1 or a0), *(b1 or b0), *(c1 or c0), *(d1 or d0)]
    return np.array(t0 + t1, dtype=np.float64)


def lp_distance(kind, q):
    """min s subject to |F_c(0,u,v)| <= s on the domain, by scipy's HiGHS."""
    linprog = pytest.importorskip("scipy.optimize").linprog
    P = np.asarray(q[:12]).reshape(4, 3)
    if kind == VF:
        A, B, C = P[0] - P[1], P[1] - P[2], P[1] - P[3]
    else:
        A, B, C = P[0] - P[2], P[1] - P[0], P[2] - P[3]
    Aub, bub = [], []
    for c in range(3):
        Aub += [[B[c], C[c], -1.0], [-B[c], -C[c], -1.0]]
        bub += [-A[c], A[c]]
    if kind == VF:
        Aub.append([1.0, 1.0, 0.0])
        bub.append(1.0)
    r = linprog([0, 0, 1], A_ub=Aub, b_ub=bub, bounds=[(0, 1), (0, 1), (0, None)],
                method="highs")
    assert r.status == 0
    return r.fun


# ---- distance ------------------------------------------------------------------

@pytest.mark.parametrize("kind", [VF, EE])
def test_distance_exact_matches_lp_solver(kind):
    rng = np.random.default_rng(3 + kind)
    for _ in range(150):
        s = 10 ** rng.uniform(-2, 2)
        q = rng.uniform(-1, 1, 24) * s
        e = float(exact.linf_distance(kind, q))
        assert abs(e - lp_distance(kind, q)) <= 1e-9 * s


@pytest.mark.parametrize("kind", [VF, EE])
def test_distance_oracle_within_rounding_of_exact(kind):
    rng = np.random.default_rng(5 + kind)
    worst = 0.0
    for _ in range(400):
        s = 10 ** rng.uniform(-2, 2)
        q = rng.uniform(-1, 1, 24) * s
        if rng.uniform() < 0.3:       # near-degenerate: nearly parallel / coplanar
            q[9:12] = q[3:6] + (q[6:9] - q[3:6]) * 0.5 + rng.normal(0, 1e-9 * s, 3)
        e = exact.linf_distance(kind, q)
        worst = max(worst, abs(oracle.linf_distance(kind, q) - float(e)) / s)
    assert worst <= 1e-13


def test_distance_closed_forms():
    h, a, b, c = 0.375, 0.25, 0.125, 0.0625
    tri = ([0, 0, 0], [1, 0, 0], [0, 1, 0])
    # point above the interior of a triangle in z = 0: |dz| = h everywhere
    q = vf_query([0.2, 0.3, h], *tri)
    assert oracle.linf_distance(VF, q) == h and exact.linf_distance(VF, q) == Fr(h)
    # point off the corner (0,0,0) along -x, -y: nearest is the corner
    q = vf_query([-a, -b, c], *tri)
    assert oracle.linf_distance(VF, q) == max(a, b, c)
    # crossing edges at vertical offset h
    q = ee_query([-1, 0, 0], [1, 0, 0], [0, -1, h], [0, 1, h])
    assert oracle.linf_distance(EE, q) == h
    # collinear edges with a gap of 1 along x
    q = ee_query([0, 0, 0], [1, 0, 0], [2, 0, 0], [3, 0, 0])
    assert oracle.linf_distance(EE, q) == 1.0
    # a point in the triangle and crossing edges: distance 0
    assert oracle.linf_distance(VF, vf_query([0.25, 0.25, 0], *tri)) == 0.0
    assert oracle.linf_distance(EE, ee_query([-1, 0, 0], [1, 0, 0], [0, -1, 0], [0, 1, 0])) == 0.0
    # L-inf, not L2: point beyond the hypotenuse of the triangle along (1,1,0)
    q = vf_query([0.75, 0.75, 0], *tri)
    assert oracle.linf_distance(VF, q) == 0.25        # the L2 distance is 0.25 * sqrt(2)


@pytest.mark.parametrize("kind", [VF, EE])
def test_distance_scales_exactly_and_bounds_samples(kind):
    rng = np.random.default_rng(11 + kind)
    for _ in range(40):
        q = np.round(rng.uniform(-1, 1, 24) * 2**20) / 2**20
        d = oracle.linf_distance(kind, q)
        assert oracle.linf_distance(kind, q * 8.0) == 8.0 * d     # power-of-two scaling is exact
        e = exact.linf_distance(kind, q)
        qf = exact.to_fr(q)
        for _ in range(30):                                       # min over the domain
            u, v = Fr(int(rng.integers(0, 65))), Fr(int(rng.integers(0, 65)))
            if kind == VF and u + v > 64:
                u, v = 64 - u, 64 - v
            F = exact.F(kind, qf, Fr(0), u / 64, v / 64)
            assert e <= max(abs(x) for x in F)


def test_distance_of_grid_queries_within_a_few_ulps():
    """On a coarse dyadic grid of unit-scale coordinates A, B, C are exact,
    so the only rounding left is that of the candidate point and the final
    few operations, a few ulps of the unit input scale."""
    rng = np.random.default_rng(17)
    for kind in (VF, EE):
        for _ in range(100):
            q = rng.integers(-8, 9, 24) / 8.0
            e = float(exact.linf_distance(kind, q))
            assert abs(oracle.linf_distance(kind, q) - e) <= 4 * np.spacing(1.0)


# ---- line-search step ----------------------------------------------------------

TRI = ([0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0])


def falling_point(h0, h1, xy=(0.25, 0.25)):
    """A point above the triangle in z = 0, moving straight from height h0 to h1."""
    return vf_query([xy[0], xy[1], h0], *TRI, p1=[xy[0], xy[1], h1])


def test_step_bounds_alpha_by_the_separated_contact():
    h0, delta = 2.0**-6, 1e-6
    q = falling_point(h0, -h0)
    r = line_search_ccd(q, np.zeros((0, 24)), p=0.5, delta=delta)
    assert r["validated"] and r["passes"] == 1
    assert r["d_i"] == h0 and r["d"] == delta          # d = min(p d_i, delta)
    t_d = (h0 - r["d"]) / (2 * h0)                    # the point reaches height d
    speed = 2 * h0
    assert 0.0 < r["alpha"] <= t_d
    assert t_d - r["alpha"] <= math.sqrt(3) * (r["delta_i"] + r["eps_i"] + r["d"]) / speed


def test_printed_cap_keeps_p_times_distance():
    """cap = max keeps d = p d_i.  delta is chosen so that the region
    |F| <= d (a square of side 2d on the triangle) takes far fewer than m_I
    boxes of width delta; otherwise the answer comes from the check limit."""
    h0, delta = 2.0**-6, 1e-4
    q = falling_point(h0, -h0)
    r = line_search_ccd(q, np.zeros((0, 24)), p=0.5, delta=delta, cap="max")
    assert r["validated"] and r["d"] == 0.5 * h0
    t_d = (h0 - r["d"]) / (2 * h0)
    speed = 2 * h0
    assert 0.0 < r["alpha"] <= t_d
    assert t_d - r["alpha"] <= 2 * math.sqrt(3) * (r["delta_i"] + r["eps_i"]) / speed


def test_p_is_halved_until_the_inequality_holds():
    """Worked example of step 4: d_i = 1.5 delta, p = 0.9, cap = min.
    d = delta fails (0.5 delta < delta + eps + rho); p = 0.45 gives
    d = 0.675 delta, which fails (0.825 delta); p = 0.225 gives
    d = 0.3375 delta and 1.1625 delta > delta + eps + rho holds."""
    delta = 2.0**-20
    q = falling_point(1.5 * delta, -1.0)
    r = line_search_ccd(q, np.zeros((0, 24)), p=0.9, delta=delta, rho=0.0)
    assert r["d_i"] == 1.5 * delta
    assert r["p"] == 0.225 and r["d"] == 0.225 * (1.5 * delta)
    assert r["alpha"] > 0.0


def test_unvalidated_when_no_p_can_work():
    """d_i < delta + eps + rho: no p satisfies the inequality.  Slow motion
    keeps alpha > 0, so the step repeats its pass (delta <- delta_i) up to
    max_passes and reports that the inequality does not hold."""
    delta = 1e-6
    q = falling_point(0.5 * delta, -1e-3)
    r = line_search_ccd(q, np.zeros((0, 24)), p=0.5, delta=delta, max_passes=3)
    assert not r["validated"]
    assert r["alpha"] == 0.0 or r["passes"] == 3


def test_touching_at_start_gives_a_zero_step():
    q = falling_point(0.0, -1.0)
    r = line_search_ccd(q, np.zeros((0, 24)), p=0.5, delta=1e-6, max_passes=4)
    assert r["d_i"] == 0.0 and r["alpha"] == 0.0 and not r["validated"]
    assert r["passes"] == 1                  # no interval left after alpha = 0


def test_empty_candidate_set_takes_the_full_step():
    z = np.zeros((0, 24))
    r = line_search_ccd(z, z, p=0.5, delta=1e-6)
    assert r["alpha"] == 1.0 and r["passes"] == 0 and r["validated"]


def test_separated_candidates_do_not_limit_the_step():
    ee = ee_query([0, 0, 0], [1, 0, 0], [0, 0, 1], [1, 0, 1], c1=[0, 0, 0.5], d1=[1, 0, 0.5])
    r = line_search_ccd(np.zeros((0, 24)), ee, p=0.5, delta=1e-6)
    assert r["validated"] and r["alpha"] == 1.0 and r["d_i"] == 1.0


def test_steps_form_a_valid_ccd_sequence():
    """Repeated steps toward a contact (Sec. 6): with the printed cap the
    separation after each step is about p times the one before, it never
    reaches zero, and the accumulated step t_i increases toward the contact.
    Each step uses delta = d_i / 256, small against the separation."""
    p = 0.5
    h, target = 2.0**-4, -2.0**-4
    t_total, dists, ts = 0.0, [], []
    for _ in range(6):
        q = falling_point(h, target)
        r = line_search_ccd(q, np.zeros((0, 24)), p=p, delta=h / 256, cap="max")
        assert r["validated"]
        h_new = h + r["alpha"] * (target - h)
        t_total += r["alpha"] * (1 - t_total)
        dists.append(h_new)
        ts.append(t_total)
        assert abs(h_new / h - p) < 0.02        # separation shrinks by about p
        h = h_new
    assert all(d > 0 for d in dists)
    assert all(a < b for a, b in zip(ts, ts[1:]))
    assert ts[-1] < 0.5                         # the contact is at t* = 0.5


def test_step_over_a_mixed_set_takes_the_earliest_candidate():
    """alpha is the minimum over VF and EE candidates of their separated
    contact times; delta_i the maximum reached tolerance."""
    h_vf, h_ee, delta = 2.0**-5, 2.0**-6, 1e-6
    vf = falling_point(h_vf, -h_vf)
    ee = ee_query([-1, 0, 0], [1, 0, 0], [0, -1, h_ee], [0, 1, h_ee],
                  c1=[0, -1, -h_ee], d1=[0, 1, -h_ee])
    r = line_search_ccd(vf, ee, p=0.5, delta=delta)
    a_vf = line_search_ccd(vf, np.zeros((0, 24)), p=0.5, delta=delta)
    a_ee = line_search_ccd(np.zeros((0, 24)), ee, p=0.5, delta=delta)
    assert r["d_i"] == h_ee
    assert r["alpha"] <= min(a_vf["alpha"], a_ee["alpha"]) + 1e-12
    assert r["alpha"] >= min(a_vf["alpha"], a_ee["alpha"]) - 1e-5


def test_distance_and_tolerance_reductions_over_the_set():
    """Over a candidate set (Algorithm 4), d_i is the smallest distance of
    the set, and one pass leaves delta_i = max(delta, the tolerances it
    reached).  Three points fall onto the triangle from different heights;
    the distances are checked against exact rational ones, and with a small
    check limit the reached tolerances exceed delta and differ, so the
    maximum is the only reduction that gives delta_i."""
    delta, max_itr = 1e-6, 40
    heights = [2.0**-5, 2.0**-7, 2.0**-6]
    vf = np.stack([falling_point(h, -h, xy=(0.2 + 0.1 * i, 0.25)) for i, h in enumerate(heights)])
    d_exact = [float(exact.linf_distance(VF, q)) for q in vf]
    assert d_exact == heights
    r = line_search_ccd(vf, np.zeros((0, 24)), p=0.5, delta=delta, max_itr=max_itr,
                        max_passes=1)
    assert r["d_i"] == min(d_exact)
    eps = oracle.err_from_bounds(VF, vf, ms_nonzero=True)
    col, toi, tol, chk = oracle.ccd_batch(VF, vf, eps, ms=r["d"], delta=delta, max_itr=max_itr)
    assert np.all(col == 1) and np.all(chk >= max_itr)      # every query cut by the limit
    assert tol.min() < tol.max() and tol.min() > delta
    assert r["delta_i"] == max(delta, float(tol.max()))
    assert r["alpha"] == float(toi.min())
