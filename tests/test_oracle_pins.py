"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

Each test ties the oracle to something other than itself: the paper's printed
constants and worked examples (tests/golden), exact-rational evaluation of the
paper's own formulas, constructed collisions with exactly known contact
times, closed-form bounds (Proposition 1, Eq. codomain), and an independent
exact-arithmetic run of Algorithm 2 that uses the literal "append + stable
sort" queue instead of the oracle's heap.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
import oracle.exact as ex
from paper_2009_13349_gb300 import workloads as W

U = Fr(1, 2**53)


# ---------------------------------------------------------------------------
# Eq. (ccd-error), Eq. (msccd-error): the filter constants
# ---------------------------------------------------------------------------

def test_filter_constants_are_the_papers_and_dyadic():
    # printed values; each is an integer multiple of 2^-52
    assert oracle.filter_constant(0, False) == 6.661338147750939e-15 == 30 * 2.0**-52
    assert oracle.filter_constant(1, False) == 6.217248937900877e-15 == 28 * 2.0**-52
    assert oracle.filter_constant(0, True) == 7.549516567451064e-15 == 34 * 2.0**-52
    assert oracle.filter_constant(1, True) == 7.105427357601002e-15 == 32 * 2.0**-52


def test_err_from_bounds_matches_formula_by_hand():
    rng = np.random.default_rng(5)
    v = rng.uniform(-3, 3, (7, 24))
    v[2, 4] = -11.5      # largest |y| of the scene (point 1, coord 1), query 2
    got = oracle.err_from_bounds(0, v)
    g = np.maximum(np.abs(v.reshape(7, 8, 3)).max(axis=(0, 1)), 1.0)
    assert g[1] == 11.5
    np.testing.assert_array_equal(got, 30 * 2.0**-52 * (g * g * g))
    per = oracle.err_from_bounds(1, v, ms_nonzero=True, per_query=True)
    gq = np.maximum(np.abs(v.reshape(7, 8, 3)).max(axis=1), 1.0)
    np.testing.assert_array_equal(per, 32 * 2.0**-52 * (gq * gq * gq))


# ---------------------------------------------------------------------------
# Forward error of the fixed F expression vs the filter constants
# ---------------------------------------------------------------------------

def _running_bound(kind, ms):
    """Rigorous forward-error bound (gamma = 1) of the oracle's operation
    order, in units of |value| <= M, with fl(a op b) = (a op b)(1 + theta)
    and fma(s, y, z) = (s y + z)(1 + theta), |theta| <= u = 2^-53, t, u, v in
    [0, 1] exact; second-order terms kept."""
    u = U

    def add(Ea, Eb, M):       # a + b, exact |result| <= M
        return Ea + Eb + u * (M + Ea + Eb)

    def fma(Ey, Ez, M):       # s y + z with an exact |s| <= 1, exact |result| <= M
        return Ey + Ez + u * (M + Ey + Ez)

    Ed = add(0, 0, 2)             # x1 - x0
    Ex = fma(Ed, 0, 1)            # fma(x1 - x0, t, x0), |x(t)| <= 1
    if kind == 0:
        Eq = add(Ex, Ex, 2)       # q = p - v1, e1, e2 alike
        Ea = fma(Eq, Eq, 2)       # fma(-u, e1, q) = p - ((1-u) v1 + u v2)
        EF = fma(Eq, Ea, 4)       # fma(-v, e2, .), |F| <= 4 off the prism
        M = 4
    else:
        Ed1 = add(Ex, Ex, 2)      # d1 = p2 - p1 (and d2)
        Eb = fma(Ed1, Ex, 1)      # fma(v, d2, p3) = (1-v) p3 + v p4
        Ec = add(Ex, Eb, 2)       # p1 - b
        EF = fma(Ed1, Ec, 2)      # fma(u, d1, p1 - b)
        M = 2
    if ms:
        EF = add(EF, 0, M + 1)    # m - d with d < gamma
    return EF


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("ms", [False, True])
def test_fixed_expression_error_bound_below_filter(kind, ms):
    bound = _running_bound(kind, ms)
    K = Fr(oracle.filter_constant(kind, ms))
    # per-product underflow (at most 6 products on a path) adds
    # < 6 * 2^-1075, far below the slack
    assert bound + 6 * Fr(1, 2**1075) < K
    # first-order coefficients: 30 u (VF), 27 u (EE) against 60 u / 56 u
    assert int(bound / U) == (30 if kind == 0 else 27) + (5 if (ms and kind == 0) else 3 if ms else 0)


@pytest.mark.parametrize("kind", [0, 1])
def test_corner_values_within_eps_of_exact(kind):
    """|fl(F) - F| <= eps at random and adversarial corners, several scales
    (the sign of F is certain when |fl(F)| > eps, Sec. 4.2)."""
    rng = np.random.default_rng(11 + kind)
    worst = Fr(0)
    for trial in range(300):
        scale = 10.0 ** rng.uniform(-2, 2)
        qv = rng.uniform(-1, 1, 24) * scale
        if trial % 3 == 0:      # adversarial: near-cancelling coordinates
            qv[12:] = qv[:12] * (1 + rng.normal(0, 1e-9, 12))
        eps = oracle.err_from_bounds(kind, qv)
        qf = ex.to_fr(qv)
        gam = np.maximum(np.abs(qv.reshape(8, 3)).max(0), 1.0)
        for _ in range(4):
            if rng.random() < 0.5:
                t, u, v = (float(x) for x in rng.random(3))
            else:
                k = rng.integers(1, 30, 3)
                t, u, v = (float(rng.integers(0, 2**kk + 1)) / 2**kk for kk in k)
            F = oracle.corner(kind, qv, t, u, v)
            Fx = ex.F(kind, qf, Fr(t), Fr(u), Fr(v))
            for c in range(3):
                err = abs(Fr(F[c]) - Fx[c])
                assert err <= Fr(eps[c]), (trial, c, float(err), eps[c])
                worst = max(worst, err / Fr(gam[c]))
    # the measured worst case stays below the proven first-order bound
    assert worst <= _running_bound(kind, False)


# ---------------------------------------------------------------------------
# Proposition 1 (B_F is an inclusion function; corners attained) and
# Eq. (codomain) (w(B) <= sum_d w(I_d) kappa_d / 3)
# ---------------------------------------------------------------------------

def _random_box(rng):
    I = []
    for _ in range(3):
        k = int(rng.integers(0, 12))
        a = int(rng.integers(0, 2**k))
        I += [Fr(a, 2**k), Fr(a + 1, 2**k)]
    return I


@pytest.mark.parametrize("kind", [0, 1])
def test_box_inclusion_and_tightness(kind):
    rng = np.random.default_rng(21 + kind)
    for trial in range(40):
        qv = rng.uniform(-1, 1, 24)
        qf = ex.to_fr(qv)
        eps = [Fr(e) for e in oracle.err_from_bounds(kind, qv)]
        I = _random_box(rng)
        m, M = oracle.box(kind, qv, [float(x) for x in I])
        # dense rational sample of the box interior and faces
        for _ in range(60):
            s = [I[2 * d] + (I[2 * d + 1] - I[2 * d]) * Fr(int(rng.integers(0, 17)), 16)
                 for d in range(3)]
            Fx = ex.F(kind, qf, *s)
            for c in range(3):
                assert Fr(m[c]) - eps[c] <= Fx[c] <= Fr(M[c]) + eps[c]
        # tightness: the exact extremes are attained at corners
        mx, Mx = ex.box(kind, qf, I)
        for c in range(3):
            assert abs(Fr(m[c]) - mx[c]) <= eps[c]
            assert abs(Fr(M[c]) - Mx[c]) <= eps[c]


@pytest.mark.parametrize("kind", [0, 1])
def test_kappa_and_codomain_width_bound(kind):
    rng = np.random.default_rng(31 + kind)
    for trial in range(40):
        qv = rng.uniform(-1, 1, 24) * (10.0 ** rng.uniform(-1, 1))
        qf = ex.to_fr(qv)
        kap = oracle.kappa(kind, qv)
        kx = ex.kappa(kind, qf)
        eps = max(oracle.err_from_bounds(kind, qv))
        for d in range(3):
            assert abs(Fr(kap[d]) - kx[d]) <= 3 * 2 * Fr(eps) + abs(kx[d]) * 4 * U
        I = _random_box(rng)
        mx, Mx = ex.box(kind, qf, I)
        w_exact = max(Mx[c] - mx[c] for c in range(3))
        rhs = sum((I[2 * d + 1] - I[2 * d]) * kx[d] for d in range(3)) / 3
        assert w_exact <= rhs
        m, M = oracle.box(kind, qv, [float(x) for x in I])
        w_fp = max(M[c] - m[c] for c in range(3))
        assert Fr(w_fp) <= rhs + 2 * Fr(eps) + Fr(2**-50) * rhs


# ---------------------------------------------------------------------------
# Constructed ground truth
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", [0, 1])
def test_constructed_collisions_and_disjoint_boxes(kind):
    b = W.unit_cube(kind, 600, seed=40 + kind)
    e = oracle.err_from_bounds(kind, b.verts)
    col, toi, tol, chk = oracle.ccd_batch(kind, b.verts, e, nthreads=4)
    hit = b.truth == 1
    assert np.all(col[hit] == 1), "false negative on a constructed collision"
    assert np.all(toi[hit] <= b.t_star[hit]), "toi later than the exact contact"
    assert np.all(b.t_star[hit] - toi[hit] <= 10 * 1e-6)
    assert np.all(tol[hit] < 1e-6) or np.all(chk[hit][tol[hit] >= 1e-6] >= 10**6)
    miss = b.truth == 0
    assert np.all(col[miss] == 0)
    assert np.all(np.isinf(toi[miss])) and np.all(tol[miss] == 0)
    if kind == 1:
        # EE root-box corners are vertex differences p_i - p_j, all of one sign
        # on the separating axis: rejected by the first check
        assert np.all(chk[miss] == 1)


def test_constructed_exactness_of_contact():
    """p(t*) = T(t*, u*, v*) holds exactly for the stored doubles."""
    for kind in (0, 1):
        b = W.unit_cube(kind, 200, seed=50 + kind)
        for i in np.nonzero(b.truth == 1)[0][:60]:
            f = ex.coplanarity_cubic(kind, b.verts[i])
            t = Fr(b.t_star[i])
            assert f[0] + f[1] * t + f[2] * t**2 + f[3] * t**3 == 0


def test_time_accuracy_static_triangle():
    """Static triangle, point with normal speed s: at the returned toi some
    F value is within delta + eps, so t* - toi <= sqrt(3)(delta + eps)/s."""
    rng = np.random.default_rng(60)
    g = 2.0**-20
    for _ in range(60):
        V = W.q(rng.uniform(-1, 1, (3, 3)), g)
        t = W.q(rng.uniform(0.05, 0.95), 2.0**-10)
        u, v = 0.25, 0.375
        X = (1 - u - v) * V[0] + u * V[1] + v * V[2]
        nrm = np.cross(V[1] - V[0], V[2] - V[0])
        nrm /= np.linalg.norm(nrm)
        D = W.q(rng.uniform(2, 4) * nrm, g)
        p0, p1 = X - t * D, X + (1 - t) * D
        qv = np.concatenate([p0, V.ravel(), p1, V.ravel()])
        e = oracle.err_from_bounds(0, qv)
        c, toi, tol, n = oracle.ccd(0, qv, e)
        s = abs(float(np.dot(D, nrm)))
        assert c and toi <= t
        assert t - toi <= np.sqrt(3) * (1e-6 + e.max()) / s * 1.001 + 1e-15


def test_special_cases():
    # contact exactly at t = 0, leaving along the normal: toi == 0
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], float)
    p0 = np.array([0.25, 0.25, 0.0])
    p1 = np.array([0.25, 0.25, 1.0])
    qv = np.concatenate([p0, V.ravel(), p1, V.ravel()])
    e = oracle.err_from_bounds(0, qv)
    c, toi, tol, n = oracle.ccd(0, qv, e)
    assert c and toi == 0.0
    # point static on a static triangle: collides from the start
    qv2 = np.concatenate([p0, V.ravel(), p0, V.ravel()])
    c, toi, tol, n = oracle.ccd(0, qv2, e)
    assert c and toi == 0.0
    # contact exactly at t = 1
    qv3 = np.concatenate([[0.25, 0.25, -1.0], V.ravel(), p0, V.ravel()])
    c, toi, tol, n = oracle.ccd(0, qv3, e)
    assert c and 1.0 - 1e-5 <= toi <= 1.0
    # static parallel edges at distance 0.5: no collision
    qe = np.array([0, 0, 0, 1, 0, 0, 0, 0.5, 0, 1, 0.5, 0] * 2, float)
    ee = oracle.err_from_bounds(1, qe)
    c, toi, tol, n = oracle.ccd(1, qe, ee)
    assert not c and np.isinf(toi) and tol == 0.0
    # a huge delta: the colliding root box terminates at level 0
    c, toi, tol, n = oracle.ccd(0, qv, e, delta=100.0)
    assert c and toi == 0.0 and n == 1
    # max_itr = 1: the first colliding check returns
    c, toi, tol, n = oracle.ccd(0, qv3, e, max_itr=1)
    assert c and toi == 0.0 and n == 1


def test_minimum_separation_distance_semantics():
    """MSCCD (Sec. 5.1): static point at L-inf distance 0.01 from a static
    triangle's plane collides iff d >= 0.01 (up to eps and delta)."""
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], float)
    p = np.array([0.25, 0.25, 0.01])
    qv = np.concatenate([p, V.ravel(), p, V.ravel()])
    for d, expect in ((0.0, False), (0.005, False), (0.0099, False), (0.0101, True), (0.02, True)):
        e = oracle.err_from_bounds(0, qv, ms_nonzero=d > 0)
        c, toi, tol, n = oracle.ccd(0, qv, e, ms=d)
        assert c == expect, d
        if expect:
            assert toi == 0.0


# ---------------------------------------------------------------------------
# Algorithm 2's second termination test, B inside C_eps (Sec. 4.2), and the
# depth guard, on inputs where they alone decide
# ---------------------------------------------------------------------------

def _tiny_static_vf():
    """A static triangle of legs 2^-50 and a point 2^-52 inside it that rises
    by 2^-51 over the step.  Every corner of the root box is an exact dyadic,
    so B_F([0,1]^3) is known in closed form: x and y span
    [-3 * 2^-52, 2^-52], z spans [0, 2^-51]; w(B) = 2^-50."""
    a, p = 2.0**-50, 2.0**-52
    V = [0.0, 0.0, 0.0, a, 0.0, 0.0, 0.0, a, 0.0]
    return np.array([p, p, 0.0, *V, p, p, 2.0**-51, *V])


def test_inside_filter_box_terminates_at_first_check():
    """With delta below w(B) the only way to stop at the root box is
    B subset of C_eps: eps_VF = 30 * 2^-52 (gamma = 1) contains every axis
    range above, so Algorithm 2 returns at check 1 with toi = 0 and the
    reached tolerance w(B) = 2^-50 >= delta."""
    qv = _tiny_static_vf()
    e = oracle.err_from_bounds(0, qv)
    assert np.all(e == 30 * 2.0**-52)
    c, toi, tol, n = oracle.ccd(0, qv, e, delta=2.0**-52)
    assert c and toi == 0.0 and n == 1 and tol == 2.0**-50
    # the same box against eps = 2^-52: B is no longer inside, and w(B) >=
    # delta, so the root box is split
    c, toi, tol, n = oracle.ccd(0, qv, np.full(3, 2.0**-52), delta=2.0**-52)
    assert c and n > 1


def test_inside_test_uses_the_enlarged_box():
    """Under minimum separation d the inside test takes the box enlarged by
    d (Sec. 5.1): with eps = 34 * 2^-52 (Eq. msccd-error, gamma = 1) the
    enlarged x range [-3 * 2^-52 - d, 2^-52 + d] lies in [-eps, eps] iff
    d <= 31 * 2^-52.  So d = 16 * 2^-52 stops at check 1 and d = 32 * 2^-52
    does not (its box still meets C_eps, and w(B) >= delta).  The reached
    tolerance is the un-enlarged width 2^-50."""
    qv = _tiny_static_vf()
    e = oracle.err_from_bounds(0, qv, ms_nonzero=True)
    assert np.all(e == 34 * 2.0**-52)
    c, toi, tol, n = oracle.ccd(0, qv, e, ms=16 * 2.0**-52, delta=2.0**-52)
    assert c and toi == 0.0 and n == 1 and tol == 2.0**-50
    c, toi, tol, n = oracle.ccd(0, qv, e, ms=32 * 2.0**-52, delta=2.0**-52)
    assert c and toi == 0.0 and n > 1


def test_depth_guard_stops_at_width_2_to_the_minus_53():
    """A static point exactly on a static triangle, eps = 0 and delta far
    below any representable width: no box ever terminates, so only the
    depth guard ends the run.  kappa_t = 0 (nothing moves), hence t is never
    split and toi = 0; u and v alternate (kappa_u = kappa_v = 3) until the
    split dimension has width 2^-53, after at most 2 * 53 levels of at most
    eight boxes.  The box then returned has x and y ranges equal to its u
    and v widths, 2^-53 or 2^-52, well above delta."""
    V = [0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0, 0.0]
    p = [0.25, 0.25, 0.0]
    qv = np.array([*p, *V, *p, *V])
    np.testing.assert_array_equal(oracle.kappa(0, qv), [0.0, 3.0, 3.0])
    c, toi, tol, n = oracle.ccd(0, qv, np.zeros(3), delta=1e-300, max_itr=10**6)
    assert c and toi == 0.0
    assert tol in (2.0**-53, 2.0**-52)
    assert n <= 2 * 53 * 8


# ---------------------------------------------------------------------------
# The paper's worked examples (tests/golden)
# ---------------------------------------------------------------------------

def test_paper_hourglass(golden):
    qv, meta = golden("hourglass_vf.txt")
    e = oracle.err_from_bounds(meta["kind"], qv)
    c, toi, tol, n = oracle.ccd(meta["kind"], qv, e)
    assert meta["truth"] == 1 and c
    t_star = 1 - Fr(0.1)
    assert Fr(toi) <= t_star and t_star - Fr(toi) < Fr(1, 10**5)


def test_paper_inflection_cubic_and_no_collision(golden):
    qv, meta = golden("inflection_vf.txt")
    cubic = [Fr(int(x)) for x in meta["cubic"].split()]
    assert ex.coplanarity_cubic(meta["kind"], qv) == cubic
    e = oracle.err_from_bounds(meta["kind"], qv)
    c, toi, tol, n = oracle.ccd(meta["kind"], qv, e)
    assert meta["truth"] == 0 and not c
    # the exact run empties its queue too: certified no root
    cx, _, _, _ = ex.solve(meta["kind"], qv, 1e-6, 5000)
    assert not cx


def test_paper_bsc_false_negative_case(golden):
    qv, meta = golden("bsc_false_negative_vf.txt")
    e = oracle.err_from_bounds(meta["kind"], qv)
    c, toi, tol, n = oracle.ccd(meta["kind"], qv, e, max_itr=10**5)
    assert meta["truth"] == 1 and c
    y0, y1 = Fr(0.57), Fr(0.28)
    t_star = (y0 - Fr(0.5)) / (y0 - y1)      # v2 meets p on the line x = 1
    assert Fr(toi) <= t_star
    assert abs(float(t_star) - 7 / 29) < 1e-12


# ---------------------------------------------------------------------------
# Algorithm 2 control logic vs an independent exact implementation
# ---------------------------------------------------------------------------

def _exact_grid_queries(rng, n, kind):
    out = []
    for _ in range(n):
        P = rng.integers(-16, 17, 24) / 8.0            # coordinates on a 1/8 grid
        if rng.random() < 0.3:                         # coplanar motion
            ax = rng.integers(0, 3)
            P.reshape(8, 3)[:, ax] = rng.integers(-8, 9) / 8.0
        if rng.random() < 0.2:                         # a static primitive
            P[12:] = P[:12]
        out.append(P)
    return out


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("ms", [0.0, 1 / 64])
def test_control_logic_matches_literal_exact_queue(kind, ms):
    """With coordinates on a coarse dyadic grid and a coarse delta every
    floating-point operation of the oracle is exact, so with eps = 0 its
    heap-based run must equal the literal list + stable-sort run in rational
    arithmetic: same flag, toi, out_tol and check count."""
    rng = np.random.default_rng(70 + kind + int(ms * 64))
    delta, max_itr = 1 / 32, 400
    for qv in _exact_grid_queries(rng, 25, kind):
        zero = np.zeros(3)
        for flags in (0, oracle.LITERAL_DROP):
            c, toi, tol, n = oracle.ccd(kind, qv, zero, ms=ms, delta=delta,
                                        max_itr=max_itr, flags=flags)
            cx, tx, wx, nx = ex.solve(kind, qv, Fr(delta), max_itr, ms=Fr(ms),
                                      literal_drop=bool(flags))
            assert (c, n) == (cx, nx)
            if c:
                assert Fr(toi) == tx and Fr(tol) == wx
            else:
                assert np.isinf(toi) and tol == 0


# ---------------------------------------------------------------------------
# No false negatives against exact roots found by brute force
# ---------------------------------------------------------------------------

def _planted_root_queries(rng, n, kind):
    """Queries on a 1/8 grid with an exact root planted at a grid point
    (t*, u*, v*), some in coplanar motion or with a static primitive."""
    out = []
    for _ in range(n):
        P = rng.integers(-8, 9, 24) / 8.0
        coplanar = rng.random() < 0.4
        if coplanar:
            ax = rng.integers(0, 3)
            P.reshape(8, 3)[:, ax] = rng.integers(-4, 5) / 8.0
        if rng.random() < 0.2:
            P[12:] = P[:12]
        t = rng.integers(0, 9) / 8.0
        u = rng.integers(0, 9) / 8.0
        v = rng.integers(0, 9 - (8 * u if kind == 0 else 0)) / 8.0 if kind == 0 else rng.integers(0, 9) / 8.0
        X = lambda i: (1 - t) * P[i * 3:i * 3 + 3] + t * P[12 + i * 3:12 + i * 3 + 3]
        if kind == 0:
            target = (1 - u - v) * X(1) + u * X(2) + v * X(3)
            D = rng.integers(-8, 9, 3) / 8.0
            if coplanar:
                D[ax] = 0.0
            P[0:3], P[12:15] = target - t * D, target + (1 - t) * D
        else:
            target = (1 - v) * X(2) + v * X(3)
            E = rng.integers(-8, 9, 3) / 8.0
            D = rng.integers(-8, 9, 3) / 8.0
            if coplanar:
                D[ax] = 0.0
                E[ax] = 0.0
            a, b = target - u * E, target + (1 - u) * E
            P[0:3], P[12:15] = a - t * D, a + (1 - t) * D
            P[3:6], P[15:18] = b - t * D, b + (1 - t) * D
        out.append(P)
    return out


@pytest.mark.parametrize("kind", [0, 1])
def test_no_false_negative_vs_bruteforce_exact_roots(kind):
    """Exact zeros of F found by brute-force rational sampling of (t, u, v)
    on the 1/8 grid certify collisions; the oracle must report each one with
    toi no later than the earliest root found."""
    rng = np.random.default_rng(80 + kind)
    grid = [Fr(i, 8) for i in range(9)]
    found = 0
    for qv in _planted_root_queries(rng, 40, kind):
        qf = ex.to_fr(qv)
        first_root = None
        for t in grid:
            P = [ex.point(qf, i, t) for i in range(4)]
            for u in grid:
                for v in grid:
                    if kind == 0 and u + v > 1:
                        continue
                    if kind == 0:
                        F = [P[0][c] - ((1 - u - v) * P[1][c] + u * P[2][c] + v * P[3][c]) for c in range(3)]
                    else:
                        F = [((1 - u) * P[0][c] + u * P[1][c]) - ((1 - v) * P[2][c] + v * P[3][c]) for c in range(3)]
                    if F == [0, 0, 0]:
                        first_root = t
                        break
                if first_root is not None:
                    break
            if first_root is not None:
                break
        assert first_root is not None      # the planted root at least
        found += 1
        e = oracle.err_from_bounds(kind, qv)
        c, toi, tol, n = oracle.ccd(kind, qv, e, max_itr=20000)
        assert c, "false negative against an exact root"
        assert toi <= float(first_root)
    assert found == 40


# ---------------------------------------------------------------------------
# SolveMSCCD's shortened time interval [0, t_max] (Sec. 6, line search)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("t_max", [0.5, 0.75])
def test_shortened_interval_control_logic_matches_exact(kind, t_max):
    rng = np.random.default_rng(90 + kind + int(8 * t_max))
    for qv in _exact_grid_queries(rng, 20, kind):
        zero = np.zeros(3)
        for ms in (0.0, 1 / 64):
            c, toi, tol, n = oracle.ccd(kind, qv, zero, ms=ms, delta=1 / 32, max_itr=400,
                                        t_max=t_max)
            cx, tx, wx, nx = ex.solve(kind, qv, Fr(1, 32), 400, ms=Fr(ms), t_max=Fr(t_max))
            assert (c, n) == (cx, nx)
            if c:
                assert Fr(toi) == tx and Fr(tol) == wx and toi <= t_max


def test_shortened_interval_sees_only_roots_before_t_max():
    """Static triangle, point crossing its plane once at t*: a collision is
    reported for t_max >= t* (toi <= t*), none for t_max well below t*."""
    rng = np.random.default_rng(95)
    g = 2.0**-20
    for _ in range(40):
        V = W.q(rng.uniform(-1, 1, (3, 3)), g)
        t = W.q(rng.uniform(0.2, 0.8), 2.0**-10)
        X = 0.5 * V[0] + 0.25 * V[1] + 0.25 * V[2]
        nrm = np.cross(V[1] - V[0], V[2] - V[0])
        nrm /= np.linalg.norm(nrm)
        D = W.q(rng.uniform(2, 4) * nrm, g)
        qv = np.concatenate([X - t * D, V.ravel(), X + (1 - t) * D, V.ravel()])
        e = oracle.err_from_bounds(0, qv)
        c1, toi1, _, _ = oracle.ccd(0, qv, e, t_max=1.0)
        c2, toi2, _, _ = oracle.ccd(0, qv, e, t_max=min(1.0, t + 0.1))
        c3, _, _, _ = oracle.ccd(0, qv, e, t_max=t - 0.1)
        assert c1 and c2 and not c3
        assert toi1 <= t and toi2 <= t
    # t_max = 1 is the plain solver
    b = W.unit_cube(1, 200, seed=96)
    e = oracle.err_from_bounds(1, b.verts)
    for x, y in zip(oracle.ccd_batch(1, b.verts, e), oracle.ccd_batch(1, b.verts, e, t_max=1.0)):
        assert np.array_equal(x, y)
