"""Exact-rational companion of the oracle (TEST INFRASTRUCTURE ONLY).

Everything here uses ``fractions.Fraction`` and the paper's own algebraic
forms, independently of the floating-point operation order in
``ccd_oracle.c``:

* ``F`` -- Eq. (F-vf) / (F-ee) as printed: barycentric / edge-parameter
  combinations of the linearly interpolated points.
* ``solve`` -- Algorithm 2 run in exact arithmetic with a Python list that is
  stably re-sorted by (level, left end of I_t) after every insertion, i.e. the
  literal "Q <- Q u {I1, I2}; sort(Q, order)" of the paper.  With eps = 0 and
  exact arithmetic, an emptied queue certifies that F has no root in the
  domain (B_F is an inclusion function, Proposition 1).
* ``coplanarity_cubic`` -- f(t) = <n(t), q(t)> of Eq. (univariate).
* ``linf_distance`` -- min over the domain of ||F(0,u,v)||_inf (Sec. 5.1
  norm), the exact optimum of that linear program by vertex enumeration.
"""
from __future__ import annotations

from fractions import Fraction as Fr
from typing import Sequence

VF, EE = 0, 1


def to_fr(query: Sequence[float]) -> list[Fr]:
    return [Fr(float(x)) for x in query]


def point(q: Sequence[Fr], i: int, t: Fr) -> list[Fr]:
    """p_i(t) = (1 - t) p_i^0 + t p_i^1 (Sec. 3)."""
    return [(1 - t) * q[i * 3 + c] + t * q[12 + i * 3 + c] for c in range(3)]


def F(kind: int, q: Sequence[Fr], t: Fr, u: Fr, v: Fr) -> list[Fr]:
    """Eq. (F-vf) for kind VF, Eq. (F-ee) for kind EE, in exact arithmetic."""
    a, b, c, d = (point(q, i, t) for i in range(4))
    if kind == VF:
        return [a[k] - ((1 - u - v) * b[k] + u * c[k] + v * d[k]) for k in range(3)]
    return [((1 - u) * a[k] + u * b[k]) - ((1 - v) * c[k] + v * d[k]) for k in range(3)]


def box(kind: int, q, I, t_max=1) -> tuple[list[Fr], list[Fr]]:
    """Exact B_F(I): per-axis min / max over the 8 corners (Eq. box); I[0:2]
    are s-values, the corner times t_max * s."""
    vals = [F(kind, q, t * t_max, u, v) for t in I[0:2] for u in I[2:4] for v in I[4:6]]
    m = [min(x[k] for x in vals) for k in range(3)]
    M = [max(x[k] for x in vals) for k in range(3)]
    return m, M


def kappa(kind: int, q, t_max=1) -> list[Fr]:
    """Eq. (kappas) in exact arithmetic over [0, t_max] x [0,1]^2."""
    one, zero = Fr(1), Fr(0)
    out = []
    for dim in range(3):
        best = Fr(0)
        for i in (zero, one):
            for j in (zero, one):
                lo = [zero, zero, zero]
                hi = [one, one, one]
                others = [k for k in range(3) if k != dim]
                lo[others[0]] = hi[others[0]] = i
                lo[others[1]] = hi[others[1]] = j
                A = F(kind, q, lo[0] * t_max, lo[1], lo[2])
                B = F(kind, q, hi[0] * t_max, hi[1], hi[2])
                best = max(best, max(abs(A[k] - B[k]) for k in range(3)))
        out.append(3 * best)
    return out


def solve(kind: int, query, delta, max_itr: int, ms=0, err=(0, 0, 0),
          literal_drop: bool = False, t_max=1):
    """Algorithm 2 in exact arithmetic.  Returns (collides, toi, w(B), checks).

    ``err`` is the per-axis half-width of C_eps (0 for a pure exact run);
    the same readings as the C oracle apply (stable order, split-anyway for a
    non-first terminating box unless ``literal_drop``, out_tol = w(B), depth
    guard at width 2^-53).
    """
    q = query if isinstance(query[0], Fr) else to_fr(query)
    delta = Fr(delta)
    ms = Fr(ms)
    err = [Fr(e) for e in err]
    t_max = Fr(t_max)
    kap = kappa(kind, q, t_max)
    Q = [(0, [Fr(0), Fr(1), Fr(0), Fr(1), Fr(0), Fr(1)])]
    n = 0
    lp = -1
    If_left = None
    while Q:
        level, I = Q.pop(0)
        m, M = box(kind, q, I, t_max)
        n += 1
        hit = all(m[c] - ms <= err[c] and M[c] + ms >= -err[c] for c in range(3))
        if not hit:
            continue
        first = level != lp
        if first:
            If_left = I[0]
        wB = max(M[c] - m[c] for c in range(3))
        if n >= max_itr:
            return True, If_left * t_max, wB, n
        inside = all(m[c] - ms >= -err[c] and M[c] + ms <= err[c] for c in range(3))
        if wB < delta or inside:
            if first:
                return True, If_left * t_max, wB, n
            if literal_drop:
                lp = level
                continue
        c = [(I[2 * d + 1] - I[2 * d]) * kap[d] for d in range(3)]
        cm = max(c)
        dim = 0 if c[0] == cm else (1 if c[1] == cm else 2)
        L, R = I[2 * dim], I[2 * dim + 1]
        if R - L <= Fr(1, 2**53):
            return True, If_left * t_max, wB, n
        mid = (L + R) / 2
        I1, I2 = list(I), list(I)
        I1[2 * dim + 1] = mid
        I2[2 * dim] = mid
        for child in (I1, I2):
            if kind == VF and child[2] + child[4] > 1:
                continue
            Q.append((level + 1, child))
        Q.sort(key=lambda e: (e[0], e[1][0]))  # stable: ties keep insertion order
        lp = level
    return False, None, Fr(0), n


def coplanarity_cubic(kind: int, query) -> list[Fr]:
    """Coefficients [c0, c1, c2, c3] of f(t) = <n(t), q(t)> (Eq. univariate):
    VF: n = (v2 - v1) x (v3 - v1), q = p - v1;
    EE: n = (p2 - p1) x (p4 - p3), q = p3 - p1."""
    q = query if isinstance(query[0], Fr) else to_fr(query)

    # Each point is affine in t: P(t) = P0 + t (P1 - P0); work with polynomials.
    def poly_point(i):
        return [[q[i * 3 + c], q[12 + i * 3 + c] - q[i * 3 + c]] for c in range(3)]

    def sub(A, B):
        return [[A[c][0] - B[c][0], A[c][1] - B[c][1]] for c in range(3)]

    def pmul(a, b):
        out = [Fr(0)] * (len(a) + len(b) - 1)
        for i, x in enumerate(a):
            for j, y in enumerate(b):
                out[i + j] += x * y
        return out

    def padd(a, b):
        n = max(len(a), len(b))
        return [(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(n)]

    def psub(a, b):
        return padd(a, [-x for x in b])

    def cross(A, B):
        return [psub(pmul(A[1], B[2]), pmul(A[2], B[1])),
                psub(pmul(A[2], B[0]), pmul(A[0], B[2])),
                psub(pmul(A[0], B[1]), pmul(A[1], B[0]))]

    P = [poly_point(i) for i in range(4)]
    if kind == VF:
        n = cross(sub(P[2], P[1]), sub(P[3], P[1]))
        qq = sub(P[0], P[1])
    else:
        n = cross(sub(P[1], P[0]), sub(P[3], P[2]))
        qq = sub(P[2], P[0])
    f = [Fr(0)]
    for c in range(3):
        f = padd(f, pmul(n[c], qq[c]))
    f = f + [Fr(0)] * (4 - len(f))
    return f[:4]


def linf_distance(kind: int, query) -> Fr:
    """Exact min over the domain (VF triangle, EE unit square) of
    max_c |F_c(0,u,v)|, with F affine in (u, v) at t = 0.  The linear program
    min s s.t. -s <= F_c(u,v) <= s, (u,v) in the domain has its optimum at a
    vertex of its feasible set: a domain corner, a point of a domain edge
    where two of the lines +-F_c cross, or an interior point where three of
    them meet (two axes zero, or s1 F_1 = s2 F_2 = s3 F_3).  Every such point
    is computed exactly and the exact objective is minimised over them."""
    q = query if isinstance(query[0], Fr) else to_fr(query)
    zero, one = Fr(0), Fr(1)

    def f(u, v):
        return F(kind, q, zero, u, v)

    def g(u, v):
        return max(abs(x) for x in f(u, v))

    def inside(u, v):
        if u < 0 or v < 0:
            return False
        return u + v <= 1 if kind == VF else (u <= 1 and v <= 1)

    A = f(zero, zero)
    Bu = [f(one, zero)[c] - A[c] for c in range(3)]
    Cv = [f(zero, one)[c] - A[c] for c in range(3)]
    pts = [(zero, zero), (one, zero), (zero, one)] + ([(one, one)] if kind == EE else [])
    edges = ([((0, 0), (1, 0)), ((0, 0), (0, 1)), ((1, 0), (-1, 1))] if kind == VF else
             [((0, 0), (1, 0)), ((0, 0), (0, 1)), ((1, 0), (0, 1)), ((0, 1), (1, 0))])
    for (pu, pv), (du, dv) in edges:
        al = [A[c] + pu * Bu[c] + pv * Cv[c] for c in range(3)]
        be = [du * Bu[c] + dv * Cv[c] for c in range(3)]
        taus = [-al[c] / be[c] for c in range(3) if be[c] != 0]
        for c1 in range(3):
            for c2 in range(c1 + 1, 3):
                for sg in (1, -1):
                    den = be[c1] - sg * be[c2]
                    if den != 0:
                        taus.append((sg * al[c2] - al[c1]) / den)
        pts += [(pu + t * du, pv + t * dv) for t in taus if 0 <= t <= 1]
    rows = []
    for c1 in range(3):
        for c2 in range(c1 + 1, 3):
            rows.append(((Bu[c1], Cv[c1], -A[c1]), (Bu[c2], Cv[c2], -A[c2])))
    for s1, s2, s3 in ((1, 1, 1), (1, 1, -1), (1, -1, 1), (-1, 1, 1)):
        s = (s1, s2, s3)
        rows.append(((s[0] * Bu[0] - s[1] * Bu[1], s[0] * Cv[0] - s[1] * Cv[1],
                      s[1] * A[1] - s[0] * A[0]),
                     (s[1] * Bu[1] - s[2] * Bu[2], s[1] * Cv[1] - s[2] * Cv[2],
                      s[2] * A[2] - s[1] * A[1])))
    for (a11, a12, b1), (a21, a22, b2) in rows:
        det = a11 * a22 - a12 * a21
        if det != 0:
            u = (b1 * a22 - a12 * b2) / det
            v = (a11 * b2 - b1 * a21) / det
            if inside(u, v):
                pts.append((u, v))
    return min(g(u, v) for u, v in pts if inside(u, v))
