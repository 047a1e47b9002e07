"""Seeded synthetic CCD workloads (inputs only: no CCD arithmetic here).

The paper's benchmark (Sec. 3.1: a handcrafted set of degenerate queries and
a simulation set of queries from elastodynamic runs) is not available, so
these generators stand in for it.  Every query is 24 doubles laid out as
index = time*12 + point*3 + coord (the four points at t0, then at t1;
Appendix A).  VF points are (p, v1, v2, v3), EE points (p1, p2, p3, p4).

Constructed collisions are exact in binary64: coordinates, times and
barycentric parameters are chosen on dyadic grids small enough that every
intermediate product and sum below is representable, so the constructed
contact p(t*) = T(t*, u*, v*) holds exactly for the stored doubles.

Each generator returns a ``Workload`` with per-kind (n, 24) float64 arrays and
per-query labels: ``truth`` 1 = constructed collision at ``t_star``,
0 = certified no collision (disjoint swept AABBs), -1 = not labelled.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

VF, EE = 0, 1


@dataclass
class Batch:
    kind: int
    verts: np.ndarray                    # (n, 24) float64
    truth: np.ndarray                    # (n,) int8
    t_star: np.ndarray                   # (n,) float64 (nan if not constructed)
    family: np.ndarray = None            # (n,) int8 family tag (generator-specific)

    @property
    def n(self) -> int:
        return self.verts.shape[0]


@dataclass
class Workload:
    name: str
    batches: list = field(default_factory=list)   # list[Batch]
    params: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return sum(b.n for b in self.batches)


def q(x, grid):
    """Round to a dyadic grid (exact for the magnitudes used here)."""
    return np.round(np.asarray(x, dtype=np.float64) / grid) * grid


def _pack(P0, P1):
    """P0, P1: (n, 4, 3) -> (n, 24)."""
    n = P0.shape[0]
    return np.concatenate([P0.reshape(n, 12), P1.reshape(n, 12)], axis=1).copy()


def _unit(v):
    return v / np.maximum(np.linalg.norm(v, axis=-1, keepdims=True), 1e-300)


def _sample_bary(rng, n, lo=0.05, hi_sum=0.95, grid=2.0**-8):
    """(u*, v*) on a grid with u*, v* >= lo and u* + v* <= hi_sum."""
    u = np.empty(n)
    v = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        a = q(rng.uniform(lo, hi_sum, todo.size), grid)
        b = q(rng.uniform(lo, hi_sum, todo.size), grid)
        ok = (a >= lo) & (b >= lo) & (a + b <= hi_sum)
        u[todo[ok]] = a[ok]
        v[todo[ok]] = b[ok]
        todo = todo[~ok]
    return u, v


def _interp(A0, A1, t):
    """(1 - t) A0 + t A1 written as A0 + t (A1 - A0); exact on the grids used."""
    return A0 + t[:, None] * (A1 - A0)


# ---------------------------------------------------------------------------
# Uniform unit-cube workload (VF: 10,000 queries, seed 0) and its EE analogue
# ---------------------------------------------------------------------------

def _vf_collide(rng, n, scale=1.0, disp=0.1, speed=(2.0, 4.0)):
    """Point moved linearly through a moving triangle's interior at t*."""
    g = 2.0**-20
    V0 = q(rng.uniform(-1, 1, (n, 3, 3)) * scale, g * scale)
    V1 = q(V0 + rng.normal(0, disp, (n, 3, 3)) * scale, g * scale)
    t = q(rng.uniform(0, 1, n), 2.0**-10)
    t = np.clip(t, 2.0**-10, 1 - 2.0**-10)
    u, v = _sample_bary(rng, n)
    Vt = _interp(V0.reshape(n, 9), V1.reshape(n, 9), t).reshape(n, 3, 3)
    X = (1 - u - v)[:, None] * Vt[:, 0] + u[:, None] * Vt[:, 1] + v[:, None] * Vt[:, 2]
    nrm = _unit(np.cross(Vt[:, 1] - Vt[:, 0], Vt[:, 2] - Vt[:, 0]))
    s = rng.uniform(*speed, n) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    D = q((s[:, None] * nrm + rng.normal(0, 0.3, (n, 3))) * scale, g * scale)
    p0 = X - t[:, None] * D
    p1 = X + (1 - t)[:, None] * D
    P0 = np.concatenate([p0[:, None], V0], axis=1)
    P1 = np.concatenate([p1[:, None], V1], axis=1)
    return _pack(P0, P1), t


def _ee_collide(rng, n, scale=1.0, disp=0.1, speed=(2.0, 4.0)):
    """Edge (p1, p2) moved rigidly through edge (p3, p4) at t*, u*, v*."""
    g = 2.0**-20
    B0 = q(rng.uniform(-1, 1, (n, 2, 3)) * scale, g * scale)
    B1 = q(B0 + rng.normal(0, disp, (n, 2, 3)) * scale, g * scale)
    t = q(rng.uniform(0, 1, n), 2.0**-10)
    t = np.clip(t, 2.0**-10, 1 - 2.0**-10)
    u = q(rng.uniform(0.05, 0.95, n), 2.0**-8)
    v = q(rng.uniform(0.05, 0.95, n), 2.0**-8)
    Bt = _interp(B0.reshape(n, 6), B1.reshape(n, 6), t).reshape(n, 2, 3)
    X = (1 - v)[:, None] * Bt[:, 0] + v[:, None] * Bt[:, 1]
    E = q(rng.uniform(-1, 1, (n, 3)) * scale, g * scale)
    a = X - u[:, None] * E
    b = X + (1 - u)[:, None] * E
    nrm = _unit(np.cross(E, Bt[:, 1] - Bt[:, 0]))
    s = rng.uniform(*speed, n) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    D = q((s[:, None] * nrm + rng.normal(0, 0.3, (n, 3))) * scale, g * scale)
    a0, a1 = a - t[:, None] * D, a + (1 - t)[:, None] * D
    b0, b1 = b - t[:, None] * D, b + (1 - t)[:, None] * D
    P0 = np.stack([a0, b0, B0[:, 0], B0[:, 1]], axis=1)
    P1 = np.stack([a1, b1, B1[:, 0], B1[:, 1]], axis=1)
    return _pack(P0, P1), t


def _disjoint(rng, n, kind, scale=1.0, disp=0.1):
    """Random primitives translated so their swept AABBs are disjoint."""
    g = 2.0**-20
    P0 = q(rng.uniform(-1, 1, (n, 4, 3)) * scale, g * scale)
    P1 = q(P0 + rng.normal(0, disp, (n, 4, 3)) * scale, g * scale)
    first = [0] if kind == VF else [0, 1]
    second = [1, 2, 3] if kind == VF else [2, 3]
    A = np.concatenate([P0[:, first], P1[:, first]], axis=1)
    B = np.concatenate([P0[:, second], P1[:, second]], axis=1)
    axis = rng.integers(0, 3, n)
    side = rng.random(n) < 0.5
    gap = q(rng.uniform(0.01, 0.5, n) * scale, g * scale)
    idx = np.arange(n)
    a_lo, a_hi = A.min(1)[idx, axis], A.max(1)[idx, axis]
    b_lo, b_hi = B.min(1)[idx, axis], B.max(1)[idx, axis]
    shift = np.where(side, b_hi + gap - a_lo, b_lo - gap - a_hi)
    shift = q(shift, g * scale)
    # after rounding the shift, make sure the gap is still positive
    shift = np.where(side, np.maximum(shift, b_hi - a_lo + g * scale),
                     np.minimum(shift, b_lo - a_hi - g * scale))
    for arr in (P0, P1):
        arr[idx[:, None], np.array(first)[None, :], axis[:, None]] += shift[:, None]
    return _pack(P0, P1)


def unit_cube(kind: int, n: int, seed: int, scale: float = 1.0) -> Batch:
    """Half constructed collisions (truth 1, exact t*), half disjoint swept
    AABBs (truth 0); triangle/edge vertices uniform in [-1,1]^3 at t0 and
    displaced by N(0, 0.1) to t1, all times ``scale``."""
    rng = np.random.default_rng(seed)
    nc = n // 2
    nd = n - nc
    if kind == VF:
        C, tc = _vf_collide(rng, nc, scale)
    else:
        C, tc = _ee_collide(rng, nc, scale)
    D = _disjoint(rng, nd, kind, scale)
    verts = np.concatenate([C, D])
    truth = np.concatenate([np.ones(nc, np.int8), np.zeros(nd, np.int8)])
    t_star = np.concatenate([tc, np.full(nd, np.nan)])
    perm = rng.permutation(n)
    return Batch(kind, verts[perm], truth[perm], t_star[perm],
                 np.zeros(n, np.int8))


def uniform_vf_10k(seed: int = 0, n: int = 10_000) -> Workload:
    """10,000 VF queries: half through the triangle interior, half disjoint."""
    return Workload("uniform-vf-10k", [unit_cube(VF, n, seed)],
                    {"seed": seed, "ms": 0.0, "delta": 1e-6, "max_itr": 10**6})


# ---------------------------------------------------------------------------
# Simulation-shaped workload: two jittered sheets of a unit-scale mesh
# ---------------------------------------------------------------------------

def _surface(xy):
    x, y = xy[..., 0], xy[..., 1]
    return 0.05 * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)


FAM_PLAIN, FAM_CONSTRUCTED, FAM_COPLANAR, FAM_PARALLEL, FAM_T0, FAM_T1, FAM_ON_EDGE, \
    FAM_COLLINEAR, FAM_VERTEX, FAM_GRAZING = range(10)


def _sim_plain(rng, n, kind, h, disp, g):
    """Nearby primitive pairs from two sheets separated by a small gap,
    every vertex displaced by N(0, disp) over the step."""
    anchor = rng.uniform(0.05, 0.95, (n, 2))
    tri_off = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    gap = h * 10.0 ** rng.uniform(-2.5, 0.5, n)
    if kind == VF:
        xy = anchor[:, None, :] + tri_off[None] * h + rng.uniform(-0.2, 0.2, (n, 3, 2)) * h
        tri = np.concatenate([xy, _surface(xy)[..., None]], axis=-1)
        pxy = anchor + rng.uniform(-0.5, 1.5, (n, 2)) * h
        pz = _surface(pxy) + gap * np.where(rng.random(n) < 0.5, -1.0, 1.0)
        pt = np.concatenate([pxy, pz[:, None]], axis=-1)
        P0 = np.concatenate([pt[:, None], tri], axis=1)
    else:
        e1 = anchor[:, None, :] + np.array([[0.0, 0.0], [1.0, 0.0]])[None] * h \
            + rng.uniform(-0.2, 0.2, (n, 2, 2)) * h
        ea = np.concatenate([e1, _surface(e1)[..., None]], axis=-1)
        c = anchor + 0.5 * h + rng.uniform(-0.5, 0.5, (n, 2)) * h
        ang = rng.uniform(0, np.pi, n)
        dxy = np.stack([np.cos(ang), np.sin(ang)], -1) * 0.5 * h
        e2 = np.stack([c - dxy, c + dxy], axis=1)
        z2 = _surface(e2) + (gap * np.where(rng.random(n) < 0.5, -1.0, 1.0))[:, None]
        eb = np.concatenate([e2, z2[..., None]], axis=-1)
        P0 = np.concatenate([ea, eb], axis=1)
    P0 = q(P0, g)
    P1 = q(P0 + rng.normal(0, disp, P0.shape), g)
    return _pack(P0, P1)


def _sim_constructed(rng, n, kind, h, disp, g):
    """Constructed collisions at mesh scale (same recipe as the unit-cube set,
    scaled to the mesh spacing, speeds ~ the step displacement)."""
    if kind == VF:
        V, t = _vf_collide(rng, n, scale=h, disp=disp / h, speed=(2.0, 4.0))
    else:
        V, t = _ee_collide(rng, n, scale=h, disp=disp / h, speed=(2.0, 4.0))
    anchor = q(rng.uniform(0.05, 0.95, (n, 3)) * np.array([1, 1, 0.05]), 2.0**-20)
    V = V + np.tile(anchor, 8)     # exact: anchors on a 2^-20 grid
    return V, t


def _sim_degenerate(rng, n, kind, h, g):
    """5 % families: coplanar motion, parallel edges, contact exactly at t=0
    or t=1, point on an edge (VF) / endpoint on an edge (EE)."""
    fam = rng.choice([FAM_COPLANAR, FAM_PARALLEL, FAM_T0, FAM_T1, FAM_ON_EDGE], n)
    out = np.empty((n, 24))
    gg = 2.0**-20
    for f in np.unique(fam):
        idx = np.nonzero(fam == f)[0]
        m = idx.size
        anchor = q(rng.uniform(0.05, 0.95, (m, 3)) * np.array([1, 1, 0.05]), gg)
        if f == FAM_COPLANAR or (f == FAM_PARALLEL and kind == VF):
            P0 = q(rng.uniform(-1, 1, (m, 4, 3)) * h, gg * h)
            P1 = q(P0 + rng.normal(0, 0.3, (m, 4, 3)) * h, gg * h)
            ax = rng.integers(0, 3, m)
            P0[np.arange(m), :, ax] = 0.0
            P1[np.arange(m), :, ax] = 0.0
            V = _pack(P0, P1)
        elif f == FAM_PARALLEL:
            a0 = q(rng.uniform(-1, 1, (m, 3)) * h, gg * h)
            d = q(rng.uniform(-1, 1, (m, 3)) * h, gg * h)
            off = q(rng.normal(0, 0.3, (m, 3)) * h, gg * h)
            mv = q(rng.normal(0, 0.3, (m, 3)) * h, gg * h)
            s = q(rng.uniform(0.2, 1.5, m), 2.0**-4)[:, None]
            P0 = np.stack([a0, a0 + d, a0 + off, a0 + off + s * d], 1)
            P1 = P0.copy()
            P1[:, 0:2] += mv[:, None]
            V = _pack(P0, P1)
        else:
            if kind == VF:
                V, t = _vf_collide(rng, m, scale=h, disp=0.3, speed=(2.0, 4.0))
            else:
                V, t = _ee_collide(rng, m, scale=h, disp=0.3, speed=(2.0, 4.0))
            P0 = V[:, :12].reshape(m, 4, 3)
            P1 = V[:, 12:].reshape(m, 4, 3)
            if f == FAM_T0:
                # contact at t = 0: move the first primitive so it touches at t0
                # and then leaves along the same velocity
                shift = None
                if kind == VF:
                    bary = _sample_bary(rng, m)
                    X0 = (1 - bary[0] - bary[1])[:, None] * P0[:, 1] + bary[0][:, None] * P0[:, 2] \
                        + bary[1][:, None] * P0[:, 3]
                    shift = X0 - P0[:, 0]
                    P0[:, 0] += shift
                    P1[:, 0] += shift
                else:
                    uu = q(rng.uniform(0.1, 0.9, m), 2.0**-8)
                    X0 = (1 - uu)[:, None] * P0[:, 2] + uu[:, None] * P0[:, 3]
                    shift = X0 - P0[:, 0]
                    P0[:, 0:2] += shift[:, None]
                    P1[:, 0:2] += shift[:, None]
            elif f == FAM_T1:
                if kind == VF:
                    bary = _sample_bary(rng, m)
                    X1 = (1 - bary[0] - bary[1])[:, None] * P1[:, 1] + bary[0][:, None] * P1[:, 2] \
                        + bary[1][:, None] * P1[:, 3]
                    shift = X1 - P1[:, 0]
                    P0[:, 0] += shift
                    P1[:, 0] += shift
                else:
                    uu = q(rng.uniform(0.1, 0.9, m), 2.0**-8)
                    X1 = (1 - uu)[:, None] * P1[:, 2] + uu[:, None] * P1[:, 3]
                    shift = X1 - P1[:, 0]
                    P0[:, 0:2] += shift[:, None]
                    P1[:, 0:2] += shift[:, None]
            else:  # on edge: the contact point lies on an edge of the second primitive
                t = q(rng.uniform(0.1, 0.9, m), 2.0**-10)
                uu = q(rng.uniform(0.1, 0.9, m), 2.0**-8)
                if kind == VF:
                    Vt = _interp(P0[:, 1:].reshape(m, 9), P1[:, 1:].reshape(m, 9), t).reshape(m, 3, 3)
                    X = (1 - uu)[:, None] * Vt[:, 1] + uu[:, None] * Vt[:, 2]   # on edge v2-v3
                    Dp = P1[:, 0] - P0[:, 0]
                    P0[:, 0] = X - t[:, None] * Dp
                    P1[:, 0] = X + (1 - t)[:, None] * Dp
                else:
                    Bt = _interp(P0[:, 2:].reshape(m, 6), P1[:, 2:].reshape(m, 6), t).reshape(m, 2, 3)
                    X = (1 - uu)[:, None] * Bt[:, 0] + uu[:, None] * Bt[:, 1]
                    Dp = P1[:, 0] - P0[:, 0]
                    shift0 = X - t[:, None] * Dp - P0[:, 0]
                    P0[:, 0:2] += shift0[:, None]
                    P1[:, 0:2] += shift0[:, None]
            V = _pack(P0, P1)
        out[idx] = V + np.tile(anchor, 8)
    return out, fam.astype(np.int8)


def simulation_mixed(n: int = 1_000_000, seed: int = 1, frac_collide: float = 0.01,
                     frac_degenerate: float = 0.05) -> Workload:
    """Simulation-shaped mixed workload (VF:EE 1:1): nearby primitive pairs on
    a jittered unit-scale mesh surface, step displacements N(0, 1e-3), ~1 %
    constructed collisions at known t*, ~5 % degenerate configurations."""
    rng = np.random.default_rng(seed)
    h = 1.0 / 64
    disp = 1e-3
    g = 2.0**-30
    batches = []
    for kind, nk in ((VF, n - n // 2), (EE, n // 2)):
        nc = int(round(nk * frac_collide))
        ndg = int(round(nk * frac_degenerate))
        npl = nk - nc - ndg
        A = _sim_plain(rng, npl, kind, h, disp, g)
        C, tc = _sim_constructed(rng, nc, kind, h, disp, g)
        Dg, fam = _sim_degenerate(rng, ndg, kind, h, g)
        verts = np.concatenate([A, C, Dg])
        truth = np.concatenate([np.full(npl, -1, np.int8), np.ones(nc, np.int8),
                                np.full(ndg, -1, np.int8)])
        t_star = np.concatenate([np.full(npl, np.nan), tc, np.full(ndg, np.nan)])
        family = np.concatenate([np.full(npl, FAM_PLAIN, np.int8),
                                 np.full(nc, FAM_CONSTRUCTED, np.int8), fam])
        perm = rng.permutation(nk)
        batches.append(Batch(kind, verts[perm], truth[perm], t_star[perm], family[perm]))
    return Workload("simulation-mixed", batches,
                    {"seed": seed, "n": n, "ms": 0.0, "delta": 1e-6, "max_itr": 10**6,
                     "mesh_spacing": h, "step_disp_sigma": disp})


# ---------------------------------------------------------------------------
# Degenerate-heavy workload on a 2^-20 grid
# ---------------------------------------------------------------------------

def _cross2(a, b):
    return a[..., 0] * b[..., 1] - a[..., 1] * b[..., 0]


def _place(L, ax):
    """Local (a, b, normal) coordinates -> global axes, the normal along ``ax``
    (a permutation of coordinates: exact)."""
    G = np.empty_like(L)
    idx = np.arange(L.shape[0])
    for k, off in enumerate((1, 2, 0)):
        G[idx, ..., (ax + off) % 3] = L[..., k]
    return G


def _grazing(rng, m, kind):
    """Tangent contact: the primitives touch at one time t* only, with zero
    normal speed there.  In local coordinates (a, b, normal) the second
    primitive (VF triangle / EE edge p3 p4) lies at t* in the plane n = c and
    its points rise at rates w = L(x) for an affine L(x) = l0 + g . x over the
    plane, while the whole scene drifts by m in (a, b).  The first primitive's
    points are placed in that plane at t* (VF: the point at barycentric
    (u*, v*) of the triangle; EE: an edge crossing p3 p4 at (u*, v*)), drift
    by m + s, and rise at L of their own position at t*.  The plane's height
    under such a point is then c + (t - t*) L(x) + (t - t*)^2 g . s, so its
    normal offset is -(t - t*)^2 g . s: zero only at t*, with zero speed.
    Grids: positions 2^-8, (u*, v*) 2^-4, l0 and g 2^-2, t* 2^-6, drifts
    2^-14, so every coordinate lies on the 2^-20 grid and the contact is
    exact in binary64.  Returns (queries, t*)."""
    t = rng.integers(1, 64, m) / 64.0
    c = q(rng.uniform(-1, 1, m), 2.0**-8)
    l0 = q(rng.uniform(-1, 1, m), 2.0**-2)
    g = q(rng.uniform(-1, 1, (m, 2)), 2.0**-2)
    drift = q(rng.normal(0, 0.3, (m, 2)), 2.0**-14)
    s = q(rng.normal(0, 0.3, (m, 2)), 2.0**-14)
    # keep g . s away from 0: the contact must be a single tangent touch
    bad = np.abs(np.sum(g * s, -1)) < 0.02
    while bad.any():
        g[bad] = q(rng.uniform(-1, 1, (bad.sum(), 2)), 2.0**-2)
        s[bad] = q(rng.normal(0, 0.3, (bad.sum(), 2)), 2.0**-14)
        bad = np.abs(np.sum(g * s, -1)) < 0.02
    Lf = lambda x: l0[:, None] + np.sum(g[:, None, :] * x, -1)   # x: (m, k, 2)
    if kind == VF:
        tri = q(rng.uniform(-1, 1, (m, 3, 2)), 2.0**-8)
        area = np.abs(_cross2(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0]))
        while (area < 0.1).any():
            k = area < 0.1
            tri[k] = q(rng.uniform(-1, 1, (k.sum(), 3, 2)), 2.0**-8)
            area = np.abs(_cross2(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0]))
        # (u*, v*) on the 2^-4 grid, u*, v* >= 1/16, u* + v* <= 15/16
        u = rng.integers(1, 15, m)
        v = rng.integers(1, 15, m)
        over = u + v > 15
        u[over], v[over] = 15 - u[over], 15 - v[over]
        u, v = u / 16.0, v / 16.0
        pt = (1 - u - v)[:, None] * tri[:, 0] + u[:, None] * tri[:, 1] + v[:, None] * tri[:, 2]
        X = np.concatenate([pt[:, None], tri], 1)              # (m, 4, 2) at t*
        vel = np.concatenate([(drift + s)[:, None], np.repeat(drift[:, None], 3, 1)], 1)
    else:
        B = q(rng.uniform(-1, 1, (m, 2, 2)), 2.0**-8)
        E = q(rng.uniform(-1, 1, (m, 2)), 2.0**-8)
        cr = np.abs(_cross2(E, B[:, 1] - B[:, 0]))
        while (cr < 0.1).any():
            k = cr < 0.1
            B[k] = q(rng.uniform(-1, 1, (k.sum(), 2, 2)), 2.0**-8)
            E[k] = q(rng.uniform(-1, 1, (k.sum(), 2)), 2.0**-8)
            cr = np.abs(_cross2(E, B[:, 1] - B[:, 0]))
        u = rng.integers(1, 16, m) / 16.0
        v = rng.integers(1, 16, m) / 16.0
        Xc = (1 - v)[:, None] * B[:, 0] + v[:, None] * B[:, 1]
        A = np.stack([Xc - u[:, None] * E, Xc + (1 - u)[:, None] * E], 1)
        X = np.concatenate([A, B], 1)
        vel = np.concatenate([np.repeat((drift + s)[:, None], 2, 1),
                              np.repeat(drift[:, None], 2, 1)], 1)
    w = Lf(X)                                                  # (m, 4) rise rates
    L0 = np.concatenate([X - t[:, None, None] * vel,
                         (c[:, None] - t[:, None] * w)[..., None]], -1)
    L1 = np.concatenate([X + (1 - t)[:, None, None] * vel,
                         (c[:, None] + (1 - t)[:, None] * w)[..., None]], -1)
    ax = rng.integers(0, 3, m)
    return _pack(_place(L0, ax), _place(L1, ax)), t


def _degenerate_family(rng, m, kind, fam):
    """One degenerate family on the 2^-20 grid.  Returns (queries, t*): t* is
    an exact contact time for the constructed families (vertex-on-vertex and
    grazing), NaN otherwise."""
    gg = 2.0**-20
    tstar = np.full(m, np.nan)
    P0 = q(rng.uniform(-1, 1, (m, 4, 3)), gg)
    P1 = q(P0 + rng.normal(0, 0.3, (m, 4, 3)), gg)
    idx = np.arange(m)
    if fam == FAM_COPLANAR:
        ax = rng.integers(0, 3, m)
        c = q(rng.uniform(-1, 1, m), gg)
        P0[idx, :, ax] = c[:, None]
        P1[idx, :, ax] = c[:, None]
    elif fam == FAM_COLLINEAR:
        # all points on one moving line: x(s) = a + s d, s on 2^-8, d on 2^-12
        a0 = q(rng.uniform(-1, 1, (m, 3)), gg)
        d0 = q(rng.uniform(-1, 1, (m, 3)), 2.0**-12)
        a1 = q(a0 + rng.normal(0, 0.3, (m, 3)), gg)
        s = q(rng.uniform(-1, 1, (m, 4)), 2.0**-8)
        P0 = a0[:, None] + s[..., None] * d0[:, None]
        s1 = q(s + rng.normal(0, 0.3, (m, 4)), 2.0**-8)
        P1 = a1[:, None] + s1[..., None] * d0[:, None]
    elif fam == FAM_PARALLEL:
        d = q(rng.uniform(-1, 1, (m, 3)), 2.0**-16)
        off = q(rng.normal(0, 0.05, (m, 3)), gg)
        sc = q(rng.uniform(0.25, 1.5, m), 2.0**-4)[:, None]
        a0 = P0[:, 0]
        P0 = np.stack([a0, a0 + d, a0 + off, a0 + off + sc * d], 1)
        mv = q(rng.normal(0, 0.05, (m, 3)), gg)
        P1 = P0.copy()
        P1[:, 0:2] += mv[:, None]
        if kind == VF:   # VF analogue: point moving parallel to edge v1-v2
            P0[:, 3] = q(P0[:, 1] + rng.uniform(-1, 1, (m, 3)), gg)
            P1[:, 3] = P0[:, 3]
    elif fam == FAM_VERTEX:
        # a vertex of the first primitive meets a vertex of the second (VF: p
        # meets v1; EE: p1 meets p3) at t* on a 2^-4 grid; positions on 2^-16
        P0 = q(P0, 2.0**-16)
        P1 = q(P1, 2.0**-16)
        t = rng.integers(1, 16, m) / 16.0
        j = 1 if kind == VF else 2
        Vt = _interp(P0[:, j], P1[:, j], t)
        Dp = P1[:, 0] - P0[:, 0]
        P0[:, 0] = Vt - t[:, None] * Dp
        P1[:, 0] = Vt + (1 - t)[:, None] * Dp
        tstar = t
    elif fam == FAM_GRAZING:
        return _grazing(rng, m, kind)
    return _pack(P0, P1), tstar


def degenerate_heavy(n: int = 100_000, seed: int = 2) -> Workload:
    """Degenerate-heavy workload on a 2^-20 grid (VF:EE 1:1): coplanar,
    collinear, parallel-edge, vertex-on-vertex and grazing-tangent motions in
    equal parts.  Vertex-on-vertex and grazing queries are constructed
    contacts (truth 1, exact t*); the others are unlabelled."""
    rng = np.random.default_rng(seed)
    fams = [FAM_COPLANAR, FAM_COLLINEAR, FAM_PARALLEL, FAM_VERTEX, FAM_GRAZING]
    batches = []
    for kind, nk in ((VF, n - n // 2), (EE, n // 2)):
        fam = np.array([fams[i % len(fams)] for i in range(nk)], np.int8)
        verts = np.empty((nk, 24))
        tstar = np.full(nk, np.nan)
        for f in fams:
            idx = np.nonzero(fam == f)[0]
            verts[idx], tstar[idx] = _degenerate_family(rng, idx.size, kind, f)
        truth = np.where(np.isnan(tstar), -1, 1).astype(np.int8)
        perm = rng.permutation(nk)
        batches.append(Batch(kind, verts[perm], truth[perm], tstar[perm], fam[perm]))
    return Workload("degenerate-heavy", batches,
                    {"seed": seed, "n": n, "ms": (0.0, 1e-4), "delta": 1e-6,
                     "max_itr": 10**6})


# ---------------------------------------------------------------------------
# Batched multi-instance workload and served request stream
# ---------------------------------------------------------------------------

def instance_sizes(rng, count=64, lo=1_000, hi=2_000_000, total=20_000_000):
    s = np.exp(rng.uniform(np.log(lo), np.log(hi), count))
    s = s * (total / s.sum())
    return np.maximum(np.round(s).astype(np.int64), 2)


def multi_instance(count: int = 64, total: int = 20_000_000, seed: int = 3,
                   size_scale: float = 1.0) -> Workload:
    """``count`` simulation instances with log-uniform query counts (sum ~
    ``total``), VF:EE 1:1, unit-cube geometry scaled by 10^U(-2, 2) per
    instance.  Each Batch is one instance-kind segment."""
    rng = np.random.default_rng(seed)
    sizes = instance_sizes(rng, count, total=int(total * size_scale))
    batches = []
    for i, s in enumerate(sizes):
        scale = float(2.0 ** np.round(np.log2(10.0 ** rng.uniform(-2, 2))))
        for kind, nk in ((VF, int(s) - int(s) // 2), (EE, int(s) // 2)):
            b = unit_cube(kind, nk, seed * 100_003 + 2 * i + kind, scale=scale)
            b.family = np.full(nk, i, np.int32)
            batches.append(b)
    return Workload("multi-instance", batches,
                    {"seed": seed, "count": count, "delta": 1e-6, "max_itr": 10**6})


def request_stream(clients: int = 16, duration_s: float = 2.0, rate_hz: float = 8.0,
                   seed: int = 4, lo: int = 100, hi: int = 500_000):
    """Poisson request arrivals per client; sizes log-uniform in [lo, hi];
    per-request delta in {1e-4, 1e-6}, ms in {0, 1e-4}.  Returns a list of
    dicts sorted by arrival time (geometry is generated lazily by
    ``request_batch``)."""
    rng = np.random.default_rng(seed)
    reqs = []
    for c in range(clients):
        t = 0.0
        while True:
            t += rng.exponential(1.0 / rate_hz)
            if t > duration_s:
                break
            size = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
            reqs.append({"client": c, "arrival": t, "size": size,
                         "kind": int(rng.integers(0, 2)),
                         "delta": float(rng.choice([1e-4, 1e-6])),
                         "ms": float(rng.choice([0.0, 1e-4])),
                         "seed": int(rng.integers(0, 2**31))})
    reqs.sort(key=lambda r: r["arrival"])
    for i, r in enumerate(reqs):
        r["id"] = i
    return reqs


def request_batch(req) -> Batch:
    return unit_cube(req["kind"], req["size"], req["seed"])


def line_search_scene(n: int = 1_000_000, seed: int = 5, h: float = 1.0 / 64,
                      approach=(0.0, 2.0), g: float = 2.0**-30) -> Workload:
    """Candidate set of one line-search step (Sec. 6, Algorithm 4), VF:EE 1:1.

    Each pair is a flat local configuration of mesh size h, tilted by up to
    30 degrees and placed in the unit cube: VF a triangle and a point above
    its interior, EE an edge and a crossing edge above it, separated by a gap
    along the normal that is log-uniform in [10^-2, 1] h.  The update dx
    moves the upper primitive toward the lower one by s times the gap,
    s ~ U(approach) (s > 1 closes the gap within the full step), plus
    N(0, (1e-3 h)^2) on every coordinate.  Coordinates are on a 2^-30 grid."""
    rng = np.random.default_rng(seed)
    batches = []
    for kind, m in ((VF, n // 2), (EE, n - n // 2)):
        # rotation: spin about z, then tilt about x by up to 30 degrees
        tx = rng.uniform(-np.pi / 6, np.pi / 6, m)
        sp = rng.uniform(0, 2 * np.pi, m)
        cx, sx, cz, sz = np.cos(tx), np.sin(tx), np.cos(sp), np.sin(sp)
        R = np.zeros((m, 3, 3))
        R[:, 0, 0], R[:, 0, 1] = cz, -sz
        R[:, 1, 0], R[:, 1, 1], R[:, 1, 2] = cx * sz, cx * cz, -sx
        R[:, 2, 0], R[:, 2, 1], R[:, 2, 2] = sx * sz, sx * cz, cx
        c = rng.uniform(0.1, 0.9, (m, 3))
        gap = h * 10.0 ** rng.uniform(-2.0, 0.0, m)
        if kind == VF:
            local = np.zeros((m, 4, 3))
            local[:, 2, :2] = [h, 0.0]
            local[:, 3, :2] = [0.0, h]
            local[:, 1:, :2] += rng.uniform(-0.2, 0.2, (m, 3, 2)) * h
            u = rng.uniform(0.1, 0.45, m)
            v = rng.uniform(0.1, 0.45, m)
            local[:, 0] = ((1 - u - v)[:, None] * local[:, 1] + u[:, None] * local[:, 2]
                           + v[:, None] * local[:, 3])
            local[:, 0, 2] = gap
            mover = [0]
        else:
            local = np.zeros((m, 4, 3))
            local[:, 0, 0], local[:, 1, 0] = -0.5 * h, 0.5 * h
            ang = rng.uniform(np.pi / 6, 5 * np.pi / 6, m)
            local[:, 2, 0], local[:, 2, 1] = -0.5 * h * np.cos(ang), -0.5 * h * np.sin(ang)
            local[:, 3, 0], local[:, 3, 1] = 0.5 * h * np.cos(ang), 0.5 * h * np.sin(ang)
            local[:, 2:, :2] += rng.uniform(-0.1, 0.1, (m, 2, 2)) * h
            local[:, 2:, 2] = gap[:, None]
            mover = [2, 3]
        L1 = local.copy()
        L1[:, mover, 2] -= (rng.uniform(approach[0], approach[1], m) * gap)[:, None]
        P0 = q(np.einsum("nij,nkj->nki", R, local) + c[:, None], g)
        P1 = q(np.einsum("nij,nkj->nki", R, L1) + c[:, None] + rng.normal(0, 1e-3 * h, L1.shape),
               g)
        batches.append(Batch(kind, _pack(P0, P1), np.full(m, -1, np.int8),
                             np.full(m, np.nan)))
    return Workload("line-search", batches, {"seed": seed, "h": h, "approach": approach})


@dataclass
class Mesh:
    x0: np.ndarray       # (nv, 3) float64 positions at t0
    x1: np.ndarray       # (nv, 3) float64 positions at t1
    faces: np.ndarray    # (nf, 3) int32 vertex ids
    edges: np.ndarray    # (ne, 2) int32 vertex ids, each edge once, a < b


def _grid_sheet(nx, spacing, origin):
    """nx x nx vertices on a square grid, two triangles per cell."""
    i, j = np.meshgrid(np.arange(nx), np.arange(nx), indexing="ij")
    xy = np.stack([i.ravel(), j.ravel()], -1) * spacing + origin
    idx = (i * nx + j)
    a, b = idx[:-1, :-1].ravel(), idx[1:, :-1].ravel()
    c, d = idx[:-1, 1:].ravel(), idx[1:, 1:].ravel()
    faces = np.concatenate([np.stack([a, b, d], -1), np.stack([a, d, c], -1)])
    return xy, faces


def _mesh_edges(faces):
    e = np.concatenate([faces[:, [0, 1]], faces[:, [1, 2]], faces[:, [0, 2]]])
    e = np.sort(e, axis=1)
    return np.unique(e, axis=0)


def cloth_scene(nx: int = 256, seed: int = 6, gap: float = 0.25, fall: float = 0.5,
                g: float = 2.0**-30) -> Mesh:
    """Two cloth-like sheets of nx x nx vertices (spacing 1 / (nx - 1)) for
    Algorithm 3's active set: sheet A lies near z = 0 with a small wave,
    sheet B starts gap spacings above it, shifted by half a cell, and moves
    down by fall + gap spacings with per-vertex jitter, so part of it passes
    through A within the step.  Both sheets also carry their own
    self-candidates (nearby primitives of one sheet)."""
    rng = np.random.default_rng(seed)
    h = 1.0 / (nx - 1)
    xy_a, f_a = _grid_sheet(nx, h, np.array([0.0, 0.0]))
    xy_b, f_b = _grid_sheet(nx, h, np.array([0.5 * h, 0.5 * h]))
    wave = lambda xy: 0.5 * h * np.sin(2 * np.pi * xy[:, 0]) * np.sin(2 * np.pi * xy[:, 1])
    za = wave(xy_a) + rng.normal(0, 0.02 * h, len(xy_a))
    zb = wave(xy_b) + gap * h + rng.normal(0, 0.02 * h, len(xy_b))
    A0 = np.concatenate([xy_a, za[:, None]], 1)
    B0 = np.concatenate([xy_b, zb[:, None]], 1)
    drop = (gap + fall) * h * (0.5 + 0.5 * np.sin(np.pi * xy_b[:, 0]))   # falls more mid-sheet
    A1 = A0 + rng.normal(0, 0.02 * h, A0.shape)
    B1 = B0 + rng.normal(0, 0.02 * h, B0.shape)
    B1[:, 2] -= drop
    x0 = q(np.concatenate([A0, B0]), g)
    x1 = q(np.concatenate([A1, B1]), g)
    faces = np.concatenate([f_a, f_b + len(xy_a)]).astype(np.int32)
    return Mesh(x0, x1, faces, _mesh_edges(faces).astype(np.int32))
