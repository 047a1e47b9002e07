"""Algorithm 4 (Sec. 6, "Line Search"), its CCD part, on the CPU oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Given the candidate set C of one line search (vertex-face queries ``vf`` and
edge-edge queries ``ee``, each n x 24 with x1 = x0 + dx already applied),
the step computes, in the paper's order:

1. d_i: the distance of the candidates at x0, in the L-infinity norm that
   MSCCD measures separation in (Sec. 5.1): the minimum over C of
   ``linf_distance``.  rho_i, its error bound, is a caller argument (the
   paper fixes 1e-9).
2. eps_i: the scene's MSCCD error (Eq. msccd-error) per kind and axis from
   the bounds of the kind's points; the scalar in the inequality below is
   its maximum over kinds and axes.
3. d <- cap(p d_i, delta) with cap = min (the text caps d at delta; the
   printed max is available as ``cap="max"``).
4. find p: while the inequality d_i - d > delta + eps_i + rho_i fails, and
   some smaller p could satisfy it, p <- p / 2 and d <- cap(p d_i, delta)
   (the printed loop condition is reversed; the text halves p "until it is
   small enough").
5. one MSCCD pass over C on the time interval [0, alpha] (SolveMSCCD with
   ms = d): alpha <- min(alpha, min toi), delta_i <- max(delta, max
   out_tol).  The printed loop updates alpha candidate by candidate, which
   makes the result depend on the (unspecified) order of C; every candidate
   of a pass uses the alpha of the pass's start instead.
6. validate after: if d_i - d > delta_i + eps_i + rho_i the step is done;
   otherwise delta <- delta_i and the step goes back to 4 (at most
   ``max_passes`` passes).

The backtracking loop on the energy E that follows in Algorithm 4 belongs to
the application and is not part of this step.  Every comparison is written
as (d_i - d) > ((delta + eps_i) + rho).
"""
from __future__ import annotations

import math

import numpy as np

from . import VF, EE, ccd_batch, err_from_bounds, linf_distance_batch


def _cap(x: float, delta: float, cap: str) -> float:
    return min(x, delta) if cap == "min" else max(x, delta)


def line_search_ccd(vf, ee, p: float, delta: float, max_itr: int = 10**6, rho: float = 1e-9,
                    max_passes: int = 16, cap: str = "min", nthreads: int = 1) -> dict:
    """Returns alpha (the step bound), the validated p, d, d_i, eps_i,
    delta_i, the number of MSCCD passes and whether the inequality holds."""
    if not (0.0 < p < 1.0) or not delta > 0.0 or rho < 0.0 or max_passes < 1:
        raise ValueError("need 0 < p < 1, delta > 0, rho >= 0, max_passes >= 1")
    if cap not in ("min", "max"):
        raise ValueError("cap is 'min' or 'max'")
    sets = [(VF, np.asarray(vf, dtype=np.float64).reshape(-1, 24)),
            (EE, np.asarray(ee, dtype=np.float64).reshape(-1, 24))]
    sets = [(k, q) for k, q in sets if q.shape[0] > 0]

    # 1. distance of the candidates at x0;  2. eps_i of the scene
    d_i = math.inf
    eps_i = 0.0
    eps = {}
    for k, q in sets:
        d_i = min(d_i, float(linf_distance_batch(k, q, nthreads).min()))
        eps[k] = err_from_bounds(k, q, ms_nonzero=True)
        eps_i = max(eps_i, float(eps[k].max()))

    alpha = 1.0
    delta_cur = float(delta)
    delta_i = delta_cur
    d = _cap(p * d_i, delta_cur, cap)
    limit = 0.0 if cap == "min" else None   # d as p -> 0
    passes = 0
    validated = (d_i - d) > ((delta_cur + eps_i) + rho)
    while sets:
        # 4. find p
        while not ((d_i - d) > ((delta_cur + eps_i) + rho)):
            lim = limit if limit is not None else delta_cur
            if not ((d_i - lim) > ((delta_cur + eps_i) + rho)) or p == 0.0:
                break   # no smaller p satisfies the inequality
            p = p / 2.0
            d = _cap(p * d_i, delta_cur, cap)
        if alpha == 0.0:
            break       # no time interval left
        # 5. one MSCCD pass over the candidate set on [0, alpha]
        delta_i = delta_cur
        alpha_pass = alpha
        for k, q in sets:
            _, toi, tol, _ = ccd_batch(k, q, eps[k], ms=d, delta=delta_cur, max_itr=max_itr,
                                       nthreads=nthreads, t_max=alpha_pass)
            alpha = min(alpha, float(toi.min()))
            delta_i = max(delta_i, float(tol.max()))
        passes += 1
        # 6. validate after
        validated = (d_i - d) > ((delta_i + eps_i) + rho)
        if validated or passes >= max_passes:
            break
        delta_cur = delta_i
    return {"alpha": alpha, "p": p, "d": d, "d_i": d_i, "eps_i": eps_i, "delta_i": delta_i,
            "passes": passes, "validated": bool(validated)}
