"""CPU oracle for the inclusion-based CCD root finder (Sec. 4, Algorithm 2).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package.  The GPU
library (``paper_2009_13349_gb300``) never imports it and shares no code,
header, helper or constant generator with it.

``ccd_oracle.c`` is a plain C implementation, compiled with
``-ffp-contract=off`` and without fast-math, so every arithmetic operation is
one IEEE double operation in the written order.  ``exact.py`` holds an
independent exact-rational (``fractions.Fraction``) run of the same
algorithm, used to certify ground truth on tiny inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ccd_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD_DIR, "libccd_oracle.so")
_LOCK = threading.Lock()
_LIB = None

VF, EE = 0, 1
LITERAL_DROP = 1  # flag: drop non-first terminating boxes (literal Algorithm 2)

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
          "-shared", "-fPIC"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build (idempotent).  The
    mutation tests set CCD_ORACLE_LIB to a library built from a deliberately
    altered copy of ccd_oracle.c; that library is then used instead."""
    override = os.environ.get("CCD_ORACLE_LIB")
    if override:
        return override
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lp = ctypes.POINTER(ctypes.c_longlong)
            up = ctypes.POINTER(ctypes.c_ubyte)
            lib.oracle_corner.argtypes = [ctypes.c_int, dp, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, dp]
            lib.oracle_corner.restype = None
            lib.oracle_box.argtypes = [ctypes.c_int, dp, dp, dp, dp]
            lib.oracle_box.restype = None
            lib.oracle_kappa.argtypes = [ctypes.c_int, dp, dp]
            lib.oracle_kappa.restype = None
            lib.oracle_filter_constant.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.oracle_filter_constant.restype = ctypes.c_double
            lib.oracle_err_from_bounds.argtypes = [ctypes.c_int, dp, ctypes.c_longlong,
                                                   ctypes.c_int, ctypes.c_int, dp]
            lib.oracle_err_from_bounds.restype = None
            lib.oracle_ccd.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_longlong, ctypes.c_int,
                                       dp, dp, lp]
            lib.oracle_ccd.restype = ctypes.c_int
            lib.oracle_ccd_batch.argtypes = [ctypes.c_int, dp, ctypes.c_longlong, dp,
                                             ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_longlong, ctypes.c_int, up, dp, dp,
                                             lp, ctypes.c_int]
            lib.oracle_ccd_batch.restype = ctypes.c_longlong
            lib.oracle_ccd_t.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_longlong, ctypes.c_double,
                                         ctypes.c_int, dp, dp, lp]
            lib.oracle_ccd_t.restype = ctypes.c_int
            lib.oracle_ccd_batch_t.argtypes = [ctypes.c_int, dp, ctypes.c_longlong, dp,
                                               ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_longlong, ctypes.c_double, ctypes.c_int,
                                               up, dp, dp, lp, ctypes.c_int]
            lib.oracle_ccd_batch_t.restype = ctypes.c_longlong
            lib.oracle_kappa_t.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp]
            lib.oracle_kappa_t.restype = None
            lib.oracle_linf_distance.argtypes = [ctypes.c_int, dp]
            lib.oracle_linf_distance.restype = ctypes.c_double
            lib.oracle_linf_distance_batch.argtypes = [ctypes.c_int, dp, ctypes.c_longlong, dp,
                                                       ctypes.c_int]
            lib.oracle_linf_distance_batch.restype = None
            _LIB = lib
        return _LIB


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _as_queries(verts) -> np.ndarray:
    v = np.ascontiguousarray(np.asarray(verts, dtype=np.float64))
    if v.ndim == 1:
        v = v.reshape(1, 24)
    v = v.reshape(v.shape[0], 24)
    return v


def corner(kind: int, query, t: float, u: float, v: float) -> np.ndarray:
    """F(t, u, v) of one query with the fixed operation order (Eq. F-vf / F-ee)."""
    q = _as_queries(query)[0]
    out = np.zeros(3)
    _lib().oracle_corner(kind, _dptr(q), t, u, v, _dptr(out))
    return out


def box(kind: int, query, interval) -> tuple[np.ndarray, np.ndarray]:
    """(m, M) of B_F(I) for I = (tL, tR, uL, uR, vL, vR) (Eq. box)."""
    q = _as_queries(query)[0]
    I = np.ascontiguousarray(np.asarray(interval, dtype=np.float64))
    m, M = np.zeros(3), np.zeros(3)
    _lib().oracle_box(kind, _dptr(q), _dptr(I), _dptr(m), _dptr(M))
    return m, M


def kappa(kind: int, query, t_max: float = 1.0) -> np.ndarray:
    """(kappa_t, kappa_u, kappa_v) of Eq. (kappas) over [0, t_max] x [0,1]^2."""
    q = _as_queries(query)[0]
    out = np.zeros(3)
    _lib().oracle_kappa_t(kind, _dptr(q), float(t_max), _dptr(out))
    return out


def filter_constant(kind: int, ms_nonzero: bool) -> float:
    return _lib().oracle_filter_constant(kind, int(bool(ms_nonzero)))


def err_from_bounds(kind: int, verts, ms_nonzero: bool = False,
                    per_query: bool = False) -> np.ndarray:
    """eps per axis (Eq. ccd-error / msccd-error), over the scene or per query."""
    v = _as_queries(verts)
    n = v.shape[0]
    out = np.zeros((n, 3) if per_query else 3)
    _lib().oracle_err_from_bounds(kind, _dptr(v), n, int(bool(ms_nonzero)),
                                  int(bool(per_query)), _dptr(out))
    return out


def ccd(kind: int, query, err, ms: float = 0.0, delta: float = 1e-6,
        max_itr: int = 10**6, flags: int = 0, t_max: float = 1.0):
    """One query -> (collides, toi, out_tol, checks); time interval [0, t_max]."""
    q = _as_queries(query)[0]
    e = np.ascontiguousarray(np.asarray(err, dtype=np.float64).reshape(3))
    toi, tol = ctypes.c_double(), ctypes.c_double()
    n = ctypes.c_longlong()
    r = _lib().oracle_ccd_t(kind, _dptr(q), _dptr(e), float(ms), float(delta),
                            int(max_itr), float(t_max), int(flags), ctypes.byref(toi),
                            ctypes.byref(tol), ctypes.byref(n))
    if r < 0:
        raise MemoryError("oracle queue allocation failed")
    return bool(r), toi.value, tol.value, n.value


def ccd_batch(kind: int, verts, err, ms: float = 0.0, delta: float = 1e-6,
              max_itr: int = 10**6, flags: int = 0, nthreads: int = 1, t_max: float = 1.0):
    """n queries (n x 24) -> (collides u8, toi f64, out_tol f64, checks i64)."""
    v = _as_queries(verts)
    n = v.shape[0]
    e = np.ascontiguousarray(np.asarray(err, dtype=np.float64))
    if e.size == 3:
        stride = 0
        e = e.reshape(3)
    else:
        stride = 3
        e = e.reshape(n, 3)
    col = np.zeros(n, dtype=np.uint8)
    toi = np.zeros(n)
    tol = np.zeros(n)
    chk = np.zeros(n, dtype=np.int64)
    fails = _lib().oracle_ccd_batch_t(
        kind, _dptr(v), n, _dptr(e), stride, float(ms), float(delta), int(max_itr),
        float(t_max), int(flags), col.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), _dptr(toi),
        _dptr(tol), chk.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), int(nthreads))
    if fails:
        raise MemoryError(f"oracle queue allocation failed for {fails} queries")
    return col, toi, tol, chk


def linf_distance(kind: int, query) -> float:
    """L-infinity distance between the primitives at t = 0 (Sec. 5.1 norm)."""
    q = _as_queries(query)[0]
    return _lib().oracle_linf_distance(kind, _dptr(q))


def linf_distance_batch(kind: int, verts, nthreads: int = 1) -> np.ndarray:
    """linf_distance of n queries (n x 24)."""
    v = _as_queries(verts)
    out = np.zeros(v.shape[0])
    _lib().oracle_linf_distance_batch(kind, _dptr(v), v.shape[0], _dptr(out), int(nthreads))
    return out
