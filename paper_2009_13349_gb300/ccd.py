"""Thin Python binding of the C ABI in ``include/ccd.h`` (argument marshalling only).

Every step of the path runs in the CUDA library ``_lib/libccd_gb300.so``;
this module converts torch tensors to device pointers, allocates the caller-
side workspace with torch, and raises if the library or a GPU is missing.
There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

VF, EE = 0, 1
STATUS = {0: "CCD_OK", -1: "CCD_ERR_ARG", -2: "CCD_ERR_WORKSPACE", -3: "CCD_ERR_TIMEOUT",
          -4: "CCD_ERR_CUDA", -5: "CCD_ERR_CAPACITY", -6: "CCD_ERR_BUSY", -7: "CCD_ERR_CANCELLED"}

_LIB = None


class CCDError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


def lib():
    """Load the CUDA library (fails loudly when it has not been built)."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing: run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        vp, dp = ctypes.c_void_p, ctypes.c_void_p
        i64, sz = ctypes.c_int64, ctypes.c_size_t
        L.ccd_workspace_bytes.argtypes = [i64, i64]
        L.ccd_workspace_bytes.restype = sz
        L.ccd_workspace_bytes_pages.argtypes = [i64, i64, i64]
        L.ccd_workspace_bytes_pages.restype = sz
        L.ccd_workspace_layout.argtypes = [i64, i64, sz, ctypes.POINTER(WorkspaceInfo)]
        L.ccd_workspace_layout.restype = ctypes.c_int
        for name in ("ccd_vf_batch", "ccd_ee_batch"):
            f = getattr(L, name)
            f.argtypes = [dp, i64, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, i64,
                          vp, dp, dp, vp, vp, sz, vp]
            f.restype = ctypes.c_int
        L.ccd_err_from_bounds.argtypes = [ctypes.c_int, dp, i64, ctypes.c_int, ctypes.c_int, dp, vp]
        L.ccd_err_from_bounds.restype = ctypes.c_int
        L.ccd_workspace_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_int32), vp]
        L.ccd_workspace_status.restype = ctypes.c_int
        L.ccd_workspace_counters.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                                             vp]
        L.ccd_workspace_counters.restype = ctypes.c_int
        L.ccd_set_stage_events.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]
        L.ccd_set_stage_events.restype = ctypes.c_int
        tp = ctypes.POINTER(Tuning)
        L.ccd_multi_workspace_bytes.argtypes = [i64, i64, tp]
        L.ccd_multi_workspace_bytes.restype = sz
        L.ccd_multi_batch.argtypes = [dp, i64, vp, ctypes.c_int32, i64, vp, dp, dp, vp, tp, vp,
                                      sz, vp]
        L.ccd_multi_batch.restype = ctypes.c_int
        L.ccd_segments_err_from_bounds.argtypes = [dp, i64, vp, ctypes.c_int32, vp]
        L.ccd_segments_err_from_bounds.restype = ctypes.c_int
        L.ccd_group_reduce.argtypes = [dp, dp, i64, vp, ctypes.c_int32, ctypes.c_int32, dp, dp,
                                       vp]
        L.ccd_group_reduce.restype = ctypes.c_int
        L.ccd_linf_distance.argtypes = [dp, i64, vp, ctypes.c_int32, ctypes.c_int32, dp, dp, vp]
        L.ccd_linf_distance.restype = ctypes.c_int
        L.ccd_line_search_workspace_bytes.argtypes = [i64, i64]
        L.ccd_line_search_workspace_bytes.restype = sz
        L.ccd_line_search.argtypes = [dp, i64, i64, ctypes.POINTER(LineSearchIO), vp, sz, vp]
        L.ccd_line_search.restype = ctypes.c_int
        L.ccd_scene_eps.argtypes = [dp, dp, i64, dp, vp, sz, vp]
        L.ccd_scene_eps.restype = ctypes.c_int
        L.ccd_broad_phase_workspace_bytes.argtypes = [i64, i64, i64, i64, i64]
        L.ccd_broad_phase_workspace_bytes.restype = sz
        L.ccd_broad_phase.argtypes = [dp, dp, i64, vp, i64, vp, i64, ctypes.c_double, vp, i64,
                                      vp, i64, ctypes.POINTER(ctypes.c_int64), vp, sz, vp]
        L.ccd_broad_phase.restype = ctypes.c_int
        L.ccd_active_set_workspace_bytes.argtypes = [i64, i64]
        L.ccd_active_set_workspace_bytes.restype = sz
        L.ccd_active_set.argtypes = [dp, dp, i64, vp, vp, vp, i64, vp, i64, ctypes.c_double,
                                     i64, vp, vp, dp, ctypes.POINTER(ctypes.c_int64), dp, vp, sz,
                                     vp]
        L.ccd_active_set.restype = ctypes.c_int
        L.ccd_aos_to_soa.argtypes = [dp, i64, dp, i64, vp]
        L.ccd_aos_to_soa.restype = ctypes.c_int
        L.ccd_status_str.argtypes = [ctypes.c_int]
        L.ccd_status_str.restype = ctypes.c_char_p
        L.ccd_fp64_peak_probe.argtypes = [ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_float), vp]
        L.ccd_fp64_peak_probe.restype = ctypes.c_int
        L.ccd_batch_begin.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
        L.ccd_batch_begin.restype = ctypes.c_int
        L.ccd_batch_submit.argtypes = [vp, ctypes.POINTER(CRequest), ctypes.POINTER(i64)]
        L.ccd_batch_submit.restype = ctypes.c_int
        L.ccd_batch_poll.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32),
                                     ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                     ctypes.c_int32]
        L.ccd_batch_poll.restype = ctypes.c_int
        L.ccd_batch_cancel.argtypes = [vp, i64]
        L.ccd_batch_cancel.restype = ctypes.c_int
        L.ccd_batch_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
        L.ccd_batch_stats.restype = ctypes.c_int
        L.ccd_batch_end.argtypes = [vp]
        L.ccd_batch_end.restype = ctypes.c_int
        _LIB = L
    return _LIB


def _check(code: int, what: str):
    if code != 0:
        raise CCDError(code, what)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _require_cuda(t: torch.Tensor, name: str, dtype):
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dtype} tensor")


def workspace_bytes(n: int, max_itr: int) -> int:
    return int(lib().ccd_workspace_bytes(int(n), int(max_itr)))


PAGE_BOXES = 32768   # boxes per frontier page of the deep tier (768 KB)


class WorkspaceInfo(ctypes.Structure):
    _fields_ = [("paged", ctypes.c_int32), ("deep_blocks", ctypes.c_int32),
                ("full_slots", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("pages", ctypes.c_int64), ("slot_boxes", ctypes.c_int64),
                ("fixed_bytes", ctypes.c_size_t), ("used_bytes", ctypes.c_size_t)]


def workspace_layout(n: int, max_itr: int, ws_bytes: int) -> dict:
    """ccd_workspace_layout: how a workspace of ws_bytes is used."""
    info = WorkspaceInfo()
    _check(lib().ccd_workspace_layout(int(n), int(max_itr), int(ws_bytes), ctypes.byref(info)),
           "ccd_workspace_layout")
    return {f: getattr(info, f) for f, _ in WorkspaceInfo._fields_ if f != "pad"}


def workspace(n: int, max_itr: int, device=None, pages: int | None = None) -> torch.Tensor:
    """Caller-owned device workspace for ``n`` queries at check limit
    ``max_itr``; ``pages`` sets the deep tier's frontier pages (default: per
    deep block, one level of the largest size a level can reach)."""
    if pages is None:
        nbytes = workspace_bytes(n, max_itr)
    else:
        nbytes = int(lib().ccd_workspace_bytes_pages(int(n), int(max_itr), int(pages)))
    if nbytes == 0:
        raise CCDError(-1, "ccd_workspace_bytes")
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


@dataclass
class Result:
    collides: torch.Tensor   # (n,) uint8
    toi: torch.Tensor        # (n,) float64
    out_tol: torch.Tensor    # (n,) float64
    checks: torch.Tensor     # (n,) int64 or None


def batch(kind: int, verts: torch.Tensor, err: torch.Tensor, ms: float = 0.0,
          delta: float = 1e-6, max_itr: int = 10**6, ws: torch.Tensor | None = None,
          out: Result | None = None, with_checks: bool = True, stream=None) -> Result:
    """ccd_vf_batch / ccd_ee_batch.  ``verts``: (24, n) float64 CUDA tensor
    (structure of arrays); ``err``: (3,) or (n, 3) float64 CUDA tensor."""
    _require_cuda(verts, "verts", torch.float64)
    if verts.dim() != 2 or verts.shape[0] != 24:
        raise ValueError("verts must have shape (24, n)")
    n = verts.shape[1]
    _require_cuda(err, "err", torch.float64)
    stride = 0 if err.numel() == 3 else 3
    if stride == 3 and err.numel() != 3 * n:
        raise ValueError("err must have 3 or 3*n elements")
    dev = verts.device
    if out is None:
        out = Result(torch.empty(n, dtype=torch.uint8, device=dev),
                     torch.empty(n, dtype=torch.float64, device=dev),
                     torch.empty(n, dtype=torch.float64, device=dev),
                     torch.empty(n, dtype=torch.int64, device=dev) if with_checks else None)
    if ws is None:
        ws = workspace(n, max_itr, dev)
    fn = lib().ccd_vf_batch if kind == VF else lib().ccd_ee_batch
    code = fn(_ptr(verts), n, _ptr(err), stride, float(ms), float(delta), int(max_itr),
              _ptr(out.collides), _ptr(out.toi), _ptr(out.out_tol), _ptr(out.checks),
              _ptr(ws), ws.numel(), _stream(stream))
    _check(code, "ccd_vf_batch" if kind == VF else "ccd_ee_batch")
    return out


def vf_batch(verts, err, **kw) -> Result:
    return batch(VF, verts, err, **kw)


def ee_batch(verts, err, **kw) -> Result:
    return batch(EE, verts, err, **kw)


def err_from_bounds(kind: int, verts: torch.Tensor, ms_nonzero: bool = False,
                    per_query: bool = False, stream=None) -> torch.Tensor:
    _require_cuda(verts, "verts", torch.float64)
    n = verts.shape[1]
    out = torch.empty((n, 3) if per_query else (3,), dtype=torch.float64, device=verts.device)
    _check(lib().ccd_err_from_bounds(kind, _ptr(verts), n, int(bool(ms_nonzero)),
                                     int(bool(per_query)), _ptr(out), _stream(stream)),
           "ccd_err_from_bounds")
    return out


def workspace_status(ws: torch.Tensor, stream=None):
    st, fb = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().ccd_workspace_status(_ptr(ws), ctypes.byref(st), ctypes.byref(fb),
                                      _stream(stream)), "ccd_workspace_status")
    return st.value, fb.value


COUNTER_NAMES = ("survivors", "deep_queries", "fallbacks", "checks_small", "checks_deep",
                 "evals_small", "evals_deep", "status", "tq_small", "tq_deep", "a_tasks_deep",
                 "split_chunks_deep", "evals_shared_deep", "mid_queries", "checks_pool",
                 "evals_pool", "tq_deep_ee", "a_tasks_deep_ee", "evals_pool_ee", "tq_small_ee",
                 "evals_small_ee", "deferred_queries", "pages_peak", "tq_pool", "tq_pool_ee",
                 "pool_iters", "pool_serial", "a_tasks_pool", "a_tasks_pool_ee",
                 "evals_pool_shared", "evals_pool_shared_ee", "evals_deep_ee",
                 "evals_shared_deep_ee")


def workspace_counters(ws: torch.Tensor, stream=None) -> dict:
    arr = (ctypes.c_int64 * len(COUNTER_NAMES))()
    _check(lib().ccd_workspace_counters(_ptr(ws), arr, len(COUNTER_NAMES), _stream(stream)),
           "ccd_workspace_counters")
    return dict(zip(COUNTER_NAMES, list(arr)))


def set_stage_events(events) -> None:
    """events: None (off) or 5 torch.cuda.Event(enable_timing=True), each
    already recorded once (so that its CUDA handle exists)."""
    if not events:
        _check(lib().ccd_set_stage_events(None, 0), "ccd_set_stage_events")
        return
    arr = (ctypes.c_void_p * 5)(*[ctypes.c_void_p(e.cuda_event) for e in events])
    _check(lib().ccd_set_stage_events(arr, 5), "ccd_set_stage_events")


def fp64_peak_probe(blocks: int, iters: int, stream=None):
    """Returns (ms, fp64 ops issued) of the FMA throughput probe."""
    ms = ctypes.c_float()
    _check(lib().ccd_fp64_peak_probe(int(blocks), int(iters), ctypes.byref(ms), _stream(stream)),
           "ccd_fp64_peak_probe")
    return ms.value, blocks * 256 * iters * 8


# ---- multi-instance batches -------------------------------------------------------

SEGMENT_DTYPE = np.dtype([("offset", "<i8"), ("count", "<i8"), ("kind", "<i4"),
                          ("group", "<i4"), ("err", "<f8", (3,)), ("ms", "<f8"),
                          ("delta", "<f8"), ("max_itr", "<i8"), ("t_max", "<f8")])
assert SEGMENT_DTYPE.itemsize == 80


class Tuning(ctypes.Structure):
    """ccd_tuning: launch shapes only (results never depend on them)."""
    _fields_ = [("deep_threads", ctypes.c_int32), ("deep_slots", ctypes.c_int32),
                ("small_blocks_per_sm", ctypes.c_int32), ("small_cap", ctypes.c_int32),
                ("pool_cap", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def _tuning_ptr(tuning):
    if tuning is None:
        return None
    if isinstance(tuning, dict):
        tuning = Tuning(**tuning)
    return ctypes.pointer(tuning)


def make_segments(counts, kinds, ms=0.0, delta=1e-6, max_itr=10**6, err=None, t_max=1.0,
                  group=0) -> np.ndarray:
    """Host segment table (structured array) tiling [0, sum(counts))."""
    counts = np.asarray(counts, dtype=np.int64)
    k = len(counts)
    seg = np.zeros(k, dtype=SEGMENT_DTYPE)
    seg["offset"] = np.concatenate([[0], np.cumsum(counts)[:-1]]) if k else []
    seg["count"] = counts
    seg["kind"] = np.broadcast_to(np.asarray(kinds, dtype=np.int32), (k,))
    seg["ms"] = np.broadcast_to(np.asarray(ms, dtype=np.float64), (k,))
    seg["delta"] = np.broadcast_to(np.asarray(delta, dtype=np.float64), (k,))
    seg["max_itr"] = np.broadcast_to(np.asarray(max_itr, dtype=np.int64), (k,))
    seg["t_max"] = np.broadcast_to(np.asarray(t_max, dtype=np.float64), (k,))
    seg["group"] = np.broadcast_to(np.asarray(group, dtype=np.int32), (k,))
    if err is not None:
        seg["err"] = np.asarray(err, dtype=np.float64).reshape(k, 3)
    return seg


def segments_to_device(seg: np.ndarray, device=None) -> torch.Tensor:
    """Copy a segment table to the device (as raw bytes)."""
    raw = torch.from_numpy(np.ascontiguousarray(seg).view(np.uint8).copy())
    return raw.to(device or "cuda")


def segments_from_device(seg_dev: torch.Tensor) -> np.ndarray:
    return seg_dev.cpu().numpy().view(SEGMENT_DTYPE).copy()


def multi_workspace_bytes(n: int, max_itr_bound: int, tuning=None) -> int:
    return int(lib().ccd_multi_workspace_bytes(int(n), int(max_itr_bound), _tuning_ptr(tuning)))


def multi_workspace(n: int, max_itr_bound: int, tuning=None, device=None) -> torch.Tensor:
    nbytes = multi_workspace_bytes(n, max_itr_bound, tuning)
    if nbytes == 0:
        raise CCDError(-1, "ccd_multi_workspace_bytes")
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def segments_err_from_bounds(verts: torch.Tensor, seg_dev: torch.Tensor, stream=None) -> None:
    _require_cuda(verts, "verts", torch.float64)
    nseg = seg_dev.numel() // SEGMENT_DTYPE.itemsize
    _check(lib().ccd_segments_err_from_bounds(_ptr(verts), verts.shape[1], _ptr(seg_dev), nseg,
                                              _stream(stream)), "ccd_segments_err_from_bounds")


def multi_batch(verts: torch.Tensor, seg_dev: torch.Tensor, max_itr_bound: int,
                ws: torch.Tensor | None = None, out: Result | None = None, tuning=None,
                with_checks: bool = True, stream=None) -> Result:
    """ccd_multi_batch over every segment of the device table ``seg_dev``."""
    _require_cuda(verts, "verts", torch.float64)
    if verts.dim() != 2 or verts.shape[0] != 24:
        raise ValueError("verts must have shape (24, n)")
    n = verts.shape[1]
    nseg = seg_dev.numel() // SEGMENT_DTYPE.itemsize
    dev = verts.device
    if out is None:
        out = Result(torch.empty(n, dtype=torch.uint8, device=dev),
                     torch.empty(n, dtype=torch.float64, device=dev),
                     torch.empty(n, dtype=torch.float64, device=dev),
                     torch.empty(n, dtype=torch.int64, device=dev) if with_checks else None)
    if ws is None:
        ws = multi_workspace(n, max_itr_bound, tuning, dev)
    code = lib().ccd_multi_batch(_ptr(verts), n, _ptr(seg_dev), nseg, int(max_itr_bound),
                                 _ptr(out.collides), _ptr(out.toi), _ptr(out.out_tol),
                                 _ptr(out.checks), _tuning_ptr(tuning), _ptr(ws), ws.numel(),
                                 _stream(stream))
    _check(code, "ccd_multi_batch")
    return out


def group_reduce(res: Result, seg_dev: torch.Tensor, ngroups: int, stream=None):
    """Per candidate set: (alpha = min toi, tol = max out_tol) device tensors
    of ngroups doubles (ccd_group_reduce)."""
    n = res.toi.numel()
    nseg = seg_dev.numel() // SEGMENT_DTYPE.itemsize
    dev = res.toi.device
    alpha = torch.empty(ngroups, dtype=torch.float64, device=dev)
    tol = torch.empty(ngroups, dtype=torch.float64, device=dev)
    _check(lib().ccd_group_reduce(_ptr(res.toi), _ptr(res.out_tol), n, _ptr(seg_dev), nseg,
                                  int(ngroups), _ptr(alpha), _ptr(tol), _stream(stream)),
           "ccd_group_reduce")
    return alpha, tol


def linf_distance(verts: torch.Tensor, seg_dev: torch.Tensor, ngroups: int = 1,
                  per_query: bool = False, stream=None):
    """L-infinity distance at t = 0 of every query (ccd_linf_distance):
    (group_min, dist or None), device tensors."""
    _require_cuda(verts, "verts", torch.float64)
    n = verts.shape[1]
    nseg = seg_dev.numel() // SEGMENT_DTYPE.itemsize
    gmin = torch.empty(ngroups, dtype=torch.float64, device=verts.device)
    dist = torch.empty(n, dtype=torch.float64, device=verts.device) if per_query else None
    _check(lib().ccd_linf_distance(_ptr(verts), n, _ptr(seg_dev), nseg, int(ngroups),
                                   _ptr(dist) if dist is not None else None, _ptr(gmin),
                                   _stream(stream)), "ccd_linf_distance")
    return gmin, dist


class LineSearchIO(ctypes.Structure):
    _fields_ = [("p", ctypes.c_double), ("delta", ctypes.c_double), ("rho", ctypes.c_double),
                ("max_itr", ctypes.c_int64), ("max_passes", ctypes.c_int32),
                ("cap_max", ctypes.c_int32), ("alpha", ctypes.c_double),
                ("p_out", ctypes.c_double), ("d", ctypes.c_double), ("d_i", ctypes.c_double),
                ("eps_i", ctypes.c_double), ("delta_i", ctypes.c_double),
                ("passes", ctypes.c_int32), ("validated", ctypes.c_int32)]


def line_search_workspace(n: int, max_itr: int, device=None) -> torch.Tensor:
    nb = lib().ccd_line_search_workspace_bytes(int(n), int(max_itr))
    if nb == 0:
        raise CCDError(-4, "ccd_line_search_workspace_bytes")
    return torch.empty(nb, dtype=torch.uint8, device=device or "cuda")


def line_search(verts: torch.Tensor, n_vf: int, n_ee: int, p: float, delta: float,
                max_itr: int = 10**6, rho: float = 1e-9, max_passes: int = 16,
                cap: str = "min", ws: torch.Tensor | None = None, stream=None) -> dict:
    """Algorithm 4's CCD step over one candidate set (ccd_line_search): the
    first n_vf columns of verts are vertex-face queries, the next n_ee
    edge-edge queries.  Returns alpha, p, d, d_i, eps_i, delta_i, passes and
    validated."""
    _require_cuda(verts, "verts", torch.float64)
    if cap not in ("min", "max"):
        raise ValueError("cap is 'min' or 'max'")
    if verts.shape[1] != n_vf + n_ee:
        raise ValueError("verts has n_vf + n_ee columns")
    if ws is None:
        ws = line_search_workspace(n_vf + n_ee, max_itr, verts.device)
    io = LineSearchIO(p=float(p), delta=float(delta), rho=float(rho), max_itr=int(max_itr),
                      max_passes=int(max_passes), cap_max=1 if cap == "max" else 0)
    code = lib().ccd_line_search(_ptr(verts), int(n_vf), int(n_ee), ctypes.byref(io), _ptr(ws),
                                 ws.numel(), _stream(stream))
    if code not in (0, -5):
        raise CCDError(code, "ccd_line_search")
    return {"alpha": io.alpha, "p": io.p_out, "d": io.d, "d_i": io.d_i, "eps_i": io.eps_i,
            "delta_i": io.delta_i, "passes": io.passes, "validated": bool(io.validated),
            "status": code}


def _mesh_args(x0, x1, faces, edges):
    for t, name, dt in ((x0, "x0", torch.float64), (x1, "x1", torch.float64),
                        (faces, "faces", torch.int32), (edges, "edges", torch.int32)):
        _require_cuda(t, name, dt)
    if x0.shape != x1.shape or x0.dim() != 2 or x0.shape[1] != 3:
        raise ValueError("x0, x1 are (nv, 3)")
    if faces.dim() != 2 or faces.shape[1] != 3 or edges.dim() != 2 or edges.shape[1] != 2:
        raise ValueError("faces are (nf, 3), edges (ne, 2)")


def scene_eps(x0: torch.Tensor, x1: torch.Tensor, stream=None) -> np.ndarray:
    """eps of the scene per kind and axis, (2, 3) on the host (ccd_scene_eps)."""
    ws = torch.empty(256, dtype=torch.uint8, device=x0.device)
    eps = (ctypes.c_double * 6)()
    _check(lib().ccd_scene_eps(_ptr(x0), _ptr(x1), x0.shape[0], eps, _ptr(ws), 256,
                               _stream(stream)), "ccd_scene_eps")
    return np.array(list(eps)).reshape(2, 3)


def broad_phase(x0, x1, faces, edges, margin: float, cap: int | None = None, stream=None):
    """Candidate pairs (vf (k, 2), ee (m, 2)) int32 device tensors, sorted
    (ccd_broad_phase); capacities grow until the lists fit."""
    _mesh_args(x0, x1, faces, edges)
    nv, nf, ne = x0.shape[0], faces.shape[0], edges.shape[0]
    cap_vf = cap_ee = int(cap if cap is not None else 4 * (nv + nf + ne) + 1024)
    while True:
        nb = lib().ccd_broad_phase_workspace_bytes(nv, nf, ne, cap_vf, cap_ee)
        if nb == 0:
            raise CCDError(-1, "ccd_broad_phase_workspace_bytes")
        ws = torch.empty(nb, dtype=torch.uint8, device=x0.device)
        vf = torch.empty((cap_vf, 2), dtype=torch.int32, device=x0.device)
        ee = torch.empty((cap_ee, 2), dtype=torch.int32, device=x0.device)
        counts = (ctypes.c_int64 * 2)()
        code = lib().ccd_broad_phase(_ptr(x0), _ptr(x1), nv, _ptr(faces), nf, _ptr(edges), ne,
                                     float(margin), _ptr(vf), cap_vf, _ptr(ee), cap_ee, counts,
                                     _ptr(ws), nb, _stream(stream))
        if code == -5:
            cap_vf, cap_ee = max(cap_vf, int(counts[0])), max(cap_ee, int(counts[1]))
            continue
        _check(code, "ccd_broad_phase")
        return vf[:counts[0]], ee[:counts[1]]


def active_set(x0, x1, faces, edges, vf, ee, delta: float = 1e-6, max_itr: int = 10**6,
               stream=None) -> dict:
    """Algorithm 3 over given candidates (ccd_active_set): kind, pairs, toi
    of the colliding candidates (device tensors) and the eps used."""
    _mesh_args(x0, x1, faces, edges)
    n = vf.shape[0] + ee.shape[0]
    nb = lib().ccd_active_set_workspace_bytes(n, int(max_itr))
    if nb == 0:
        raise CCDError(-1, "ccd_active_set_workspace_bytes")
    dev = x0.device
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    kind = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    pairs = torch.empty((max(n, 1), 2), dtype=torch.int32, device=dev)
    toi = torch.empty(max(n, 1), dtype=torch.float64, device=dev)
    na = ctypes.c_int64()
    eps = (ctypes.c_double * 6)()
    vfc, eec = vf.contiguous(), ee.contiguous()
    code = lib().ccd_active_set(_ptr(x0), _ptr(x1), x0.shape[0], _ptr(faces), _ptr(edges),
                                _ptr(vfc), vfc.shape[0], _ptr(eec), eec.shape[0], float(delta),
                                int(max_itr), _ptr(kind), _ptr(pairs), _ptr(toi),
                                ctypes.byref(na), eps, _ptr(ws), nb, _stream(stream))
    if code not in (0, -5):
        raise CCDError(code, "ccd_active_set")
    m = na.value
    return {"kind": kind[:m], "pairs": pairs[:m], "toi": toi[:m],
            "eps": np.array(list(eps)).reshape(2, 3), "status": code}


def construct_active_set(x0, x1, faces, edges, delta: float = 1e-6, max_itr: int = 10**6,
                         margin: float | None = None, stream=None) -> dict:
    """Algorithm 3 end to end: scene eps, broad phase with margin (default
    the largest eps), CCD of every candidate, the colliding ones."""
    if margin is None:
        margin = float(scene_eps(x0, x1, stream).max())
    vf, ee = broad_phase(x0, x1, faces, edges, margin, stream=stream)
    out = active_set(x0, x1, faces, edges, vf, ee, delta, max_itr, stream)
    out.update({"vf_candidates": vf, "ee_candidates": ee, "margin": margin})
    return out


def aos_to_soa(aos: torch.Tensor, soa: torch.Tensor, col: int = 0, stream=None) -> None:
    """Device (n, 24) array of structures into columns [col, col + n) of a
    (24, ld) structure-of-arrays tensor (ccd_aos_to_soa)."""
    _require_cuda(aos, "aos", torch.float64)
    _require_cuda(soa, "soa", torch.float64)
    n, ld = aos.shape[0], soa.shape[1]
    if aos.dim() != 2 or aos.shape[1] != 24 or soa.shape[0] != 24 or col < 0 or col + n > ld:
        raise ValueError("shape mismatch")
    ptr = ctypes.c_void_p(soa.data_ptr() + 8 * col)
    _check(lib().ccd_aos_to_soa(_ptr(aos), n, ptr, ld, _stream(stream)), "ccd_aos_to_soa")


def to_soa(verts_aos, device="cuda") -> torch.Tensor:
    """(n, 24) host array -> (24, n) contiguous float64 device tensor."""
    t = torch.as_tensor(verts_aos, dtype=torch.float64)
    return t.t().contiguous().to(device)


# ---- the served form (ccd_batch_begin / submit / poll / cancel / end) -----------

class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("lanes", ctypes.c_int32),
                ("max_requests", ctypes.c_int32), ("max_batch", ctypes.c_int64),
                ("inbox_queries", ctypes.c_int64), ("max_segments", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("max_itr_bound", ctypes.c_int64),
                ("deep_slice_us", ctypes.c_int64)]


class CRequest(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pad", ctypes.c_int32), ("n", ctypes.c_int64),
                ("verts", ctypes.c_void_p), ("ms", ctypes.c_double), ("delta", ctypes.c_double),
                ("max_itr", ctypes.c_int64), ("collides", ctypes.c_void_p),
                ("toi", ctypes.c_void_p), ("out_tol", ctypes.c_void_p),
                ("checks", ctypes.c_void_p)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("cancelled", ctypes.c_int64), ("busy_rejections", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("deep_rounds", ctypes.c_int64),
                ("yields", ctypes.c_int64),
                ("inbox_peak_queries", ctypes.c_int64), ("pages", ctypes.c_int64),
                ("pages_peak", ctypes.c_int32), ("lanes_busy_peak", ctypes.c_int32),
                ("arena_bytes", ctypes.c_size_t)]


class NativeServer:
    """Marshalling for the C server: host numpy arrays in and out."""

    def __init__(self, **config):
        cfg = ServerConfig(**config)
        h = ctypes.c_void_p()
        _check(lib().ccd_batch_begin(ctypes.byref(cfg), ctypes.byref(h)), "ccd_batch_begin")
        self.h = h

    def submit(self, kind, verts_aos: np.ndarray, ms, delta, max_itr, col, toi, tol, chk=None):
        """Returns the ticket, or None when the server has no room now."""
        n = int(verts_aos.shape[0])
        req = CRequest(kind=int(kind), n=n, verts=verts_aos.ctypes.data, ms=float(ms),
                       delta=float(delta), max_itr=int(max_itr), collides=col.ctypes.data,
                       toi=toi.ctypes.data, out_tol=tol.ctypes.data,
                       checks=chk.ctypes.data if chk is not None else None)
        t = ctypes.c_int64()
        code = lib().ccd_batch_submit(self.h, ctypes.byref(req), ctypes.byref(t))
        if code == -6:
            return None
        _check(code, "ccd_batch_submit")
        return t.value

    def poll(self, cap=256, wait_us=0):
        done = (ctypes.c_int64 * cap)()
        st = (ctypes.c_int32 * cap)()
        nd = ctypes.c_int32()
        _check(lib().ccd_batch_poll(self.h, done, st, cap, ctypes.byref(nd), int(wait_us)),
               "ccd_batch_poll")
        return [(done[i], st[i]) for i in range(nd.value)]

    def cancel(self, ticket) -> int:
        return lib().ccd_batch_cancel(self.h, int(ticket))

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib().ccd_batch_stats(self.h, ctypes.byref(s)), "ccd_batch_stats")
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self.h:
            _check(lib().ccd_batch_end(self.h), "ccd_batch_end")
            self.h = None
