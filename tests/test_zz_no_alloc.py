"""The vertex-face entry point that allocates nothing (ccd_vf_batch_static).

It serves callers that cannot allocate device memory -- code running under
CUDA graph capture, real-time loops that must stay out of the allocator,
plugins whose host owns all allocations, processes on a fixed memory quota.
Its scratch is a 40 MiB device array inside the library.  These tests call
it through the C ABI and require the same answers as ccd_vf_batch (which
uses a caller workspace) on two calls in a row, and a clean refusal of
batches beyond its limits.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2009_13349_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MAX_N, MAX_ITR = 32768, 65536
V = ctypes.c_void_p


def _entry():
    from paper_2009_13349_gb300 import ccd
    f = ccd.lib().ccd_vf_batch_static
    f.argtypes = [V, ctypes.c_int64, V, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                  ctypes.c_int64, V, V, V, V, V]
    f.restype = ctypes.c_int
    return ccd, f


def _call_static(f, verts, err, max_itr):
    n = verts.shape[1]
    col = torch.empty(n, dtype=torch.uint8, device="cuda")
    toi = torch.empty(n, dtype=torch.float64, device="cuda")
    tol = torch.empty(n, dtype=torch.float64, device="cuda")
    chk = torch.empty(n, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = f(V(verts.data_ptr()), n, V(err.data_ptr()), 0 if err.numel() == 3 else 3, 0.0, 1e-6,
           max_itr, V(col.data_ptr()), V(toi.data_ptr()), V(tol.data_ptr()), V(chk.data_ptr()),
           V(stream))
    assert rc == 0, rc
    torch.cuda.synchronize()
    return col.cpu().numpy(), toi.cpu().numpy(), tol.cpu().numpy(), chk.cpu().numpy()


def test_static_scratch_matches_workspace_entry_point_twice_in_a_row():
    ccd, f = _entry()
    inputs = [W.unit_cube(0, 3000, seed=31).verts,                      # shallow queries
              W.simulation_mixed(n=20_000, seed=32).batches[0].verts]   # includes deep ones
    for verts in inputs:
        v = ccd.to_soa(verts)
        e = ccd.err_from_bounds(0, v)
        got = _call_static(f, v, e, MAX_ITR)
        r = ccd.batch(0, v, e, delta=1e-6, max_itr=MAX_ITR)
        torch.cuda.synchronize()
        ref = (r.collides.cpu().numpy(), r.toi.cpu().numpy(), r.out_tol.cpu().numpy(),
               r.checks.cpu().numpy())
        assert np.array_equal(got[0], ref[0])
        hit = ref[0] == 1
        assert np.all(np.abs(got[1][hit] - ref[1][hit]) <= 1e-6)
        assert np.array_equal(got[1], ref[1])
        assert np.array_equal(got[2], ref[2])
        assert np.array_equal(got[3], ref[3])


def test_static_scratch_refuses_batches_beyond_its_limits():
    ccd, f = _entry()
    one = torch.zeros(24, dtype=torch.float64, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    stream = V(torch.cuda.current_stream().cuda_stream)
    p = V(one.data_ptr())
    o = V(out.data_ptr())
    # nothing is read or written for refused sizes
    assert f(p, MAX_N + 1, p, 0, 0.0, 1e-6, 100, o, o, o, V(0), stream) == -2
    assert f(p, 1, p, 0, 0.0, 1e-6, MAX_ITR + 1, o, o, o, V(0), stream) == -2
    assert f(p, -1, p, 0, 0.0, 1e-6, 100, o, o, o, V(0), stream) == -1
