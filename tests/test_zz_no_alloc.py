"""The vertex-face entry point that allocates nothing (ccd_vf_batch_static).

It serves callers that cannot allocate device memory -- real-time loops that
must stay out of the allocator, plugins whose host owns all allocations,
processes on a fixed memory quota.  Its scratch is a 40 MiB device array
inside the library.  These tests call it through the C ABI, twice in a row
on each input, and require the answers of ccd_vf_batch (which uses a caller
workspace) and of the CPU oracle, with and without minimum separation and
at two check limits; one input sends queries to the deep tier.  Batches
beyond its limits are refused before any work.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
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


def _call_static(f, verts, err, ms, max_itr):
    n = verts.shape[1]
    col = torch.empty(n, dtype=torch.uint8, device="cuda")
    toi = torch.empty(n, dtype=torch.float64, device="cuda")
    tol = torch.empty(n, dtype=torch.float64, device="cuda")
    chk = torch.empty(n, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = f(V(verts.data_ptr()), n, V(err.data_ptr()), 0 if err.numel() == 3 else 3, float(ms),
           1e-6, max_itr, V(col.data_ptr()), V(toi.data_ptr()), V(tol.data_ptr()),
           V(chk.data_ptr()), V(stream))
    assert rc == 0, rc
    torch.cuda.synchronize()
    return col.cpu().numpy(), toi.cpu().numpy(), tol.cpu().numpy(), chk.cpu().numpy()


@pytest.mark.parametrize("ms", [0.0, 1e-4])
@pytest.mark.parametrize("max_itr", [50, MAX_ITR])
def test_static_scratch_matches_workspace_entry_point_and_oracle(ms, max_itr):
    ccd, f = _entry()
    rng = np.random.default_rng(33)
    inputs = [W.unit_cube(0, 3000, seed=31).verts,                      # shallow queries
              W.degenerate_heavy(n=4000, seed=32).batches[0].verts]     # deep frontiers
    for which, verts in enumerate(inputs):
        v = ccd.to_soa(verts)
        e = ccd.err_from_bounds(0, v, ms_nonzero=ms > 0)
        ws = ccd.workspace(verts.shape[0], max_itr)
        r = ccd.batch(0, v, e, ms=ms, delta=1e-6, max_itr=max_itr, ws=ws)
        torch.cuda.synchronize()
        ref = (r.collides.cpu().numpy(), r.toi.cpu().numpy(), r.out_tol.cpu().numpy(),
               r.checks.cpu().numpy())
        if which == 1 and max_itr == MAX_ITR:
            # frontiers beyond 256 boxes reach ccd_vf_batch's deep tier; the
            # static path's one-warp slots hold 256, so they reach its deep tier
            assert ccd.workspace_counters(ws)["deep_queries"] > 0
        for _ in range(2):                                              # two calls in a row
            got = _call_static(f, v, e, ms, max_itr)
            assert np.array_equal(got[0], ref[0])
            hit = ref[0] == 1
            assert np.all(np.abs(got[1][hit] - ref[1][hit]) <= 1e-6)
            for x, y in zip(got[1:], ref[1:]):
                assert np.array_equal(x, y)
        eo = oracle.err_from_bounds(0, verts, ms_nonzero=ms > 0)
        assert np.array_equal(e.cpu().numpy(), eo)
        idx = np.sort(rng.choice(verts.shape[0], 400, replace=False))
        o = oracle.ccd_batch(0, verts[idx], eo, ms=ms, delta=1e-6, max_itr=max_itr, nthreads=8)
        for x, y in zip(got, o):
            assert np.array_equal(x[idx], y)


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
