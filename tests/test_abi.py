"""The C ABI library loads and exports every symbol include/ccd.h declares;
host-side argument checks return before any device work (CPU only)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2009_13349_gb300 import build as B

HEADER = os.path.join(B.ROOT, "include", "ccd.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ccd_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    return B.build()


def test_header_declares_the_boundary():
    names = declared()
    for must in ("ccd_vf_batch", "ccd_ee_batch", "ccd_workspace_bytes", "ccd_err_from_bounds",
                 "ccd_workspace_status", "ccd_status_str"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (ccd_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    L = ctypes.CDLL(lib_path)
    for n in declared():
        getattr(L, n)


def test_host_argument_validation_without_device(lib_path):
    L = ctypes.CDLL(lib_path)
    f = L.ccd_vf_batch
    f.restype = ctypes.c_int
    V = ctypes.c_void_p
    f.argtypes = [V, ctypes.c_int64, V, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                  ctypes.c_int64, V, V, V, V, V, ctypes.c_size_t, V]
    one = V(16)   # never dereferenced: every call below fails argument checks
    args = dict(verts=one, n=1, err=one, stride=0, ms=0.0, delta=1e-6, mi=10, col=one,
                toi=one, tol=one, chk=V(0), ws=one, wsb=1 << 20, st=V(0))

    def call(**kw):
        a = dict(args, **kw)
        return f(a["verts"], a["n"], a["err"], a["stride"], a["ms"], a["delta"], a["mi"],
                 a["col"], a["toi"], a["tol"], a["chk"], a["ws"], a["wsb"], a["st"])

    assert call(n=-1) == -1
    assert call(delta=0.0) == -1
    assert call(delta=float("nan")) == -1
    assert call(mi=0) == -1
    assert call(ms=-1.0) == -1
    assert call(stride=1) == -1
    assert call(verts=V(0)) == -1
    assert call(ws=V(0)) == -2
    L.ccd_status_str.restype = ctypes.c_char_p
    assert L.ccd_status_str(-5).startswith(b"frontier")
