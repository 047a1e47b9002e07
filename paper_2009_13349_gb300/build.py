"""Build the sm_103a CUDA library (``_lib/libccd_gb300.so``) in-tree with nvcc.

Flags: ``-gencode arch=compute_103a,code=sm_103a -O3 -lineinfo -fmad=false``.
The kernels spell every FP64 add and multiply as a round-to-nearest
intrinsic; ``-fmad=false`` additionally forbids contraction anywhere else.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc", "ccd.cu")
SRCS = [SRC, os.path.join(HERE, "csrc", "activeset.cu"), os.path.join(HERE, "csrc", "serve.cu")]
INCLUDE = os.path.join(ROOT, "include")
LIB_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIB_DIR, "libccd_gb300.so")

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo",
              "-fmad=false", "-std=c++17", "-Xcompiler", "-fPIC"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return [*SRCS, os.path.join(INCLUDE, "ccd.h"), os.path.join(HERE, "csrc", "internal.h"),
            os.path.join(HERE, "csrc", "serve_queue.h")]


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    os.makedirs(LIB_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(s) for s in sources())):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    objs, procs = [], []
    for src in SRCS:   # translation units compile in parallel, then one link
        obj = os.path.join(LIB_DIR, os.path.basename(src) + f".{os.getpid()}.o")
        cmd = [nvcc(), *NVCC_FLAGS, *extra, "-I", INCLUDE, "-I", os.path.join(HERE, "csrc"), "-c",
               "-o", obj, src]
        if verbose:
            print(" ".join(cmd))
        procs.append((subprocess.Popen(cmd), cmd))
        objs.append(obj)
    for proc, cmd in procs:
        if proc.wait() != 0:
            raise subprocess.CalledProcessError(proc.returncode, cmd)
    link = [nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp, *objs]
    subprocess.run(link, check=True)
    for obj in objs:
        os.remove(obj)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
