"""Builds the CUDA library libpa.so in-tree for sm_103a (GB300) with nvcc.

The translation units are compiled in parallel, then linked into a shared
library next to this file.  Nothing here needs a GPU: nvcc cross-compiles.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libpa.so")
BUILD_DIR = os.path.join(HERE, "_build")
UNITS = ["pa_api.cu", "pa_forward.cu", "pa_adjoint.cu", "pa_misc.cu", "pa_noalloc.cu", "pa_image.cu", "pa_probe.cu",
         "pa_order.cu"]
HEADERS = [os.path.join(CSRC, "pa_common.cuh"), os.path.join(CSRC, "pa_internal.h"),
           os.path.join(ROOT, "include", "pa.h")]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-gencode", "arch=compute_103a,code=sm_103a",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    srcs = [os.path.join(CSRC, u) for u in UNITS] + HEADERS + [os.path.abspath(__file__)]
    return any(os.path.getmtime(s) > t for s in srcs)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    bdir = os.path.join(BUILD_DIR, str(os.getpid()))
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    procs = []
    for u in UNITS:
        obj = os.path.join(bdir, u.replace(".cu", ".o"))
        cmd = [nvcc, *NVCC_FLAGS, "-c", os.path.join(CSRC, u), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((u, obj, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    objs = []
    failed = []
    for u, obj, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((u, out))
        objs.append(obj)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(f"--- {u}\n{o}" for u, o in failed))
    tmp = f"{LIB}.{os.getpid()}.tmp"
    cmd = [nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp, *objs]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout)
    os.replace(tmp, LIB)
    for obj in objs:
        os.remove(obj)
    os.rmdir(bdir)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
