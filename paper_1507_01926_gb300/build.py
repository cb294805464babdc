"""Builds libmf.so (the C-ABI solver library) in-tree with nvcc for sm_103a.

Translation units are compiled in parallel (only those whose source or headers changed) and linked into
``paper_1507_01926_gb300/libmf.so``.
Nothing is installed; the library is loaded from this directory.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(PKG, "libmf.so")
BUILD = os.path.join(PKG, "_build")
# the same library with every gather index of the solver checked (MF_CHECK_BOUNDS), for tests
OUT_CHECK = os.path.join(PKG, "libmf_check.so")
BUILD_CHECK = os.path.join(PKG, "_build_check")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["mf_kernels_m0.cu", "mf_kernels_m1.cu", "mf_kernels_s0.cu", "mf_kernels_s1.cu", "mf_solver.cu", "mf_api.cu", "mf_batch.cu", "mf_service.cu", "mf_noalloc.cu", "mf_tune.cu"]
CPP_SOURCES = ["mf_csr.cpp"]
HEADERS = ["mf_solver.cuh", "mf_device.cuh", "mf_internal.h"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmf.so")


def _inputs():
    srcs = [os.path.join(CSRC, f) for f in CU_SOURCES + CPP_SOURCES + HEADERS]
    return srcs + [os.path.join(INCLUDE, "mf.h"), os.path.abspath(__file__)]


def up_to_date(out: str = OUT) -> bool:
    if not os.path.exists(out):
        return False
    t = os.path.getmtime(out)
    return all(os.path.getmtime(p) <= t for p in _inputs())


def build(force: bool = False, verbose: bool = False, check: bool = False) -> str:
    """Builds libmf.so, or with check=True libmf_check.so (the solver compiled with MF_CHECK_BOUNDS: a gather
    index outside its array is reported as MF_ERR_INTERNAL with the source line and the index, no trap)."""
    out, build_dir = (OUT_CHECK, BUILD_CHECK) if check else (OUT, BUILD)
    if not force and up_to_date(out):
        return out
    os.makedirs(build_dir, exist_ok=True)
    nv = nvcc()
    common = ["-O3", "-std=c++17", "-I", INCLUDE, "-I", CSRC] + (["-DMF_CHECK_BOUNDS"] if check else [])
    procs = []
    objs = []
    # an object is rebuilt when its source, a header or this script is newer than it (or force)
    deps = max(os.path.getmtime(p) for p in [os.path.join(CSRC, h) for h in HEADERS]
               + [os.path.join(INCLUDE, "mf.h"), os.path.abspath(__file__)])

    def stale(src, obj):
        return force or not os.path.exists(obj) or os.path.getmtime(obj) < max(deps, os.path.getmtime(src))

    for f in CU_SOURCES:
        o = os.path.join(build_dir, f + ".o")
        objs.append(o)
        if not stale(os.path.join(CSRC, f), o):
            continue
        cmd = [nv, *ARCH, "-lineinfo", *common, "-Xcompiler", "-fPIC", "-c", os.path.join(CSRC, f), "-o", o]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for f in CPP_SOURCES:
        o = os.path.join(build_dir, f + ".o")
        objs.append(o)
        if not stale(os.path.join(CSRC, f), o):
            continue
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-I", INCLUDE, "-I", CSRC, "-c", os.path.join(CSRC, f), "-o", o]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        log, _ = p.communicate()
        if verbose or p.returncode:
            sys.stderr.write(log.decode(errors="replace"))
        if p.returncode:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("libmf build failed:\n" + "\n".join(failed))
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call([nv, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"])
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
