"""Builds the solver's shared libraries in-tree.

    libns3d.so            the CUDA library behind include/ns3d.h (sm_103a)
    libns3d_hostcheck.so  CPU emulation of the kernels' block bodies, used only
                          by the index-logic tests

Every CUDA translation unit is compiled separately and in parallel, then
linked with nvcc.  Objects go to _build/ at the repository root and are
rebuilt only when a source or header is newer.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libns3d.so")
HOSTLIB = os.path.join(PKG, "libns3d_hostcheck.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# host-only constexpr functions called from device code are errors, not warnings
NVFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                  "--diag-error", "20013,20014,20015", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def build_cuda(jobs: int | None = None, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdrs = _headers()
    objs, todo = [], []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if _stale(o, [s] + hdrs):
            todo.append((s, o))
    nv = _nvcc()
    jobs = jobs or max(1, min(len(todo), os.cpu_count() or 4))
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        outs = list(ex.map(lambda so: _run([nv] + NVFLAGS + ["-c", so[0], "-o", so[1]]), todo))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    if todo or _stale(LIB, objs):
        _run([nv] + ARCH + ["-shared", "-o", LIB] + objs)
    return LIB


def build_hostcheck() -> str:
    src = os.path.join(CSRC, "hostcheck.cpp")
    if _stale(HOSTLIB, [src] + _headers()):
        cxx = os.environ.get("CXX", "g++")
        _run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, "-o", HOSTLIB, src])
    return HOSTLIB


def build_all(verbose: bool = False):
    build_hostcheck()
    return build_cuda(verbose=verbose)


if __name__ == "__main__":
    print(build_all(verbose="-v" in sys.argv))
