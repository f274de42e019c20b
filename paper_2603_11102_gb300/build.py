"""Build libgks.so in-tree with nvcc for sm_103a.

Each CUDA translation unit is compiled in parallel, then linked into
``paper_2603_11102_gb300/_build/libgks.so``. Run ``python -m
paper_2603_11102_gb300.build`` or call :func:`build`. ``build(debug=True)``
(or ``--debug-bounds``) builds ``_build/debug/libgks_debug.so`` with
GKS_DEBUG_BOUNDS: kernels check their data-dependent indices and the calls
report GKS_ERR_DEBUG_BOUNDS instead of touching memory outside a buffer;
``gks.load`` takes it when the environment variable GKS_DEBUG_BOUNDS=1.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libgks.so")
OUT_DEBUG = os.path.join(OUT, "debug")
LIB_DEBUG = os.path.join(OUT_DEBUG, "libgks_debug.so")
SOURCES = ["gks_api.cu", "gks_stencil.cu", "gks_forcing.cu", "gks_noalloc.cu", "gks_adjoint.cu", "gks_peak.cu"]
HEADERS = ["gks_internal.h", "gks_device.cuh", os.path.join(ROOT, "include", "gks_api.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
                   "-I", CSRC] + list(extra)


def _stale(lib=LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + [h if os.path.isabs(h) else os.path.join(CSRC, h)
                                                       for h in HEADERS]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, extra=(), debug: bool = False) -> str:
    lib, out = (LIB_DEBUG, OUT_DEBUG) if debug else (LIB, OUT)
    if debug:
        extra = list(extra) + ["-DGKS_DEBUG_BOUNDS"]
    if not force and not _stale(lib):
        return lib
    os.makedirs(out, exist_ok=True)
    cc = nvcc()
    procs = []
    objs = []
    for s in SOURCES:
        obj = os.path.join(out, s.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [cc] + flags(extra) + ["-c", os.path.join(CSRC, s), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((s, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for s, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append("%s:\n%s" % (s, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"))
    if errors:
        raise RuntimeError("nvcc failed\n" + "\n".join(errors))
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else (), debug="--debug-bounds" in sys.argv))
