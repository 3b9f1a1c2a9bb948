"""Compile libawpm.so (CUDA, sm_103a) in-tree with nvcc.

The translation units are compiled in parallel and linked into
``paper_1801_09809_gb300/libawpm.so``; objects go to ``_build/`` at the
repository root.  Only sm_103a code is generated.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJDIR = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libawpm.so")
SOURCES = ["awpm_kernels.cu", "awpm_api.cu", "awpm_serve.cu", "awpm_noalloc.cu"]
HEADERS = [os.path.join(CSRC, "awpm_internal.h"), os.path.join(CSRC, "awpm_ctx.h"),
           os.path.join(INCLUDE, "awpm.h")]

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-fmad=false", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
         "-I" + INCLUDE, "-I" + CSRC]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OBJDIR, exist_ok=True)
    procs, objs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OBJDIR, os.path.splitext(src)[0] + ".o")
        objs.append(o)
        if force or _stale(o, [s] + HEADERS):
            cmd = [NVCC, *ARCH, *FLAGS, "-c", s, "-o", o]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                                stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd) + "\n" + out.decode())
    if force or procs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call([NVCC, "-shared", *ARCH, *objs, "-o", tmp])
        os.replace(tmp, LIB)
    return LIB


def build_debug(lib: str, objdir: str) -> str:
    """The same library compiled with AWPM_DEBUG_BOUNDS (device index checks
    that report AWPM_ERR_INTERNAL instead of touching memory out of range),
    written to `lib`; objects go to `objdir`.  Not part of build(): tests that
    need it build it themselves and load it through AWPM_LIBRARY."""
    os.makedirs(objdir, exist_ok=True)
    procs, objs = [], []
    for src in SOURCES:
        o = os.path.join(objdir, os.path.splitext(src)[0] + ".o")
        objs.append(o)
        cmd = [NVCC, *ARCH, *FLAGS, "-DAWPM_DEBUG_BOUNDS", "-c", os.path.join(CSRC, src), "-o", o]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                            stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd) + "\n" + out.decode())
    subprocess.check_call([NVCC, "-shared", *ARCH, *objs, "-o", lib])
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
