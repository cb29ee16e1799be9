"""Build of the renderer's shared library (libvr.so) for sm_103a.

Each CUDA translation unit is compiled by nvcc in parallel into
``paper_1012_2909_gb300/_build/`` and linked into ``paper_1012_2909_gb300/libvr.so``
with the CUDA runtime linked statically, so the library loads by path with no
search-path set-up.  Nothing is rebuilt when every object is newer than its
sources and headers.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libvr.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvr.so")
    return exe


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                   "-I", CSRC, "--expt-relaxed-constexpr", *extra]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False, extra_flags=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    hdrs = _headers()
    srcs = sources()
    objs = [os.path.join(BUILD, os.path.basename(s)[:-3] + ".o") for s in srcs]
    exe = nvcc()

    def compile_one(pair):
        src, obj = pair
        if not force and not _stale(obj, [src, *hdrs, __file__]):
            return None
        tmp = obj + f".{os.getpid()}.tmp"
        cmd = [exe, *_flags(extra_flags), "-c", src, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stderr}")
        os.replace(tmp, obj)
        return r.stderr if verbose else None

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs)) or 1) as ex:
        for msg in ex.map(compile_one, zip(srcs, objs)):
            if msg:
                print(msg)
    if force or _stale(LIB, objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [exe, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of libvr.so failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


def ptxas_report(src_name: str) -> str:
    """Register / shared-memory usage of one translation unit (-Xptxas -v)."""
    src = os.path.join(CSRC, src_name)
    out = os.path.join(BUILD, "ptxas_probe.o")
    os.makedirs(BUILD, exist_ok=True)
    r = subprocess.run([nvcc(), *_flags(["-Xptxas", "-v"]), "-c", src, "-o", out],
                       capture_output=True, text=True)
    return r.stderr


if __name__ == "__main__":
    print(build(verbose=True))
