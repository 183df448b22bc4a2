"""Builds the CUDA library ``_lib/libsht.so`` for sm_103a with nvcc.

The translation units are compiled in parallel, then linked against the
shared CUDA runtime (the one PyTorch also loads).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libsht.so")
LIBDIR_CHECK = os.path.join(HERE, "_lib_check")
SOURCES = ["sht_plan.cu", "legendre.cu", "legendre_tc.cu", "legendre_df.cu", "ringfft.cu", "diag.cu", "noalloc.cu", "spin.cu", "batch.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "sht.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Build _lib/libsht.so; with checked=True the bounds-checked variant (nvcc -DSHT_CHECK:
    out-of-bounds kernel accesses are skipped and reported in bit 1 of the plan status word)
    into _lib_check/libsht.so instead."""
    libdir = LIBDIR_CHECK if checked else LIBDIR
    lib = os.path.join(libdir, "libsht.so")
    if not force and not _stale(lib):
        return lib
    os.makedirs(libdir, exist_ok=True)
    cc = nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(libdir, os.path.splitext(src)[0] + ".o")
        cmd = [cc] + _flags() + (["-DSHT_CHECK"] if checked else []) + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for obj, err in ex.map(compile_one, SOURCES):
            objs.append(obj)
            if verbose and err:
                print(err)
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [cc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
