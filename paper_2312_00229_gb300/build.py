"""Builds the CUDA library ``_build/libwdweno.so`` for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked into one shared
library with the C ABI of ``include/wdweno.h``.  The library is built in-tree
(the ``_build`` directory next to this file) and is rebuilt when a source or
header is newer than it.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libwdweno.so")
SOURCES = ["wd_api.cu", "wd_fwd.cu", "wd_fwd_typed.cu", "wd_fwd_typed_b2r.cu", "wd_batched.cu",
           "wd_batched2.cu", "wd_bwd.cu",
           "wd_resample.cu", "wd_noalloc.cu", "wd_cascade.cu", "wd_probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libwdweno.so")


def _sources():
    return [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "wdweno.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, extra_flags=(), lib_path=None) -> str:
    """Compiles every translation unit and links LIB (or `lib_path`)."""
    target = lib_path or LIB
    if not force and lib_path is None and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I", INCLUDE, "-I", CSRC] + list(extra_flags)

    def compile_one(src):
        obj = os.path.join(os.path.dirname(target), src.replace(".cu", f".{os.getpid()}.o"))
        cmd = [cc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    srcs = _sources()
    objs = [os.path.join(os.path.dirname(target), s.replace(".cu", f".{os.getpid()}.o"))
            for s in srcs]
    try:
        with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
            list(ex.map(compile_one, srcs))
        tmp = target + f".tmp{os.getpid()}"
        cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, target)
    finally:
        for o in objs:  # the per-process object files are not kept
            if os.path.exists(o):
                os.remove(o)
    return target


if __name__ == "__main__":
    print(build(force=True, verbose=True))
