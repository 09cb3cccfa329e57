"""Builds the CUDA library ``libffs.so`` in-tree (``paper_1903_10741_gb300/_build``).

nvcc, one ``-gencode`` for sm_103a, translation units compiled in parallel, linked
into a shared library that exports the C ABI of ``include/ffs.h``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libffs.so")
# The bounds-checked variant (FFS_CHECKED): device indices into shared and global buffers
# are checked, counted and clamped instead of used out of range; for tests, not for speed.
BUILD_CHECKED = os.path.join(PKG, "_build_checked")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
_lock = threading.Lock()


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libffs")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                   "--expt-relaxed-constexpr", *extra]


def build(force: bool = False, verbose: bool = False, extra=(), checked: bool = False) -> str:
    out_dir = BUILD_CHECKED if checked else BUILD
    lib_path = os.path.join(out_dir, "libffs.so")
    if checked:
        extra = tuple(extra) + ("-DFFS_CHECKED",)
    with _lock:
        if not force and up_to_date(lib_path):
            return lib_path
        os.makedirs(out_dir, exist_ok=True)
        nv = nvcc()
        srcs = _sources()

        def compile_one(src):
            obj = os.path.join(out_dir, os.path.basename(src) + ".o")
            cmd = [nv, *flags(extra), "-c", src, "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
            if verbose and r.stderr:
                print(r.stderr)
            return obj

        with cf.ThreadPoolExecutor(max_workers=max(1, len(srcs))) as ex:
            objs = list(ex.map(compile_one, srcs))
        tmp = lib_path + f".tmp{os.getpid()}"
        r = subprocess.run([nv, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
        os.replace(tmp, lib_path)
        return lib_path


if __name__ == "__main__":
    print(build(force=True, verbose=True))
