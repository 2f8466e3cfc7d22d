"""Builds libges.so in-tree with nvcc for sm_103a (GB300).

Translation units are compiled in parallel, then linked into one shared
library under paper_2411_09156_gb300/_build/. A stamp of the sources and flags
skips the rebuild when nothing changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libges.so")
SOURCES = ["api.cu", "preprocess.cu", "binning.cu", "render.cu", "noalloc.cu", "loss.cu", "knn.cu", "gsr.cu", "levelset.cu", "peaks.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the GES CUDA library cannot be built")


def lib_path(debug: bool = False) -> str:
    """The release library, or the debug build (GES_DEBUG: device-side bounds checks) beside it."""
    return os.path.join(BUILD, "debug", "libges.so") if debug else LIB


def _stamp(flags) -> str:
    h = hashlib.sha256()
    for f in sorted(os.listdir(CSRC)) + ["../../include/ges.h"]:
        p = os.path.normpath(os.path.join(CSRC, f))
        if os.path.isfile(p):
            h.update(f.encode())
            with open(p, "rb") as fh:
                h.update(fh.read())
    h.update(" ".join(ARCH + flags).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compiles and links the library (or its debug build) unless the sources and flags are
    unchanged since the last build; returns its path."""
    out_dir = os.path.join(BUILD, "debug") if debug else BUILD
    lib = lib_path(debug)
    flags = FLAGS + (["-DGES_DEBUG"] if debug else [])
    os.makedirs(out_dir, exist_ok=True)
    stamp_path = os.path.join(out_dir, "libges.stamp")
    stamp = _stamp(flags)
    if not force and os.path.exists(lib) and os.path.exists(stamp_path):
        with open(stamp_path) as fh:
            if fh.read().strip() == stamp:
                return lib
    nvcc = _nvcc()
    # -fvisibility=hidden: only the GES_API functions of include/ges.h are exported
    def compile_one(src):
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        cmd = [nvcc] + ARCH + flags + ["-I" + INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    with open(stamp_path, "w") as fh:
        fh.write(stamp)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
