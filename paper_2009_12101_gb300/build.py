"""Build the CUDA library libcbgmres.so for sm_103a (GB300) in-tree.

Each translation unit (one per basis format, the FP64-input SpMV, the host driver) is
compiled by its own nvcc process in parallel, then linked into one shared library in
``paper_2009_12101_gb300/_lib``.  No cmake, no torch extension machinery: the library
has a plain C ABI (include/cbgmres.h).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libcbgmres.so")
# debug variant (-DCBG_DEBUG): guard tails on the solver's device allocations, checked
# after every solve, and column-index checks in the SpMV kernels
LIB_DEBUG = os.path.join(OUT_DIR, "libcbgmres_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["solver.cu", "spmv_f64.cu", "noalloc.cu", "batched.cu", "learned.cu", "mlp_tc.cu", "multi.cu",
           "multi_tc.cu"] + [f"basis_{f}.cu" for f in
                                          ("f64", "f32", "f16", "bf16", "e4m3", "i32", "i16")]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcbgmres")
    return cand


def _newest_source_mtime() -> float:
    t = 0.0
    for f in os.listdir(CSRC):
        t = max(t, os.path.getmtime(os.path.join(CSRC, f)))
    return max(t, os.path.getmtime(os.path.join(ROOT, "include", "cbgmres.h")))


def build(force: bool = False, verbose: bool = False, jobs: int | None = None, debug: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    lib = LIB_DEBUG if debug else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _newest_source_mtime():
        return lib
    nvcc = _nvcc()
    obj_dir = os.path.join(OUT_DIR, "obj_debug" if debug else "obj")
    os.makedirs(obj_dir, exist_ok=True)
    flags = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                    "-I", os.path.join(ROOT, "include")] + (["-DCBG_DEBUG"] if debug else [])
    if verbose:
        flags += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(obj_dir, src.replace(".cu", ".o"))
        cmd = [nvcc] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    jobs = jobs or min(len(SOURCES), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for (_, err), src in zip(results, SOURCES):
            sys.stderr.write(f"== {src}\n{err}")
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results] + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
