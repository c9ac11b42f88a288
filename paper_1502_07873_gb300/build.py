"""Build liboed.so (the sm_103a CUDA library behind include/oed.h) in-tree.

Each translation unit is compiled by nvcc in parallel and linked into
``paper_1502_07873_gb300/liboed.so``.  Objects go to ``_build/`` next to this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "liboed.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["api.cu", "source.cu", "stencil.cu", "stream_tma.cu", "stream_tma2.cu", "resident.cu", "hessian.cu", "logdet.cu", "dlmc.cu", "adjoint.cu",
           "noalloc.cu", "smolyak.cpp", "server.cpp"]
HEADERS = [os.path.join(CSRC, "oed_internal.cuh"), os.path.join(CSRC, "stencil_cell.cuh"),
           os.path.join(CSRC, "nvtx_range.h"), os.path.join(CSRC, "pair_math.cuh"),
           os.path.join(CSRC, "tma_sync.cuh"),
           os.path.join(ROOT, "include", "oed.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    jobs = []
    objs = []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        if force or _stale(obj, [path] + HEADERS):
            if src.endswith(".cu"):
                cmd = [cc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                       "-Xptxas", "-v" if verbose else "-O3", *extra_flags, "-c", path, "-o", obj]
            else:
                cmd = [cc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-c", path, "-o", obj]
            jobs.append(cmd)

    def run(cmd):
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("compile failed: " + " ".join(cmd) + "\n" + p.stderr)
        return p.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for log in ex.map(run, jobs):
            if verbose and log:
                print(log)
    if force or jobs or _stale(OUT, objs):
        tmp = OUT + f".tmp{os.getpid()}"
        run([cc, *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
