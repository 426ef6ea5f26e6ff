"""Builds libgws.so in-tree for sm_103a (nvcc; translation units compiled in parallel).

Two variants of the same sources: ``libgws.so`` (the product) and ``libgws_check.so``, compiled
with GWS_CHECK_BOUNDS: its kernels check their tile, list and record indices (an index out of
range is recorded in the device status word and its access skipped) and its workspace carries
canary words after every sub-buffer, checked at the end of each call.  The checking variant is
the stand-in for a memory checker in the GPU tests; nothing else loads it.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libgws.so")
LIB_CHECK = os.path.join(OUT, "libgws_check.so")
SOURCES = ["gws_api.cu", "gws_prep.cu", "gws_sort.cu", "gws_splat.cu", "gws_bwd.cu", "gws_noalloc.cu", "gws_exact.cu",
           "gws_front.cu", "gws_tri.cu"]
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden"]
VARIANTS = {"": (LIB, OUT, []), "check": (LIB_CHECK, os.path.join(OUT, "check"), ["-DGWS_CHECK_BOUNDS"])}


def _deps():
    return ([os.path.join(CSRC, s) for s in SOURCES] + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "gws.h")])


def stale(variant: str = "") -> bool:
    lib = VARIANTS[variant][0]
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in _deps() if os.path.exists(d))


def _compile(job) -> str:
    src, objdir, defs = job
    obj = os.path.join(objdir, os.path.splitext(src)[0] + ".o")
    cmd = [NVCC, *ARCH, *FLAGS, *defs, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def _link(lib: str, objs) -> None:
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, "-shared", *objs, "-o", tmp, "-lcufft", "-cudart", "static",
           "-Xlinker", f"-rpath,{os.path.join(CUDA_HOME, 'lib64')}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)


def build(force: bool = False, variants=("", "check")) -> str:
    """Compiles every CUDA translation unit of the requested variants (all in parallel) and links
    each library (static cudart, cuFFT).  Returns the product library's path."""
    todo = [v for v in variants if force or stale(v)]
    if todo:
        jobs = []
        for v in todo:
            _, objdir, defs = VARIANTS[v]
            os.makedirs(objdir, exist_ok=True)
            jobs += [(src, objdir, defs) for src in SOURCES]
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 8)) as ex:
            objs = list(ex.map(_compile, jobs))
        for i, v in enumerate(todo):
            _link(VARIANTS[v][0], objs[i * len(SOURCES):(i + 1) * len(SOURCES)])
    return LIB


if __name__ == "__main__":
    print(build(force=True))
