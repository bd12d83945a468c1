"""Builds the CUDA libraries of the package in-tree for sm_103a (GB300):

    libsirius.so          the C-ABI hot path (include/sirius.h)
    libsirius_datagen.so  the CUDA twin of the seeded input generator

Each .cu file compiles to an object in parallel; objects are relinked only when a source or
header is newer.  Plain nvcc, no CMake.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shlex
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OBJ = os.path.join(PKG, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
         "--expt-relaxed-constexpr"]

LIBS = {
    "libsirius.so": ["api.cu", "filter.cu", "hashjoin.cu", "groupby.cu", "pipeline.cu", "batch.cu", "topn.cu", "sortgroup.cu", "strings.cu"],
    "libsirius_datagen.so": ["datagen.cu"],
}


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build libsirius")


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "sirius.h")]


def _newer(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(nvcc: str, src: str, obj: str, verbose: bool):
    # SIRIUS_NVCC_FLAGS: extra nvcc flags, e.g. -D overrides of the kernels' build-time tunables
    cmd = [nvcc, *ARCH, *FLAGS, *shlex.split(os.environ.get("SIRIUS_NVCC_FLAGS", "")), "-c", src, "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(verbose: bool = False, force: bool = False) -> dict:
    """Compile and link every library; returns {library name: path}."""
    nvcc = _nvcc()
    os.makedirs(OBJ, exist_ok=True)
    hdrs = _headers()
    jobs = {}
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        for lib, srcs in LIBS.items():
            for s in srcs:
                src = os.path.join(CSRC, s)
                obj = os.path.join(OBJ, s.replace(".cu", ".o"))
                if force or _newer(obj, [src, *hdrs]):
                    jobs[obj] = ex.submit(_compile, nvcc, src, obj, verbose)
        for f in jobs.values():
            f.result()
    out = {}
    for lib, srcs in LIBS.items():
        target = os.path.join(PKG, lib)
        objs = [os.path.join(OBJ, s.replace(".cu", ".o")) for s in srcs]
        if force or _newer(target, objs):
            cmd = [nvcc, *ARCH, "-shared", "-o", target, *objs]
            if verbose:
                print(" ".join(cmd), flush=True)
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link of {lib} failed:\n{r.stdout}\n{r.stderr}")
        out[lib] = target
    return out


if __name__ == "__main__":
    for k, v in build(verbose=True).items():
        print(k, "->", v)
