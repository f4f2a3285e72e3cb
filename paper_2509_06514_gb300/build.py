"""Builds libimpir.so in-tree: every CUDA/C++ unit compiled for sm_103a in parallel, then
linked into one shared library. Also builds the input generator helper. With --bounds it
builds the debug library libimpir_bounds.so instead: the same units compiled with
-DIMPIR_BOUNDS, whose kernels check every index against its buffer (see impir_bounds_status).

    python -m paper_2509_06514_gb300.build [--verbose-ptxas] [--bounds]
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libimpir.so")
BUILD_BOUNDS = os.path.join(HERE, "_build_bounds")
LIB_BOUNDS = os.path.join(HERE, "libimpir_bounds.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = ["fused_q1.cu", "fused_q2.cu", "fused_q4.cu", "fused_q8.cu", "fused_q16.cu", "fused_add.cu", "setup.cu", "noalloc.cu", "aes_bench.cu", "combine.cu", "host_aes.cpp", "impir_host.cpp",
         "serve.cpp"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libimpir")


def _sources():
    return [os.path.join(CSRC, u) for u in UNITS]


def _deps():
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "impir.h"))
    return deps


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps() + [__file__])


def _compile(src: str, verbose_ptxas: bool, bounds: bool = False) -> str:
    obj = os.path.join(BUILD_BOUNDS if bounds else BUILD, os.path.basename(src) + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
           "-I", os.path.join(HERE, "..", "include"), "-c", src, "-o", obj]
    if bounds:
        cmd.append("-DIMPIR_BOUNDS")
    if verbose_ptxas and src.endswith(".cu"):
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    if verbose_ptxas:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose_ptxas: bool = False, bounds: bool = False) -> str:
    """Builds libimpir.so (or, with bounds=True, the debug library libimpir_bounds.so)."""
    lib = LIB_BOUNDS if bounds else LIB
    if not force and not verbose_ptxas and up_to_date(lib):
        return lib
    os.makedirs(BUILD_BOUNDS if bounds else BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=min(len(UNITS), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose_ptxas, bounds), _sources()))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    from . import workloads
    workloads.build_inputs()
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose_ptxas="--verbose-ptxas" in sys.argv, bounds="--bounds" in sys.argv))
