"""Builds libphylograd.so in-tree with nvcc for sm_103a (GB300).

Each .cu file under csrc/ is compiled to an object in parallel, then linked into one shared
library against the shared CUDA runtime (so a process that already loaded PyTorch's runtime
uses that one).  ``python -m paper_1905_12146_gb300.build`` or ``build()``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJDIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libphylograd.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# code-generation flags of every translation unit (explicit fmaf calls are the only contractions)
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libphylograd.so")


def _cuda_libdir(nvcc: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")


def _compile(nvcc: str, src: str, extra: list[str]) -> str:
    obj = os.path.join(OBJDIR, os.path.basename(src) + ".o")
    cmd = [nvcc, *ARCH, *FLAGS, "-Xcompiler", "-fPIC,-O2",
           "-I", INCLUDE, "-I", CSRC, *extra, "-c", src, "-o", obj]
    subprocess.run(cmd, check=True)
    return obj


def _stale(sources: list[str]) -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")) + [__file__]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    if not force and not _stale(sources):
        return LIB
    nvcc = _nvcc()
    os.makedirs(OBJDIR, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(sources), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(lambda s: _compile(nvcc, s, extra), sources))
    tmp = LIB + f".{os.getpid()}.tmp"
    libdir = _cuda_libdir(nvcc)
    subprocess.run([nvcc, *ARCH, "-shared", "-cudart", "shared", "-Xlinker", "--no-undefined", "-o", tmp, *objs,
                    "-Xlinker", f"-rpath,{libdir}"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose_ptxas="-v" in sys.argv))
