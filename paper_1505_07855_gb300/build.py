"""Build libaln_gb300.so in-tree: nvcc for the CUDA sources (sm_103a only), g++
for the host index builder, linked into one shared library."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libaln_gb300.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["aln_kernels.cu", "aln_capi.cu", "index_gpu.cu", "aln_pair.cu"]
CPP_SOURCES = ["index_build.cpp", "aln_server.cpp"]
HEADERS = ["aln_device.cuh", "aln_search.cuh", "aln_flat.cuh", "aln_internal.h", "aln_scan.cuh"]


def _newer(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, extra: list[str], out_dir: str = BUILD) -> str:
    obj = os.path.join(out_dir, os.path.basename(src) + ".o")
    deps = [os.path.join(CSRC, src)] + [os.path.join(CSRC, h) for h in HEADERS] + \
        [os.path.join(INCLUDE, "aln_gb300.h")]
    if not _newer(obj, deps):
        return obj
    if src.endswith(".cu"):
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-I", INCLUDE, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    else:
        cmd = ["g++", "-O3", "-std=c++17", "-fPIC", "-pthread", "-Wall", "-I", INCLUDE,
               "-I", os.path.join(CUDA_HOME, "include"), *extra,
               "-c", os.path.join(CSRC, src), "-o", obj]
    subprocess.run(cmd, check=True)
    return obj


def build(force: bool = False, verbose: bool = False, stats: bool = False, variant: str = "",
          defines: tuple = ()) -> str:
    """Compile every source for sm_103a and link the library; returns its path.
    stats=True builds the instrumented variant (event counters) into _build/stats;
    variant/defines build a tuning variant into _build/<variant>."""
    out_dir = os.path.join(BUILD, "stats" if stats else variant) if (stats or variant) else BUILD
    lib = os.path.join(out_dir, "libaln_gb300.so")
    if force and os.path.isdir(out_dir):
        shutil.rmtree(out_dir)
    os.makedirs(out_dir, exist_ok=True)
    srcs = CU_SOURCES + CPP_SOURCES
    defs = (["-DALN_STATS"] if stats else []) + [f"-D{d}" for d in defines]
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(lambda s: _compile(s, defs + (["-Xptxas", "-v"] if verbose and s.endswith(".cu") else []),
                                              out_dir), srcs))
    if _newer(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [NVCC, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
               "-Xlinker", "-rpath", "-Xlinker", os.path.join(CUDA_HOME, "lib64"), "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
