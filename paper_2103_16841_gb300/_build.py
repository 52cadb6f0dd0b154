"""Builds the CUDA library libstbem.so in-tree for sm_103a with nvcc.

Each translation unit is compiled in parallel; the shared object is linked
with nvcc. Nothing is installed outside the package directory.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libstbem.so")
SOURCES = ["stbem_core.cu", "stbem_matvec.cu", "stbem_solver.cu", "stbem_gmres.cu", "stbem_capi.cu", "stbem_noalloc.cu", "stbem_server.cu", "stbem_batch.cu", "stbem_peaks.cu", "stbem_spmm_tc.cu", "stbem_tune.cu", "stbem_littree.cu"]
HEADERS = ["stbem_quad.cuh", "stbem_internal.h", "stbem_tc.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# The quadrature translation unit: FP32 division and square root to within a
# few ulp (the hardware approximations). The mixed quadrature's error target
# is 1e-7 relative, formed from cancellation-free expressions, and the FP64
# arithmetic (cone geometry, the FP64 path, the sparsity contract) is
# unaffected by these flags. (Flushing FP32 denormals as well measured slower
# for both the quadrature and the pattern kernels.)
SOURCE_FLAGS = {"stbem_core.cu": ["-prec-div=false", "-prec-sqrt=false"]}


def nvcc() -> str:
    for c in [os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")]:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags(extra=()):
    return ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
            "-I", os.path.join(HERE, "..", "include"), *extra]


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src, os.path.abspath(__file__)] + [os.path.join(CSRC, h) for h in HEADERS] + \
        [os.path.join(HERE, "..", "include", "stbem.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nv = nvcc()
    jobs = []
    objs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, src):
            extra = (["-Xptxas", "-v"] if ptxas_v else []) + SOURCE_FLAGS.get(s, [])
            jobs.append([nv, *_flags(extra), "-c", src, "-o", obj])

    def run(cmd):
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + p.stdout + p.stderr)
        return p.stdout + p.stderr

    logs = []
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 1)) as ex:
            logs = list(ex.map(run, jobs))
    if jobs or force or not os.path.exists(LIB):
        tmp = LIB + f".{os.getpid()}.tmp"
        run([nv, "-shared", *ARCH, "-o", tmp, *objs, "-lcudart"])
        os.replace(tmp, LIB)
    if verbose:
        for l in logs:
            print(l)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="--ptxas" in sys.argv))
