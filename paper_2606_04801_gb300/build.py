"""Build the in-tree shared library libcp_gb300.so for sm_103a.

nvcc compiles every kernel source for ``-gencode arch=compute_103a,code=sm_103a``
(one translation unit per process, in parallel); g++ compiles the host-side
lookup-table builder; nvcc links the shared library next to this file
(``_build/``).  Sources are rebuilt only when newer than their objects.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libcp_gb300.so")
CU = ["cp_prune.cu", "cp_sort.cu", "cp_uf.cu", "cp_emit.cu", "cp_api.cu", "cp_noalloc.cu", "cp_tfilt.cu", "cp_h1.cu"]
CPP = ["cp_lut.cpp"]
HEADERS = ["cp_common.cuh", "cp_grid.cuh", "cp_kernels.h", "cp_lut.h", os.path.join("..", "..", "include", "cubical_persistence.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, h) for h in HEADERS]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    nvcc = _nvcc()
    os.makedirs(OUT, exist_ok=True)
    jobs = []
    for f in CU:
        src, obj = os.path.join(CSRC, f), os.path.join(OUT, f.replace(".cu", ".o"))
        if force or _stale(obj, src):
            jobs.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-c", src, "-o", obj])
    for f in CPP:
        src, obj = os.path.join(CSRC, f), os.path.join(OUT, f.replace(".cpp", ".o"))
        if force or _stale(obj, src):
            jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"build failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(OUT, f.replace(".cu", ".o")) for f in CU] + [os.path.join(OUT, f.replace(".cpp", ".o")) for f in CPP]
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + f".{os.getpid()}.tmp"
        run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
