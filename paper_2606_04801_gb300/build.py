"""Build the in-tree shared library libcp_gb300.so for sm_103a.

nvcc compiles every kernel source for ``-gencode arch=compute_103a,code=sm_103a``
(one translation unit per process, in parallel); g++ compiles the host-side
lookup-table builder; nvcc links the shared library next to this file
(``_build/``).  Sources are rebuilt only when newer than their objects.

``checked=True`` builds the same sources with ``-DCP_CHECKED`` into
``_build_checked/libcp_gb300_checked.so``: every data-dependent index into a
device array is tested against the array's size first, and a bad one sets a
status bit (the call returns CP_ERR_INTERNAL) instead of being used.  The
binding loads it when the environment has CP_LIB_VARIANT=checked.
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
OUT_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(OUT_CHECKED, "libcp_gb300_checked.so")
CU = ["cp_prune.cu", "cp_sort.cu", "cp_uf.cu", "cp_emit.cu", "cp_api.cu", "cp_noalloc.cu", "cp_tfilt.cu", "cp_h1.cu", "cp_slab.cu", "cp_boruvka.cu"]
CPP = ["cp_lut.cpp"]
HEADERS = ["cp_common.cuh", "cp_grid.cuh", "cp_kernels.h", "cp_lut.h", "cp_mask3.cuh", "cp_pairs.cuh",
           os.path.join("..", "..", "include", "cubical_persistence.h")]
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


def _jobs(nvcc: str, out: str, defs, force: bool):
    jobs = []
    for f in CU:
        src, obj = os.path.join(CSRC, f), os.path.join(out, f.replace(".cu", ".o"))
        if force or _stale(obj, src):
            jobs.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", *defs, "-Xcompiler", "-fPIC", "-c", src, "-o", obj])
    for f in CPP:
        src, obj = os.path.join(CSRC, f), os.path.join(out, f.replace(".cpp", ".o"))
        if force or _stale(obj, src):
            jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-c", src, "-o", obj])
    return jobs


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Builds the library (checked=True: the bounds-checked variant) and
    returns its path."""
    nvcc = _nvcc()
    out, lib = (OUT_CHECKED, LIB_CHECKED) if checked else (OUT, LIB)
    os.makedirs(out, exist_ok=True)
    jobs = _jobs(nvcc, out, ["-DCP_CHECKED"] if checked else [], force)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"build failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(out, f.replace(".cu", ".o")) for f in CU] + [os.path.join(out, f.replace(".cpp", ".o")) for f in CPP]
    if force or jobs or not os.path.exists(lib):
        tmp = lib + f".{os.getpid()}.tmp"
        run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs])
        os.replace(tmp, lib)
    return lib


def build_all(force: bool = False) -> None:
    """Both variants, their translation units compiled in parallel."""
    with ThreadPoolExecutor(max_workers=2) as ex:
        list(ex.map(lambda c: build(force=force, checked=c), (False, True)))


if __name__ == "__main__":
    print(build(verbose=True))
