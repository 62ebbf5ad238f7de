"""CPU oracle for V- and T-filtration cubical persistence (H0 + top dimension,
and H1 of volumes).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product package never imports
this module, and this module imports nothing from the product package.

The arithmetic lives in ``cp_oracle.c`` (plain C, single thread, no pruning,
no lookup table); this file only compiles it with gcc and marshals arguments
through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cp_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libcp_oracle.so")
_lock = threading.Lock()
_lib = None

PAIR_DTYPE = np.dtype(
    [
        ("birth", np.float32),
        ("death", np.float32),
        ("birth_cell", np.int64),
        ("death_cell", np.int64),
        ("birth_pixel", np.int64),
        ("death_pixel", np.int64),
        ("dim", np.int32),
        ("pad", np.int32),
    ]
)

ERRORS = {-1: "bad argument", -2: "non-finite input", -3: "capacity", -4: "out of memory"}


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (gcc -O2, portable flags)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_persistence.restype = ctypes.c_int64
            lib.oracle_persistence.argtypes = [
                ctypes.c_void_p,
                ctypes.c_int,
                ctypes.c_void_p,
                ctypes.c_int,
                ctypes.c_void_p,
                ctypes.c_int64,
            ]
            lib.oracle_persistence_t.restype = ctypes.c_int64
            lib.oracle_persistence_t.argtypes = lib.oracle_persistence.argtypes
            lib.oracle_persistence_full.restype = ctypes.c_int64
            lib.oracle_persistence_full.argtypes = lib.oracle_persistence.argtypes
            lib.oracle_cell_key.restype = ctypes.c_int
            lib.oracle_cell_key.argtypes = [
                ctypes.c_void_p,
                ctypes.c_int,
                ctypes.c_void_p,
                ctypes.c_int64,
                ctypes.POINTER(ctypes.c_float),
                ctypes.POINTER(ctypes.c_int64),
                ctypes.POINTER(ctypes.c_int32),
            ]
            _lib = lib
    return _lib


def _call(fn, img, keep_zero):
    a = np.ascontiguousarray(img, dtype=np.float32)
    if a.ndim not in (2, 3):
        raise ValueError("image must be 2D or 3D")
    dims = np.asarray(a.shape, dtype=np.int64)
    n = fn(a.ctypes.data, a.ndim, dims.ctypes.data, int(keep_zero), None, 0)
    if n < 0:
        raise ValueError(f"oracle: {ERRORS.get(int(n), n)}")
    out = np.zeros(int(n), dtype=PAIR_DTYPE)
    m = fn(a.ctypes.data, a.ndim, dims.ctypes.data, int(keep_zero), out.ctypes.data, int(n))
    if m != n:
        raise RuntimeError("oracle: pair count changed between calls")
    return out


def persistence(img, keep_zero: bool = False) -> np.ndarray:
    """Persistence pairs of a 2D (H, W) or 3D (D, H, W) float32 image.

    Returns a structured array (PAIR_DTYPE) sorted by (dim, birth_cell).
    Cell indices are doubled-grid indices; the essential H0 class has
    death = +inf and death_cell = death_pixel = -1.
    """
    return _call(_load().oracle_persistence, img, keep_zero)


def persistence_full(img, keep_zero: bool = False) -> np.ndarray:
    """As ``persistence``, plus the H1 pairs of a volume (dim 1), from the
    column reduction of the square-edge boundary matrix.  Equal to
    ``persistence`` for a 2D image."""
    return _call(_load().oracle_persistence_full, img, keep_zero)


def persistence_t(img, keep_zero: bool = False) -> np.ndarray:
    """Persistence pairs of a 2D or 3D float32 image under the T-filtration
    (pixel values on the top cells; see ``cp_oracle.c``).

    Same output as ``persistence``; cells are indices in the doubled grid of
    the T-complex (extents 2n+1), pixels the top cells the cells enter with.
    """
    return _call(_load().oracle_persistence_t, img, keep_zero)


def cell_key(img, cell: int):
    """Refined key (f(m), m, dim) of one doubled-grid cell."""
    lib = _load()
    a = np.ascontiguousarray(img, dtype=np.float32)
    dims = np.asarray(a.shape, dtype=np.int64)
    fm = ctypes.c_float()
    m = ctypes.c_int64()
    d = ctypes.c_int32()
    rc = lib.oracle_cell_key(a.ctypes.data, a.ndim, dims.ctypes.data, int(cell), ctypes.byref(fm), ctypes.byref(m), ctypes.byref(d))
    if rc:
        raise ValueError("bad cell")
    return float(fm.value), int(m.value), int(d.value)
