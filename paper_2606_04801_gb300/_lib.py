"""ctypes binding of libcp_gb300.so (argument marshalling only).

Every function here forwards to the C-ABI declared in
include/cubical_persistence.h; no computation happens in Python.  Loading
fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB, LIB_CHECKED

CP_OK = 0
CP_ERR_ARG = -1
CP_ERR_NONFINITE = -2
CP_ERR_CAPACITY = -3
CP_ERR_CUDA = -4
CP_ERR_TIMEOUT = -5
CP_ERR_INTERNAL = -6
CP_MAX_ITEMS = 128

# The C struct cp_pair (32 bytes).
PAIR_DTYPE = np.dtype(
    [
        ("birth", np.float32),
        ("death", np.float32),
        ("birth_cell", np.int32),
        ("death_cell", np.int32),
        ("birth_pixel", np.int32),
        ("death_pixel", np.int32),
        ("dim", np.int32),
        ("item", np.int32),
    ]
)


class CpStats(ctypes.Structure):
    _fields_ = [
        ("n_pixels", ctypes.c_int64),
        ("h0_survivors", ctypes.c_int64),
        ("top_survivors", ctypes.c_int64),
        ("h0_roots", ctypes.c_int64),
        ("top_roots", ctypes.c_int64),
        ("h0_rounds", ctypes.c_int64),
        ("top_rounds", ctypes.c_int64),
        ("pairs", ctypes.c_int64),
        ("status", ctypes.c_uint32),
        ("mst_rounds", ctypes.c_uint32),
    ]


class CpSlabStats(ctypes.Structure):
    _fields_ = [
        (name, ctypes.c_int64 * 2)
        for name in ("survivors", "internal", "crossing", "committed", "final_pairs", "merged", "rounds_slab",
                     "rounds_merge")
    ]


# name -> (restype, argtypes); must match include/cubical_persistence.h
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_SIGS = {
    "cp_version": (ctypes.c_int, []),
    "cp_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "cp_lut_num_classes": (ctypes.c_int, [ctypes.c_int]),
    "cp_lut_lookup": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint32, _P, _P]),
    "cp_lut_check_layout": (ctypes.c_int, [_P]),
    "cubical_persistence_workspace_size": (ctypes.c_size_t, [ctypes.c_int, _P, _I64]),
    "cubical_persistence_2d": (ctypes.c_int, [_P, _P, _P, _I64, _P, _P, _P, ctypes.c_size_t, _I64, _P]),
    "cubical_persistence_3d": (ctypes.c_int, [_P, _P, _P, _I64, _P, _P, _P, ctypes.c_size_t, _I64, _P]),
    "cubical_persistence_slabs_workspace_size": (ctypes.c_size_t, [ctypes.c_int, _P, ctypes.c_int, _I64]),
    "cubical_persistence_slabs": (
        ctypes.c_int,
        [ctypes.c_int, _P, _P, ctypes.c_int, _P, _I64, _P, _P, _P, ctypes.c_size_t, _I64, _P,
         ctypes.POINTER(CpSlabStats)],
    ),
    "cubical_persistence_t_workspace_size": (ctypes.c_size_t, [ctypes.c_int, _P, _I64]),
    "cubical_persistence_t_2d": (ctypes.c_int, [_P, _P, _P, _I64, _P, _P, _P, ctypes.c_size_t, _I64, _P]),
    "cubical_persistence_t_3d": (ctypes.c_int, [_P, _P, _P, _I64, _P, _P, _P, ctypes.c_size_t, _I64, _P]),
    "cubical_persistence_t_batched_workspace_size": (ctypes.c_size_t, [ctypes.c_int, _P, _P, _I64]),
    "cubical_persistence_t_batched": (
        ctypes.c_int,
        [ctypes.c_int, _P, _P, _P, _P, _I64, _P, _P, _P, ctypes.c_size_t, _I64, _P],
    ),
    "cubical_persistence_batched_workspace_size": (ctypes.c_size_t, [ctypes.c_int, _P, _P, _I64]),
    "cubical_persistence_batched": (
        ctypes.c_int,
        [ctypes.c_int, _P, _P, _P, _P, _I64, _P, _P, _P, ctypes.c_size_t, _I64, _P],
    ),
    "cubical_persistence_full_workspace_size": (ctypes.c_size_t, [ctypes.c_int, _P, _I64, _I64]),
    "cubical_persistence_full_3d": (ctypes.c_int, [_P, _P, _P, _I64, _P, _P, _P, ctypes.c_size_t, _I64, _I64, _P]),
    "cubical_persistence_full_batched_workspace_size": (ctypes.c_size_t, [ctypes.c_int, _P, _P, _I64, _I64]),
    "cubical_persistence_full_batched": (
        ctypes.c_int,
        [ctypes.c_int, _P, _P, _P, _P, _I64, _P, _P, _P, ctypes.c_size_t, _I64, _I64, _P],
    ),
    "cubical_persistence_full_info": (
        ctypes.c_int,
        [_P, ctypes.c_int, _P, _P, _I64, _I64, _P, ctypes.c_int, _P],
    ),
    "cubical_persistence_stats": (ctypes.c_int, [_P, ctypes.POINTER(CpStats), _P]),
    "cubical_persistence_backward_workspace_size": (ctypes.c_size_t, [_I64]),
    "cubical_persistence_backward": (ctypes.c_int, [_P, _I64, _P, _P, _P, _P, _I64, _P, ctypes.c_size_t, _P]),
    "cubical_persistence_loss_backward_workspace_size": (ctypes.c_size_t, [_I64]),
    "cubical_persistence_loss_backward": (
        ctypes.c_int,
        [_P, _I64, _P, ctypes.c_float, _P, _P, _P, _I64, _P, ctypes.c_size_t, _P],
    ),
    "cubical_persistence_backward_noalloc_max_pixels": (ctypes.c_int64, []),
    "cubical_persistence_backward_noalloc": (ctypes.c_int, [_P, _I64, _P, _P, _P, _P, _I64, _P]),
    "cubical_persistence_uf_trace": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int, _P]),
    "cubical_persistence_uf_trace2": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, ctypes.c_int, _P]),
    "cubical_persistence_debug_prune": (ctypes.c_int, [ctypes.c_int, _P, _P, _P, _P, ctypes.c_size_t, _I64, _P]),
    "cubical_persistence_debug_layout": (ctypes.c_int, [ctypes.c_int, _P, _P, _I64, _P, ctypes.c_int]),
    "cubical_persistence_debug_wait_timeout": (ctypes.c_int, [_P, ctypes.c_size_t, _I64, _P]),
    "cp_set_tuning": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    "cp_get_tuning": (ctypes.c_int, [ctypes.c_int]),
    "cp_launch_count": (ctypes.c_longlong, []),
    "cp_profile": (ctypes.c_int, [ctypes.c_int]),
    "cp_stage_times": (ctypes.c_int, [_P, ctypes.c_int]),
}

_lib = None


def load():
    """Load the library (it must have been built: see paper_2606_04801_gb300.build).
    CP_LIB_VARIANT=checked in the environment loads the bounds-checked build."""
    global _lib
    if _lib is None:
        path = LIB_CHECKED if os.environ.get("CP_LIB_VARIANT") == "checked" else LIB
        if not os.path.exists(path):
            raise RuntimeError(
                f"{os.path.basename(path)} is missing ({path}); build it first with "
                "`python -c 'import __graft_entry__ as g; g.build()'` or `python -m paper_2606_04801_gb300.build`"
            )
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


def error_string(code: int) -> str:
    return load().cp_error_string(int(code)).decode()


class CpError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = int(code)
        super().__init__(f"{what}: {error_string(code)} ({code})" if what else f"{error_string(code)} ({code})")
