"""Autotuner for the pruning pass (K1).

Picks the 3D task depth (planes per task), the number of 3D pruning CTAs per
SM and the rows per 2D task by timing the lookup + pruning pass alone
(cubical_persistence_debug_prune) on the given inputs, and caches the winner
per GPU and shape bucket in a JSON file (default
~/.cache/cp_gb300/autotune.json, or $CP_AUTOTUNE_CACHE).  The pairs never
depend on these settings; only the time does.

    from paper_2606_04801_gb300 import autotune
    cfg = autotune.autotune([vol])      # tunes (or loads), then applies
"""
from __future__ import annotations

import ctypes
import json
import os
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib

ZCHUNK_3D, CTAS_PER_SM, ROWS_2D = 1, 2, 3
CAND_ZCHUNK = (16, 32, 64, 128, 256)
CAND_CTAS = (0, 2, 3)
CAND_ROWS = (16, 32, 64, 128)


def _cache_path() -> str:
    return os.environ.get("CP_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "cp_gb300", "autotune.json"))


def bucket(shapes: Sequence[Sequence[int]]) -> str:
    """Shape bucket: number of 2D/3D items and the powers of two of their sizes."""
    n2 = [int(np.prod(s)) for s in shapes if len(s) == 2]
    n3 = [int(np.prod(s)) for s in shapes if len(s) == 3]
    d3 = [int(s[0]) for s in shapes if len(s) == 3]

    def p2(v):
        return int(np.ceil(np.log2(max(1, v))))

    return f"2d:{len(n2)}x{p2(sum(n2))}|3d:{len(n3)}x{p2(sum(n3))}|depth:{p2(max(d3) if d3 else 0)}"


def current() -> dict:
    lib = _lib.load()
    return {"zchunk3d": lib.cp_get_tuning(ZCHUNK_3D), "ctas3d": lib.cp_get_tuning(CTAS_PER_SM),
            "rows2d": lib.cp_get_tuning(ROWS_2D)}


def apply(cfg: dict) -> None:
    lib = _lib.load()
    for key, name in ((ZCHUNK_3D, "zchunk3d"), (CTAS_PER_SM, "ctas3d"), (ROWS_2D, "rows2d")):
        if name in cfg and lib.cp_set_tuning(key, int(cfg[name])) != 0:
            raise ValueError(f"bad tuning value {name}={cfg[name]}")


def _time_prune(inputs: Sequence[torch.Tensor], repeats: int) -> float:
    lib = _lib.load()
    k = len(inputs)
    ptrs = (ctypes.c_void_p * k)(*[t.data_ptr() for t in inputs])
    ndims = (ctypes.c_int32 * k)(*[t.dim() for t in inputs])
    flat = []
    for t in inputs:
        flat += ([1] + list(t.shape)) if t.dim() == 2 else list(t.shape)
    dims = (ctypes.c_int64 * (3 * k))(*flat)
    wsb = lib.cubical_persistence_batched_workspace_size(k, ndims, dims, 0)
    ws = torch.empty(wsb, dtype=torch.uint8, device=inputs[0].device)
    stream = torch.cuda.current_stream(inputs[0].device)
    sp = ctypes.c_void_p(int(stream.cuda_stream))
    wp = ctypes.c_void_p(ws.data_ptr())

    def once():
        rc = lib.cubical_persistence_debug_prune(k, ptrs, ndims, dims, wp, wsb, 0, sp)
        if rc != 0:
            raise _lib.CpError(rc, "prune")

    once()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(repeats):
        once()
    e1.record(stream)
    torch.cuda.synchronize(inputs[0].device)
    return e0.elapsed_time(e1) / repeats


def tune(inputs: Sequence[torch.Tensor], repeats: int = 5) -> dict:
    """Time every candidate on these inputs; returns the fastest setting."""
    has2 = any(t.dim() == 2 for t in inputs)
    has3 = any(t.dim() == 3 for t in inputs)
    saved = current()
    best, best_ms = dict(saved), float("inf")
    trials = []
    try:
        for zc in CAND_ZCHUNK if has3 else (saved["zchunk3d"],):
            for ctas in CAND_CTAS if has3 else (saved["ctas3d"],):
                for rows in CAND_ROWS if has2 else (saved["rows2d"],):
                    cfg = {"zchunk3d": zc, "ctas3d": ctas, "rows2d": rows}
                    apply(cfg)
                    ms = _time_prune(inputs, repeats)
                    trials.append((ms, cfg))
                    if ms < best_ms:
                        best, best_ms = cfg, ms
    finally:
        apply(saved)
    best = dict(best)
    best["ms"] = best_ms
    best["trials"] = len(trials)
    return best


def autotune(inputs: Sequence[torch.Tensor], cache: Optional[str] = None, retune: bool = False) -> dict:
    """Load the cached setting for this GPU and shape bucket, or tune and cache it; then apply it."""
    path = cache or _cache_path()
    dev = inputs[0].device
    key = f"{torch.cuda.get_device_name(dev)}|{bucket([tuple(t.shape) for t in inputs])}"
    table = {}
    if os.path.exists(path):
        try:
            with open(path) as fh:
                table = json.load(fh)
        except Exception:
            table = {}
    if retune or key not in table:
        table[key] = tune(inputs)
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = f"{path}.{os.getpid()}.tmp"
            with open(tmp, "w") as fh:
                json.dump(table, fh, indent=1, sort_keys=True)
            os.replace(tmp, path)
        except OSError:
            pass
    apply(table[key])
    return dict(table[key], key=key)
