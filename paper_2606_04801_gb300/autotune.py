"""Autotuner for the pruning pass (K1) and the union-find design.

Picks the 3D task depth (planes per task), the number of 3D pruning CTAs per
SM and the rows per 2D task by timing the lookup + pruning pass alone
(cubical_persistence_debug_prune) on the given inputs; then the union-find
design (reservation rounds over every survivor, or Borůvka's spanning forest
first and the rounds over its edges) by timing whole forward calls with
each.  Which design is faster depends on the data (i.i.d. noise leaves many
survivors that close cycles, which Borůvka drops early; smooth fields leave
few), so the cache key holds the survivor fraction's power of two besides
the shape bucket.  The winners are cached per GPU and key in a JSON file
(default ~/.cache/cp_gb300/autotune.json, or $CP_AUTOTUNE_CACHE).  The pairs
never depend on these settings; only the time does.

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

ZCHUNK_3D, CTAS_PER_SM, ROWS_2D, UF_VARIANT = 1, 2, 3, 7
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
            "rows2d": lib.cp_get_tuning(ROWS_2D), "uf_variant": lib.cp_get_tuning(UF_VARIANT)}


def apply(cfg: dict) -> None:
    lib = _lib.load()
    for key, name in ((ZCHUNK_3D, "zchunk3d"), (CTAS_PER_SM, "ctas3d"), (ROWS_2D, "rows2d"),
                      (UF_VARIANT, "uf_variant")):
        if name in cfg and lib.cp_set_tuning(key, int(cfg[name])) != 0:
            raise ValueError(f"bad tuning value {name}={cfg[name]}")


def _marshal(inputs: Sequence[torch.Tensor]):
    k = len(inputs)
    ptrs = (ctypes.c_void_p * k)(*[t.data_ptr() for t in inputs])
    ndims = (ctypes.c_int32 * k)(*[t.dim() for t in inputs])
    flat = []
    for t in inputs:
        flat += ([1] + list(t.shape)) if t.dim() == 2 else list(t.shape)
    dims = (ctypes.c_int64 * (3 * k))(*flat)
    return k, ptrs, ndims, dims


def _time_prune(inputs: Sequence[torch.Tensor], repeats: int) -> float:
    lib = _lib.load()
    k, ptrs, ndims, dims = _marshal(inputs)
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


def survivor_fraction(inputs: Sequence[torch.Tensor]) -> float:
    """Survivors of the pruning pass (both lists) per voxel, from one
    forward call."""
    lib = _lib.load()
    k, ptrs, ndims, dims = _marshal(inputs)
    wsb = lib.cubical_persistence_batched_workspace_size(k, ndims, dims, 0)
    ws = torch.empty(wsb, dtype=torch.uint8, device=inputs[0].device)
    n = sum(int(t.numel()) for t in inputs)
    cap = 2 * n + 65536
    out = torch.empty((cap, 8), dtype=torch.int32, device=inputs[0].device)
    sp = ctypes.c_void_p(int(torch.cuda.current_stream(inputs[0].device).cuda_stream))
    cnt = ctypes.c_int64(0)
    rc = lib.cubical_persistence_batched(k, ptrs, ndims, dims, ctypes.c_void_p(out.data_ptr()), cap, ctypes.byref(cnt),
                                         None, ctypes.c_void_p(ws.data_ptr()), wsb, 0, sp)
    st = _lib.CpStats()
    lib.cubical_persistence_stats(ctypes.c_void_p(ws.data_ptr()), ctypes.byref(st), sp)
    if rc not in (0, _lib.CP_ERR_CAPACITY):
        raise _lib.CpError(rc, "forward")
    return (st.h0_survivors + st.top_survivors) / max(1, n)


def _time_forward(inputs: Sequence[torch.Tensor], repeats: int) -> float:
    """Whole forward calls on the inputs (the union-find design in force when
    the workspace is sized)."""
    lib = _lib.load()
    k, ptrs, ndims, dims = _marshal(inputs)
    n = sum(int(t.numel()) for t in inputs)
    ms = 0
    for _ in range(4):  # grow the survivor bound as the binding does
        wsb = lib.cubical_persistence_batched_workspace_size(k, ndims, dims, ms)
        ws = torch.empty(wsb, dtype=torch.uint8, device=inputs[0].device)
        cap = 2 * n + 65536
        out = torch.empty((cap, 8), dtype=torch.int32, device=inputs[0].device)
        stream = torch.cuda.current_stream(inputs[0].device)
        sp = ctypes.c_void_p(int(stream.cuda_stream))
        wp = ctypes.c_void_p(ws.data_ptr())
        op = ctypes.c_void_p(out.data_ptr())
        cnt = ctypes.c_int64(0)
        rc = lib.cubical_persistence_batched(k, ptrs, ndims, dims, op, cap, ctypes.byref(cnt), None, wp, wsb, ms, sp)
        if rc == _lib.CP_ERR_CAPACITY:
            st = _lib.CpStats()
            lib.cubical_persistence_stats(wp, ctypes.byref(st), sp)
            ms = int(1.25 * max(st.h0_survivors, st.top_survivors, 2 * st.h0_roots, 2 * st.top_roots)) + 65536
            continue
        if rc != 0:
            raise _lib.CpError(rc, "forward")
        break
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(repeats):
        lib.cubical_persistence_batched(k, ptrs, ndims, dims, op, cap, None, None, wp, wsb, ms, sp)
    e1.record(stream)
    torch.cuda.synchronize(inputs[0].device)
    st = _lib.CpStats()
    if lib.cubical_persistence_stats(wp, ctypes.byref(st), sp) != 0:
        raise _lib.CpError(st.status, "forward")
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
                    cfg = {"zchunk3d": zc, "ctas3d": ctas, "rows2d": rows, "uf_variant": saved["uf_variant"]}
                    apply(cfg)
                    ms = _time_prune(inputs, repeats)
                    trials.append((ms, cfg))
                    if ms < best_ms:
                        best, best_ms = cfg, ms
        # the union-find design, on whole forward calls with the best pruning setting
        uf_ms = {}
        for var in (0, 1):
            cfg = dict(best, uf_variant=var)
            apply(cfg)
            uf_ms[var] = _time_forward(inputs, repeats)
        best = dict(best, uf_variant=min(uf_ms, key=uf_ms.get))
    finally:
        apply(saved)
    best = dict(best)
    best["ms"] = best_ms
    best["forward_ms"] = {str(v): round(t, 4) for v, t in uf_ms.items()}
    best["trials"] = len(trials) + 2
    return best


def autotune(inputs: Sequence[torch.Tensor], cache: Optional[str] = None, retune: bool = False) -> dict:
    """Load the cached setting for this GPU and shape bucket, or tune and cache it; then apply it."""
    path = cache or _cache_path()
    dev = inputs[0].device
    frac = survivor_fraction(inputs)
    sbin = int(np.floor(np.log2(max(frac, 1e-9))))
    key = f"{torch.cuda.get_device_name(dev)}|{bucket([tuple(t.shape) for t in inputs])}|surv:{sbin}"
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
