"""PyTorch-facing API.  PyTorch supplies device memory and streams; every
step of the computation runs in the library's CUDA kernels.

    d = persistence(img)               # img: CUDA float32 (H, W) or (D, H, W)
    d.birth, d.death, d.dim, ...       # views of the pairs on the device
    d.numpy()                          # structured array (cp_pair layout)

    ds = persistence_batched([img0, vol1, ...])   # pairs carry `item`

    birth, death, dim = diagram(img)   # differentiable in img (autograd)
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import CP_ERR_CAPACITY, CP_OK, CpError, CpStats, PAIR_DTYPE


def _stream_ptr(device) -> int:
    return int(torch.cuda.current_stream(device).cuda_stream)


def _check_image(img: torch.Tensor, min_extent: int = 2):
    if not isinstance(img, torch.Tensor) or not img.is_cuda:
        raise TypeError("image must be a CUDA tensor")
    if img.dtype != torch.float32:
        raise TypeError("image must be float32")
    if img.dim() not in (2, 3):
        raise ValueError("image must be 2D (H, W) or 3D (D, H, W)")
    if any(s < min_extent for s in img.shape):
        raise ValueError(f"every axis must be at least {min_extent} long")


@dataclass
class Diagram:
    """Persistence pairs on the device: raw is an int32 (P, 8) view of cp_pair records."""

    raw: torch.Tensor
    stats: Optional[dict] = None

    def __len__(self):
        return int(self.raw.shape[0])

    @property
    def birth(self):
        return self.raw[:, 0].view(torch.float32)

    @property
    def death(self):
        return self.raw[:, 1].view(torch.float32)

    @property
    def birth_cell(self):
        return self.raw[:, 2]

    @property
    def death_cell(self):
        return self.raw[:, 3]

    @property
    def birth_pixel(self):
        return self.raw[:, 4]

    @property
    def death_pixel(self):
        return self.raw[:, 5]

    @property
    def dim(self):
        return self.raw[:, 6]

    @property
    def item(self):
        return self.raw[:, 7]

    def numpy(self) -> np.ndarray:
        return self.raw.contiguous().cpu().numpy().view(PAIR_DTYPE).reshape(-1)


def _stats(ws: torch.Tensor) -> dict:
    st = CpStats()
    rc = _lib.load().cubical_persistence_stats(
        ctypes.c_void_p(ws.data_ptr()), ctypes.byref(st), ctypes.c_void_p(_stream_ptr(ws.device))
    )
    d = {k: int(getattr(st, k)) for k, _ in CpStats._fields_ if k != "pad"}
    d["rc"] = int(rc)
    return d


def _grow(st: dict, ms: int, n_total: int) -> int:
    need = max(st["h0_survivors"], st["top_survivors"], 2 * st["h0_roots"], 2 * st["top_roots"], ms)
    return int(need * 1.25) + 65536


def persistence(img: torch.Tensor, max_survivors: int = 0, with_stats: bool = False, filtration: str = "V") -> Diagram:
    """Exact H0 and top-dimension pairs of one image or volume (sorted by (dim, birth cell)).

    filtration "V": pixels are the vertices, a cell takes the largest value of
    its vertices.  "T": pixels are the top cells, a cell takes the smallest
    value of the top cells that contain it (cells then index the T doubled
    grid, extents 2n+1; every extent may be 1)."""
    if filtration not in ("V", "T"):
        raise ValueError("filtration must be 'V' or 'T'")
    _check_image(img, min_extent=1 if filtration == "T" else 2)
    lib = _lib.load()
    img = img.contiguous()
    nd = img.dim()
    dims = (ctypes.c_int64 * nd)(*img.shape)
    n = img.numel()
    tmode = filtration == "T"
    if tmode:
        fn = lib.cubical_persistence_t_2d if nd == 2 else lib.cubical_persistence_t_3d
        wsize = lib.cubical_persistence_t_workspace_size
        n_all = n + int(np.prod([s + 1 for s in img.shape]))
        n_j = int(np.prod([s + 2 for s in img.shape]))
    else:
        fn = lib.cubical_persistence_2d if nd == 2 else lib.cubical_persistence_3d
        wsize = lib.cubical_persistence_workspace_size
        n_all = n + int(np.prod([s - 1 for s in img.shape])) + 1
        n_j = n
    ms = int(max_survivors)
    for _ in range(4):
        ws_bytes = wsize(nd, dims, ms)
        if ws_bytes == 0:
            raise CpError(_lib.CP_ERR_ARG, "workspace size")
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=img.device)
        eff = ms if ms > 0 else n_j // 2 + 65536
        cap = min(n_all, eff + 4096)
        out = torch.empty((cap, 8), dtype=torch.int32, device=img.device)
        cnt = ctypes.c_int64(0)
        rc = fn(
            ctypes.c_void_p(img.data_ptr()), dims, ctypes.c_void_p(out.data_ptr()), cap, ctypes.byref(cnt), None,
            ctypes.c_void_p(ws.data_ptr()), ws_bytes, ms, ctypes.c_void_p(_stream_ptr(img.device)),
        )
        if rc == CP_ERR_CAPACITY:
            ms = _grow(_stats(ws), eff, n_j)
            continue
        if rc != CP_OK:
            raise CpError(rc, "cubical_persistence" + ("_t" if tmode else ""))
        return Diagram(out[: cnt.value], _stats(ws) if with_stats else None)
    raise CpError(CP_ERR_CAPACITY, "cubical_persistence (after growing the workspace)")


def persistence_slabs(img: torch.Tensor, n_slabs: int, max_survivors: int = 0) -> Diagram:
    """The pairs of ``persistence(img)``, with the union-finds split into
    ``n_slabs`` slabs along the slowest axis: each slab's union-find over the
    survivors inside it, then one union-find over what the slabs committed and
    the survivors between slabs.  ``stats`` holds the split's counts
    (per list: [H0, top dimension])."""
    _check_image(img)
    if int(n_slabs) < 1:
        raise ValueError("n_slabs must be at least 1")
    lib = _lib.load()
    img = img.contiguous()
    nd = img.dim()
    dims = (ctypes.c_int64 * nd)(*img.shape)
    n = img.numel()
    n_all = n + int(np.prod([s - 1 for s in img.shape])) + 1
    ms = int(max_survivors)
    for _ in range(4):
        ws_bytes = lib.cubical_persistence_slabs_workspace_size(nd, dims, int(n_slabs), ms)
        if ws_bytes == 0:
            raise CpError(_lib.CP_ERR_ARG, "slabs workspace size")
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=img.device)
        eff = ms if ms > 0 else n // 2 + 65536
        cap = min(n_all, eff + 4096)
        out = torch.empty((cap, 8), dtype=torch.int32, device=img.device)
        cnt = ctypes.c_int64(0)
        sst = _lib.CpSlabStats()
        rc = lib.cubical_persistence_slabs(
            nd, ctypes.c_void_p(img.data_ptr()), dims, int(n_slabs), ctypes.c_void_p(out.data_ptr()), cap,
            ctypes.byref(cnt), None, ctypes.c_void_p(ws.data_ptr()), ws_bytes, ms,
            ctypes.c_void_p(_stream_ptr(img.device)), ctypes.byref(sst),
        )
        if rc == CP_ERR_CAPACITY:
            st = _stats(ws)
            # the two survivor lists sit side by side in the scratch lists
            ms = max(_grow(st, eff, n), int(1.25 * (st["h0_survivors"] + st["top_survivors"])) + 65536)
            continue
        if rc != CP_OK:
            raise CpError(rc, "cubical_persistence_slabs")
        stats = {k: [int(v) for v in getattr(sst, k)] for k, _ in _lib.CpSlabStats._fields_}
        return Diagram(out[: cnt.value], stats)
    raise CpError(CP_ERR_CAPACITY, "cubical_persistence_slabs (after growing the workspace)")


def persistence_batched(imgs: Sequence[torch.Tensor], max_survivors: int = 0, with_stats: bool = False,
                        filtration: str = "V") -> Diagram:
    """Pairs of many images and volumes in one pass; each pair carries its item index.
    filtration as for persistence()."""
    if not imgs:
        raise ValueError("empty batch")
    if filtration not in ("V", "T"):
        raise ValueError("filtration must be 'V' or 'T'")
    tmode = filtration == "T"
    lib = _lib.load()
    imgs = [im.contiguous() for im in imgs]
    for im in imgs:
        _check_image(im, min_extent=1 if tmode else 2)
    dev = imgs[0].device
    k = len(imgs)
    if k > _lib.CP_MAX_ITEMS:
        raise ValueError(f"at most {_lib.CP_MAX_ITEMS} items per call")
    ptrs = (ctypes.c_void_p * k)(*[im.data_ptr() for im in imgs])
    ndims = (ctypes.c_int32 * k)(*[im.dim() for im in imgs])
    flat = []
    for im in imgs:
        flat += ([1] + list(im.shape)) if im.dim() == 2 else list(im.shape)
    dims = (ctypes.c_int64 * (3 * k))(*flat)
    if tmode:
        n = sum(int(np.prod([s + 2 for s in im.shape])) for im in imgs)  # the dual images' vertices
        t = sum(im.numel() + int(np.prod([s + 1 for s in im.shape])) for im in imgs)
        wsize, fn = lib.cubical_persistence_t_batched_workspace_size, lib.cubical_persistence_t_batched
    else:
        n = sum(im.numel() for im in imgs)
        t = n + sum(int(np.prod([s - 1 for s in im.shape])) + 1 for im in imgs)
        wsize, fn = lib.cubical_persistence_batched_workspace_size, lib.cubical_persistence_batched
    ms = int(max_survivors)
    for _ in range(4):
        ws_bytes = wsize(k, ndims, dims, ms)
        if ws_bytes == 0:
            raise CpError(_lib.CP_ERR_ARG, "batched workspace size")
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        eff = ms if ms > 0 else n // 2 + 65536
        cap = min(t, eff + 2 * k + 4096)
        out = torch.empty((cap, 8), dtype=torch.int32, device=dev)
        cnt = ctypes.c_int64(0)
        rc = fn(
            k, ptrs, ndims, dims, ctypes.c_void_p(out.data_ptr()), cap, ctypes.byref(cnt), None,
            ctypes.c_void_p(ws.data_ptr()), ws_bytes, ms, ctypes.c_void_p(_stream_ptr(dev)),
        )
        if rc == CP_ERR_CAPACITY:
            ms = _grow(_stats(ws), eff, n)
            continue
        if rc != CP_OK:
            raise CpError(rc, "cubical_persistence_batched" + ("_t" if tmode else ""))
        return Diagram(out[: cnt.value], _stats(ws) if with_stats else None)
    raise CpError(CP_ERR_CAPACITY, "cubical_persistence_batched (after growing the workspace)")


# Volumes beyond this many voxels (in all) need allow_large=True for H1: the
# cross-star rounds grow with the area of the longest-lived loops, not with
# the voxel count (smooth fields, one GB300: 0.11 s at 128^3, 0.84 s at
# 256^3; at 512^3 the growing columns outran a 45 GB workspace).  The device
# stops the rounds once cp_get_tuning(CP_TUNE_H1_BUDGET_MS) is spent, whatever
# the size.
H1_PRACTICAL_VOXELS = 256 ** 3


def _full_call(imgs: Sequence[torch.Tensor], single: bool, max_survivors: int, pool_entries: int,
               with_stats: bool, allow_large: bool = False) -> Diagram:
    """The whole diagram (H0, H1 of the volumes, top dimension) of one volume
    (single) or of a batch; grows the survivor bound, the column pool and the
    output until they fit."""
    nvol = sum(im.numel() for im in imgs if im.dim() == 3)
    if nvol > H1_PRACTICAL_VOXELS and not allow_large:
        raise ValueError(
            f"H1 of {nvol} voxels: above the practical bound of {H1_PRACTICAL_VOXELS} voxels "
            "(pass allow_large=True; the rounds stop with CP_ERR_TIMEOUT once the H1 time budget is spent)")
    lib = _lib.load()
    dev = imgs[0].device
    k = len(imgs)
    ptrs = (ctypes.c_void_p * k)(*[im.data_ptr() for im in imgs])
    ndims = (ctypes.c_int32 * k)(*[im.dim() for im in imgs])
    flat = []
    for im in imgs:
        flat += ([1] + list(im.shape)) if im.dim() == 2 else list(im.shape)
    dims = (ctypes.c_int64 * (3 * k))(*flat)
    n = sum(im.numel() for im in imgs)
    bound = 0  # pairs before the zero-persistence filter: every edge and top cell, plus one
    for im in imgs:
        sh = list(im.shape)
        edges = sum(int(np.prod([s - (1 if a == b else 0) for b, s in enumerate(sh)])) for a in range(len(sh)))
        bound += edges + int(np.prod([s - 1 for s in sh])) + 1
    ms, pool = int(max_survivors), int(pool_entries)
    cap = min(bound, n + 2 * k + 4096)
    sp = ctypes.c_void_p(_stream_ptr(dev))
    for _ in range(8):
        if single:
            ws_bytes = lib.cubical_persistence_full_workspace_size(3, dims, ms, pool)
        else:
            ws_bytes = lib.cubical_persistence_full_batched_workspace_size(k, ndims, dims, ms, pool)
        if ws_bytes == 0:
            raise CpError(_lib.CP_ERR_ARG, "full workspace size")
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        out = torch.empty((cap, 8), dtype=torch.int32, device=dev)
        cnt = ctypes.c_int64(0)
        wsp = ctypes.c_void_p(ws.data_ptr())
        if single:
            rc = lib.cubical_persistence_full_3d(
                ctypes.c_void_p(imgs[0].data_ptr()), dims, ctypes.c_void_p(out.data_ptr()), cap, ctypes.byref(cnt),
                None, wsp, ws_bytes, ms, pool, sp,
            )
        else:
            rc = lib.cubical_persistence_full_batched(
                k, ptrs, ndims, dims, ctypes.c_void_p(out.data_ptr()), cap, ctypes.byref(cnt), None, wsp, ws_bytes,
                ms, pool, sp,
            )
        if rc == CP_ERR_CAPACITY:
            grew = False
            info = (ctypes.c_int64 * 4)()  # the H1 stage of this call (its layout needs this call's bounds)
            info_rc = lib.cubical_persistence_full_info(wsp, k, ndims, dims, ms, pool, info, 4, sp)
            st = _stats(ws)
            eff = ms if ms > 0 else n // 2 + 65536
            need = max(st["h0_survivors"], st["top_survivors"], 2 * st["h0_roots"], 2 * st["top_roots"])
            if need > eff:
                ms = _grow(st, eff, n)
                grew = True
            if info_rc == CP_OK and info[2] > info[3]:
                pool = 2 * max(int(info[2]), int(info[3]))
                grew = True
            if cnt.value > cap:
                cap = int(cnt.value) + 1024
                grew = True
            if not grew:
                raise CpError(rc, "cubical_persistence_full")
            continue
        if rc != CP_OK:
            raise CpError(rc, "cubical_persistence_full")
        return Diagram(out[: cnt.value], _stats(ws) if with_stats else None)
    raise CpError(CP_ERR_CAPACITY, "cubical_persistence_full (after growing the workspace)")


def persistence_full(img: torch.Tensor, max_survivors: int = 0, pool_entries: int = 0,
                     with_stats: bool = False, allow_large: bool = False) -> Diagram:
    """Every dimension of one volume: H0, H1 and H2 pairs (V-filtration,
    sorted by (dim, birth cell)); a 2D image gets its plain diagram.  H1 comes
    from the F2 reduction of the squares not paired in H2 over the edges not
    paired in H0, on the device; pool_entries sizes its column pool (0: the
    default, grown on demand).  Volumes above H1_PRACTICAL_VOXELS need
    allow_large=True."""
    _check_image(img)
    if img.dim() == 2:
        return persistence(img, max_survivors, with_stats)
    return _full_call([img.contiguous()], True, max_survivors, pool_entries, with_stats, allow_large)


def persistence_full_batched(imgs: Sequence[torch.Tensor], max_survivors: int = 0, pool_entries: int = 0,
                             with_stats: bool = False, allow_large: bool = False) -> Diagram:
    """persistence_full over many images and volumes in one pass (pairs carry their item index)."""
    if not imgs:
        raise ValueError("empty batch")
    if len(imgs) > _lib.CP_MAX_ITEMS:
        raise ValueError(f"at most {_lib.CP_MAX_ITEMS} items per call")
    imgs = [im.contiguous() for im in imgs]
    for im in imgs:
        _check_image(im)
    return _full_call(imgs, False, max_survivors, pool_entries, with_stats, allow_large)


def pairs_backward(raw: torch.Tensor, grad_birth: torch.Tensor, grad_death: torch.Tensor, n_pixels: int,
                   item_offsets: Optional[torch.Tensor] = None) -> torch.Tensor:
    """dL/dimage (flat, float32) from dL/dbirth and dL/ddeath of each pair."""
    lib = _lib.load()
    dev = raw.device
    gb = grad_birth.contiguous().to(torch.float32)
    gd = grad_death.contiguous().to(torch.float32)
    grad = torch.empty(n_pixels, dtype=torch.float32, device=dev)
    ws_bytes = lib.cubical_persistence_backward_workspace_size(n_pixels)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    offs = None if item_offsets is None else ctypes.c_void_p(item_offsets.data_ptr())
    rc = lib.cubical_persistence_backward(
        ctypes.c_void_p(raw.data_ptr()), raw.shape[0], ctypes.c_void_p(gb.data_ptr()), ctypes.c_void_p(gd.data_ptr()),
        offs, ctypes.c_void_p(grad.data_ptr()), n_pixels, ctypes.c_void_p(ws.data_ptr()), ws_bytes,
        ctypes.c_void_p(_stream_ptr(dev)),
    )
    if rc != CP_OK:
        raise CpError(rc, "cubical_persistence_backward")
    return grad


class _DiagramFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, img, max_survivors, filtration, full):
        if full:
            if filtration != "V":
                raise ValueError("the full diagram is computed for the V-filtration")
            d = persistence_full(img.detach(), max_survivors)
        else:
            d = persistence(img.detach(), max_survivors, filtration=filtration)
        ctx.save_for_backward(d.raw)
        ctx.shape = img.shape
        ctx.mark_non_differentiable(d.raw)
        return d.birth.clone(), d.death.clone(), d.raw

    @staticmethod
    def backward(ctx, gb, gd, _graw):
        (raw,) = ctx.saved_tensors
        n = int(np.prod(ctx.shape))
        if gb is None:
            gb = torch.zeros(raw.shape[0], dtype=torch.float32, device=raw.device)
        if gd is None:
            gd = torch.zeros(raw.shape[0], dtype=torch.float32, device=raw.device)
        g = pairs_backward(raw, gb, gd, n)
        return g.view(ctx.shape), None, None, None


def diagram(img: torch.Tensor, max_survivors: int = 0, filtration: str = "V", full: bool = False):
    """(birth, death, raw): birth and death are differentiable in img (V or T
    filtration; full=True adds the H1 pairs of a volume, V only)."""
    return _DiagramFn.apply(img, max_survivors, filtration, full)
