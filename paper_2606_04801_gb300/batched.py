"""Batched forward + backward over many images and volumes of uneven sizes.

A `BatchedPersistence` owns every buffer of a fixed batch of shapes (inputs
packed in one device array, workspace, pairs, loss, gradient) and enqueues
the whole step -- lookup + pruning of all items, one sort and one union-find
per dimension for the whole batch, emission, the total-persistence loss and
its backward scatter -- with no host round trip.  With `graph=True` the step
is captured once into a CUDA graph and each `step()` is a single graph
launch.

    bp = BatchedPersistence([(512, 384), (128, 96, 80), ...], tau=0.05)   # filtration="T" as well
    bp.load([img0, vol1, ...])        # copies the inputs in
    loss, grad = bp.step()            # device tensors (grad packed per item)
    pairs = bp.pairs()                # Diagram with an `item` field
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import CP_ERR_CAPACITY, CP_OK, CpError
from .api import Diagram, _stats


class BatchedPersistence:
    def __init__(self, shapes: Sequence[Sequence[int]], tau: float = 0.05, device=None, max_survivors: int = 0,
                 graph: bool = True, filtration: str = "V"):
        if not shapes or len(shapes) > _lib.CP_MAX_ITEMS:
            raise ValueError(f"between 1 and {_lib.CP_MAX_ITEMS} items")
        if filtration not in ("V", "T"):
            raise ValueError("filtration must be 'V' or 'T'")
        self.tmode = filtration == "T"
        self.lib = _lib.load()
        self.dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        for s in self.shapes:
            if len(s) not in (2, 3) or min(s) < (1 if self.tmode else 2):
                raise ValueError(f"bad shape {s}")
        self.tau = float(tau)
        self.k = len(self.shapes)
        self.sizes = [int(np.prod(s)) for s in self.shapes]
        offs = np.concatenate([[0], np.cumsum(self.sizes)[:-1]]).astype(np.int64)
        self.total = int(sum(self.sizes))
        self.x = torch.empty(self.total, dtype=torch.float32, device=self.dev)
        self.views = [self.x[o : o + n].view(s) for o, n, s in zip(offs, self.sizes, self.shapes)]
        self.item_offsets = torch.from_numpy(offs).to(self.dev)
        self._ptrs = (ctypes.c_void_p * self.k)(*[v.data_ptr() for v in self.views])
        self._ndims = (ctypes.c_int32 * self.k)(*[len(s) for s in self.shapes])
        flat = []
        for s in self.shapes:
            flat += ([1] + list(s)) if len(s) == 2 else list(s)
        self._dims = (ctypes.c_int64 * (3 * self.k))(*flat)
        self.d_count = torch.zeros(1, dtype=torch.int64, device=self.dev)
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.dev)
        self.grad = torch.empty(self.total, dtype=torch.float32, device=self.dev)
        bws = self.lib.cubical_persistence_loss_backward_workspace_size(self.total)
        self.bws = torch.empty(bws, dtype=torch.uint8, device=self.dev)
        self.use_graph = graph
        self.graph = None
        self._plan(int(max_survivors))

    def _plan(self, ms: int):
        self.ms = ms
        wsize = (self.lib.cubical_persistence_t_batched_workspace_size if self.tmode
                 else self.lib.cubical_persistence_batched_workspace_size)
        ws = wsize(self.k, self._ndims, self._dims, ms)
        if ws == 0:
            raise CpError(_lib.CP_ERR_ARG, "batched workspace size")
        self.ws = torch.empty(ws, dtype=torch.uint8, device=self.dev)
        if self.tmode:  # the dual images' vertices; T vertices + top cells per item
            nv = sum(int(np.prod([v + 2 for v in s])) for s in self.shapes)
            bound = sum(int(np.prod(s)) + int(np.prod([v + 1 for v in s])) for s in self.shapes)
        else:
            nv = self.total
            bound = self.total + sum(int(np.prod([v - 1 for v in s])) + 1 for s in self.shapes)
        eff = ms if ms > 0 else nv // 2 + 65536
        self.cap = min(bound, eff + 2 * self.k + 4096)
        self.out = torch.empty((self.cap, 8), dtype=torch.int32, device=self.dev)
        self.graph = None

    def load(self, inputs: Sequence[torch.Tensor]):
        if len(inputs) != self.k:
            raise ValueError("wrong number of items")
        for v, a in zip(self.views, inputs):
            v.copy_(torch.as_tensor(a).reshape(v.shape), non_blocking=True)

    def _enqueue(self, stream_ptr: int):
        lib = self.lib
        sp = ctypes.c_void_p(stream_ptr)
        fn = lib.cubical_persistence_t_batched if self.tmode else lib.cubical_persistence_batched
        rc = fn(
            self.k, self._ptrs, self._ndims, self._dims, ctypes.c_void_p(self.out.data_ptr()), self.cap, None,
            ctypes.c_void_p(self.d_count.data_ptr()), ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(), self.ms, sp,
        )
        if rc != CP_OK:
            raise CpError(rc, "cubical_persistence_batched" + ("_t" if self.tmode else ""))
        rc = lib.cubical_persistence_loss_backward(
            ctypes.c_void_p(self.out.data_ptr()), self.cap, ctypes.c_void_p(self.d_count.data_ptr()),
            ctypes.c_float(self.tau), ctypes.c_void_p(self.loss.data_ptr()),
            ctypes.c_void_p(self.item_offsets.data_ptr()), ctypes.c_void_p(self.grad.data_ptr()), self.total,
            ctypes.c_void_p(self.bws.data_ptr()), self.bws.numel(), sp,
        )
        if rc != CP_OK:
            raise CpError(rc, "cubical_persistence_loss_backward")

    def _eager_checked(self):
        """One eager step; grows the workspace until the survivors fit."""
        for _ in range(4):
            self._enqueue(int(torch.cuda.current_stream(self.dev).cuda_stream))
            st = _stats(self.ws)
            if st["rc"] == CP_OK:
                return st
            if st["rc"] != CP_ERR_CAPACITY:
                raise CpError(st["rc"], "batched step")
            need = max(st["h0_survivors"], st["top_survivors"], 2 * st["h0_roots"], 2 * st["top_roots"], self.ms)
            self._plan(int(need * 1.25) + 65536)
        raise CpError(CP_ERR_CAPACITY, "batched step (after growing the workspace)")

    def capture(self):
        """Run one eager step (sizes the workspace, sets up lazy state), then capture the step."""
        self._eager_checked()
        torch.cuda.synchronize(self.dev)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._enqueue(int(torch.cuda.current_stream(self.dev).cuda_stream))
        self.graph = g

    def step(self):
        """Forward + loss + backward of the loaded batch; returns (loss, grad) on the device."""
        if self.use_graph:
            if self.graph is None:
                self.capture()
            self.graph.replay()
        else:
            self._enqueue(int(torch.cuda.current_stream(self.dev).cuda_stream))
        return self.loss, self.grad

    def status(self) -> dict:
        return _stats(self.ws)

    def pairs(self) -> Diagram:
        n = int(self.d_count.item())
        return Diagram(self.out[:n])

    def grads(self):
        """Per-item gradient views of the packed gradient."""
        return [self.grad[o : o + n].view(s) for o, n, s in zip(self.item_offsets.tolist(), self.sizes, self.shapes)]
