"""Host side of the slab split across processes (the parallelisation that
Sec. 6 leaves to future work): which slab an element belongs to, and the one
exchange step, which brings every rank's merge records to the rank that runs
the merge union-find.

A merge record is one survivor that stage 1 of the split hands to stage 2:
a survivor that its slab's union-find committed, or one whose endpoint
classes lie in two slabs.  It carries

  key    the survivor's processing key (H0: its key; top dimension: the
         complement of its key, so that ascending order is the dual's
         descending filtration order), unique over the whole image;
  age_a  the age key of its first endpoint class, which names the class on
         every rank (the class's root vertex, or for the dual the vertex whose
         lower star holds the root top cell; an outside vertex is all ones);
  age_b  the same for the second endpoint.

The merge union-find takes the records in ascending key order, identifies
classes by their age keys, and kills the younger class at each commit (H0:
larger age; dual: smaller age).  ``cubical_persistence_slabs`` runs both
stages on one GPU; across processes each rank runs stage 1 for its slabs and
``exchange`` gathers the records.
"""
from __future__ import annotations

import numpy as np

RECORD_DTYPE = np.dtype([("key", "<u8"), ("age_a", "<u8"), ("age_b", "<u8")])


def slab_of(coord, extent: int, n_slabs: int):
    """Slab of an element at `coord` along an axis of `extent` elements cut
    into `n_slabs` slabs: coord * n_slabs // extent (as the library computes
    it; slabs differ in extent by at most one element)."""
    if extent < 1 or n_slabs < 1:
        raise ValueError("extent and n_slabs must be positive")
    return np.asarray(coord, dtype=np.int64) * n_slabs // extent


def exchange(records: np.ndarray, group=None, dst: int = 0):
    """Gathers every rank's merge records (RECORD_DTYPE) on rank `dst` of the
    process group and returns them there in ascending key order (None on the
    other ranks).  The group must carry CPU tensors (gloo).  Raises if two
    records share a key: every survivor belongs to exactly one slab's list."""
    import torch
    import torch.distributed as dist

    rec = np.ascontiguousarray(records, dtype=RECORD_DTYPE).reshape(-1)
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    n = torch.tensor([rec.shape[0]], dtype=torch.int64)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    m = max(int(s.item()) for s in sizes)
    buf = torch.zeros((max(m, 1), 3), dtype=torch.int64)
    if rec.shape[0]:
        buf[: rec.shape[0]] = torch.from_numpy(rec.view(np.int64).reshape(-1, 3).copy())
    parts = [torch.zeros_like(buf) for _ in range(world)] if rank == dst else None
    dist.gather(buf, gather_list=parts, dst=dst, group=group)
    if rank != dst:
        return None
    cols = [p[: int(s.item())].numpy() for p, s in zip(parts, sizes)]
    merged = np.ascontiguousarray(np.concatenate(cols)).view(RECORD_DTYPE).reshape(-1)
    merged = merged[np.argsort(merged["key"], kind="stable")]
    if merged.shape[0] > 1 and np.any(merged["key"][1:] == merged["key"][:-1]):
        raise ValueError("two merge records share a key")
    return merged
