"""CPU restatement of the slab split of the union-finds, on the whole
(unpruned) cubical complex of a small image.

Each slab runs the elder-rule union-find (Sec. 4.1 steps 3 and 5, Sec. 4.2
steps 2 and 3) over the cells whose two endpoint classes lie in it; what it
commits, and the cells between slabs, go to one merge union-find in
filtration order, which writes the pairs.  Here every vertex (top cell) is its
own class, so a class's slab is that of its vertex (of the top cell's
largest vertex; the outside vertex belongs to slab 0), as the library does
for the roots of its pruned forests.

Exchanged records carry the cell's processing key and the age keys of its two
endpoint classes: the age key names a class uniquely on every rank, so the
merge needs no rank-local ids.  Keys: ord(f(m)) << 32 | m << 5 | n, with m
the cell's largest vertex in (value, index) order and n its stencil offset
from m, the order of the doubled-grid index among the cells of one lower
star; the dual list is processed in descending order, so its processing key
is the complement.

Shares nothing with the CUDA path or the oracle; test infrastructure only.
"""
from __future__ import annotations

import numpy as np

OUTSIDE = np.uint64(0xFFFFFFFFFFFFFFFF)


def ord_bits(f: np.ndarray) -> np.ndarray:
    """Order-preserving unsigned bits of float32 values (-0 reads as +0)."""
    b = np.ascontiguousarray(f, dtype=np.float32).view(np.uint32).copy()
    b[(b << np.uint32(1)) == 0] = 0
    neg = (b & np.uint32(0x80000000)) != 0
    return np.where(neg, ~b, b | np.uint32(0x80000000)).astype(np.uint64)


class Complex:
    """The H0 graph (vertices, edges) and the dual graph (top cells plus an
    outside vertex, facets) of a 2D or 3D image, with refined keys."""

    def __init__(self, img: np.ndarray):
        f = np.asarray(img, dtype=np.float32)
        if f.ndim == 2:
            f = f[None]
            self.ndim = 2
        else:
            self.ndim = 3
        self.f = f
        D, H, W = f.shape
        self.shape = (D, H, W)
        n = D * H * W
        ords = ord_bits(f.reshape(-1))
        idx = np.arange(n, dtype=np.uint64)
        self.vkey = (ords << np.uint64(32)) | (idx << np.uint64(5))  # (value, index) order of the vertices
        self.fflat = f.reshape(-1)
        self.vz = np.arange(n) // (H * W)
        self.vy = (np.arange(n) // W) % H
        self._cells()

    def _stencil(self, dz, dy, dx):
        if self.ndim == 3:
            return 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1)
        return 3 * (dy + 1) + (dx + 1)

    def _cell_key(self, verts, center):
        """Key of the cell with these corner vertices and doubled-grid centre."""
        m = max(verts, key=lambda v: int(self.vkey[v]))
        D, H, W = self.shape
        mz, my, mx = m // (H * W), (m // W) % H, m % W
        cz, cy, cx = center
        n = self._stencil(cz - 2 * mz, cy - 2 * my, cx - 2 * mx)
        return (self.vkey[m] | np.uint64(n)), m

    def doubled(self, center):
        D, H, W = self.shape
        cz, cy, cx = center
        if self.ndim == 2:
            return cy * (2 * W - 1) + cx
        return (cz * (2 * H - 1) + cy) * (2 * W - 1) + cx

    def _cells(self):
        D, H, W = self.shape
        vid = lambda z, y, x: (z * H + y) * W + x  # noqa: E731
        axes = [(0, 0, 1), (0, 1, 0)] + ([(1, 0, 0)] if self.ndim == 3 else [])
        # edges
        edges = []
        for z in range(D):
            for y in range(H):
                for x in range(W):
                    for dz, dy, dx in axes:
                        if z + dz < D and y + dy < H and x + dx < W:
                            a, b = vid(z, y, x), vid(z + dz, y + dy, x + dx)
                            c = (2 * z + dz, 2 * y + dy, 2 * x + dx)
                            key, m = self._cell_key((a, b), c)
                            edges.append((key, a, b, m, c))
        self.edges = edges
        # top cells (lowest corner (z, y, x)) and their keys
        tz = D - 1 if self.ndim == 3 else 1
        self.top = {}
        for z in range(tz):
            for y in range(H - 1):
                for x in range(W - 1):
                    zs = (z, z + 1) if self.ndim == 3 else (z,)
                    verts = [vid(a, b, c) for a in zs for b in (y, y + 1) for c in (x, x + 1)]
                    c = (2 * z + 1 if self.ndim == 3 else 0, 2 * y + 1, 2 * x + 1)
                    key, m = self._cell_key(verts, c)
                    self.top[(z, y, x)] = (key, m, c)
        # facets: codimension-1 cells, with the top cells on their two sides
        facets = []
        if self.ndim == 3:
            for normal in range(3):  # 0: x, 1: y, 2: z
                for z in range(D if normal != 2 else D):
                    for y in range(H):
                        for x in range(W):
                            span = [(1, 1, 0), (1, 0, 1), (0, 1, 1)][normal]  # extents along (z, y, x)
                            sz, sy, sx = span
                            if z + sz >= D or y + sy >= H or x + sx >= W:
                                continue
                            verts = [vid(z + a, y + b, x + c) for a in range(sz + 1) for b in range(sy + 1)
                                     for c in range(sx + 1)]
                            c = (2 * z + sz, 2 * y + sy, 2 * x + sx)
                            key, m = self._cell_key(verts, c)
                            lo = (z - (normal == 2), y - (normal == 1), x - (normal == 0))
                            hi = (z, y, x)
                            facets.append((key, self.top.get(lo), self.top.get(hi), m, c))
        else:
            for dz, dy, dx in axes:
                for y in range(H):
                    for x in range(W):
                        if y + dy >= H or x + dx >= W:
                            continue
                        a, b = vid(0, y, x), vid(0, y + dy, x + dx)
                        c = (0, 2 * y + dy, 2 * x + dx)
                        key, m = self._cell_key((a, b), c)
                        # a horizontal edge (dx) separates the squares above and below it
                        lo = (0, y - 1, x) if dx else (0, y, x - 1)
                        hi = (0, y, x)
                        facets.append((key, self.top.get(lo), self.top.get(hi), m, c))
        self.facets = facets

    def slab_of_vertex(self, v, S):
        D, H, W = self.shape
        if self.ndim == 3:
            return int(self.vz[v]) * S // D
        return int(self.vy[v]) * S // H

    def h0_records(self):
        """(processing key, class age a, class age b, key vertex) of every edge."""
        return [(int(k), int(self.vkey[a]), int(self.vkey[b]), m) for k, a, b, m, _ in self.edges]

    def dual_records(self):
        """The same for every facet; a missing side is the outside vertex."""
        out = []
        for k, lo, hi, m, _ in self.facets:
            ka = int(lo[0]) if lo else int(OUTSIDE)
            kb = int(hi[0]) if hi else int(OUTSIDE)
            out.append((int(~np.uint64(k)), ka, kb, m))
        return out


def class_slab(cx: Complex, age: int, S: int) -> int:
    """Slab of a class from its age key (the vertex it names; outside: 0)."""
    if age == int(OUTSIDE):
        return 0
    return cx.slab_of_vertex((age >> 5) & ((1 << 27) - 1), S)


def union_find(records, dual: bool):
    """Elder-rule union-find over records (key, age a, age b, ...) taken in
    ascending processing-key order.  H0: the class with the larger age dies;
    dual: the smaller.  Returns the committed records, each with the ages of
    the class it killed and of the class that absorbed it (both roots)."""
    parent = {}

    def find(x):
        root = x
        while parent.get(root, root) != root:
            root = parent[root]
        while parent.get(x, x) != root:
            parent[x], x = root, parent[x]
        return root

    commits = []
    for rec in sorted(records, key=lambda r: r[0]):
        ra, rb = find(rec[1]), find(rec[2])
        if ra == rb:
            continue
        young, old = (max(ra, rb), min(ra, rb)) if not dual else (min(ra, rb), max(ra, rb))
        parent[young] = old
        commits.append((rec, young, old))
    return commits


def slab_records(cx: Complex, S: int, slabs, dual: bool, reduce: bool = False):
    """Stage 1 for the slabs in `slabs`: each slab's union-find over its
    internal records.  Returns (sent, final): what those slabs send to the
    merge, and the commits whose pairs they write themselves.

    reduce=False: every commit is sent as it is, with the crossing records
    whose key vertex lies in the slab.
    reduce=True: a class is a boundary class when one of its vertices (top
    cells) is an endpoint of a crossing record.  A commit whose dying class is
    not a boundary class at its time is final: the whole image's union-find
    sees exactly that class then (no record leads out of it), and the other
    class there contains the slab's surviving class, so it is at least as old;
    the same class dies with the same pair, and the slab writes it.  Nothing
    of the dead class reaches the merge again.  The other commits are sent
    with their endpoints replaced by the two classes' roots at that time (the
    age keys of their oldest members): the merge does not see the final
    commits, so a record's own endpoints may lie in classes it never joined."""
    recs = cx.dual_records() if dual else cx.h0_records()
    crossing = [r for r in recs if class_slab(cx, r[1], S) != class_slab(cx, r[2], S)]
    touched = {r[1] for r in crossing} | {r[2] for r in crossing}
    sent, final = [], []
    for s in slabs:
        internal = [r for r in recs if class_slab(cx, r[1], S) == s and class_slab(cx, r[2], S) == s]
        commits = union_find(internal, dual)
        if not reduce:
            sent += [rec for rec, _, _ in commits]
        else:
            boundary = {}  # root -> its class touches a crossing record
            for rec, young, old in commits:
                by = boundary.get(young, young in touched)
                bo = boundary.get(old, old in touched)
                if not by:
                    final.append((rec, young, old))
                else:
                    sent.append((rec[0], young, old, rec[3]))
                boundary[old] = by or bo
        sent += [r for r in crossing if cx.slab_of_vertex(r[3], S) == s]
    return sent, final


def pairs_from_commits(cx: Complex, commits, dual: bool):
    """(dim, birth, death, birth cell, death cell) of the nonzero commits."""
    out = []
    D, H, W = cx.shape
    byvkey = {int(k): v for v, k in enumerate(cx.vkey)}
    bytop = {int(t[0]): t for t in cx.top.values()}
    cells = {}
    for lst in (cx.edges, cx.facets):
        for rec in lst:
            cells[int(rec[0])] = rec
    for rec, young, *_ in commits:
        key = int(~np.uint64(rec[0])) if dual else rec[0]
        cell = cells[key]
        fcell = float(cx.fflat[cell[3]])
        if not dual:
            v = byvkey[young]
            birth, death = float(cx.fflat[v]), fcell
            bc = cx.doubled((2 * (v // (H * W)), 2 * ((v // W) % H), 2 * (v % W)))
            dc = cx.doubled(cell[4])
            dim = 0
        else:
            t = bytop[young]
            birth, death = fcell, float(cx.fflat[t[1]])
            bc, dc = cx.doubled(cell[4]), cx.doubled(t[2])
            dim = cx.ndim - 1
        if birth != death:
            out.append((dim, birth, death, bc, dc))
    return out


def split_pairs(img, S: int, reduce: bool = False):
    """The pairs of the slab split (stage 1 per slab, stage 2 over the union
    of what the slabs send), without the essential class."""
    cx = Complex(img)
    out = []
    for dual in (False, True):
        sent, final = slab_records(cx, S, range(S), dual, reduce)
        out += pairs_from_commits(cx, final, dual)
        out += pairs_from_commits(cx, union_find(sent, dual), dual)
    return sorted(out)


def whole_pairs(img):
    """The pairs of one union-find over the whole complex (no split)."""
    cx = Complex(img)
    out = []
    for dual in (False, True):
        recs = cx.dual_records() if dual else cx.h0_records()
        out += pairs_from_commits(cx, union_find(recs, dual), dual)
    return sorted(out)


def oracle_pairs(pairs):
    """The oracle's finite pairs in the same form."""
    out = []
    for p in pairs:
        if np.isinf(p["death"]):
            continue
        out.append((int(p["dim"]), float(p["birth"]), float(p["death"]), int(p["birth_cell"]), int(p["death_cell"])))
    return sorted(out)
