"""Brute-force persistence by F2 boundary-matrix reduction (Sec. 2.1).

An independent check of the oracle: it builds the whole cubical complex of a
tiny image, orders every cell by the fully refined V-filtration order
(Sec. 2.2-2.3, with the tie-break readings stated in the oracle) and runs the
textbook column reduction over F2 with Python integers as bit-set columns.
It shares nothing with the oracle or with the CUDA path.

Only for tiny inputs (a few hundred cells).
"""
from __future__ import annotations

import itertools

import numpy as np


def _cells(shape):
    """All cells of the cubical complex on a grid of vertex extents `shape`.

    A cell is the tuple of its doubled coordinates; coordinate 2k is the
    vertex coordinate k, coordinate 2k+1 the unit interval [k, k+1].
    """
    ranges = [range(2 * n - 1) for n in shape]
    return list(itertools.product(*ranges))


def _vertices(cell):
    choices = [(c // 2,) if c % 2 == 0 else (c // 2, c // 2 + 1) for c in cell]
    return list(itertools.product(*choices))


def _facets(cell):
    out = []
    for ax, c in enumerate(cell):
        if c % 2 == 1:
            for s in (-1, 1):
                f = list(cell)
                f[ax] = c + s
                out.append(tuple(f))
    return out


def _linear(coord, shape):
    idx = 0
    for c, n in zip(coord, shape):
        idx = idx * n + c
    return idx


def reduce_pairs(img):
    """Cell-level persistence pairs of the refined V-filtration, all dimensions.

    Returns (pairs, essential): pairs is a list of (birth_cell, death_cell,
    birth_dim) with cells as doubled-grid linear indices, essential the list
    of unpaired (birth_cell, dim).  Zero-persistence pairs are included.
    """
    f = np.asarray(img, dtype=np.float64)
    f = np.where(f == 0.0, 0.0, f)  # -0 reads as +0
    shape = f.shape
    dshape = tuple(2 * n - 1 for n in shape)
    cells = _cells(shape)

    def vkey(v):
        return (f[v], _linear(v, shape))

    def order_key(cell):
        m = max(_vertices(cell), key=vkey)
        dim = sum(c % 2 for c in cell)
        return (f[m], _linear(m, shape), dim, _linear(cell, dshape))

    cells.sort(key=order_key)
    pos = {c: i for i, c in enumerate(cells)}
    dims = [sum(c % 2 for c in cell) for cell in cells]
    cols = []
    for cell in cells:
        b = 0
        for fc in _facets(cell):
            b ^= 1 << pos[fc]
        cols.append(b)
    low_owner = {}
    pairs = []
    paired = set()
    for j in range(len(cells)):
        col = cols[j]
        while col:
            low = col.bit_length() - 1
            k = low_owner.get(low)
            if k is None:
                break
            col ^= cols[k]
        cols[j] = col
        if col:
            low = col.bit_length() - 1
            low_owner[low] = j
            pairs.append((_linear(cells[low], dshape), _linear(cells[j], dshape), dims[low]))
            paired.add(low)
            paired.add(j)
    essential = [(_linear(cells[i], dshape), dims[i]) for i in range(len(cells)) if i not in paired]
    return pairs, essential


def _pixels_t(cell, shape):
    """Top cells (pixels) of the T-complex that contain a cell: along each
    axis one pixel at an odd doubled coordinate, the ones on either side at an
    even one."""
    choices = []
    for c, n in zip(cell, shape):
        if c % 2 == 1:
            choices.append(((c - 1) // 2,))
        else:
            choices.append(tuple(k for k in (c // 2 - 1, c // 2) if 0 <= k < n))
    return list(itertools.product(*choices))


def reduce_pairs_t(img):
    """Cell-level persistence pairs of the T-filtration (pixel values on the
    top cells of the lattice complex, a cell taking the smallest value of the
    top cells that contain it), refined by (value, pixel index) of that top
    cell, then dimension, then doubled-grid index; all dimensions,
    zero-persistence pairs included.  Same output form as reduce_pairs, with
    cells indexed in the T doubled grid (extents 2n+1)."""
    f = np.asarray(img, dtype=np.float64)
    f = np.where(f == 0.0, 0.0, f)
    shape = f.shape
    dshape = tuple(2 * n + 1 for n in shape)
    cells = list(itertools.product(*[range(m) for m in dshape]))

    def order_key(cell):
        p = min(_pixels_t(cell, shape), key=lambda q: (f[q], _linear(q, shape)))
        dim = sum(c % 2 for c in cell)
        return (f[p], _linear(p, shape), dim, _linear(cell, dshape))

    cells.sort(key=order_key)
    pos = {c: i for i, c in enumerate(cells)}
    dims = [sum(c % 2 for c in cell) for cell in cells]
    cols = []
    for cell in cells:
        b = 0
        for fc in _facets(cell):
            b ^= 1 << pos[fc]
        cols.append(b)
    low_owner = {}
    pairs = []
    paired = set()
    for j in range(len(cells)):
        col = cols[j]
        while col:
            low = col.bit_length() - 1
            k = low_owner.get(low)
            if k is None:
                break
            col ^= cols[k]
        cols[j] = col
        if col:
            low = col.bit_length() - 1
            low_owner[low] = j
            pairs.append((_linear(cells[low], dshape), _linear(cells[j], dshape), dims[low]))
            paired.add(low)
            paired.add(j)
    essential = [(_linear(cells[i], dshape), dims[i]) for i in range(len(cells)) if i not in paired]
    return pairs, essential
