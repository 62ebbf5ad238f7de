"""Host-side checks of the CUDA library (no GPU needed).

- the shared library loads and exports every symbol include/*.h declares;
- the lookup table has the paper's 15,935 3D configurations (Sec. 3.3) and
  47 in 2D, and its collapse agrees with an independent enumeration;
- a plain restatement of the pruned pipeline, driven by the library's own
  table entries (cp_lut_lookup), gives the oracle's pairs: every pruning
  predicate in the table is a union-find invariant.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2606_04801_gb300 as cp
from paper_2606_04801_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def lib():
    from paper_2606_04801_gb300 import build

    build.build()
    return _lib.load()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "cubical_persistence.h")).read()
    declared = set(re.findall(r"^\s*(?:int|int64_t|size_t|long long|const char \*)\s*\**\s*(\w+)\s*\(", hdr, re.M))
    assert declared, "no declarations parsed"
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(_lib.exported_symbols())
    assert lib.cp_version() > 0
    assert lib.cp_error_string(-3).decode() == "capacity exceeded"


def test_lut_class_counts(lib):
    # Sec. 3.3 prints 15,935 configurations in 3D after the collapse
    with open(os.path.join(GOLDEN, "lut_counts.txt")) as fh:
        want = {int(l.split()[0]): int(l.split()[1]) for l in fh if l.strip() and not l.startswith("#")}
    assert lib.cp_lut_num_classes(3) == want[3] == 15935
    assert lib.cp_lut_num_classes(2) == want[2]
    assert lib.cp_lut_num_classes(4) == -1


def test_kernel_mask_layout(lib):
    """The 3D pruning kernel collapses its comparison mask in its own bit
    layout with multiplications and masks; on all 2^26 raw masks that
    collapse equals the sub-offset rule of Sec. 3.3 (the library's
    definition, itself pinned by the class counts above and by the pruned
    restatement against the oracle below)."""
    n = ctypes.c_uint64(1)
    assert lib.cp_lut_check_layout(ctypes.byref(n)) == 0
    assert n.value == 0
    assert lib.cp_lut_check_layout(None) == _lib.CP_ERR_ARG


def _offsets(ndim):
    n = 27 if ndim == 3 else 9
    if ndim == 3:
        return [(b // 9 - 1, (b // 3) % 3 - 1, b % 3 - 1) for b in range(n)]
    return [(0, b // 3 - 1, b % 3 - 1) for b in range(n)]


def _collapse_numpy(ndim):
    """Independent enumeration: every raw mask -> relevant mask, vectorised."""
    offs = _offsets(ndim)
    center = 13 if ndim == 3 else 4
    nb = len(offs)
    raw = np.arange(1 << nb, dtype=np.uint32)
    raw = raw[(raw >> center) & 1 == 0]
    rel = np.zeros_like(raw)
    for b, o in enumerate(offs):
        if b == center:
            continue
        need = np.uint32(0)
        for c, q in enumerate(offs):
            if c == center:
                continue
            if all(qa == 0 or qa == oa for qa, oa in zip(q, o)):
                need |= np.uint32(1 << c)
        rel |= np.where((raw & need) == need, np.uint32(1 << b), np.uint32(0)).astype(np.uint32)
    return raw, rel


def test_collapse_matches_independent_enumeration(lib):
    raw2, rel2 = _collapse_numpy(2)
    assert len(np.unique(rel2)) == 47
    r = ctypes.c_uint32()
    for m, want in zip(raw2, rel2):
        assert lib.cp_lut_lookup(2, int(m), ctypes.byref(r), None) == 0
        assert r.value == int(want)
    # 3D: count the distinct collapsed masks over all 2^26 raw masks
    raw3, rel3 = _collapse_numpy(3)
    seen = np.zeros(1 << 27, dtype=bool)
    seen[rel3] = True
    assert int(seen.sum()) == 15935
    rng = np.random.default_rng(0)
    for m in rng.choice(raw3, 3000, replace=False):
        assert lib.cp_lut_lookup(3, int(m), ctypes.byref(r), None) == 0
        assert r.value == int(rel3[np.searchsorted(raw3, m)])


# ---------------------------------------------------------------- restatement
from prune_restatement import Pruned


def _pruned_pipeline(lib, img, cross=False):
    return Pruned(lib, img, cross=cross).pairs()


def _oracle_rows(img):
    p = oracle.persistence(img)
    return sorted(
        (int(r["dim"]), int(r["birth_cell"]), int(r["death_cell"]), float(r["birth"]), float(r["death"]))
        for r in p
        if r["death_cell"] >= 0
    )


@pytest.mark.parametrize("cross", [False, True])
@pytest.mark.parametrize("seed", range(4))
def test_pruned_restatement_matches_oracle_2d(lib, seed, cross):
    """Both forms of the 2D top dimension (cross-pruned after H0, or at once
    with every dual survivor of the table) give the oracle's pairs."""
    rng = np.random.default_rng(200 + seed)
    for _ in range(25):
        shape = tuple(int(v) for v in rng.integers(2, 10, 2))
        img = rng.integers(0, 3, shape).astype(np.float32) if rng.random() < 0.5 else rng.random(shape, dtype=np.float32)
        assert _pruned_pipeline(lib, img, cross) == _oracle_rows(img)


@pytest.mark.parametrize("seed", range(3))
def test_pruned_restatement_matches_oracle_3d(lib, seed):
    rng = np.random.default_rng(300 + seed)
    for _ in range(8):
        shape = tuple(int(v) for v in rng.integers(2, 7, 3))
        img = rng.integers(0, 3, shape).astype(np.float32) if rng.random() < 0.5 else rng.random(shape, dtype=np.float32)
        assert _pruned_pipeline(lib, img) == _oracle_rows(img)


def test_tuning_arguments(lib):
    keys = {1: (64, [4, 16, 256], [0, 3, 5000]), 2: (0, [0, 2, 4], [-1, 9]), 3: (64, [4, 37, 4096], [0, 3, 4097]),
            4: (30000, [0, 1, 3600000], [-1, 3600001]), 5: (0, [0, 1], [-1, 2]), 6: (16, [0, 1, 1024], [-1, 1025]),
            7: (0, [0, 1], [-1, 2])}
    for key, (default, good, bad) in keys.items():
        old = lib.cp_get_tuning(key)
        try:
            for v in good:
                assert lib.cp_set_tuning(key, v) == 0 and lib.cp_get_tuning(key) == v
            for v in bad:
                assert lib.cp_set_tuning(key, v) == -1
        finally:
            assert lib.cp_set_tuning(key, old) == 0
    assert lib.cp_get_tuning(99) == -1 and lib.cp_set_tuning(99, 1) == -1


def test_t_workspace_sizes(lib):
    """The T-filtration workspace holds the V workspace of the padded dual
    image plus the image itself; every extent may be 1; bad arguments give 0."""
    import ctypes

    def size(fn, *dims):
        d = (ctypes.c_int64 * len(dims))(*dims)
        return getattr(lib, fn)(len(dims), d, 0)

    for dims in [(1, 1), (1, 7), (5, 3), (64, 64), (1, 1, 1), (3, 1, 4), (20, 30, 40)]:
        padded = tuple(n + 2 for n in dims)
        t = size("cubical_persistence_t_workspace_size", *dims)
        v = size("cubical_persistence_workspace_size", *padded)
        assert v > 0 and t >= v + 4 * int(np.prod(padded)), (dims, t, v)
    assert size("cubical_persistence_t_workspace_size", 0, 5) == 0
    assert size("cubical_persistence_t_workspace_size", 4, 0, 5) == 0
    # the padded volume must stay within 2^27 vertices: 510^3 pads to 512^3
    assert size("cubical_persistence_t_workspace_size", 511, 511, 511) == 0
    assert size("cubical_persistence_t_workspace_size", 510, 510, 510) > 0


def test_full_workspace_sizes(lib):
    """The full-diagram workspace adds the H1 stage to the plain one for a
    volume (bitmaps, columns, pivots, pool: it grows with the pool); a 2D
    image has no H1 stage; bad arguments give 0."""
    import ctypes

    def full(dims, pool=0):
        d = (ctypes.c_int64 * len(dims))(*dims)
        return lib.cubical_persistence_full_workspace_size(len(dims), d, 0, pool)

    def plain(dims):
        d = (ctypes.c_int64 * len(dims))(*dims)
        return lib.cubical_persistence_workspace_size(len(dims), d, 0)

    for dims in [(2, 2, 2), (3, 4, 5), (20, 30, 40)]:
        D, H, W = dims
        cols = D * H * (W - 1) + D * (H - 1) * W + (D - 1) * H * W - D * H * W + 1
        f, p = full(dims), plain(dims)
        # at least: per edge or square id a mask, an offset, a length and a
        # pivot; three column lists; the default pool
        assert f >= p + 3 * D * H * W * 24 + 12 * cols + 8 * (4 * cols + 2**20), (dims, f, p)
        assert full(dims, 10**6) - full(dims, 1) >= 8 * (10**6 - 1) - 256
    assert full((17, 19)) == plain((17, 19))
    assert full((1, 5, 5)) == 0 and full((4, 0, 5)) == 0
    assert full((3, 4, 5), -1) == 0
    n = (ctypes.c_int32 * 2)(3, 2)
    d = (ctypes.c_int64 * 6)(4, 5, 6, 1, 7, 8)
    assert lib.cubical_persistence_full_batched_workspace_size(2, n, d, 0, 0) > lib.cubical_persistence_batched_workspace_size(2, n, d, 0)


def test_full_entry_argument_errors(lib):
    """The full-diagram entries reject bad arguments before touching a device."""
    import ctypes

    dims3 = (ctypes.c_int64 * 3)(3, 4, 5)
    flat = (ctypes.c_int64 * 3)(1, 4, 5)
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: every call below fails its checks first
    full = lib.cubical_persistence_full_3d
    assert full(None, dims3, fake, 10, None, None, fake, 1 << 30, 0, 0, None) == -1  # no image
    assert full(fake, dims3, fake, 10, None, None, None, 1 << 30, 0, 0, None) == -1  # no workspace
    assert full(fake, flat, fake, 10, None, None, fake, 1 << 30, 0, 0, None) == -1  # an extent of 1
    assert full(fake, dims3, fake, 10, None, None, fake, 1 << 30, 0, -5, None) == -1  # a negative pool
    need = lib.cubical_persistence_full_workspace_size(3, dims3, 0, 0)
    assert full(fake, dims3, fake, 10, None, None, fake, need - 1, 0, 0, None) == -1  # workspace too small
    assert full(fake, dims3, None, 10, None, None, fake, need, 0, 0, None) == -1  # no output with capacity
    nd = (ctypes.c_int32 * 1)(3)
    ptrs = (ctypes.c_void_p * 1)(0x1000)
    fb = lib.cubical_persistence_full_batched
    assert fb(0, ptrs, nd, dims3, fake, 10, None, None, fake, 1 << 30, 0, 0, None) == -1
    assert fb(1, None, nd, dims3, fake, 10, None, None, fake, 1 << 30, 0, 0, None) == -1
    # the info entry: bad arguments, and a call without volumes has no H1 stage (nothing read)
    info = (ctypes.c_int64 * 4)()
    assert lib.cubical_persistence_full_info(None, 1, nd, dims3, 0, 0, info, 4, None) == -1
    assert lib.cubical_persistence_full_info(fake, 1, nd, dims3, 0, 0, info, 3, None) == -1
    nd2 = (ctypes.c_int32 * 1)(2)
    assert lib.cubical_persistence_full_info(fake, 1, nd2, flat, 0, 0, info, 4, None) == 0
    assert list(info) == [0, 0, 0, 0]


def test_t_entry_argument_errors(lib):
    """The T-filtration entries reject bad arguments before touching a device."""
    import ctypes

    dims2 = (ctypes.c_int64 * 2)(4, 5)
    dims3 = (ctypes.c_int64 * 3)(3, 4, 5)
    bad2 = (ctypes.c_int64 * 2)(0, 5)
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: every call below fails its checks first
    # null image / null workspace
    assert lib.cubical_persistence_t_2d(None, dims2, fake, 10, None, None, fake, 1 << 20, 0, None) == -1
    assert lib.cubical_persistence_t_3d(fake, dims3, fake, 10, None, None, None, 1 << 20, 0, None) == -1
    # an extent of 0
    assert lib.cubical_persistence_t_2d(fake, bad2, fake, 10, None, None, fake, 1 << 20, 0, None) == -1
    # a workspace smaller than the size the entry asks for
    need = lib.cubical_persistence_t_workspace_size(2, dims2, 0)
    assert lib.cubical_persistence_t_2d(fake, dims2, fake, 10, None, None, fake, need - 1, 0, None) == -1
    # batched: no items, too many items, a bad rank
    nd = (ctypes.c_int32 * 1)(4)
    d3 = (ctypes.c_int64 * 3)(1, 4, 5)
    ptrs = (ctypes.c_void_p * 1)(0x1000)
    assert lib.cubical_persistence_t_batched(0, ptrs, nd, d3, fake, 10, None, None, fake, 1 << 20, 0, None) == -1
    assert lib.cubical_persistence_t_batched(1, ptrs, nd, d3, fake, 10, None, None, fake, 1 << 20, 0, None) == -1
    assert lib.cubical_persistence_t_batched_workspace_size(129, nd, d3, 0) == 0
