"""Stage test of the pruning kernel (K1) against the host restatement.

After the lookup + pruning pass alone (cubical_persistence_debug_prune), the
workspace must hold exactly the restatement's survivors (H0 edges and dual
facets, as order keys), exactly its roots, and forests whose every vertex /
top cell reaches the same root as in the restatement's forests (the kernel
may shortcut H0 links along a vertex's own descent chain, so parents may
differ, roots may not).
"""
import ctypes

import numpy as np
import pytest

import workloads
from prune_restatement import Pruned

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
TAG = 0x80000000


@pytest.fixture(scope="module")
def cp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_04801_gb300 as cp

    return cp


def _roots(par):
    """Root of every node, by pointer doubling (paths on plateaus can be long)."""
    r = np.asarray(par, dtype=np.int64).copy()
    for _ in range(64):
        nr = r[r]
        if np.array_equal(nr, r):
            return r
        r = nr
    raise AssertionError("forest does not converge")


def _kernel_stage(cp, img):
    lib = cp.load()
    t = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    nd = img.ndim
    ptrs = (ctypes.c_void_p * 1)(t.data_ptr())
    ndims = (ctypes.c_int32 * 1)(nd)
    dims = (ctypes.c_int64 * 3)(*(([1] + list(img.shape)) if nd == 2 else list(img.shape)))
    off = (ctypes.c_int64 * 13)()
    assert lib.cubical_persistence_debug_layout(1, ndims, dims, 0, off, 13) == 13
    ws_bytes = lib.cubical_persistence_batched_workspace_size(1, ndims, dims, 0)
    ws = torch.zeros(ws_bytes, dtype=torch.uint8, device="cuda")
    rc = lib.cubical_persistence_debug_prune(1, ptrs, ndims, dims, ctypes.c_void_p(ws.data_ptr()), ws_bytes, 0, None)
    assert rc == 0
    torch.cuda.synchronize()
    w = ws.cpu().numpy()
    ctr = w[off[0] : off[0] + 24].view(np.uint32)
    assert ctr[0] == 0, f"status {ctr[0]}"
    n_s0, n_st, n_r0, n_rt = (int(v) for v in ctr[1:5])
    ntot, ttot = off[7], off[8]
    uf0 = w[off[1] : off[1] + 4 * ntot].view(np.uint32).astype(np.int64)
    uft = w[off[2] : off[2] + 4 * ttot].view(np.uint32).astype(np.int64)
    s0 = np.sort(w[off[3] : off[3] + 8 * n_s0].view(np.uint64))
    st = np.sort(~w[off[4] : off[4] + 8 * n_st].view(np.uint64))
    _check.tma_tasks = int(w[off[12] : off[12] + 4].view(np.uint32)[0])
    return uf0, uft, s0, st, n_r0, n_rt


def _check(cp, lib, img, cross=False):
    ref = Pruned(lib, img, cross=cross)
    uf0, uft, s0, st, n_r0, n_rt = _kernel_stage(cp, img)
    assert s0.tolist() == ref.s0_keys()
    assert st.tolist() == ref.st_keys()
    # roots: tagged words; the restatement's roots are self-parents
    k_roots0 = set(np.flatnonzero(uf0 & TAG).tolist())
    r_roots0 = {v for v, p in enumerate(ref.par0) if p == v}
    assert k_roots0 == r_roots0 and n_r0 == len(r_roots0)
    k_rootst = set(np.flatnonzero(uft & TAG).tolist())
    r_rootst = {t for t, p in enumerate(ref.part) if p == t}  # includes the outside vertex
    assert k_rootst == r_rootst and n_rt == len(r_rootst)
    # same root for every vertex / top cell
    p0 = np.where(uf0 & TAG, np.arange(len(uf0)), uf0)
    pt = np.where(uft & TAG, np.arange(len(uft)), uft)
    assert np.array_equal(_roots(p0), _roots(ref.par0))
    assert np.array_equal(_roots(pt), _roots(ref.part))


@pytest.mark.parametrize("seed", range(3))
def test_prune_stage_2d(cp, seed):
    lib = cp.load()
    rng = np.random.default_rng(400 + seed)
    for _ in range(8):
        shape = tuple(int(v) for v in rng.integers(2, 40, 2))
        img = rng.integers(0, 3, shape).astype(np.float32) if rng.random() < 0.5 else rng.random(shape, dtype=np.float32)
        _check(cp, lib, img)


def test_prune_stage_2d_cross_pruning(cp):
    """Under cross-pruning (CP_TUNE_CROSS_PRUNE_2D = 1) the H0 survivors that
    the dual needs carry the flag bit and stay out of the dual list."""
    lib = cp.load()
    rng = np.random.default_rng(430)
    assert lib.cp_set_tuning(5, 1) == 0
    try:
        for _ in range(8):
            shape = tuple(int(v) for v in rng.integers(2, 40, 2))
            img = rng.integers(0, 3, shape).astype(np.float32) if rng.random() < 0.5 else rng.random(shape, dtype=np.float32)
            _check(cp, lib, img, cross=True)
    finally:
        assert lib.cp_set_tuning(5, 0) == 0


@pytest.mark.parametrize("seed", range(3))
def test_prune_stage_3d(cp, seed):
    lib = cp.load()
    rng = np.random.default_rng(500 + seed)
    for _ in range(5):
        shape = tuple(int(v) for v in rng.integers(2, 14, 3))
        img = rng.integers(0, 3, shape).astype(np.float32) if rng.random() < 0.5 else rng.random(shape, dtype=np.float32)
        _check(cp, lib, img)
    # a smooth volume deeper than one z chunk of the kernel (chains across chunks)
    _check(cp, lib, workloads.blurred((70, 9, 12), 2.0, 510 + seed))


@pytest.mark.parametrize("seed", range(2))
def test_prune_stage_3d_tma_planes(cp, seed):
    """Volumes whose width is a multiple of 4 (and planes at least one 40 x 11
    box) load their planes by TMA (out-of-image positions NaN); ragged tiles in
    every axis; ties.  The same data one column wider (41: cp.async path) must
    give the same survivors and roots."""
    lib = cp.load()
    rng = np.random.default_rng(600 + seed)
    for shape in [(13, 12, 40), (9, 21, 44), (70, 11, 48)]:
        img = rng.integers(0, 3, shape).astype(np.float32) if seed == 0 else workloads.blurred(shape, 1.5, 610 + seed)
        _check(cp, lib, img)
        D, H, W = shape
        zc = lib.cp_get_tuning(1)
        tasks = -(-W // 31) * -(-H // 8) * -(-D // zc)
        assert _check.tma_tasks == tasks, ("TMA path not taken", _check.tma_tasks, tasks)
    img = rng.random((10, 12, 41), dtype=np.float32)
    _check(cp, lib, img)
    assert _check.tma_tasks == 0
