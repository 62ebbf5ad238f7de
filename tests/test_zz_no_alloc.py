"""The backward entry point that allocates nothing.

Callers that cannot allocate device memory (for example code inside another
framework's hooks without access to its allocator, or deployments whose
device memory is reserved up front by another component) use
cubical_persistence_backward_noalloc, which keeps its accumulators in a fixed
array inside the library instead of a workspace.  These tests call it through
the C-ABI and check it against cubical_persistence_backward on the same pairs
and gradients, twice in a row with different gradients (the shared array must
be cleared between calls), for one image and for a batch with item offsets.
"""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
RTOL = 1e-6  # the gradient tests' tolerance


@pytest.fixture(scope="module")
def cp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_04801_gb300 as cp

    return cp


def _with_workspace(lib, raw, gb, gd, offs, n_pixels):
    grad = torch.full((n_pixels,), float("nan"), dtype=torch.float32, device="cuda")
    ws_bytes = lib.cubical_persistence_backward_workspace_size(n_pixels)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    rc = lib.cubical_persistence_backward(
        ctypes.c_void_p(raw.data_ptr()), raw.shape[0], ctypes.c_void_p(gb.data_ptr()), ctypes.c_void_p(gd.data_ptr()),
        None if offs is None else ctypes.c_void_p(offs.data_ptr()), ctypes.c_void_p(grad.data_ptr()), n_pixels,
        ctypes.c_void_p(ws.data_ptr()), ws_bytes, None,
    )
    assert rc == 0
    return grad


def _no_alloc(lib, raw, gb, gd, offs, n_pixels):
    grad = torch.full((n_pixels,), float("nan"), dtype=torch.float32, device="cuda")
    rc = lib.cubical_persistence_backward_noalloc(
        ctypes.c_void_p(raw.data_ptr()), raw.shape[0], ctypes.c_void_p(gb.data_ptr()), ctypes.c_void_p(gd.data_ptr()),
        None if offs is None else ctypes.c_void_p(offs.data_ptr()), ctypes.c_void_p(grad.data_ptr()), n_pixels, None,
    )
    assert rc == 0
    return grad


def _compare(a, b):
    a = a.cpu().numpy()
    b = b.cpu().numpy()
    assert np.isfinite(a).all() and np.isfinite(b).all()
    scale = max(1.0, float(np.abs(b).max()))
    np.testing.assert_allclose(a, b, rtol=RTOL, atol=RTOL * scale)


def test_no_alloc_matches_workspace_backward_single(cp):
    lib = cp.load()
    img = torch.from_numpy(workloads.rank_spaced(workloads.blurred((96, 80), 2.0, 21))).cuda()
    d = cp.persistence(img)
    rng = np.random.default_rng(0)
    for _ in range(2):  # two calls in a row, different gradients
        gb = torch.from_numpy(rng.standard_normal(len(d)).astype(np.float32)).cuda()
        gd = torch.from_numpy(rng.standard_normal(len(d)).astype(np.float32)).cuda()
        want = _with_workspace(lib, d.raw, gb, gd, None, img.numel())
        got = _no_alloc(lib, d.raw, gb, gd, None, img.numel())
        torch.cuda.synchronize()
        _compare(got, want)


def test_no_alloc_matches_workspace_backward_batched(cp):
    lib = cp.load()
    items = [
        workloads.rank_spaced(workloads.blurred((40, 57), 2.0, 22)),
        workloads.rank_spaced(workloads.blurred((12, 14, 11), 1.5, 23)),
        workloads.uniform((33, 31), 24),
    ]
    tens = [torch.from_numpy(a).cuda() for a in items]
    d = cp.persistence_batched(tens)
    sizes = [a.size for a in items]
    offs = torch.tensor(np.concatenate([[0], np.cumsum(sizes)[:-1]]), dtype=torch.int64, device="cuda")
    n = int(sum(sizes))
    rng = np.random.default_rng(1)
    for _ in range(2):
        gb = torch.from_numpy(rng.standard_normal(len(d)).astype(np.float32)).cuda()
        gd = torch.from_numpy(rng.standard_normal(len(d)).astype(np.float32)).cuda()
        want = _with_workspace(lib, d.raw, gb, gd, offs, n)
        got = _no_alloc(lib, d.raw, gb, gd, offs, n)
        torch.cuda.synchronize()
        _compare(got, want)


def test_no_alloc_rejects_too_many_pixels(cp):
    lib = cp.load()
    mx = lib.cubical_persistence_backward_noalloc_max_pixels()
    assert mx == 1 << 22
    raw = torch.zeros((1, 8), dtype=torch.int32, device="cuda")
    g = torch.zeros(1, dtype=torch.float32, device="cuda")
    rc = lib.cubical_persistence_backward_noalloc(
        ctypes.c_void_p(raw.data_ptr()), 1, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(g.data_ptr()), None,
        ctypes.c_void_p(g.data_ptr()), mx + 1, None,
    )
    assert rc == -3  # CP_ERR_CAPACITY
