"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle,
element by element and bit-exact: values are copies of input pixels and
cells/pixels are integers, so every field must be identical.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
FIELDS = ("birth", "death", "birth_cell", "death_cell", "birth_pixel", "death_pixel", "dim")


@pytest.fixture(scope="module")
def cp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_04801_gb300 as cp

    return cp


def _assert_same(got, want, what=""):
    assert len(got) == len(want), f"{what}: {len(got)} pairs vs oracle {len(want)}"
    for k in FIELDS:
        g, w = got[k], want[k]
        if not np.array_equal(g, w):
            i = int(np.argmax(g != w))
            raise AssertionError(f"{what}: field {k} differs at pair {i}: {got[i]} vs {want[i]}")


def _check(cp, img, what="", **kw):
    d = cp.persistence(torch.from_numpy(np.ascontiguousarray(img)).cuda(), **kw)
    got = d.numpy()
    _assert_same(got, oracle.persistence(img), what or str(img.shape))
    assert (got["item"] == 0).all()
    return got


def test_config_2d_64_uniform(cp):
    (img,) = workloads.config("2d_64_uniform")
    _check(cp, img, "64x64 uniform")


SHAPES_2D = [(2, 2), (2, 7), (7, 2), (3, 3), (31, 33), (32, 32), (33, 31), (64, 65), (65, 64), (40, 97), (1, 2)][:-1]


@pytest.mark.parametrize("shape", SHAPES_2D)
def test_small_2d_shapes(cp, shape):
    rng = np.random.default_rng(sum(shape))
    _check(cp, rng.random(shape, dtype=np.float32), f"uniform {shape}")
    _check(cp, rng.integers(0, 3, shape).astype(np.float32), f"3 levels {shape}")
    _check(cp, rng.integers(0, 2, shape).astype(np.float32), f"binary {shape}")


def test_random_2d(cp):
    rng = np.random.default_rng(11)
    for _ in range(60):
        shape = tuple(int(v) for v in rng.integers(2, 90, 2))
        img = rng.integers(0, 4, shape).astype(np.float32) if rng.random() < 0.5 else rng.random(shape, dtype=np.float32)
        _check(cp, img)


SHAPES_3D = [(2, 2, 2), (2, 3, 4), (4, 3, 2), (8, 8, 32), (9, 9, 33), (7, 8, 31), (17, 9, 40), (3, 17, 65), (20, 12, 5)]


@pytest.mark.parametrize("shape", SHAPES_3D)
def test_small_3d_shapes(cp, shape):
    rng = np.random.default_rng(sum(shape) + 1)
    _check(cp, rng.random(shape, dtype=np.float32), f"uniform {shape}")
    _check(cp, rng.integers(0, 3, shape).astype(np.float32), f"3 levels {shape}")


def test_random_3d(cp):
    rng = np.random.default_rng(12)
    for _ in range(30):
        shape = tuple(int(v) for v in rng.integers(2, 24, 3))
        img = rng.integers(0, 4, shape).astype(np.float32) if rng.random() < 0.5 else rng.random(shape, dtype=np.float32)
        _check(cp, img)


def test_special_values(cp):
    img = np.array([[-0.0, 1e-38, -1e-38], [3.4e38, -3.4e38, 0.0], [1.0, -0.0, 2.0]], dtype=np.float32)
    got = _check(cp, img)
    assert not np.signbit(got["birth"][got["birth"] == 0]).any()
    _check(cp, np.full((5, 6), 7.0, dtype=np.float32), "constant")
    _check(cp, np.full((4, 3, 5), -1.0, dtype=np.float32), "constant 3d")
    idx = np.indices((9, 10)).sum(axis=0)
    _check(cp, (idx % 2).astype(np.float32), "checkerboard 2d")
    idx = np.indices((5, 6, 7)).sum(axis=0)
    _check(cp, (idx % 2).astype(np.float32), "checkerboard 3d")
    _check(cp, np.arange(60, dtype=np.float32).reshape(6, 10), "ramp")
    _check(cp, -np.arange(60, dtype=np.float32).reshape(3, 4, 5), "reverse ramp 3d")


def test_config_2d_2048(cp):
    for img, name in zip(workloads.config("2d_2048_grf"), ("grf", "quantised")):
        _check(cp, img, f"2048^2 {name}")


def test_config_2d_cross_pruning(cp):
    """The paper's sequential 2D order (CP_TUNE_CROSS_PRUNE_2D = 1: the dual
    list takes the H0-positive edges after the H0 union-find) gives the same
    pairs as the default, where both dimensions run at once."""
    lib = cp.load()
    assert lib.cp_set_tuning(5, 1) == 0
    try:
        for img, name in zip(workloads.config("2d_2048_grf"), ("grf", "quantised")):
            _check(cp, img, f"2048^2 {name}, cross-pruned")
        _check(cp, workloads.uniform((64, 64), 0), "64x64 uniform, cross-pruned")
        rng = np.random.default_rng(19)
        for _ in range(20):
            shape = tuple(int(v) for v in rng.integers(2, 60, 2))
            img = rng.integers(0, 3, shape).astype(np.float32) if rng.random() < 0.5 else rng.random(shape, dtype=np.float32)
            _check(cp, img, f"{shape}, cross-pruned")
        _batch_check(cp, workloads.batch(0, n2d=8, n3d=2, scale=0.2))
    finally:
        assert lib.cp_set_tuning(5, 0) == 0


def test_config_3d_128(cp):
    for img, name in zip(workloads.config("3d_128"), ("uniform", "blurred")):
        _check(cp, img, f"128^3 {name}")


def _batch_check(cp, items):
    d = cp.persistence_batched([torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in items])
    got = d.numpy()
    assert (np.diff(got["item"]) >= 0).all()
    for i, a in enumerate(items):
        _assert_same(got[got["item"] == i], oracle.persistence(a), f"item {i} {a.shape}")


def test_batched_mixed(cp):
    rng = np.random.default_rng(13)
    items = []
    for i in range(20):
        if i % 3 == 2:
            shape = tuple(int(v) for v in rng.integers(2, 14, 3))
        else:
            shape = tuple(int(v) for v in rng.integers(2, 60, 2))
        items.append(rng.integers(0, 3, shape).astype(np.float32) if i % 2 else rng.random(shape, dtype=np.float32))
    _batch_check(cp, items)


def test_batched_workload_recipe_scaled(cp):
    _batch_check(cp, workloads.batch(0, n2d=12, n3d=3, scale=0.25))


def test_deterministic(cp):
    img = workloads.quantised(workloads.blurred((300, 257), 3.0, 5))
    t = torch.from_numpy(img).cuda()
    a = cp.persistence(t).raw.cpu()
    for _ in range(3):
        assert torch.equal(cp.persistence(t).raw.cpu(), a)


def test_capacity_growth(cp):
    """A tiny survivor capacity forces CP_ERR_CAPACITY, then the binding grows the workspace."""
    idx = np.indices((40, 40)).sum(axis=0)
    img = (idx % 2).astype(np.float32)  # every 1-pixel has 4 separate lower groups
    _check(cp, img, "checkerboard small capacity", max_survivors=16)
    vol = np.random.default_rng(3).random((12, 13, 14), dtype=np.float32)
    _check(cp, vol, "3d small capacity", max_survivors=64)


def test_joint_union_find_one_after_the_other(cp):
    """Volumes run both union-finds in one launch with their active lists side by
    side; when the two lists do not fit the scratch together, the launch runs
    them one after the other.  Both must give the oracle's pairs."""
    vol = workloads.blurred((40, 44, 48), 1.5, 17)
    want = oracle.persistence(vol)
    d = cp.persistence(torch.from_numpy(vol).cuda(), with_stats=True)
    _assert_same(d.numpy(), want, "joint, side by side")
    st = d.stats
    ms = max(st["h0_survivors"], st["top_survivors"], 2 * st["h0_roots"], 2 * st["top_roots"]) + 16
    assert st["h0_survivors"] + st["top_survivors"] > ms  # the lists do not fit side by side
    d2 = cp.persistence(torch.from_numpy(vol).cuda(), max_survivors=ms, with_stats=True)
    _assert_same(d2.numpy(), want, "joint, one after the other")
    assert d2.stats["h0_rounds"] == st["h0_rounds"] and d2.stats["top_rounds"] == st["top_rounds"]


def test_errors_through_c_abi(cp):
    lib = cp.load()
    img = torch.zeros((8, 8), device="cuda")
    img[3, 4] = float("nan")
    with pytest.raises(cp.CpError) as e:
        cp.persistence(img)
    assert e.value.code == -2
    img[3, 4] = float("inf")
    with pytest.raises(cp.CpError) as e:
        cp.persistence(img)
    assert e.value.code == -2
    dims = (ctypes.c_int64 * 2)(1, 8)
    assert lib.cubical_persistence_workspace_size(2, dims, 0) == 0
    out = torch.empty((4, 8), dtype=torch.int32, device="cuda")
    cnt = ctypes.c_int64()
    dims = (ctypes.c_int64 * 2)(1, 8)
    rc = lib.cubical_persistence_2d(ctypes.c_void_p(img.data_ptr()), dims, ctypes.c_void_p(out.data_ptr()), 4,
                                    ctypes.byref(cnt), None, None, 0, 0, None)
    assert rc == -1
    # output capacity too small: the count is still reported
    good = torch.from_numpy(workloads.uniform((32, 32), 4)).cuda()
    dims = (ctypes.c_int64 * 2)(32, 32)
    ws_bytes = lib.cubical_persistence_workspace_size(2, dims, 0)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    rc = lib.cubical_persistence_2d(ctypes.c_void_p(good.data_ptr()), dims, ctypes.c_void_p(out.data_ptr()), 4,
                                    ctypes.byref(cnt), None, ctypes.c_void_p(ws.data_ptr()), ws_bytes, 0, None)
    assert rc == -3
    assert cnt.value == len(oracle.persistence(workloads.uniform((32, 32), 4)))
    # undersized workspace
    rc = lib.cubical_persistence_2d(ctypes.c_void_p(good.data_ptr()), dims, ctypes.c_void_p(out.data_ptr()), 4,
                                    ctypes.byref(cnt), None, ctypes.c_void_p(ws.data_ptr()), ws_bytes - 1, 0, None)
    assert rc == -1
