"""GPU parity of the whole diagram of volumes (H0, H1, H2) against the
oracle's full diagram, element by element and bit-exact, through the C-ABI
entry points cubical_persistence_full_3d / _full_batched: values are copies
of input values, cells and pixels are integers.  The CUDA path reduces only
the squares not paired in H2 over the edges not paired in H0, in parallel
rounds; the oracle reduces every square over every edge in sequence.
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


def _compare(got, want, what):
    assert len(got) == len(want), f"{what}: {len(got)} pairs vs oracle {len(want)}"
    for k in FIELDS:
        if not np.array_equal(got[k], want[k]):
            i = int(np.argmax(got[k] != want[k]))
            raise AssertionError(f"{what}: field {k} differs at pair {i}: {got[i]} vs {want[i]}")


def _check(cp, img, what="", **kw):
    got = cp.persistence_full(torch.from_numpy(np.ascontiguousarray(img)).cuda(), **kw).numpy()
    _compare(got, oracle.persistence_full(img), what or str(img.shape))
    assert (got["item"] == 0).all()
    return got


@pytest.mark.parametrize("shape", [(2, 2, 2), (2, 3, 2), (3, 4, 5), (2, 9, 9), (9, 9, 33), (17, 9, 40), (20, 12, 5)])
def test_full_shapes(cp, shape):
    rng = np.random.default_rng(sum(shape) + 800)
    _check(cp, rng.random(shape, dtype=np.float32), f"uniform {shape}")
    _check(cp, rng.integers(0, 3, shape).astype(np.float32), f"3 levels {shape}")
    _check(cp, rng.integers(0, 2, shape).astype(np.float32), f"binary {shape}")


def test_full_random(cp):
    rng = np.random.default_rng(801)
    for _ in range(40):
        shape = tuple(int(v) for v in rng.integers(2, 16, 3))
        img = rng.integers(0, 4, shape).astype(np.float32) if rng.random() < 0.5 else rng.random(shape, dtype=np.float32)
        if rng.random() < 0.3:
            img = img - 0.5
        _check(cp, img)


def test_full_exhaustive_binary_2x2x2(cp):
    for code in range(256):
        img = np.array([(code >> i) & 1 for i in range(8)], dtype=np.float32).reshape(2, 2, 2)
        _check(cp, img, f"binary 2x2x2 #{code}")


def test_full_larger_volumes(cp):
    """Several pruning tiles and tasks; long reductions in the smooth field."""
    _check(cp, workloads.blurred((48, 48, 48), 2.0, 802), "blurred 48^3")
    _check(cp, np.random.default_rng(803).random((40, 33, 29), dtype=np.float32), "uniform 40x33x29")
    _check(cp, workloads.blurred((64, 40, 48), 3.0, 804), "blurred 64x40x48")


def test_full_solid_torus(cp):
    img = np.full((3, 5, 5), 9.0, dtype=np.float32)
    img[1, 1:4, 1:4] = 0.0
    img[1, 2, 2] = 5.0
    got = _check(cp, img, "solid torus")
    h1 = got[got["dim"] == 1]
    assert len(h1) == 1 and (h1[0]["birth"], h1[0]["death"], h1[0]["death_pixel"]) == (0.0, 5.0, 37)


def test_full_constant_and_signed_zero(cp):
    _check(cp, np.full((4, 5, 6), 1.5, dtype=np.float32), "constant")
    img = np.random.default_rng(805).integers(0, 2, (5, 6, 7)).astype(np.float32)
    img[img == 0] = -0.0
    got = _check(cp, img, "signed zeros")
    assert not np.signbit(got["birth"]).any()


def test_full_equals_plain_outside_h1(cp):
    """The H0 and H2 pairs are those of the plain call; 2D images get the plain diagram."""
    img = workloads.blurred((30, 31, 32), 2.0, 806)
    x = torch.from_numpy(img).cuda()
    full = cp.persistence_full(x).numpy()
    plain = cp.persistence(x).numpy()
    assert np.array_equal(full[full["dim"] != 1], plain)
    im2 = torch.from_numpy(np.random.default_rng(807).random((40, 50), dtype=np.float32)).cuda()
    assert np.array_equal(cp.persistence_full(im2).numpy(), cp.persistence(im2).numpy())


def test_full_pool_growth(cp):
    """A pool with no room for merged columns: the call reports capacity and
    the binding grows it until the reduction fits; the result is unchanged."""
    img = np.random.default_rng(808).random((14, 15, 16), dtype=np.float32)
    lib = cp.load()
    x = torch.from_numpy(img).cuda()
    dims = (ctypes.c_int64 * 3)(*img.shape)
    ws_bytes = lib.cubical_persistence_full_workspace_size(3, dims, 0, 1)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    cap = 100000
    out = torch.empty((cap, 8), dtype=torch.int32, device="cuda")
    cnt = ctypes.c_int64(0)
    sp = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.cubical_persistence_full_3d(ctypes.c_void_p(x.data_ptr()), dims, ctypes.c_void_p(out.data_ptr()), cap,
                                         ctypes.byref(cnt), None, ctypes.c_void_p(ws.data_ptr()), ws_bytes, 0, 1, sp)
    assert rc == -3  # CP_ERR_CAPACITY
    info = (ctypes.c_int64 * 4)()
    one = (ctypes.c_int32 * 1)(3)
    d3 = (ctypes.c_int64 * 3)(*img.shape)
    assert lib.cubical_persistence_full_info(ctypes.c_void_p(ws.data_ptr()), 1, one, d3, 0, 1, info, 4, sp) == 0
    assert info[2] > info[3]
    _check(cp, img, "after pool growth", pool_entries=1)
    # the context stays usable and the default pool fits
    _check(cp, img, "default pool")


def test_full_info_counts(cp):
    """One column per edge not paired in H0: E - N + 1."""
    img = workloads.blurred((20, 21, 22), 2.0, 809)
    lib = cp.load()
    x = torch.from_numpy(img).cuda()
    D, H, W = img.shape
    dims = (ctypes.c_int64 * 3)(D, H, W)
    ws_bytes = lib.cubical_persistence_full_workspace_size(3, dims, 0, 0)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    cap = 200000
    out = torch.empty((cap, 8), dtype=torch.int32, device="cuda")
    cnt = ctypes.c_int64(0)
    sp = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.cubical_persistence_full_3d(ctypes.c_void_p(x.data_ptr()), dims, ctypes.c_void_p(out.data_ptr()), cap,
                                         ctypes.byref(cnt), None, ctypes.c_void_p(ws.data_ptr()), ws_bytes, 0, 0, sp)
    assert rc == 0
    info = (ctypes.c_int64 * 4)()
    one = (ctypes.c_int32 * 1)(3)
    assert lib.cubical_persistence_full_info(ctypes.c_void_p(ws.data_ptr()), 1, one, dims, 0, 0, info, 4, sp) == 0
    E = D * H * (W - 1) + D * (H - 1) * W + (D - 1) * H * W
    assert info[0] == E - D * H * W + 1
    assert info[1] >= 1 and 0 <= info[2] <= info[3]


def test_full_batched_mixed(cp):
    """Images and volumes of uneven sizes in one call: each item's pairs equal
    the oracle's full diagram for that item, in (item, dim, birth cell) order."""
    rng = np.random.default_rng(810)
    items = []
    for k in range(12):
        if k % 3 == 0:
            shape = tuple(int(v) for v in rng.integers(2, 40, 2))
        else:
            shape = tuple(int(v) for v in rng.integers(2, 14, 3))
        img = rng.integers(0, 3, shape).astype(np.float32) if rng.random() < 0.4 else rng.random(shape, dtype=np.float32)
        items.append(img)
    items.append(workloads.blurred((33, 29, 31), 2.0, 811))
    got = cp.persistence_full_batched([torch.from_numpy(a).cuda() for a in items]).numpy()
    assert np.all(np.diff(got["item"]) >= 0)
    for i, a in enumerate(items):
        _compare(got[got["item"] == i], oracle.persistence_full(a), f"item {i} {a.shape}")


def test_full_gradient(cp):
    """dL/dimage of the full diagram scatters to the birth and death pixels of
    every finite pair, H1 included."""
    img = np.random.default_rng(812).random((7, 8, 9), dtype=np.float32)
    x = torch.from_numpy(img).cuda().requires_grad_()
    birth, death, raw = cp.diagram(x, full=True)
    fin = torch.isfinite(death)
    ((death - birth)[fin] ** 2).sum().backward()
    want = np.zeros(img.size, dtype=np.float64)
    for r in oracle.persistence_full(img):
        if r["death_cell"] < 0:
            continue
        g = 2.0 * (float(r["death"]) - float(r["birth"]))
        want[r["death_pixel"]] += g
        want[r["birth_pixel"]] -= g
    assert int((raw[:, 6] == 1).sum()) > 0
    np.testing.assert_allclose(x.grad.cpu().numpy().ravel(), want.astype(np.float32), rtol=1e-6, atol=1e-6)


def test_full_nonfinite(cp):
    bad = torch.rand((6, 7, 8), device="cuda")
    bad[2, 3, 4] = float("nan")
    with pytest.raises(cp.CpError):
        cp.persistence_full(bad)
    _check(cp, np.random.default_rng(813).random((5, 6, 7), dtype=np.float32), "after an error")


def test_full_time_budget(cp):
    """The cross-star rounds run in one non-preemptible launch; their
    wall-clock budget (CP_TUNE_H1_BUDGET_MS) stops them at a round boundary
    with CP_ERR_TIMEOUT, and the context stays usable.  Budget 0 stops after
    the first round; this blurred volume needs many more."""
    from paper_2606_04801_gb300._lib import CP_ERR_TIMEOUT, CpError

    lib = cp.load()
    img = workloads.blurred((40, 36, 44), 2.0, 17)
    x = torch.from_numpy(img).cuda()
    old = lib.cp_get_tuning(4)
    assert old == 30000
    assert lib.cp_set_tuning(4, -1) != 0 and lib.cp_set_tuning(4, 3600001) != 0
    assert lib.cp_set_tuning(4, 0) == 0
    try:
        with pytest.raises(CpError) as e:
            cp.persistence_full(x)
        assert e.value.code == CP_ERR_TIMEOUT
    finally:
        assert lib.cp_set_tuning(4, old) == 0
    _check(cp, img, "after a spent budget")
    # volumes above the practical bound need an explicit opt-in
    side = round(cp.api.H1_PRACTICAL_VOXELS ** (1 / 3))
    assert side ** 3 == cp.api.H1_PRACTICAL_VOXELS
    with pytest.raises(ValueError):
        cp.persistence_full(torch.zeros((side + 1, side, side), device="cuda"))


@pytest.mark.parametrize("solo", [0, 1, 8, 1024])
def test_full_solo_rounds(cp, solo):
    """The cross-star rounds give the same pairs whether the grid runs every
    round (0), or the first CTA runs the rounds with few columns alone and
    wakes the grid again (1, 8), or runs nearly all of them alone (1024)."""
    from paper_2606_04801_gb300 import _lib

    lib = _lib.load()
    old = lib.cp_get_tuning(6)
    try:
        assert lib.cp_set_tuning(6, solo) == 0
        for seed, (shape, sigma) in enumerate([((24, 20, 22), 1.5), ((33, 17, 19), 2.0)]):
            _check(cp, workloads.blurred(shape, sigma, seed), f"blurred {shape} solo={solo}")
        rng = np.random.default_rng(900 + solo)
        _check(cp, rng.random((14, 15, 16), dtype=np.float32), f"uniform solo={solo}")
    finally:
        lib.cp_set_tuning(6, old)
