"""GPU parity of the T-filtration (pixel values on the top cells) against the
T oracle, element by element and bit-exact, through the C-ABI entry points
cubical_persistence_t_2d / _t_3d: values are copies of input pixels, cells
and pixels are integers.  The CUDA path runs the V pipeline on the dual image
and maps the pairs back; the oracle builds the T-complex directly.
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


def _check(cp, img, what=""):
    got = cp.persistence(torch.from_numpy(np.ascontiguousarray(img)).cuda(), filtration="T").numpy()
    want = oracle.persistence_t(img)
    what = what or str(img.shape)
    assert len(got) == len(want), f"{what}: {len(got)} pairs vs oracle {len(want)}"
    for k in FIELDS:
        if not np.array_equal(got[k], want[k]):
            i = int(np.argmax(got[k] != want[k]))
            raise AssertionError(f"{what}: field {k} differs at pair {i}: {got[i]} vs {want[i]}")
    assert (got["item"] == 0).all()
    return got


@pytest.mark.parametrize("shape", [(1, 1), (1, 2), (2, 1), (1, 9), (5, 1), (2, 2), (3, 3), (31, 33), (40, 97), (64, 64)])
def test_t_2d_shapes(cp, shape):
    rng = np.random.default_rng(sum(shape) + 500)
    _check(cp, rng.random(shape, dtype=np.float32), f"uniform {shape}")
    _check(cp, rng.integers(0, 3, shape).astype(np.float32), f"3 levels {shape}")
    _check(cp, rng.integers(0, 2, shape).astype(np.float32), f"binary {shape}")


def test_t_2d_random(cp):
    rng = np.random.default_rng(501)
    for _ in range(40):
        shape = tuple(int(v) for v in rng.integers(1, 80, 2))
        img = rng.integers(0, 4, shape).astype(np.float32) if rng.random() < 0.5 else rng.random(shape, dtype=np.float32)
        if rng.random() < 0.3:
            img = img - 0.5
        _check(cp, img)


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 1), (1, 4, 4), (2, 2, 2), (3, 4, 5), (9, 9, 33), (17, 9, 40), (20, 12, 5)])
def test_t_3d_shapes(cp, shape):
    rng = np.random.default_rng(sum(shape) + 600)
    _check(cp, rng.random(shape, dtype=np.float32), f"uniform {shape}")
    _check(cp, rng.integers(0, 3, shape).astype(np.float32), f"3 levels {shape}")


def test_t_3d_random_and_blurred(cp):
    rng = np.random.default_rng(601)
    for _ in range(12):
        shape = tuple(int(v) for v in rng.integers(1, 24, 3))
        img = rng.integers(0, 3, shape).astype(np.float32) if rng.random() < 0.5 else rng.random(shape, dtype=np.float32)
        _check(cp, img)
    _check(cp, workloads.blurred((70, 9, 12), 2.0, 602), "blurred 70x9x12")
    _check(cp, workloads.blurred((48, 48, 48), 2.0, 603), "blurred 48^3")


def test_t_larger_volume(cp):
    """Several 3D pruning tiles and z chunks of the padded image, smooth field."""
    _check(cp, workloads.blurred((96, 96, 96), 3.0, 604), "blurred 96^3")


def test_t_2d_config_sizes(cp):
    (img,) = workloads.config("2d_64_uniform")
    _check(cp, img, "64x64 uniform")
    _check(cp, workloads.blurred((256, 300), 4.0, 605), "blurred 256x300")


def test_t_signed_zero_and_constant(cp):
    img = np.zeros((6, 7), dtype=np.float32)
    img[::2, ::3] = -0.0
    got = _check(cp, img, "signed zeros")
    assert not np.signbit(got["birth"]).any() and not np.signbit(got["death"]).any()
    _check(cp, np.full((5, 4, 3), 2.5, dtype=np.float32), "constant 3D")
    _check(cp, -np.abs(np.random.default_rng(606).random((9, 11), dtype=np.float32)), "non-positive")


def test_t_ring_hand_case(cp):
    img = np.array([[0, 0, 0], [0, 5, 0], [0, 0, 0]], dtype=np.float32)
    got = _check(cp, img, "ring")
    assert len(got) == 2 and got[1]["dim"] == 1 and got[1]["birth"] == 0.0 and got[1]["death"] == 5.0


def test_t_errors(cp):
    lib = cp.load()
    x = torch.zeros((4, 4), device="cuda")
    dims = (ctypes.c_int64 * 2)(4, 4)
    assert lib.cubical_persistence_t_workspace_size(2, dims, 0) > lib.cubical_persistence_workspace_size(2, dims, 0)
    bad = torch.rand((6, 6), device="cuda")
    bad[2, 3] = float("nan")
    with pytest.raises(cp.CpError):
        cp.persistence(bad, filtration="T")
    big = torch.rand((6, 6), device="cuda")
    big[1, 1] = float(np.finfo(np.float32).max)  # the frame would have to lie below -FLT_MAX
    with pytest.raises(cp.CpError):
        cp.persistence(big, filtration="T")
    # the context stays usable
    _check(cp, np.random.default_rng(607).random((7, 5), dtype=np.float32), "after errors")


def test_t_gradient(cp):
    """dL/dimage scatters to the top cells the birth and death cells enter with."""
    rng = np.random.default_rng(608)
    img = rng.random((13, 17), dtype=np.float32)
    x = torch.from_numpy(img).cuda().requires_grad_()
    birth, death, raw = cp.diagram(x, filtration="T")
    fin = torch.isfinite(death)
    loss = ((death - birth)[fin] ** 2).sum()
    loss.backward()
    want = np.zeros(img.size, dtype=np.float64)
    for r in oracle.persistence_t(img):
        if r["death_cell"] < 0:
            continue
        g = 2.0 * (float(r["death"]) - float(r["birth"]))
        want[r["death_pixel"]] += g
        want[r["birth_pixel"]] -= g
    np.testing.assert_allclose(x.grad.cpu().numpy().ravel(), want.astype(np.float32), rtol=1e-6, atol=1e-6)


def test_t_batched_mixed(cp):
    """Images and volumes of uneven sizes (extents of 1 included) in one
    T-filtration call: each item's pairs equal the oracle's for that item,
    in (item, dim, birth cell) order."""
    rng = np.random.default_rng(609)
    items = []
    for k in range(14):
        if k % 3 == 2:
            shape = tuple(int(v) for v in rng.integers(1, 14, 3))
        else:
            shape = tuple(int(v) for v in rng.integers(1, 60, 2))
        img = rng.integers(0, 3, shape).astype(np.float32) if rng.random() < 0.4 else rng.random(shape, dtype=np.float32)
        items.append(img)
    items.append(workloads.blurred((40, 33, 29), 2.0, 610))
    d = cp.persistence_batched([torch.from_numpy(a).cuda() for a in items], filtration="T")
    got = d.numpy()
    assert np.all(np.diff(got["item"]) >= 0)
    for i, a in enumerate(items):
        g = got[got["item"] == i]
        w = oracle.persistence_t(a)
        assert len(g) == len(w), (i, a.shape, len(g), len(w))
        for k in FIELDS:
            assert np.array_equal(g[k], w[k]), (i, a.shape, k)


def test_t_batched_graph_step(cp):
    """The batched forward + loss + backward of the T-filtration as one CUDA
    graph: pairs per item equal the oracle's, the loss is their total
    persistence above tau, and the gradient scatters to their pixels."""
    rng = np.random.default_rng(611)
    items = [rng.random((23, 31), dtype=np.float32), workloads.blurred((12, 14, 10), 1.5, 612),
             rng.integers(0, 3, (1, 17)).astype(np.float32), rng.random((5, 1, 7), dtype=np.float32)]
    tau = 0.05
    bp = cp.BatchedPersistence([a.shape for a in items], tau=tau, filtration="T", graph=True)
    bp.load([torch.from_numpy(a) for a in items])
    loss, grad = bp.step()
    loss, grad = bp.step()  # a replay of the captured graph
    torch.cuda.synchronize()
    got = bp.pairs().numpy()
    want_loss = 0.0
    grads = bp.grads()
    for i, a in enumerate(items):
        g = got[got["item"] == i]
        w = oracle.persistence_t(a)
        assert len(g) == len(w)
        for k in FIELDS:
            assert np.array_equal(g[k], w[k]), (i, k)
        ref = np.zeros(a.size, dtype=np.float64)
        for r in w:
            if r["death_cell"] < 0:
                continue
            pers = float(r["death"]) - float(r["birth"])
            if pers > float(np.float32(tau)):  # the library compares in double against the float threshold
                want_loss += pers * pers
                ref[r["death_pixel"]] += 2.0 * pers
                ref[r["birth_pixel"]] -= 2.0 * pers
        np.testing.assert_allclose(grads[i].cpu().numpy().ravel(), ref.astype(np.float32), rtol=1e-6, atol=1e-6)
    assert abs(float(loss.item()) - want_loss) <= 1e-9 * max(1.0, want_loss)
