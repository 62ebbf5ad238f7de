"""GPU parity of the slab split of the union-finds (cubical_persistence_slabs):
bit-exact against the oracle on small volumes and images for many slab
counts (ragged slabs, more slabs than planes), identical to the unsplit call
on larger inputs (the unsplit call is itself compared with the oracle at the
same sizes in test_gpu_parity.py and test_gpu_zz_full_parity.py), and the
split's counts are consistent."""
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


def _same(got, want, what):
    assert len(got) == len(want), f"{what}: {len(got)} pairs vs {len(want)}"
    for k in FIELDS:
        if not np.array_equal(got[k], want[k]):
            i = int(np.argmax(got[k] != want[k]))
            raise AssertionError(f"{what}: field {k} differs at pair {i}: {got[i]} vs {want[i]}")


def _stats_ok(st, S):
    for q in range(2):
        assert st["internal"][q] + st["crossing"][q] == st["survivors"][q]
        assert st["merged"][q] == st["committed"][q] - st["final_pairs"][q] + st["crossing"][q]
        assert st["final_pairs"][q] <= st["committed"][q] <= st["internal"][q]
        if S == 1:
            assert st["crossing"][q] == 0


SHAPES_3D = [(2, 2, 2), (5, 9, 33), (17, 9, 40), (20, 12, 5), (33, 16, 16)]


@pytest.mark.parametrize("shape", SHAPES_3D)
@pytest.mark.parametrize("S", [1, 2, 3, 5, 8, 64])
def test_volumes_equal_oracle(cp, shape, S):
    rng = np.random.default_rng(sum(shape) * 7 + S)
    for kind, img in (
        ("uniform", rng.random(shape, dtype=np.float32)),
        ("3 levels", rng.integers(0, 3, shape).astype(np.float32)),
        ("blurred", workloads.blurred(shape, 1.5, S)),
    ):
        d = cp.persistence_slabs(torch.from_numpy(img).cuda(), S)
        _same(d.numpy(), oracle.persistence(img), f"{kind} {shape} S={S}")
        _stats_ok(d.stats, S)


@pytest.mark.parametrize("shape", [(2, 5), (31, 33), (64, 65), (97, 40)])
@pytest.mark.parametrize("S", [1, 2, 7, 100])
def test_images_equal_oracle(cp, shape, S):
    rng = np.random.default_rng(sum(shape) + S)
    for img in (rng.random(shape, dtype=np.float32), rng.integers(0, 4, shape).astype(np.float32)):
        d = cp.persistence_slabs(torch.from_numpy(img).cuda(), S)
        _same(d.numpy(), oracle.persistence(img), f"{shape} S={S}")
        _stats_ok(d.stats, S)


@pytest.mark.parametrize("S", [2, 8, 152])
def test_equals_unsplit_call(cp, S):
    for img in (workloads.blurred((128, 128, 128), 3.0, 1), workloads.uniform((96, 80, 72), 2)):
        x = torch.from_numpy(img).cuda()
        a = cp.persistence(x).raw
        d = cp.persistence_slabs(x, S)
        assert torch.equal(a, d.raw), f"S={S} {img.shape}"
        _stats_ok(d.stats, S)
        assert d.stats["crossing"][0] > 0 and d.stats["committed"][0] > 0


def test_survivor_lists_grow(cp):
    """The two survivor lists sit side by side in the scratch lists: with
    max_survivors between the longer list and their sum the call reports
    CP_ERR_CAPACITY, and the binding grows the workspace."""
    import ctypes

    from paper_2606_04801_gb300 import _lib

    img = workloads.uniform((40, 36, 33), 9)
    x = torch.from_numpy(img).cuda()
    st = cp.persistence_slabs(x, 4).stats
    n0, n1 = st["survivors"]
    ms = max(n0, n1) + 16
    assert ms < n0 + n1
    lib = _lib.load()
    dims = (ctypes.c_int64 * 3)(*img.shape)
    wsb = lib.cubical_persistence_slabs_workspace_size(3, dims, 4, ms)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    cap = img.size + 40000
    out = torch.empty((cap, 8), dtype=torch.int32, device="cuda")
    cnt = ctypes.c_int64(0)
    rc = lib.cubical_persistence_slabs(3, ctypes.c_void_p(x.data_ptr()), dims, 4, ctypes.c_void_p(out.data_ptr()),
                                       cap, ctypes.byref(cnt), None, ctypes.c_void_p(ws.data_ptr()), wsb, ms, None,
                                       None)
    assert rc == _lib.CP_ERR_CAPACITY
    d = cp.persistence_slabs(x, 4, max_survivors=ms)
    _same(d.numpy(), oracle.persistence(img), "uniform 40x36x33 S=4, grown")


def test_full_size_volume_equals_unsplit(cp):
    """The 512^3 blurred volume (sigma 3) that the benchmark times."""
    img = workloads.blurred((512, 512, 512), 3.0, 0)
    x = torch.from_numpy(img).cuda()
    a = cp.persistence(x).raw
    for S in (4, 16):
        d = cp.persistence_slabs(x, S)
        assert torch.equal(a, d.raw), f"S={S}"
        _stats_ok(d.stats, S)
    del x
    torch.cuda.empty_cache()
