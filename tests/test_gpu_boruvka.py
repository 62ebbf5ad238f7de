"""The Borůvka design of the union-finds (CP_TUNE_UF_VARIANT = 1: the
minimum spanning forest of the survivor graph first, then the elder-rule
rounds over its edges alone) gives the oracle's pairs bit for bit, on
images, volumes, batches and the T-filtration, and the same pairs as the
reservation rounds on large inputs; its forest has exactly as many edges as
the union-find commits."""
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


@pytest.fixture()
def boruvka():
    from paper_2606_04801_gb300 import _lib

    lib = _lib.load()
    old = lib.cp_get_tuning(7)
    assert lib.cp_set_tuning(7, 1) == 0
    yield lib
    lib.cp_set_tuning(7, old)


def _same(got, want, what):
    assert len(got) == len(want), f"{what}: {len(got)} pairs vs {len(want)}"
    for k in FIELDS:
        if not np.array_equal(got[k], want[k]):
            i = int(np.argmax(got[k] != want[k]))
            raise AssertionError(f"{what}: field {k} differs at pair {i}: {got[i]} vs {want[i]}")


@pytest.mark.parametrize("shape", [(2, 2), (31, 33), (64, 65), (2, 2, 2), (9, 9, 33), (17, 9, 40), (20, 12, 5)])
def test_equals_oracle(cp, boruvka, shape):
    rng = np.random.default_rng(sum(shape) + 70)
    for img in (rng.random(shape, dtype=np.float32), rng.integers(0, 3, shape).astype(np.float32)):
        d = cp.persistence(torch.from_numpy(img).cuda(), with_stats=True)
        _same(d.numpy(), oracle.persistence(img), f"{shape}")
        if d.stats["h0_survivors"] + d.stats["top_survivors"] > 0:
            assert d.stats["mst_rounds"] >= 1


def test_t_filtration_and_batch(cp, boruvka):
    rng = np.random.default_rng(71)
    img = rng.random((12, 11, 10), dtype=np.float32)
    _same(cp.persistence(torch.from_numpy(img).cuda(), filtration="T").numpy(), oracle.persistence_t(img), "T")
    items = [rng.random(s, dtype=np.float32) for s in [(40, 50), (9, 10, 11), (33, 31), (16, 8, 12)]]
    ds = cp.persistence_batched([torch.from_numpy(a).cuda() for a in items])
    got = ds.numpy()
    for i, a in enumerate(items):
        _same(got[got["item"] == i], oracle.persistence(a), f"batch item {i}")


def test_equals_reservation_rounds(cp, boruvka):
    for img in (workloads.blurred((512, 512, 512), 3.0, 0), workloads.uniform((96, 80, 72), 2),
                workloads.blurred((1024, 1024), 4.0, 3)):
        x = torch.from_numpy(img).cuda()
        a = cp.persistence(x, with_stats=True)
        assert boruvka.cp_set_tuning(7, 0) == 0
        b = cp.persistence(x, with_stats=True)
        assert boruvka.cp_set_tuning(7, 1) == 0
        assert torch.equal(a.raw, b.raw), img.shape
        assert a.stats["mst_rounds"] >= 1 and b.stats["mst_rounds"] == 0
        del x
    torch.cuda.empty_cache()


def test_with_h1_and_slabs(cp, boruvka):
    """Calls with H1 keep the reservation rounds, and the slab split keeps its
    own stages, whatever the setting: both still give the oracle's pairs."""
    rng = np.random.default_rng(72)
    img = rng.random((11, 12, 13), dtype=np.float32)
    _same(cp.persistence_full(torch.from_numpy(img).cuda()).numpy(), oracle.persistence_full(img), "full")
    d = cp.persistence_slabs(torch.from_numpy(img).cuda(), 3)
    _same(d.numpy(), oracle.persistence(img), "slabs")
    assert d.stats["crossing"][0] > 0
