"""Pins for the T-filtration oracle: checks against things other than itself.

- an independent brute-force F2 boundary-matrix reduction of the T-complex on
  tiny images (cell-level equality, zero-persistence pairs included),
  random and exhaustive;
- Betti numbers of every sublevel complex by labelling: a union of closed
  pixels is connected through shared vertices (8-/26-neighbourhood), and its
  holes (2D) or voids (3D) are the face-connected components of the pixels
  above the threshold that do not touch the image border;
- hand-computed diagrams and pair-count identities.
"""
import itertools

import numpy as np
import pytest

import oracle
from brute_force import reduce_pairs_t


def _oracle_cells(img):
    p = oracle.persistence_t(img, keep_zero=True)
    finite = {(int(r["birth_cell"]), int(r["death_cell"]), int(r["dim"])) for r in p if r["death_cell"] >= 0}
    ess = [(int(r["birth_cell"]), int(r["dim"])) for r in p if r["death_cell"] < 0]
    return finite, ess


def _brute_cells(img):
    pairs, ess = reduce_pairs_t(img)
    top = img.ndim - 1
    finite = {(b, d, dim) for b, d, dim in pairs if dim in (0, top)}
    ess0 = [(c, dim) for c, dim in ess if dim == 0]
    return finite, ess0


@pytest.mark.parametrize("seed", range(5))
def test_t_random_small_2d(seed):
    rng = np.random.default_rng(300 + seed)
    for _ in range(30):
        shape = tuple(int(v) for v in rng.integers(1, 6, 2))
        img = rng.integers(0, 3, shape).astype(np.float32) if rng.random() < 0.5 else rng.random(shape, dtype=np.float32)
        assert _oracle_cells(img) == _brute_cells(img)


@pytest.mark.parametrize("seed", range(3))
def test_t_random_small_3d(seed):
    rng = np.random.default_rng(310 + seed)
    for _ in range(10):
        shape = tuple(int(v) for v in rng.integers(1, 4, 3))
        img = rng.integers(0, 3, shape).astype(np.float32) if rng.random() < 0.5 else rng.random(shape, dtype=np.float32)
        assert _oracle_cells(img) == _brute_cells(img)


def test_t_exhaustive_2x3_three_levels():
    """Every 2x3 image over {0, 1, 2}: 729 tie-heavy cases."""
    for v in itertools.product((0.0, 1.0, 2.0), repeat=6):
        img = np.array(v, dtype=np.float32).reshape(2, 3)
        assert _oracle_cells(img) == _brute_cells(img)


def test_t_exhaustive_binary_3x3():
    for v in itertools.product((0.0, 1.0), repeat=9):
        img = np.array(v, dtype=np.float32).reshape(3, 3)
        assert _oracle_cells(img) == _brute_cells(img)


def test_t_exhaustive_binary_2x2x2():
    for v in itertools.product((0.0, 1.0), repeat=8):
        img = np.array(v, dtype=np.float32).reshape(2, 2, 2)
        assert _oracle_cells(img) == _brute_cells(img)


# ---------------------------------------------------------------- Betti numbers by labelling
def _betti0_t(img, t):
    from scipy import ndimage

    _, n = ndimage.label(img <= t, structure=np.ones((3,) * img.ndim, dtype=bool))
    return n


def _betti_top_t(img, t):
    from scipy import ndimage

    lab, n = ndimage.label(img > t, structure=ndimage.generate_binary_structure(img.ndim, 1))
    border = np.zeros(img.shape, dtype=bool)
    for ax in range(img.ndim):
        sl0 = [slice(None)] * img.ndim
        sl1 = [slice(None)] * img.ndim
        sl0[ax] = 0
        sl1[ax] = -1
        border[tuple(sl0)] = True
        border[tuple(sl1)] = True
    touching = set(np.unique(lab[border & (lab > 0)]).tolist())
    return n - len(touching)


def _alive(p, dim, t):
    sel = (p["dim"] == dim) & (p["birth"] <= t) & (t < p["death"])
    return int(sel.sum())


@pytest.mark.parametrize(
    "img",
    [
        np.random.default_rng(17).random((19, 21), dtype=np.float32),
        np.random.default_rng(18).integers(0, 4, (16, 13)).astype(np.float32),
        np.random.default_rng(19).random((7, 6, 8), dtype=np.float32),
        np.random.default_rng(20).integers(0, 3, (6, 5, 7)).astype(np.float32),
    ],
    ids=["2d_uniform", "2d_levels", "3d_uniform", "3d_levels"],
)
def test_t_betti_numbers_at_every_threshold(img):
    p = oracle.persistence_t(img)
    top = img.ndim - 1
    for t in np.unique(img):
        assert _alive(p, 0, t) == _betti0_t(img, t)
        assert _alive(p, top, t) == _betti_top_t(img, t)


# ---------------------------------------------------------------- hand cases and counts
def test_t_ring_2d():
    """A ring of 0 around a 5: one hole born when the ring closes, filled at 5;
    the ring's last pixel (index 8, bottom right) closes it through the centre
    pixel's bottom edge (doubled (4, 3) = 31), whose first top cell is pixel 7."""
    img = np.array([[0, 0, 0], [0, 5, 0], [0, 0, 0]], dtype=np.float32)
    p = oracle.persistence_t(img)
    assert len(p) == 2
    e, h = p[0], p[1]
    assert (e["dim"], e["birth"], e["death"], e["birth_cell"], e["death_cell"], e["birth_pixel"]) == (0, 0.0, np.inf, 0, -1, 0)
    assert (h["dim"], h["birth"], h["death"], h["death_cell"], h["death_pixel"]) == (1, 0.0, 5.0, 24, 4)


def test_t_hollow_cube_3d():
    """A shell of 1 around a 7 in a 3x3x3 volume: one void (H2) from 1 to 7."""
    img = np.ones((3, 3, 3), dtype=np.float32)
    img[1, 1, 1] = 7.0
    p = oracle.persistence_t(img)
    voids = p[p["dim"] == 2]
    assert len(voids) == 1 and voids[0]["birth"] == 1.0 and voids[0]["death"] == 7.0
    assert voids[0]["death_cell"] == (3 * 7 + 3) * 7 + 3 and voids[0]["death_pixel"] == 13
    assert int((p["dim"] == 0).sum()) == 1  # only the essential class


@pytest.mark.parametrize("shape", [(1, 1), (1, 5), (4, 3), (1, 1, 1), (2, 3, 1), (3, 2, 4)])
def test_t_pair_counts_before_filtering(shape):
    """Every vertex but the oldest dies in H0; every top cell dies in the dual."""
    img = np.random.default_rng(sum(shape)).random(shape, dtype=np.float32)
    p = oracle.persistence_t(img, keep_zero=True)
    nv = int(np.prod([n + 1 for n in shape]))
    assert int(((p["dim"] == 0) & (p["death_cell"] >= 0)).sum()) == nv - 1
    assert int(((p["dim"] == 0) & (p["death_cell"] < 0)).sum()) == 1
    assert int((p["dim"] == img.ndim - 1).sum()) == img.size


def test_t_values_follow_pixels_and_rejects_nonfinite():
    img = np.random.default_rng(5).integers(0, 6, (7, 9)).astype(np.float32)
    p = oracle.persistence_t(img)
    flat = img.ravel()
    assert np.all(p["birth"] == flat[p["birth_pixel"]])
    fin = p["death_cell"] >= 0
    assert np.all(p["death"][fin] == flat[p["death_pixel"][fin]])
    bad = img.copy()
    bad[3, 4] = np.nan
    with pytest.raises(ValueError):
        oracle.persistence_t(bad)
