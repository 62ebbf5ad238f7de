"""Pins for the oracle's H1 of volumes (the middle dimension in 3D): checks
against things other than itself.

- the brute-force F2 reduction of the whole complex (all dimensions in one
  matrix, Python bit-set columns) on tiny volumes, random and exhaustive,
  cell-level with zero-persistence pairs kept;
- Betti numbers at every threshold: b1(t) = b0(t) + b2(t) - chi(t), with b0
  by face-connected labelling of {f <= t}, b2 by the components of the
  complement (Alexander duality) and chi counted from the cells of K_t;
- pair-count identities, a hand-computed solid torus, and the hand-derived
  whole diagrams of tests/golden/h1_hand_cases.txt (rings, a notched ring, a
  capped ring, a hollow cube);
- metamorphic checks (an increasing map keeps the cells, a flip keeps the
  values).
"""
import itertools

import numpy as np
import pytest

import oracle
from brute_force import reduce_pairs
from test_oracle_pins import _alive, _betti0, _betti_top, _build_case, _parse_cases


def _cells_full(img):
    p = oracle.persistence_full(img, keep_zero=True)
    return {(int(r["birth_cell"]), int(r["death_cell"]), int(r["dim"])) for r in p if r["death_cell"] >= 0}


def _check_brute(img):
    pairs, ess = reduce_pairs(img)
    assert _cells_full(img) == set(pairs)
    assert [d for _, d in ess] == [0]  # a box: only the essential H0 class


@pytest.mark.parametrize("seed", range(4))
def test_h1_random_small_volumes(seed):
    rng = np.random.default_rng(700 + seed)
    for _ in range(12):
        shape = tuple(int(v) for v in rng.integers(2, 5, 3))
        img = rng.integers(0, 3, shape).astype(np.float32) if rng.random() < 0.5 else rng.random(shape, dtype=np.float32)
        _check_brute(img)


@pytest.mark.parametrize("shape", [(2, 2, 2), (2, 2, 3)])
def test_h1_exhaustive_binary(shape):
    n = int(np.prod(shape))
    for v in itertools.product((0.0, 1.0), repeat=n):
        _check_brute(np.array(v, dtype=np.float32).reshape(shape))


def _block_max(a, axes):
    out = a
    for ax in axes:
        sl0 = [slice(None)] * a.ndim
        sl1 = [slice(None)] * a.ndim
        sl0[ax] = slice(0, -1)
        sl1[ax] = slice(1, None)
        out = np.maximum(out[tuple(sl0)], out[tuple(sl1)])
    return out


def _euler(img, t):
    """chi(K_t): cells by dimension, a cell's value the max of its vertices."""
    chi = 0
    for k in range(4):
        for axes in itertools.combinations(range(3), k):
            chi += (-1) ** k * int((_block_max(img, axes) <= t).sum())
    return chi


@pytest.mark.parametrize(
    "img",
    [
        np.random.default_rng(701).random((6, 7, 5), dtype=np.float32),
        np.random.default_rng(702).integers(0, 4, (7, 6, 6)).astype(np.float32),
        np.random.default_rng(703).integers(0, 2, (5, 5, 8)).astype(np.float32),
    ],
    ids=["uniform", "levels", "binary"],
)
def test_h1_betti_numbers_at_every_threshold(img):
    p = oracle.persistence_full(img)
    for t in np.unique(img):
        b0, b2 = _betti0(img, t), _betti_top(img, t)
        assert _alive(p, 0, t) == b0
        assert _alive(p, 2, t) == b2
        assert _alive(p, 1, t) == b0 + b2 - _euler(img, t)


@pytest.mark.parametrize("shape", [(2, 2, 2), (3, 4, 5), (4, 3, 2), (5, 5, 5)])
def test_h1_pair_counts_before_filtering(shape):
    """Every edge that closes a cycle dies in H1 (a box has no essential H1):
    E - N + 1 pairs, with N - 1 finite H0 pairs and one H2 pair per cube."""
    img = np.random.default_rng(sum(shape) + 710).random(shape, dtype=np.float32)
    p = oracle.persistence_full(img, keep_zero=True)
    D, H, W = shape
    N = D * H * W
    E = D * H * (W - 1) + D * (H - 1) * W + (D - 1) * H * W
    assert int((p["dim"] == 1).sum()) == E - N + 1
    assert int(((p["dim"] == 0) & (p["death_cell"] >= 0)).sum()) == N - 1
    assert int((p["dim"] == 2).sum()) == (D - 1) * (H - 1) * (W - 1)


def test_h1_solid_torus():
    """A ring of 0 in the middle plane of a 3x5x5 volume of 9, around a 5:
    one loop, born when the ring's last vertex (1,3,3) = 43 joins through its
    edge to (1,3,2) (doubled (2,6,5) = 221), filled when the centre
    (1,2,2) = 37 enters."""
    img = np.full((3, 5, 5), 9.0, dtype=np.float32)
    img[1, 1:4, 1:4] = 0.0
    img[1, 2, 2] = 5.0
    p = oracle.persistence_full(img)
    h1 = p[p["dim"] == 1]
    assert len(h1) == 1
    r = h1[0]
    assert (r["birth"], r["death"], r["birth_pixel"], r["death_pixel"], r["birth_cell"]) == (0.0, 5.0, 43, 37, 221)
    assert int((p["dim"] == 2).sum()) == 0 and int((p["dim"] == 0).sum()) == 1


def test_h1_equals_plain_diagram_elsewhere():
    """The H0 and H2 pairs of the full diagram are those of the plain call,
    and a 2D image gets the plain diagram."""
    img = np.random.default_rng(720).random((5, 6, 7), dtype=np.float32)
    full = oracle.persistence_full(img)
    plain = oracle.persistence(img)
    assert np.array_equal(full[full["dim"] != 1], plain)
    im2 = np.random.default_rng(721).random((9, 8), dtype=np.float32)
    assert np.array_equal(oracle.persistence_full(im2), oracle.persistence(im2))


def _h1_values(p):
    h = p[p["dim"] == 1]
    return sorted(zip(h["birth"].tolist(), h["death"].tolist()))


def test_h1_metamorphic():
    rng = np.random.default_rng(722)
    img = rng.integers(0, 6, (6, 5, 7)).astype(np.float32)
    base = oracle.persistence_full(img)
    inc = oracle.persistence_full(img * 2.0 + 3.0)
    for k in ("birth_cell", "death_cell", "birth_pixel", "death_pixel", "dim"):
        assert np.array_equal(base[k], inc[k])
    for ax in range(3):
        assert _h1_values(oracle.persistence_full(np.flip(img, ax).copy())) == _h1_values(base)
    assert _h1_values(oracle.persistence_full(np.transpose(img, (2, 0, 1)).copy())) == _h1_values(base)


H1_CASES = _parse_cases("h1_hand_cases.txt")


@pytest.mark.parametrize("case", H1_CASES, ids=[c["name"] for c in H1_CASES])
def test_h1_hand_case(case):
    img = _build_case(case)
    got = {}
    for r in oracle.persistence_full(img):
        k = (int(r["dim"]), float(r["birth"]), float(r["death"]))
        got[k] = got.get(k, 0) + 1
    assert got == {(d, b, e): n for d, b, e, n in case["expect"]}
    if img.size <= 125:
        _check_brute(img)
