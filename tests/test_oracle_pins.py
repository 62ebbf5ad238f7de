"""Pins for the CPU oracle: checks against things other than itself.

- an independent brute-force F2 boundary-matrix reduction (Sec. 2.1) on tiny
  images, random and exhaustive (cell-level equality, zero-persistence pairs
  included);
- hand-computed diagrams (tests/golden/hand_cases.txt);
- Betti numbers of every sublevel complex counted by flood fill (scipy
  labelling / graph components), and the Euler characteristic;
- pair-count identities and metamorphic properties.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from brute_force import reduce_pairs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _oracle_cells(img, keep_zero=True):
    p = oracle.persistence(img, keep_zero=keep_zero)
    finite = {(int(r["birth_cell"]), int(r["death_cell"]), int(r["dim"])) for r in p if r["death_cell"] >= 0}
    ess = [(int(r["birth_cell"]), int(r["dim"])) for r in p if r["death_cell"] < 0]
    return finite, ess


def _brute_cells(img):
    pairs, ess = reduce_pairs(img)
    top = img.ndim - 1
    finite = {(b, d, dim) for b, d, dim in pairs if dim in (0, top)}
    ess0 = [(c, dim) for c, dim in ess if dim == 0]
    return finite, ess0


def _check_against_brute(img):
    assert _oracle_cells(img) == _brute_cells(img)


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("seed", range(6))
def test_random_small_2d(seed):
    rng = np.random.default_rng(seed)
    for _ in range(40):
        shape = tuple(int(v) for v in rng.integers(2, 7, 2))
        if rng.random() < 0.5:
            img = rng.integers(0, 3, shape).astype(np.float32)  # heavy ties
        else:
            img = rng.random(shape, dtype=np.float32)
        _check_against_brute(img)


@pytest.mark.parametrize("seed", range(4))
def test_random_small_3d(seed):
    rng = np.random.default_rng(100 + seed)
    for _ in range(15):
        shape = tuple(int(v) for v in rng.integers(2, 5, 3))
        if rng.random() < 0.5:
            img = rng.integers(0, 3, shape).astype(np.float32)
        else:
            img = rng.random(shape, dtype=np.float32)
        _check_against_brute(img)


def test_exhaustive_3x3_three_levels():
    """Every 3x3 image over {0, 1, 2}: 19,683 tie-heavy cases."""
    vals = np.array(list(itertools.product((0.0, 1.0, 2.0), repeat=9)), dtype=np.float32)
    for v in vals:
        _check_against_brute(v.reshape(3, 3))


@pytest.mark.parametrize("shape", [(2, 2, 2), (2, 2, 3)])
def test_exhaustive_small_binary_volumes(shape):
    n = int(np.prod(shape))
    for bits in range(1 << n):
        img = np.array([(bits >> i) & 1 for i in range(n)], dtype=np.float32).reshape(shape)
        _check_against_brute(img)


def test_negative_zero_and_signs():
    img = np.array([[-0.0, 0.0, -1.5], [2.0, -0.0, 0.25], [1.0, -3.0, 0.0]], dtype=np.float32)
    _check_against_brute(img)
    # -0.0 is the smallest value and the first pixel: the essential class is born there
    img2 = np.array([[-0.0, 1.0, 0.0], [2.0, -0.0, 3.0], [1.0, 0.5, -0.0]], dtype=np.float32)
    for im in (img, img2):
        p = oracle.persistence(im)
        for k in ("birth", "death"):
            assert not np.signbit(p[k][p[k] == 0]).any()
    p = oracle.persistence(img2)
    ess = p[p["death_cell"] < 0]
    assert ess["birth_pixel"][0] == 0 and ess["birth"][0] == 0.0


def _cell_vertices(cell, shape):
    dsh = [2 * n - 1 for n in shape]
    coords = []
    for g in reversed(dsh):
        coords.append(cell % g)
        cell //= g
    coords = coords[::-1]
    choices = [(c // 2,) if c % 2 == 0 else (c // 2, c // 2 + 1) for c in coords]
    return [int(np.ravel_multi_index(v, shape)) for v in itertools.product(*choices)]


def _argmax_vertex(img, cell):
    flat = np.where(img.ravel() == 0, 0.0, img.ravel())
    return max(_cell_vertices(cell, img.shape), key=lambda v: (flat[v], v))


@pytest.mark.parametrize("shape", [(9, 11), (4, 5, 6)])
def test_pixels_and_values_follow_cells(shape):
    """birth/death pixel = largest vertex of the birth/death cell; values are copied from those pixels."""
    rng = np.random.default_rng(17)
    for img in (rng.random(shape, dtype=np.float32), rng.integers(0, 3, shape).astype(np.float32)):
        p = oracle.persistence(img)
        flat = img.ravel()
        for r in p:
            assert r["birth_pixel"] == _argmax_vertex(img, int(r["birth_cell"]))
            assert r["birth"] == flat[r["birth_pixel"]]
            if r["death_cell"] >= 0:
                assert r["death_pixel"] == _argmax_vertex(img, int(r["death_cell"]))
                assert r["death"] == flat[r["death_pixel"]]
            else:
                assert r["death_pixel"] == -1 and np.isinf(r["death"])


# ---------------------------------------------------------------- hand cases
def _parse_cases(name="hand_cases.txt"):
    cases, cur = [], None
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "case":
                cur = {"name": tok[1], "set": [], "expect": []}
            elif tok[0] == "shape":
                cur["shape"] = tuple(int(t) for t in tok[1:])
            elif tok[0] == "fill":
                cur["fill"] = float(tok[1])
            elif tok[0] == "set":
                cur["set"].append((tuple(int(t) for t in tok[1:-1]), float(tok[-1])))
            elif tok[0] == "checker":
                cur["checker"] = (float(tok[1]), float(tok[2]))
            elif tok[0] == "expect":
                cur["expect"].append((int(tok[1]), float(tok[2]), float(tok[3]), int(tok[4])))
            elif tok[0] == "end":
                cases.append(cur)
    return cases


def _build_case(c):
    if "checker" in c:
        lo, hi = c["checker"]
        idx = np.indices(c["shape"]).sum(axis=0)
        img = np.where(idx % 2 == 0, lo, hi).astype(np.float32)
    else:
        img = np.full(c["shape"], c["fill"], dtype=np.float32)
    for coord, v in c["set"]:
        img[coord] = v
    return img


CASES = _parse_cases()


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_hand_case(case):
    img = _build_case(case)
    p = oracle.persistence(img)
    got = {}
    for r in p:
        k = (int(r["dim"]), float(r["birth"]), float(r["death"]))
        got[k] = got.get(k, 0) + 1
    want = {(d, b, e): n for d, b, e, n in case["expect"]}
    assert got == want
    if img.size <= 125:
        _check_against_brute(img)


# ---------------------------------------------------------------- invariants
def _betti0(img, t):
    from scipy import ndimage

    struct = ndimage.generate_binary_structure(img.ndim, 1)  # face adjacency
    _, n = ndimage.label(img <= t, structure=struct)
    return n


def _betti_top(img, t):
    """Bounded components of the complement of K_t (Alexander duality).

    Nodes: top cells with value > t plus the outside; two nodes are joined by
    every facet with value > t between them.
    """
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components

    d = img.ndim
    # value of each top cell and of each facet: the max of its vertices
    def block_max(a, axes):
        out = a
        for ax in axes:
            sl0 = [slice(None)] * d
            sl1 = [slice(None)] * d
            sl0[ax] = slice(0, -1)
            sl1[ax] = slice(1, None)
            out = np.maximum(out[tuple(sl0)], out[tuple(sl1)])
        return out

    top = block_max(img, range(d))
    tshape = top.shape
    ntop = top.size
    OUT = ntop
    alive = np.append(top.ravel() > t, True)
    rows, cols = [], []
    tid = np.arange(ntop).reshape(tshape)
    for ax in range(d):
        # facets orthogonal to axis ax: their vertices span the other axes
        fac = block_max(img, [a for a in range(d) if a != ax])  # extent along ax = n_ax
        for k in range(img.shape[ax]):
            sl = [slice(None)] * d
            sl[ax] = k
            fv = fac[tuple(sl)] > t
            lo = tid.take(k - 1, axis=ax) if k - 1 >= 0 else None
            hi = tid.take(k, axis=ax) if k < tshape[ax] else None
            a = lo if lo is not None else np.full(fv.shape, OUT)
            b = hi if hi is not None else np.full(fv.shape, OUT)
            m = fv
            rows.append(a[m])
            cols.append(b[m])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    g = coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(ntop + 1, ntop + 1))
    _, lab = connected_components(g, directed=False)
    return len(np.unique(lab[alive])) - 1


def _alive(p, dim, t):
    sel = (p["dim"] == dim) & (p["birth"] <= t) & (t < p["death"])
    return int(sel.sum())


@pytest.mark.parametrize(
    "img",
    [
        np.random.default_rng(7).random((17, 23), dtype=np.float32),
        np.random.default_rng(8).integers(0, 5, (19, 14)).astype(np.float32),
        np.random.default_rng(9).random((6, 7, 5), dtype=np.float32),
        np.random.default_rng(10).integers(0, 4, (5, 6, 6)).astype(np.float32),
    ],
    ids=["2d_uniform", "2d_levels", "3d_uniform", "3d_levels"],
)
def test_betti_numbers_at_every_threshold(img):
    p = oracle.persistence(img)
    top = img.ndim - 1
    for t in np.unique(img):
        assert _alive(p, 0, t) == _betti0(img, t)
        assert _alive(p, top, t) == _betti_top(img, t)


def test_euler_characteristic_2d():
    img = np.random.default_rng(11).integers(0, 6, (15, 12)).astype(np.float32)
    p = oracle.persistence(img)
    for t in np.unique(img):
        v = img <= t
        ex = v[:, :-1] & v[:, 1:]
        ey = v[:-1, :] & v[1:, :]
        sq = v[:-1, :-1] & v[:-1, 1:] & v[1:, :-1] & v[1:, 1:]
        chi = int(v.sum()) - int(ex.sum()) - int(ey.sum()) + int(sq.sum())
        assert chi == _alive(p, 0, t) - _alive(p, 1, t)


def test_euler_characteristic_3d_with_brute_h1():
    """chi(K_t) = b0 - b1 + b2, with b1 from the brute-force reduction of the whole complex."""
    rng = np.random.default_rng(12)
    for _ in range(4):
        img = rng.integers(0, 4, (3, 4, 3)).astype(np.float32)
        p = oracle.persistence(img)
        pairs, ess = reduce_pairs(img)
        f = img
        for t in np.unique(img):
            # count cells of K_t by dimension through the doubled grid
            D, H, W = f.shape
            chi = 0
            for Z in range(2 * D - 1):
                for Y in range(2 * H - 1):
                    for X in range(2 * W - 1):
                        vs = [
                            f[z, y, x]
                            for z in {Z // 2, (Z + 1) // 2}
                            for y in {Y // 2, (Y + 1) // 2}
                            for x in {X // 2, (X + 1) // 2}
                        ]
                        if max(vs) <= t:
                            chi += (-1) ** ((Z % 2) + (Y % 2) + (X % 2))
            # b1 from the brute-force pairs: cell values are max over vertices
            shape = f.shape
            dsh = tuple(2 * n - 1 for n in shape)

            def val(c):
                Z, rem = divmod(c, dsh[1] * dsh[2])
                Y, X = divmod(rem, dsh[2])
                return max(
                    f[z, y, x]
                    for z in {Z // 2, (Z + 1) // 2}
                    for y in {Y // 2, (Y + 1) // 2}
                    for x in {X // 2, (X + 1) // 2}
                )

            b1 = sum(1 for b, d, dim in pairs if dim == 1 and val(b) <= t < val(d))
            b1 += sum(1 for c, dim in ess if dim == 1 and val(c) <= t)
            assert chi == _alive(p, 0, t) - b1 + _alive(p, 2, t)


def test_pair_counts_before_filtering():
    """With zero-persistence pairs kept: N-1 finite H0 pairs and one top pair per top cell."""
    for shape in [(9, 13), (4, 5, 6)]:
        img = np.random.default_rng(13).random(shape, dtype=np.float32)
        p = oracle.persistence(img, keep_zero=True)
        n = img.size
        ntop = int(np.prod([s - 1 for s in shape]))
        assert int(((p["dim"] == 0) & (p["death_cell"] >= 0)).sum()) == n - 1
        assert int((p["dim"] == img.ndim - 1).sum()) == ntop


def test_refined_order_is_a_filtration():
    """Every face precedes its cofaces under the refined key (Sec. 2.3 reading)."""
    rng = np.random.default_rng(14)
    img = rng.integers(0, 3, (4, 3, 5)).astype(np.float32)
    D, H, W = img.shape
    dsh = (2 * D - 1, 2 * H - 1, 2 * W - 1)
    for c in range(int(np.prod(dsh))):
        Z, rem = divmod(c, dsh[1] * dsh[2])
        Y, X = divmod(rem, dsh[2])
        kc = oracle.cell_key(img, c)
        for ax, C in enumerate((Z, Y, X)):
            if C % 2:
                for s in (-1, 1):
                    q = [Z, Y, X]
                    q[ax] += s
                    face = (q[0] * dsh[1] + q[1]) * dsh[2] + q[2]
                    kf = oracle.cell_key(img, face)
                    assert (kf[0], kf[1], kf[2], face) < (kc[0], kc[1], kc[2], c)


def _value_diagram(p):
    return sorted((int(r["dim"]), float(r["birth"]), float(r["death"])) for r in p)


def test_strictly_increasing_map_keeps_cell_pairs():
    rng = np.random.default_rng(15)
    for shape in [(12, 9), (5, 4, 6)]:
        img = rng.integers(0, 4, shape).astype(np.float32)
        a = oracle.persistence(img)
        b = oracle.persistence(img * np.float32(2.0) + np.float32(8.0))  # exact and order preserving here
        for k in ("birth_cell", "death_cell", "birth_pixel", "death_pixel", "dim"):
            assert (a[k] == b[k]).all()


def test_flips_keep_value_diagram():
    """Flips reverse the first-order tie-break on tie-heavy images; the value diagram must not change."""
    rng = np.random.default_rng(16)
    for shape in [(11, 8), (5, 6, 4)]:
        img = rng.integers(0, 3, shape).astype(np.float32)
        base = _value_diagram(oracle.persistence(img))
        for axes in [(0,), (img.ndim - 1,), tuple(range(img.ndim))]:
            assert _value_diagram(oracle.persistence(np.flip(img, axes).copy())) == base
        assert _value_diagram(oracle.persistence(np.ascontiguousarray(img.T))) == base


def test_rejects_nonfinite_and_small():
    with pytest.raises(ValueError):
        oracle.persistence(np.array([[0.0, np.nan], [1.0, 2.0]], dtype=np.float32))
    with pytest.raises(ValueError):
        oracle.persistence(np.array([[0.0, np.inf], [1.0, 2.0]], dtype=np.float32))
    with pytest.raises(ValueError):
        oracle.persistence(np.zeros((1, 5), dtype=np.float32))


def _betti_top_by_vertices(img, t):
    """Top Betti number from the vertices above t: the complement of K_t is the
    union of the open stars of those vertices, and two stars meet exactly when
    the vertices share a top cell (8-/26-adjacency); components touching the
    border are joined to the outside."""
    from scipy import ndimage

    lab, n = ndimage.label(img > t, structure=np.ones((3,) * img.ndim, dtype=bool))
    border = set()
    for ax in range(img.ndim):
        border |= set(np.unique(np.take(lab, 0, axis=ax)).tolist())
        border |= set(np.unique(np.take(lab, -1, axis=ax)).tolist())
    border.discard(0)
    return n - len(border)


@pytest.mark.parametrize("shape", [(13, 17), (6, 7, 5)])
def test_top_betti_vertex_formulation(shape):
    """Pins the formulation the full-size GPU test uses, against the facet-graph count and the oracle."""
    rng = np.random.default_rng(18)
    for img in (rng.random(shape, dtype=np.float32), rng.integers(0, 4, shape).astype(np.float32)):
        p = oracle.persistence(img)
        for t in np.unique(img):
            assert _betti_top_by_vertices(img, t) == _betti_top(img, t) == _alive(p, img.ndim - 1, t)
