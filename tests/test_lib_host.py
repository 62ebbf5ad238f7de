"""Host-side checks of the CUDA library (no GPU needed).

- the shared library loads and exports every symbol include/*.h declares;
- the lookup table has the paper's 15,935 3D configurations (Sec. 3.3) and
  47 in 2D, and its collapse agrees with an independent enumeration;
- a plain restatement of the pruned pipeline, driven by the library's own
  table entries (cp_lut_lookup), gives the oracle's pairs: every pruning
  predicate in the table is a union-find invariant.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2606_04801_gb300 as cp
from paper_2606_04801_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def lib():
    from paper_2606_04801_gb300 import build

    build.build()
    return _lib.load()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "cubical_persistence.h")).read()
    declared = set(re.findall(r"^\s*(?:int|int64_t|size_t|long long|const char \*)\s*\**\s*(\w+)\s*\(", hdr, re.M))
    assert declared, "no declarations parsed"
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(_lib.exported_symbols())
    assert lib.cp_version() > 0
    assert lib.cp_error_string(-3).decode() == "capacity exceeded"


def test_lut_class_counts(lib):
    # Sec. 3.3 prints 15,935 configurations in 3D after the collapse
    with open(os.path.join(GOLDEN, "lut_counts.txt")) as fh:
        want = {int(l.split()[0]): int(l.split()[1]) for l in fh if l.strip() and not l.startswith("#")}
    assert lib.cp_lut_num_classes(3) == want[3] == 15935
    assert lib.cp_lut_num_classes(2) == want[2]
    assert lib.cp_lut_num_classes(4) == -1


def _offsets(ndim):
    n = 27 if ndim == 3 else 9
    if ndim == 3:
        return [(b // 9 - 1, (b // 3) % 3 - 1, b % 3 - 1) for b in range(n)]
    return [(0, b // 3 - 1, b % 3 - 1) for b in range(n)]


def _collapse_numpy(ndim):
    """Independent enumeration: every raw mask -> relevant mask, vectorised."""
    offs = _offsets(ndim)
    center = 13 if ndim == 3 else 4
    nb = len(offs)
    raw = np.arange(1 << nb, dtype=np.uint32)
    raw = raw[(raw >> center) & 1 == 0]
    rel = np.zeros_like(raw)
    for b, o in enumerate(offs):
        if b == center:
            continue
        need = np.uint32(0)
        for c, q in enumerate(offs):
            if c == center:
                continue
            if all(qa == 0 or qa == oa for qa, oa in zip(q, o)):
                need |= np.uint32(1 << c)
        rel |= np.where((raw & need) == need, np.uint32(1 << b), np.uint32(0)).astype(np.uint32)
    return raw, rel


def test_collapse_matches_independent_enumeration(lib):
    raw2, rel2 = _collapse_numpy(2)
    assert len(np.unique(rel2)) == 47
    r = ctypes.c_uint32()
    for m, want in zip(raw2, rel2):
        assert lib.cp_lut_lookup(2, int(m), ctypes.byref(r), None) == 0
        assert r.value == int(want)
    # 3D: count the distinct collapsed masks over all 2^26 raw masks
    raw3, rel3 = _collapse_numpy(3)
    seen = np.zeros(1 << 27, dtype=bool)
    seen[rel3] = True
    assert int(seen.sum()) == 15935
    rng = np.random.default_rng(0)
    for m in rng.choice(raw3, 3000, replace=False):
        assert lib.cp_lut_lookup(3, int(m), ctypes.byref(r), None) == 0
        assert r.value == int(rel3[np.searchsorted(raw3, m)])


# ---------------------------------------------------------------- restatement
def _entry(lib, ndim, raw):
    e = ctypes.c_uint64()
    assert lib.cp_lut_lookup(ndim, raw, None, ctypes.byref(e)) == 0
    return e.value


def _pruned_pipeline(lib, img):
    """Sequential restatement of the pruned method using the library's table.

    Forest links from the table, survivors sorted by the refined order,
    sequential elder-rule union-find, 2D cross-pruning; returns pairs as the
    oracle does (value-filtered, sorted by (dim, birth_cell)).
    """
    nd = img.ndim
    f = np.where(img == 0, 0.0, img).astype(np.float64)
    shape = img.shape if nd == 3 else (1,) + img.shape
    D, H, W = shape
    f3 = f.reshape(shape)
    N = D * H * W
    offs = _offsets(nd)
    faces = [b for b, o in enumerate(offs) if sum(x != 0 for x in o) == 1]
    facets = [b for b, o in enumerate(offs) if sum(x != 0 for x in o) == nd - 1]
    tops = [b for b, o in enumerate(offs) if sum(x != 0 for x in o) == nd]
    TD = D - 1 if nd == 3 else 1
    T = TD * (H - 1) * (W - 1)
    OUT = T
    GH, GW = 2 * H - 1, 2 * W - 1

    def K(v):
        z, r = divmod(v, H * W)
        y, x = divmod(r, W)
        return (f3[z, y, x], v)

    def vid(z, y, x):
        return (z * H + y) * W + x

    def top_of(z, y, x, o):
        cz = z + (o[0] < 0 and -1 or 0) if nd == 3 else 0
        cy, cx = y + (-1 if o[1] < 0 else 0), x + (-1 if o[2] < 0 else 0)
        if cy < 0 or cy >= H - 1 or cx < 0 or cx >= W - 1 or (nd == 3 and (cz < 0 or cz >= D - 1)):
            return OUT
        return (cz * (H - 1) + cy) * (W - 1) + cx

    par0 = list(range(N))
    part = list(range(T + 1))
    tage = {}  # dual root -> (K(m), slot)
    s0, st = [], []
    for z in range(D):
        for y in range(H):
            for x in range(W):
                v = vid(z, y, x)
                kv = K(v)
                raw = 0
                for b, o in enumerate(offs):
                    if o == (0, 0, 0):
                        continue
                    zz, yy, xx = z + o[0], y + o[1], x + o[2]
                    if 0 <= zz < D and 0 <= yy < H and 0 <= xx < W and K(vid(zz, yy, xx)) < kv:
                        raw |= 1 << b
                e = _entry(lib, nd, raw)
                direct = e & 7
                if direct != 7:
                    o = offs[faces[direct]]
                    par0[v] = vid(z + o[0], y + o[1], x + o[2])
                h0s, ds = (e >> 3) & 0x3F, (e >> 41) & 0xFFF
                for s, b in enumerate(faces):
                    if (h0s >> s) & 1:
                        s0.append((kv, b, v, bool((ds >> s) & 1) if nd == 2 else False))
                for s, b in enumerate(facets):
                    if (ds >> s) & 1 and not (nd == 2 and (h0s >> s) & 1):
                        st.append((kv, b, v))
                for t, b in enumerate(tops):
                    code = (e >> (9 + 4 * t)) & 15
                    if code == 15:
                        continue
                    me = top_of(z, y, x, offs[b])
                    if code == 8:
                        tage[me] = (kv, b)
                    else:
                        part[me] = top_of(z, y, x, offs[tops[code]])

    def find(p, a):
        while p[a] != a:
            p[a] = p[p[a]]
            a = p[a]
        return a

    def dcell(z, y, x, o):
        return ((2 * z + o[0]) * GH + 2 * y + o[1]) * GW + 2 * x + o[2]

    def coords(v):
        z, r = divmod(v, H * W)
        return z, r // W, r % W

    out = []
    for kv, b, v, flag in sorted(s0):
        z, y, x = coords(v)
        o = offs[b]
        u = vid(z + o[0], y + o[1], x + o[2])
        ra, rb = find(par0, v), find(par0, u)
        if ra == rb:
            if flag:
                st.append((kv, b, v))
            continue
        yv = ra if K(ra) > K(rb) else rb
        par0[yv] = rb if yv == ra else ra
        if K(yv)[0] != kv[0]:
            out.append((0, dcell(*coords(yv), (0, 0, 0)), dcell(z, y, x, o), K(yv)[0], kv[0]))
    for kv, b, v in sorted(st, reverse=True):
        z, y, x = coords(v)
        o = offs[b]
        ax = [a for a in range(3 - nd, 3) if o[a] == 0][0]
        sides = []
        for sgn in (-1, 1):
            q = list(o)
            q[ax] = sgn
            sides.append(top_of(z, y, x, q))
        ra, rb = find(part, sides[0]), find(part, sides[1])
        if ra == rb:
            continue
        if ra == OUT:
            yv = rb
        elif rb == OUT:
            yv = ra
        else:
            yv = ra if tage[ra] < tage[rb] else rb
        part[yv] = rb if yv == ra else ra
        (km, bm) = tage[yv]
        if km[0] != kv[0]:
            out.append((nd - 1, dcell(z, y, x, o), dcell(*coords(km[1]), offs[bm]), kv[0], km[0]))
    return sorted(out)


def _oracle_rows(img):
    p = oracle.persistence(img)
    return sorted(
        (int(r["dim"]), int(r["birth_cell"]), int(r["death_cell"]), float(r["birth"]), float(r["death"]))
        for r in p
        if r["death_cell"] >= 0
    )


@pytest.mark.parametrize("seed", range(4))
def test_pruned_restatement_matches_oracle_2d(lib, seed):
    rng = np.random.default_rng(200 + seed)
    for _ in range(25):
        shape = tuple(int(v) for v in rng.integers(2, 10, 2))
        img = rng.integers(0, 3, shape).astype(np.float32) if rng.random() < 0.5 else rng.random(shape, dtype=np.float32)
        assert _pruned_pipeline(lib, img) == _oracle_rows(img)


@pytest.mark.parametrize("seed", range(3))
def test_pruned_restatement_matches_oracle_3d(lib, seed):
    rng = np.random.default_rng(300 + seed)
    for _ in range(8):
        shape = tuple(int(v) for v in rng.integers(2, 7, 3))
        img = rng.integers(0, 3, shape).astype(np.float32) if rng.random() < 0.5 else rng.random(shape, dtype=np.float32)
        assert _pruned_pipeline(lib, img) == _oracle_rows(img)
