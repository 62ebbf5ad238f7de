"""The H1 stage's decomposition, restated in Python and checked against the
oracle's full diagram (CPU).  The device path (csrc/cp_h1.cu) classifies
cells and reduces columns in two parts; each part's claim is checked here on
small volumes, with the oracle's zero-persistence pairs as the truth:

1. H2 births that one lower star settles: the squares of L(m), in
   descending order, with a union-find over its octant cubes (cubes outside
   the star and the outside vertex count as older classes of unknown
   connectivity); a join of two classes of which at least one reaches
   nothing outside the star is an H2 birth.  Every square so marked is an H2
   birth, and every other H2 birth is a dual survivor of the pruning pass
   (restated from the library's own lookup table), so the union-find's
   commits complete the set.
2. The reduction inside each lower star, on the columns of the squares not
   paired in H2 over the edges not paired in H0: a column whose lowest entry
   stays an edge through m pairs with that edge, as in the oracle; the
   columns whose lowest entry leaves the star include every pair of nonzero
   persistence, and are exactly those when the values are distinct.
3. The rounds across stars (bids with the oldest key winning, every loser or
   displaced holder adding its row's winner at once), in shuffled orders:
   the final lowest entries are the oracle's pairs, zero persistence
   included.
"""
import numpy as np
import pytest

import oracle
import workloads

SQ_DESC = [(1, 1, 0), (1, 0, 1), (1, 0, -1), (1, -1, 0), (0, 1, 1), (0, 1, -1),
           (0, -1, 1), (0, -1, -1), (-1, 1, 0), (-1, 0, 1), (-1, 0, -1), (-1, -1, 0)]
FACES = [(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 1), (0, 1, 0), (1, 0, 0)]


class Vol:
    def __init__(self, img):
        self.img = img
        self.D, self.H, self.W = img.shape
        self.f = np.where(img == 0, 0.0, img).astype(np.float64).ravel()
        self.GH, self.GW = 2 * self.H - 1, 2 * self.W - 1

    def key(self, v):
        return (self.f[v], v)

    def coords(self, v):
        return v // (self.H * self.W), (v // self.W) % self.H, v % self.W

    def inside(self, z, y, x):
        return 0 <= z < self.D and 0 <= y < self.H and 0 <= x < self.W

    def vid(self, z, y, x):
        return (z * self.H + y) * self.W + x

    def lower(self, m, o):
        z, y, x = self.coords(m)
        zz, yy, xx = z + o[0], y + o[1], x + o[2]
        return self.inside(zz, yy, xx) and self.key(self.vid(zz, yy, xx)) < self.key(m)

    def cell(self, m, o2):
        """Doubled index of the cell at doubled offset o2 from vertex m."""
        z, y, x = self.coords(m)
        return ((2 * z + o2[0]) * self.GH + 2 * y + o2[1]) * self.GW + 2 * x + o2[2]

    def square_in_star(self, m, o):
        subs = [(a, b, c) for a in ({0, o[0]}) for b in ({0, o[1]}) for c in ({0, o[2]}) if (a, b, c) != (0, 0, 0)]
        return all(self.lower(m, s) for s in subs)


def _truth(img):
    p = oracle.persistence_full(img, keep_zero=True)
    neg_e = set(int(c) for c in p["death_cell"][(p["dim"] == 0) & (p["death_cell"] >= 0)])
    pos_q = set(int(c) for c in p["birth_cell"][p["dim"] == 2])
    h1 = p[p["dim"] == 1]
    return p, neg_e, pos_q, {int(r["death_cell"]): int(r["birth_cell"]) for r in h1}, h1


def _star_births(v):
    out = set()
    for m in range(v.D * v.H * v.W):
        z, y, x = v.coords(m)
        node, ext = {}, [False] * 9
        for oc in range(8):
            s = (1 if oc & 4 else -1, 1 if oc & 2 else -1, 1 if oc & 1 else -1)
            c = (z + min(s[0], 0), y + min(s[1], 0), x + min(s[2], 0))
            if not (0 <= c[0] < v.D - 1 and 0 <= c[1] < v.H - 1 and 0 <= c[2] < v.W - 1):
                node[oc] = 8
                continue
            node[oc] = oc
            ext[oc] = not all(v.lower(m, (a * s[0], b * s[1], cc * s[2]))
                              for a in (0, 1) for b in (0, 1) for cc in (0, 1) if (a, b, cc) != (0, 0, 0))
        ext[8] = True
        par = list(range(9))

        def find(a):
            while par[a] != a:
                a = par[a]
            return a

        for o in SQ_DESC:
            if not v.square_in_star(m, o):
                continue
            ax = [i for i in range(3) if o[i] == 0][0]
            sides = []
            for s in (-1, 1):
                t = list(o)
                t[ax] = s
                sides.append(node[(4 if t[0] > 0 else 0) | (2 if t[1] > 0 else 0) | (1 if t[2] > 0 else 0)])
            ra, rb = find(sides[0]), find(sides[1])
            if ra == rb:
                continue
            if not (ext[ra] and ext[rb]):
                out.add(v.cell(m, o))
            par[ra] = rb
            ext[rb] = ext[rb] or ext[ra]
    return out


def _volumes():
    rng = np.random.default_rng(950)
    vols = []
    for t in range(24):
        shape = tuple(int(s) for s in rng.integers(2, 6, 3))
        vols.append(rng.integers(0, 3, shape).astype(np.float32) if t % 3 == 0 else rng.random(shape, dtype=np.float32))
    vols.append(workloads.blurred((12, 11, 10), 1.5, 951))
    return vols


@pytest.fixture(scope="module")
def lib():
    import paper_2606_04801_gb300 as cp

    return cp.load()


def test_star_rule_marks_h2_births_and_survivors_cover_the_rest(lib):
    from prune_restatement import Pruned, offsets

    offs = offsets(3)
    for img in _volumes():
        v = Vol(img)
        _, _, pos_q, _, _ = _truth(img)
        marked = _star_births(v)
        assert marked <= pos_q, img.shape
        pr = Pruned(lib, img)
        surv = {v.cell(m, offs[b]) for _, b, m in pr.st}
        assert pos_q - marked <= surv, (img.shape, sorted(pos_q - marked - surv)[:4])


def test_star_local_reduction(lib):
    for img in _volumes():
        v = Vol(img)
        _, neg_e, pos_q, death_to_birth, h1 = _truth(img)
        nonzero = {int(r["death_cell"]) for r in h1 if r["birth"] != r["death"]}
        left = set()
        for m in range(v.D * v.H * v.W):
            # rows through m: lower face neighbours whose edge does not merge in H0
            rows = [v.lower(m, fc) and v.cell(m, fc) not in neg_e for fc in FACES]
            owner, cols = [None] * 6, {}
            for o in reversed(SQ_DESC):  # ascending stencil order
                if not v.square_in_star(m, o) or v.cell(m, o) in pos_q:
                    continue
                nz = [i for i in range(3) if o[i]]
                u1 = [0, 0, 0]
                u2 = [0, 0, 0]
                u1[nz[0]] = o[nz[0]]
                u2[nz[1]] = o[nz[1]]
                col = set()
                for st, dr in ((u1, u2), (u2, u1)):
                    f = FACES.index(tuple(st))
                    if rows[f]:
                        col.add(("m", f))
                    far = v.cell(m, tuple(2 * st[i] + dr[i] for i in range(3)))
                    if far not in neg_e:
                        col.add(("far", far))
                # the sequential reduction while the lowest entry is an edge through m
                while any(e[0] == "m" for e in col):
                    f = max(e[1] for e in col if e[0] == "m")
                    if owner[f] is None:
                        owner[f] = o
                        break
                    col ^= cols[owner[f]]
                cols[o] = col
                sq = v.cell(m, o)
                if any(e[0] == "m" for e in col):
                    # stays in the star: pairs with that edge, as in the oracle
                    f = max(e[1] for e in col if e[0] == "m")
                    assert death_to_birth[sq] == v.cell(m, FACES[f]), (img.shape, m, o)
                else:
                    left.add(sq)
        # every pair of nonzero persistence leaves its star; with distinct
        # values nothing else does (equal values let a zero-persistence pair
        # span two stars)
        assert nonzero <= left, (img.shape, sorted(nonzero - left))
        if len(np.unique(img)) == img.size:
            assert left == nonzero, (img.shape, len(left), len(nonzero))


def _refined(v, cell):
    """(f(m), m, doubled index) of a cell: the order inside one dimension."""
    Z, Y, X = cell // (v.GH * v.GW), (cell // v.GW) % v.GH, cell % v.GW
    best = None
    for z in {Z // 2, (Z + 1) // 2}:
        for y in {Y // 2, (Y + 1) // 2}:
            for x in {X // 2, (X + 1) // 2}:
                m = v.vid(z, y, x)
                if best is None or v.key(m) > best:
                    best = v.key(m)
    return (best[0], best[1], cell)


def test_cross_star_rounds_match_oracle(lib):
    """The rounds of the device path, restated: columns that left their star
    bid for their lowest row (the oldest key wins; star pivots hold theirs
    from the start), every loser or displaced holder adds the winner of its
    row, all at once, and bids again; processed in shuffled orders, the final
    lowest entries are the oracle's pairs, zero persistence included."""
    rng = np.random.default_rng(960)
    for img in _volumes():
        v = Vol(img)
        _, neg_e, pos_q, death_to_birth, _ = _truth(img)
        cols, pivot, left = {}, {}, []
        for m in range(v.D * v.H * v.W):
            rows = [v.lower(m, fc) and v.cell(m, fc) not in neg_e for fc in FACES]
            owner = [None] * 6
            for o in reversed(SQ_DESC):
                sq = v.cell(m, o)
                if not v.square_in_star(m, o) or sq in pos_q:
                    continue
                nz = [i for i in range(3) if o[i]]
                u1, u2 = [0, 0, 0], [0, 0, 0]
                u1[nz[0]] = o[nz[0]]
                u2[nz[1]] = o[nz[1]]
                col = set()
                for st, dr in ((u1, u2), (u2, u1)):
                    if rows[FACES.index(tuple(st))]:
                        col.add(v.cell(m, tuple(st)))
                    far = v.cell(m, tuple(2 * st[i] + dr[i] for i in range(3)))
                    if far not in neg_e:
                        col.add(far)
                through = {v.cell(m, fc) for fc in FACES}
                while col & through:
                    low = max(col & through, key=lambda e: _refined(v, e))
                    f = [v.cell(m, fc) for fc in FACES].index(low)
                    if owner[f] is None:
                        owner[f] = sq
                        pivot[low] = sq  # a star pivot: final
                        break
                    col ^= cols[owner[f]]
                cols[sq] = col
                if not (col & through):
                    left.append(sq)
        key = {q: _refined(v, q) for q in cols}

        def low(q):
            return max(cols[q], key=lambda e: _refined(v, e))

        chg = list(left)
        for _ in range(100000):
            rng.shuffle(chg)
            work = []
            for q in chg:
                e = low(q)
                old = pivot.get(e)
                if old is None or key[q] < key[old]:
                    pivot[e] = q
                    if old is not None:
                        work.append(old)
                else:
                    work.append(q)
            if not work:
                break
            rng.shuffle(work)
            snapshot = {q: set(cols[q]) for q in work}
            for q in work:
                p = pivot[low(q)]
                assert key[p] < key[q] and p not in snapshot
                cols[q] = snapshot[q] ^ cols[p]
                assert cols[q], "a column of a square not paired in H2 cannot vanish"
            chg = work
        got = {q: low(q) for q in cols}
        assert got == death_to_birth, img.shape
