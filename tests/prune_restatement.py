"""Plain sequential restatement of the pruned method, driven by the library's
own lookup-table entries (cp_lut_lookup, host side).  Test infrastructure:
used to check the table's predicates against the oracle (CPU) and the
pruning kernel's outputs stage by stage (GPU).
"""
import ctypes

import numpy as np


def offsets(ndim):
    if ndim == 3:
        return [(b // 9 - 1, (b // 3) % 3 - 1, b % 3 - 1) for b in range(27)]
    return [(0, b // 3 - 1, b % 3 - 1) for b in range(9)]


def entry(lib, ndim, raw):
    e = ctypes.c_uint64()
    assert lib.cp_lut_lookup(ndim, raw, None, ctypes.byref(e)) == 0
    return e.value


def ord_bits(x):
    b = int(np.float32(x).view(np.uint32))
    if (b << 1) & 0xFFFFFFFF == 0:
        b = 0
    return (~b & 0xFFFFFFFF) if b & 0x80000000 else (b | 0x80000000)


class Pruned:
    """K1's outputs for one image, computed one vertex at a time.

    cross: 2D cross-pruning (the dual list takes an H0 survivor only once the
    H0 union-find finds it positive); otherwise every dual survivor of the
    table goes to the dual list at once, where one that kills an H0 class
    closes a dual cycle (a no-op)."""

    def __init__(self, lib, img, cross=False):
        nd = img.ndim
        self.nd = nd
        self.cross = bool(cross) and nd == 2
        f = np.where(img == 0, 0.0, img).astype(np.float64)
        shape = img.shape if nd == 3 else (1,) + img.shape
        D, H, W = shape
        self.shape = (D, H, W)
        f3 = f.reshape(shape)
        self.f3 = f3
        N = D * H * W
        offs = offsets(nd)
        self.offs = offs
        self.faces = [b for b, o in enumerate(offs) if sum(x != 0 for x in o) == 1]
        self.facets = [b for b, o in enumerate(offs) if sum(x != 0 for x in o) == nd - 1]
        self.tops = [b for b, o in enumerate(offs) if sum(x != 0 for x in o) == nd]
        T = (D - 1 if nd == 3 else 1) * (H - 1) * (W - 1)
        self.T = T
        self.OUT = T
        self.par0 = list(range(N))
        self.part = list(range(T + 1))
        self.tage = {}
        self.s0 = []  # (K(v), n, v, flag)
        self.st = []  # (K(v), n, v)
        for z in range(D):
            for y in range(H):
                for x in range(W):
                    self._vertex(lib, z, y, x)

    def K(self, v):
        D, H, W = self.shape
        z, r = divmod(v, H * W)
        y, x = divmod(r, W)
        return (self.f3[z, y, x], v)

    def vid(self, z, y, x):
        D, H, W = self.shape
        return (z * H + y) * W + x

    def top_of(self, z, y, x, o):
        D, H, W = self.shape
        cz = z + (-1 if o[0] < 0 else 0) if self.nd == 3 else 0
        cy, cx = y + (-1 if o[1] < 0 else 0), x + (-1 if o[2] < 0 else 0)
        if cy < 0 or cy >= H - 1 or cx < 0 or cx >= W - 1 or (self.nd == 3 and (cz < 0 or cz >= D - 1)):
            return self.OUT
        return (cz * (H - 1) + cy) * (W - 1) + cx

    def _vertex(self, lib, z, y, x):
        D, H, W = self.shape
        nd, offs = self.nd, self.offs
        v = self.vid(z, y, x)
        kv = self.K(v)
        raw = 0
        for b, o in enumerate(offs):
            if o == (0, 0, 0):
                continue
            zz, yy, xx = z + o[0], y + o[1], x + o[2]
            if 0 <= zz < D and 0 <= yy < H and 0 <= xx < W and self.K(self.vid(zz, yy, xx)) < kv:
                raw |= 1 << b
        e = entry(lib, nd, raw)
        direct = e & 7
        if direct != 7:
            o = offs[self.faces[direct]]
            self.par0[v] = self.vid(z + o[0], y + o[1], x + o[2])
        h0s, ds = (e >> 3) & 0x3F, (e >> 41) & 0xFFF
        for s, b in enumerate(self.faces):
            if (h0s >> s) & 1:
                self.s0.append((kv, b, v, bool((ds >> s) & 1) if self.cross else False))
        for s, b in enumerate(self.facets):
            if (ds >> s) & 1 and not (self.cross and (h0s >> s) & 1):
                self.st.append((kv, b, v))
        for t, b in enumerate(self.tops):
            code = (e >> (9 + 4 * t)) & 15
            if code == 15:
                continue
            me = self.top_of(z, y, x, offs[b])
            if code == 8:
                self.tage[me] = (kv, b)
            else:
                self.part[me] = self.top_of(z, y, x, offs[self.tops[code]])

    # keys in the kernel's encoding: ord << 32 | v << 5 | low
    def key(self, kv, n, v, flag=False):
        low = n if self.nd == 3 else ((n << 1) | int(flag))
        return (ord_bits(kv[0]) << 32) | (v << 5) | low

    def s0_keys(self):
        return sorted(self.key(kv, n, v, fl) for kv, n, v, fl in self.s0)

    def st_keys(self):
        return sorted(self.key(kv, n, v) for kv, n, v in self.st)

    def pairs(self):
        """Sequential elder-rule union-finds over the survivors (with 2D
        cross-pruning when chosen)."""
        nd, offs = self.nd, self.offs
        D, H, W = self.shape
        GH, GW = 2 * H - 1, 2 * W - 1
        par0 = list(self.par0)
        part = list(self.part)
        st = list(self.st)

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
        for kv, b, v, flag in sorted(self.s0):
            z, y, x = coords(v)
            o = offs[b]
            u = self.vid(z + o[0], y + o[1], x + o[2])
            ra, rb = find(par0, v), find(par0, u)
            if ra == rb:
                if flag:
                    st.append((kv, b, v))
                continue
            yv = ra if self.K(ra) > self.K(rb) else rb
            par0[yv] = rb if yv == ra else ra
            if self.K(yv)[0] != kv[0]:
                out.append((0, dcell(*coords(yv), (0, 0, 0)), dcell(z, y, x, o), self.K(yv)[0], kv[0]))
        for kv, b, v in sorted(st, reverse=True):
            z, y, x = coords(v)
            o = offs[b]
            ax = [a for a in range(3 - nd, 3) if o[a] == 0][0]
            sides = []
            for sgn in (-1, 1):
                q = list(o)
                q[ax] = sgn
                sides.append(self.top_of(z, y, x, q))
            ra, rb = find(part, sides[0]), find(part, sides[1])
            if ra == rb:
                continue
            if ra == self.OUT:
                yv = rb
            elif rb == self.OUT:
                yv = ra
            else:
                yv = ra if self.tage[ra] < self.tage[rb] else rb
            part[yv] = rb if yv == ra else ra
            (km, bm) = self.tage[yv]
            if km[0] != kv[0]:
                out.append((nd - 1, dcell(z, y, x, o), dcell(*coords(km[1]), offs[bm]), kv[0], km[0]))
        return sorted(out)
