// Builds the neighbourhood lookup table of Sec. 3.3 once, at library load.
// See cp_lut.h for the entry layout.  Every predicate stored here is a
// union-find invariant: dropping or pre-applying what the table says never
// changes the pairs that the full union-find would produce.
//
//  H0 (Sec. 3.2, Sec. 4.1 steps 1-3): the edges of L(v) enter right after v,
//  in slot order.  The first one joins the singleton v to an older class and
//  kills v at zero persistence (a direct pair).  A later edge v-u whose u is
//  joined, through vertices and edges of the lower link of v (all of which
//  precede L(v)), to the endpoint of an earlier edge of L(v) closes a loop:
//  it is positive and is dropped.  What is left is the first edge of every
//  local group other than the direct one.
//
//  Top dimension (Sec. 3.1, Sec. 3.2 dual pruning): in the reversed order the
//  top cells of L(v) appear before the facets of L(v), and the facets of
//  L(v) arrive in descending slot order after every facet around v that is
//  not in L(v).  Top cells around v that are not in L(v) are older than every
//  top cell of L(v).  A local union-find over the 2^d top cells around v,
//  seeded with the facets around v that are not in L(v), therefore sees a
//  subset of the true dual connectivity:
//    - a facet whose sides are already joined is a dual cycle (dropped);
//    - a facet joining a class made only of top cells of L(v) kills that
//      class's representative at zero persistence (a local dual pair, applied
//      as a forest link to the top cell across the facet);
//    - a facet joining two classes that each hold an older top cell is left
//      for the global dual union-find.
#include "cp_lut.h"
#include "cp_mask3.cuh"

#include <algorithm>
#include <cstring>

namespace cp {

static Stencil make_stencil(int ndim) {
    Stencil st;
    std::memset(&st, 0, sizeof(st));
    st.ndim = ndim;
    st.nbits = ndim == 3 ? 27 : 9;
    st.center = ndim == 3 ? 13 : 4;
    for (int n = 0; n < st.nbits; ++n) {
        if (ndim == 3) {
            st.off[n][0] = n / 9 - 1;
            st.off[n][1] = (n / 3) % 3 - 1;
            st.off[n][2] = n % 3 - 1;
        } else {
            st.off[n][0] = 0;
            st.off[n][1] = n / 3 - 1;
            st.off[n][2] = n % 3 - 1;
        }
    }
    for (int n = 0; n < st.nbits; ++n) {
        if (n == st.center) continue;
        int nz = (st.off[n][0] != 0) + (st.off[n][1] != 0) + (st.off[n][2] != 0);
        if (nz == 1) st.face_n[st.nfaces++] = n;
        if (nz == ndim - 1) st.facet_n[st.nfacets++] = n;
        if (nz == ndim) st.top_n[st.ntops++] = n;
        // nonzero sub-offsets: zero out any subset of the nonzero coordinates
        uint32_t sub = 0;
        for (int m = 0; m < st.nbits; ++m) {
            if (m == st.center) continue;
            bool ok = true;
            for (int a = 0; a < 3; ++a)
                if (st.off[m][a] != 0 && st.off[m][a] != st.off[n][a]) ok = false;
            if (ok) sub |= 1u << m;
        }
        st.sub[n] = sub;
    }
    // the two top cells on either side of each facet: set its zero coordinate
    // (on one of the image's axes) to -1 and +1
    for (int f = 0; f < st.nfacets; ++f) {
        const int* o = st.off[st.facet_n[f]];
        int k = 0;
        for (int a = 3 - ndim; a < 3; ++a) {
            if (o[a] != 0) continue;
            for (int s = -1; s <= 1; s += 2) {
                int q[3] = {o[0], o[1], o[2]};
                q[a] = s;
                for (int t = 0; t < st.ntops; ++t) {
                    const int* p = st.off[st.top_n[t]];
                    if (p[0] == q[0] && p[1] == q[1] && p[2] == q[2]) st.facet_tops[f][k++] = t;
                }
            }
        }
    }
    return st;
}

const Stencil& stencil(int ndim) {
    static const Stencil s2 = make_stencil(2);
    static const Stencil s3 = make_stencil(3);
    return ndim == 3 ? s3 : s2;
}

uint32_t collapse(const Stencil& st, uint32_t raw) {
    uint32_t rel = 0;
    for (int n = 0; n < st.nbits; ++n) {
        if (n == st.center) continue;
        if ((raw & st.sub[n]) == st.sub[n]) rel |= 1u << n;
    }
    return rel;
}

static int l1(const Stencil& st, int a, int b) {
    int d = 0;
    for (int k = 0; k < 3; ++k) d += std::abs(st.off[a][k] - st.off[b][k]);
    return d;
}

uint64_t classify(const Stencil& st, uint32_t rel) {
    // ---- H0: local groups of the lower link ----
    int comp[27];
    for (int n = 0; n < 27; ++n) comp[n] = -1;
    int ncomp = 0;
    for (int n = 0; n < st.nbits; ++n) {
        if (!((rel >> n) & 1) || comp[n] >= 0) continue;
        int stack[27], sp = 0;
        stack[sp++] = n;
        comp[n] = ncomp;
        while (sp) {
            int a = stack[--sp];
            for (int b = 0; b < st.nbits; ++b)
                if (((rel >> b) & 1) && comp[b] < 0 && l1(st, a, b) == 1) {
                    comp[b] = ncomp;
                    stack[sp++] = b;
                }
        }
        ++ncomp;
    }
    int direct = 7;
    uint32_t h0_surv = 0;
    bool seen[27] = {false};
    for (int s = 0; s < st.nfaces; ++s) {
        int n = st.face_n[s];
        if (!((rel >> n) & 1)) continue;
        if (direct == 7) {
            direct = s;
            seen[comp[n]] = true;
        } else if (!seen[comp[n]]) {
            seen[comp[n]] = true;
            h0_surv |= 1u << s;
        }
    }
    // ---- top dimension: local dual union-find over the top cells around v ----
    int par[8];
    bool has_old[8];
    int max_slot[8];
    bool in_l[8];
    for (int t = 0; t < st.ntops; ++t) {
        par[t] = t;
        in_l[t] = (rel >> st.top_n[t]) & 1;
        has_old[t] = !in_l[t];
        max_slot[t] = in_l[t] ? t : -1;
    }
    auto find = [&](int x) {
        while (par[x] != x) x = par[x];
        return x;
    };
    auto unite = [&](int a, int b) {  // a, b roots; keep a
        par[b] = a;
        has_old[a] = has_old[a] || has_old[b];
        max_slot[a] = std::max(max_slot[a], max_slot[b]);
    };
    for (int f = 0; f < st.nfacets; ++f) {
        if ((rel >> st.facet_n[f]) & 1) continue;  // facet not in L(v): processed earlier
        int ra = find(st.facet_tops[f][0]), rb = find(st.facet_tops[f][1]);
        if (ra != rb) unite(ra, rb);
    }
    uint32_t dual_code[8];
    for (int t = 0; t < 8; ++t) dual_code[t] = 15;
    for (int t = 0; t < st.ntops; ++t)
        if (in_l[t]) dual_code[t] = 8;
    uint32_t dual_surv = 0;
    for (int f = st.nfacets - 1; f >= 0; --f) {
        if (!((rel >> st.facet_n[f]) & 1)) continue;
        int A = st.facet_tops[f][0], B = st.facet_tops[f][1];
        int ra = find(A), rb = find(B);
        if (ra == rb) continue;  // dual cycle
        if (has_old[ra] && has_old[rb]) {
            dual_surv |= 1u << f;
            unite(ra, rb);
            continue;
        }
        int young;
        if (has_old[ra]) young = rb;
        else if (has_old[rb]) young = ra;
        else young = max_slot[ra] < max_slot[rb] ? ra : rb;
        int dying = max_slot[young];  // representative of a class of L(v) top cells
        int across = (find(A) == young) ? B : A;
        dual_code[dying] = uint32_t(across);
        if (young == ra) unite(rb, ra);
        else unite(ra, rb);
    }
    uint64_t e = uint64_t(direct) | (uint64_t(h0_surv) << 3);
    uint32_t in_mask = 0;
    for (int t = 0; t < 8; ++t) {
        e |= uint64_t(dual_code[t]) << (9 + 4 * t);
        if (dual_code[t] != 15) in_mask |= 1u << t;
    }
    e |= uint64_t(dual_surv) << 41;
    e |= uint64_t(in_mask) << 53;
    return e;
}

std::vector<uint32_t> relevant_masks(const Stencil& st) {
    std::vector<uint32_t> out;
    // enumerate by faces, then each allowed higher offset, recursively:
    // a relevant mask is closed under nonzero sub-offsets
    std::vector<int> order;  // offsets by number of nonzero coordinates
    for (int k = 1; k <= 3; ++k)
        for (int n = 0; n < st.nbits; ++n) {
            if (n == st.center) continue;
            int nz = (st.off[n][0] != 0) + (st.off[n][1] != 0) + (st.off[n][2] != 0);
            if (nz == k) order.push_back(n);
        }
    struct Rec {
        const Stencil& st;
        const std::vector<int>& order;
        std::vector<uint32_t>& out;
        void go(size_t i, uint32_t m) {
            if (i == order.size()) {
                out.push_back(m);
                return;
            }
            int n = order[i];
            go(i + 1, m);
            uint32_t need = st.sub[n] & ~(1u << n);
            if ((m & need) == need) go(i + 1, m | (1u << n));
        }
    } rec{st, order, out};
    rec.go(0, 0);
    std::sort(out.begin(), out.end());
    return out;
}

// the hash takes a mask in the pruning kernel's bit layout (cp_mask3.cuh)
static inline uint32_t hash_bucket(uint32_t m) { return (mask3_from_canonical(m) * kH1) >> (32 - kLog2Buckets); }
static inline uint32_t hash_slot(uint32_t m, uint32_t d) {
    return ((mask3_from_canonical(m) ^ (d * kD)) * kH2) >> (32 - kLog2Slots);
}

bool build_lut3d(Lut3D& out) {
    const Stencil& st = stencil(3);
    std::vector<uint32_t> masks = relevant_masks(st);
    const int nb = 1 << kLog2Buckets, ns = 1 << kLog2Slots;
    std::vector<std::vector<uint32_t>> buckets(nb);
    for (uint32_t m : masks) buckets[hash_bucket(m)].push_back(m);
    std::vector<int> order(nb);
    for (int i = 0; i < nb; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return buckets[a].size() > buckets[b].size(); });
    out.disp.assign(nb, 0);
    out.entry.assign(ns, 0);
    out.key.assign(ns, 0xFFFFFFFFu);
    std::vector<uint32_t> slots;
    for (int b : order) {
        const auto& keys = buckets[b];
        if (keys.empty()) continue;
        bool placed = false;
        for (uint32_t d = 0; d < 65536 && !placed; ++d) {
            slots.clear();
            bool ok = true;
            for (uint32_t m : keys) {
                uint32_t s = hash_slot(m, d);
                if (out.key[s] != 0xFFFFFFFFu || std::find(slots.begin(), slots.end(), s) != slots.end()) {
                    ok = false;
                    break;
                }
                slots.push_back(s);
            }
            if (!ok) continue;
            for (size_t i = 0; i < keys.size(); ++i) {
                out.key[slots[i]] = keys[i];
                out.entry[slots[i]] = classify(st, keys[i]);
            }
            out.disp[b] = uint16_t(d);
            placed = true;
        }
        if (!placed) return false;
    }
    out.nclasses = int(masks.size());
    return true;
}

uint64_t check_mask3_layout() {
    const Stencil& st = stencil(3);
    // the layout one byte of the canonical mask at a time
    uint32_t perm[4][256];
    for (int b = 0; b < 4; ++b)
        for (uint32_t v = 0; v < 256; ++v) perm[b][v] = mask3_from_canonical((v << (8 * b)) & 0x7FFDFFFu);
    auto dev = [&](uint32_t raw) {
        return perm[0][raw & 255u] | perm[1][(raw >> 8) & 255u] | perm[2][(raw >> 16) & 255u] | perm[3][raw >> 24];
    };
    uint64_t bad = 0;
    for (uint32_t raw = 0; raw < (1u << 27); ++raw) {
        if (raw & (1u << 13)) continue;
        if (collapse3_lattice(dev(raw)) != dev(collapse(st, raw))) ++bad;
    }
    return bad;
}

void build_lut2d(std::vector<uint64_t>& out, int* nclasses) {
    const Stencil& st = stencil(2);
    out.assign(256, 0);
    for (uint32_t r = 0; r < 256; ++r) {
        uint32_t raw = (r & 0xFu) | ((r >> 4) << 5);  // skip the centre bit 4
        out[r] = classify(st, collapse(st, raw));
    }
    if (nclasses) *nclasses = int(relevant_masks(st).size());
}

}  // namespace cp
