// H1 of volumes: the middle dimension of a 3D image, by an F2 matrix
// reduction whose rows are the edges not paired in H0 and whose columns are
// the squares not paired in H2, with the zero-persistence pairs that one
// lower star settles taken out first (Sec. 4.2, 3D steps 4-5).
//
// Over F2 the 1-dimensional pairs come from the column reduction (Sec. 2.1)
// of the boundary matrix of the squares (columns) over the edges (rows), both
// in the fully refined order (Sec. 2.3).  Two restrictions keep every pair:
//   - a square that creates a 2-cycle (a merging facet of the dual graph,
//     paired in H2) has a column that reduces to zero: it is left out;
//   - an edge that merges two H0 classes is never the lowest entry of a
//     column during the reduction (every column is a 1-cycle, and the
//     youngest edge of a cycle joins vertices that the rest of the cycle
//     already connects, so it does not merge), hence deleting those rows
//     changes no lowest entry and no column addition: they are left out.
// One column per square not paired in H2, one row per edge not paired in H0:
// equally many (the Euler characteristic of a box is 1), and every column
// reduces to a nonzero column whose lowest entry is its partner.
//
// Which cells those are: what the pruning pass settles inside one lower
// star, recomputed here from the image (each vertex's first lower face
// neighbour gives a merging edge; the squares of a lower star that join two
// classes of its cubes, at most one of which reaches outside the star, merge
// in the dual graph), and the survivors that the union-finds commit, which
// they mark in the same bitmaps.  The counts are checked: N - 1 merging edges
// and (D-1)(H-1)(W-1) squares paired in H2 per volume.
//
// The reduction runs in two parts.  Inside each lower star L(m) first: its
// cells are consecutive in the filtration order, and no column of an earlier
// star holds an edge of L(m), so the sequential reduction of L(m)'s columns
// (in order, each adding the earlier column that holds its lowest entry)
// is exact for as long as a column's lowest entry is an edge through m.  One
// thread per vertex does it on 32-bit masks over the 30 edges of the star
// (6 through m, 24 that miss it).  A column that ends holding an edge
// through m is final: its pair has zero persistence, and the column is the
// pivot of that edge.  The others (their lowest entry left the star: every
// pair of nonzero persistence, and with distinct values only those) are
// reduced across stars in rounds
// inside one cooperative kernel (the last rounds, once few columns change,
// in its first CTA alone, with CTA barriers): every column whose lowest entry changed
// bids for that row with an atomic minimum of its key (the filtration order)
// in a per-edge pivot word; every column that loses a bid, or is displaced
// by an older one, then adds the winner of its row (all such additions at
// once), so its lowest entry drops, and it bids again in the next round.
// Adding an older column with the same lowest entry is a left-to-right
// column operation, so once all lowest entries are distinct the pairs are
// those of the sequential reduction, whatever the order of additions.
// Rounds end when no bid is lost.  Every wait is bounded; pool overflow and
// failed checks set a status bit and stop the rounds.
#include <atomic>

#include "cp_common.cuh"
#include "cp_grid.cuh"
#include "cp_kernels.h"

namespace cp {
namespace {

constexpr int kHT = 256;  // threads per CTA of the element-wise kernels
constexpr int kRT = 512;  // threads per CTA of the reduction
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kMaxRounds = 1u << 20;
// Once at most solo_cols columns enter a round, CTA 0 runs the rounds alone
// while the other CTAs wait parked (a grid barrier costs microseconds, a CTA
// barrier a fraction of one, and the long tails of rounds carry few
// columns); when more than twice as many enter a round again, CTA 0 wakes
// the grid.
constexpr int kSoloDefault = kRT / 32;
// A bounded wait that gave up earlier leaves the sorted columns unreliable;
// non-finite input leaves the order unreliable: the call fails anyway.
constexpr uint32_t kStSkip = kStTimeout | kStNonfinite;

// Vertex order inside an item: (ord f, local id).
__device__ __forceinline__ uint64_t vkey(const float* img, int64_t v) {
    return (uint64_t(ord_bits(__ldg(img + v))) << 32) | uint64_t(v);
}

__device__ __forceinline__ int n3(int dz, int dy, int dx) { return (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1); }

__device__ __forceinline__ void set_bit(uint32_t* map, uint32_t id) { atomicOr(map + (id >> 5), 1u << (id & 31u)); }
__device__ __forceinline__ bool get_bit(const uint32_t* map, uint32_t id) {
    return (__ldg(map + (id >> 5)) >> (id & 31u)) & 1u;
}

__device__ __forceinline__ int64_t axis_step(const Item& it, int a) {
    return a == 0 ? 1 : (a == 1 ? int64_t(it.W) : int64_t(it.W) * it.H);
}

// Key of the edge from local vertex u along axis a.
__device__ __forceinline__ uint64_t edge_key(const Item& it, int64_t u, int a) {
    const int64_t w = u + axis_step(it, a);
    const uint64_t ku = vkey(it.img, u), kw = vkey(it.img, w);
    const bool hi = kw > ku;  // m is the far end: the edge lies on its -a side
    const int64_t m = hi ? w : u;
    const int s = hi ? -1 : 1;
    const int n = n3(a == 2 ? s : 0, a == 1 ? s : 0, a == 0 ? s : 0);
    return make_key(uint32_t((hi ? kw : ku) >> 32), uint64_t(it.voff + m), uint32_t(n));
}

// Key of the square with lowest corner u (local) and normal axis a.
__device__ __forceinline__ uint64_t square_key(const Item& it, int64_t u, int a) {
    const int p = a == 0 ? 1 : 0, q = a == 2 ? 1 : 2;  // the spanned axes
    const int64_t sp = axis_step(it, p), sq = axis_step(it, q);
    uint64_t km = 0;
    int bp = 0, bq = 0;
    for (int c = 0; c < 4; ++c) {
        const int cp = c & 1, cq = c >> 1;
        const uint64_t k = vkey(it.img, u + cp * sp + cq * sq);
        if (c == 0 || k > km) {
            km = k;
            bp = cp;
            bq = cq;
        }
    }
    int o[3] = {0, 0, 0};  // offset of the square's centre from m, per axis (x, y, z)
    o[p] = bp ? -1 : 1;
    o[q] = bq ? -1 : 1;
    const int64_t m = u + bp * sp + bq * sq;
    return make_key(uint32_t(km >> 32), uint64_t(it.voff + m), uint32_t(n3(o[2], o[1], o[0])));
}

__device__ __forceinline__ uint32_t edge_id(const ItemTable& tab, uint64_t key) {
    return cell_id3(tab.it[item_of_vertex(tab, key_vertex(key))], key, false);
}

__device__ __forceinline__ int32_t cell_index(const Item& it, uint64_t key) {
    const int64_t lv = int64_t(key_vertex(key)) - it.voff;
    const int x = int(lv % it.W), y = int((lv / it.W) % it.H), z = int(lv / (int64_t(it.W) * it.H));
    int dz, dy, dx;
    stencil_off(3, int(key_low(key)), dz, dy, dx);
    return int32_t(doubled_index(it, z, y, x, dz, dy, dx));
}

// ---- the direct pairs' cells, from the image
__global__ void __launch_bounds__(kHT) k_h1_direct(const __grid_constant__ ItemTable tab, H1Bufs b, int64_t v0,
                                                   int64_t v1) {
    for (int64_t g = v0 + int64_t(blockIdx.x) * kHT + threadIdx.x; g < v1; g += int64_t(gridDim.x) * kHT) {
        const Item& it = tab.it[item_of_vertex(tab, uint32_t(g))];
        const int64_t W = it.W, HW = int64_t(it.H) * it.W;
        const int64_t v = g - it.voff;
        const int x = int(v % W), y = int((v / W) % it.H), z = int(v / HW);
        const uint64_t kv = vkey(it.img, v);
        // the first lower face neighbour (by stencil index) gives the edge
        // that merges v into an older class
        {
            const int fz[6] = {-1, 0, 0, 0, 0, 1}, fy[6] = {0, -1, 0, 0, 1, 0}, fx[6] = {0, 0, -1, 1, 0, 0};
            for (int k = 0; k < 6; ++k) {
                const int nz = z + fz[k], ny = y + fy[k], nx = x + fx[k];
                if (nz < 0 || nz >= it.D || ny < 0 || ny >= it.H || nx < 0 || nx >= it.W) continue;
                const int64_t u = v + fz[k] * HW + fy[k] * W + fx[k];
                if (vkey(it.img, u) < kv) {
                    const int axis = fx[k] ? 0 : (fy[k] ? 1 : 2);
                    set_bit(b.neg_e, uint32_t(3 * (it.voff + (u < v ? u : v)) + axis));
                    break;
                }
            }
        }
        // the lower star of v: its squares in descending order, with a
        // union-find over its 8 octant cubes (a cube outside the box is the
        // outside vertex); cubes not in the star and the outside are older
        // than every cube in it and their classes are not known here.  The
        // star's cells are consecutive in the filtration order and its cubes
        // enter it as singletons, so a square that joins two classes of which
        // at least one has touched nothing outside the star merges them: a
        // 2-cycle is born (Sec. 3.1 dual graph).  Joins of two classes that
        // both reach outside are left to the dual union-find's survivors.
        uint32_t low = 0;  // bit n3(o): the neighbour at offset o is lower
        for (int n = 0; n < 27; ++n) {
            const int dz = n / 9 - 1, dy = (n / 3) % 3 - 1, dx = n % 3 - 1;
            const int nz = z + dz, ny = y + dy, nx = x + dx;
            if (n == 13 || nz < 0 || nz >= it.D || ny < 0 || ny >= it.H || nx < 0 || nx >= it.W) continue;
            if (vkey(it.img, v + dz * HW + dy * W + dx) < kv) low |= 1u << n;
        }
        if (low == 0u) continue;
        uint8_t node[8];   // octant (bit 2: +z, bit 1: +y, bit 0: +x) -> union-find node (8: the outside)
        uint8_t par[9];
        uint16_t ext = 1u << 8;  // bit k: node k's class reaches outside the star
        for (int oc = 0; oc < 8; ++oc) {
            const int sz = (oc & 4) ? 1 : -1, sy = (oc & 2) ? 1 : -1, sx = (oc & 1) ? 1 : -1;
            const int cz = z + (sz < 0 ? -1 : 0), cy = y + (sy < 0 ? -1 : 0), cx = x + (sx < 0 ? -1 : 0);
            par[oc] = uint8_t(oc);
            if (cz < 0 || cz >= it.D - 1 || cy < 0 || cy >= it.H - 1 || cx < 0 || cx >= it.W - 1) {
                node[oc] = 8;
                continue;
            }
            node[oc] = uint8_t(oc);
            bool in_star = true;  // its 7 other corners are lower
            for (int c = 1; c < 8; ++c)
                in_star = in_star && ((low >> n3((c >> 2) * sz, ((c >> 1) & 1) * sy, (c & 1) * sx)) & 1u);
            if (!in_star) ext |= uint16_t(1u << oc);
        }
        par[8] = 8;
        // the 12 squares through v by stencil index, descending
        const int8_t sqo[12][3] = {{1, 1, 0},  {1, 0, 1},  {1, 0, -1},  {1, -1, 0},  {0, 1, 1},   {0, 1, -1},
                                   {0, -1, 1}, {0, -1, -1}, {-1, 1, 0}, {-1, 0, 1}, {-1, 0, -1}, {-1, -1, 0}};
        for (int k = 0; k < 12; ++k) {
            const int oz = sqo[k][0], oy = sqo[k][1], ox = sqo[k][2];
            // in the star: its three other corners are lower (and in the box)
            const bool in_star = ((low >> n3(oz, oy, ox)) & 1u) && ((low >> n3(oz, 0, 0)) & 1u || oz == 0) &&
                                 ((low >> n3(0, oy, 0)) & 1u || oy == 0) && ((low >> n3(0, 0, ox)) & 1u || ox == 0);
            if (!in_star) continue;
            const int a = oz == 0 ? 2 : (oy == 0 ? 1 : 0);  // normal axis
            // its two cubes: the normal component at -1 and at +1
            const int base = (oz > 0 ? 4 : 0) | (oy > 0 ? 2 : 0) | (ox > 0 ? 1 : 0);
            const int bit = a == 2 ? 4 : (a == 1 ? 2 : 1);
            int ra = node[base & ~bit], rb = node[base | bit];
            while (par[ra] != ra) ra = par[ra];
            while (par[rb] != rb) rb = par[rb];
            if (ra == rb) continue;
            if (!(((ext >> ra) & 1u) && ((ext >> rb) & 1u))) {
                const int64_t lo = v + (oz < 0 ? -HW : 0) + (oy < 0 ? -W : 0) + (ox < 0 ? -1 : 0);
                set_bit(b.pos_q, uint32_t(3 * (it.voff + lo) + a));
            }
            par[ra] = uint8_t(rb);
            if ((ext >> ra) & 1u) ext |= uint16_t(1u << rb);
        }
    }
}

// ---- the slots of a lower star L(m): the 6 edges through m (slot 24 + f,
// faces by stencil index ascending) and, for each of the 12 squares through
// m (k by stencil index ascending), its two edges that miss m (slots 2k and
// 2k + 1).  Edges through m come after every edge that misses m in the
// filtration order, and among themselves in face order.
__device__ const int8_t kSqA[12][3] = {{-1, -1, 0}, {-1, 0, -1}, {-1, 0, 1}, {-1, 1, 0}, {0, -1, -1}, {0, -1, 1},
                                       {0, 1, -1},  {0, 1, 1},   {1, -1, 0}, {1, 0, -1}, {1, 0, 1},  {1, 1, 0}};
__device__ const int8_t kFace[6][3] = {{-1, 0, 0}, {0, -1, 0}, {0, 0, -1}, {0, 0, 1}, {0, 1, 0}, {1, 0, 0}};
constexpr uint32_t kThrough = 0x3Fu << 24;

__device__ __forceinline__ int face_of(int dz, int dy, int dx) {
    return dz < 0 ? 0 : (dy < 0 ? 1 : (dx < 0 ? 2 : (dx > 0 ? 3 : (dy > 0 ? 4 : 5))));
}

// Edge from local vertex a along the unit offset (dz, dy, dx): its id and key.
__device__ __forceinline__ uint32_t edge_id_at(const Item& it, int64_t a, int dz, int dy, int dx) {
    const int64_t lo = a + (dz < 0 ? -int64_t(it.H) * it.W : 0) + (dy < 0 ? -int64_t(it.W) : 0) + (dx < 0 ? -1 : 0);
    return uint32_t(3 * (it.voff + lo) + (dx ? 0 : (dy ? 1 : 2)));
}
__device__ __forceinline__ uint64_t edge_key_at(const Item& it, int64_t a, int dz, int dy, int dx) {
    const int64_t lo = a + (dz < 0 ? -int64_t(it.H) * it.W : 0) + (dy < 0 ? -int64_t(it.W) : 0) + (dx < 0 ? -1 : 0);
    return edge_key(it, lo, dx ? 0 : (dy ? 1 : 2));
}
__device__ __forceinline__ int64_t step_of(const Item& it, int dz, int dy, int dx) {
    return dz * int64_t(it.H) * it.W + dy * int64_t(it.W) + dx;
}

// The two unit offsets of square k and its far edge j: (start vertex offset, direction).
__device__ __forceinline__ void far_edge(int k, int j, int& sz, int& sy, int& sx, int& dz, int& dy, int& dx) {
    const int o[3] = {kSqA[k][0], kSqA[k][1], kSqA[k][2]};
    const int i1 = o[0] ? 0 : 1, i2 = o[2] ? 2 : 1;  // the two nonzero components
    int u1[3] = {0, 0, 0}, u2[3] = {0, 0, 0};
    u1[i1] = o[i1];
    u2[i2] = o[i2];
    const int* st = j == 0 ? u1 : u2;
    const int* dr = j == 0 ? u2 : u1;
    sz = st[0];
    sy = st[1];
    sx = st[2];
    dz = dr[0];
    dy = dr[1];
    dx = dr[2];
}

// Key of slot sl of L(m).
__device__ __forceinline__ uint64_t slot_key(const Item& it, int64_t m, int sl) {
    if (sl >= 24) return edge_key_at(it, m, kFace[sl - 24][0], kFace[sl - 24][1], kFace[sl - 24][2]);
    int sz, sy, sx, dz, dy, dx;
    far_edge(sl >> 1, sl & 1, sz, sy, sx, dz, dy, dx);
    return edge_key_at(it, m + step_of(it, sz, sy, sx), dz, dy, dx);
}

// Keys of the edges of a star column (mask over the slots of L(m)),
// descending, decoded by a whole warp: lane l computes slot l's key (the
// image loads of all slots in flight together), and each key goes to its
// rank among the column's keys (all distinct).  Returns the count.
__device__ uint32_t warp_decode(const Item& it, int64_t m, uint32_t mask, uint64_t* keys) {
    const unsigned lane = lane_id();
    const bool has = lane < 30u && ((mask >> lane) & 1u);
    const uint64_t k = has ? slot_key(it, m, int(lane)) : 0ull;
    uint32_t rank = 0;
#pragma unroll
    for (int j = 0; j < 30; ++j) {
        const uint64_t kj = __shfl_sync(0xFFFFFFFFu, k, j);
        rank += (((mask >> j) & 1u) && kj > k) ? 1u : 0u;
    }
    if (has) keys[rank] = k;
    __syncwarp();
    return uint32_t(__popc(mask & 0x3FFFFFFFu));
}

// The lowest entry (largest key) of a star column: its last edge through m
// if it holds one (those come after every edge that misses m, in slot
// order), else the largest of its other edges' keys.
__device__ __forceinline__ uint64_t star_low(const Item& it, int64_t m, uint32_t mask) {
    mask &= 0x3FFFFFFFu;
    if (mask & kThrough) return slot_key(it, m, 31 - __clz(mask));
    uint64_t best = 0;
#pragma unroll
    for (int sl = 0; sl < 24; ++sl)
        if ((mask >> sl) & 1u) best = max(best, slot_key(it, m, sl));
    return best;
}

// The column of square id q: its key, the item, and its star vertex m (local).
__device__ __forceinline__ uint64_t column_key(const ItemTable& tab, uint32_t q, const Item*& itp, int64_t& m) {
    const Item& it = tab.it[item_of_vertex(tab, q / 3u)];
    itp = &it;
    const uint64_t k = square_key(it, int64_t(q / 3u) - it.voff, int(q % 3u));
    m = int64_t(key_vertex(k)) - it.voff;
    return k;
}

// Pool offset of column q's entries (its current region), or ~0 while the
// column is still its star mask.
__device__ __forceinline__ uint64_t column_at(const H1Bufs& b, uint32_t q) {
    const uint64_t o = __ldcg(b.coff + q);
    const uint32_t c = __ldcg(b.ccap + q);  // both loads in flight together
    if (o == ~0ull) return o;
    return o + ((c >> 31) ? uint64_t(c & 0x7FFFFFFFu) : 0ull);
}

__device__ __forceinline__ uint64_t column_low(const H1Bufs& b, const Item& it, int64_t m, uint32_t q) {
    const uint64_t o = column_at(b, q);
    if (o != ~0ull) return __ldcg(b.pool + o);
    return star_low(it, m, __ldcg(b.cmask + q));
}

// ---- every lower star: its columns (squares not paired in H2) reduced
// among themselves, and the check counts
__global__ void __launch_bounds__(kHT) k_h1_local(const __grid_constant__ ItemTable tab, H1Bufs b, int64_t v0,
                                                  int64_t v1) {
    uint32_t ne = 0, pe = 0, pq = 0, nm = 0;
    const unsigned lane = lane_id();
    for (int64_t base = v0 + int64_t(blockIdx.x) * kHT; base < v1; base += int64_t(gridDim.x) * kHT) {
        const int64_t g = base + threadIdx.x;
        const bool live = g < v1;
        uint32_t nonlocal[12];
        uint32_t nn = 0;
        if (live) {
            const Item& it = tab.it[item_of_vertex(tab, uint32_t(g))];
            const int64_t W = it.W, HW = int64_t(it.H) * it.W;
            const int64_t m = g - it.voff;
            const int x = int(m % W), y = int((m / W) % it.H), z = int(m / HW);
            const bool room[3] = {x < it.W - 1, y < it.H - 1, z < it.D - 1};
            for (int a = 0; a < 3; ++a) {  // cells whose lowest corner is m
                const uint32_t id = uint32_t(3 * g + a);
                if (room[a]) {
                    if (get_bit(b.neg_e, id)) ++ne;
                    else ++pe;
                }
                if (room[a == 0 ? 1 : 0] && room[a == 2 ? 1 : 2] && get_bit(b.pos_q, id)) ++pq;
            }
            const uint64_t km = vkey(it.img, m);
            uint32_t low = 0;
            for (int n = 0; n < 27; ++n) {
                const int dz = n / 9 - 1, dy = (n / 3) % 3 - 1, dx = n % 3 - 1;
                const int nz = z + dz, ny = y + dy, nx = x + dx;
                if (n == 13 || nz < 0 || nz >= it.D || ny < 0 || ny >= it.H || nx < 0 || nx >= it.W) continue;
                if (vkey(it.img, m + dz * HW + dy * W + dx) < km) low |= 1u << n;
            }
            // the edges through m that are rows: lower neighbour, not merging in H0
            uint32_t rows = 0;
            for (int f = 0; f < 6; ++f)
                if (((low >> n3(kFace[f][0], kFace[f][1], kFace[f][2])) & 1u) &&
                    !get_bit(b.neg_e, edge_id_at(it, m, kFace[f][0], kFace[f][1], kFace[f][2])))
                    rows |= 1u << (24 + f);
            uint32_t colmask[12];
            int8_t owner[6] = {-1, -1, -1, -1, -1, -1};
            const uint32_t ordm = uint32_t(km >> 32);
            for (int k = 0; k < 12; ++k) {
                colmask[k] = 0;
                const int oz = kSqA[k][0], oy = kSqA[k][1], ox = kSqA[k][2];
                const bool in_star = ((low >> n3(oz, oy, ox)) & 1u) && (oz == 0 || ((low >> n3(oz, 0, 0)) & 1u)) &&
                                     (oy == 0 || ((low >> n3(0, oy, 0)) & 1u)) && (ox == 0 || ((low >> n3(0, 0, ox)) & 1u));
                if (!in_star) continue;
                const int a = oz == 0 ? 2 : (oy == 0 ? 1 : 0);
                const int64_t lo = m + (oz < 0 ? -HW : 0) + (oy < 0 ? -W : 0) + (ox < 0 ? -1 : 0);
                const uint32_t q = uint32_t(3 * (it.voff + lo) + a);
                if (get_bit(b.pos_q, q)) continue;  // paired in H2: its column reduces to zero
                ++nm;
                // its four edges, the rows among them
                uint32_t mask = 0;
                for (int j = 0; j < 2; ++j) {
                    int sz, sy, sx, dz, dy, dx;
                    far_edge(k, j, sz, sy, sx, dz, dy, dx);
                    mask |= (1u << (24 + face_of(sz, sy, sx))) & rows;  // the edge from m to the start
                    if (!get_bit(b.neg_e, edge_id_at(it, m + step_of(it, sz, sy, sx), dz, dy, dx))) mask |= 1u << (2 * k + j);
                }
                // the sequential reduction inside the star: the owner of a row
                // through m is a column of this star, already final
                while (mask & kThrough) {
                    const int f = 31 - __clz(mask) - 24;
                    if (owner[f] < 0) {
                        owner[f] = int8_t(k);
                        b.pivot[edge_id_at(it, m, kFace[f][0], kFace[f][1], kFace[f][2])] =
                            make_key(ordm, uint64_t(it.voff + m), uint32_t(n3(oz, oy, ox)));
                        break;
                    }
                    mask ^= colmask[owner[f]];
                }
                colmask[k] = mask;
                b.cmask[q] = mask;
                b.coff[q] = ~0ull;
                if (!(mask & kThrough)) nonlocal[nn++] = q;  // (mask 0 only with inconsistent marks: flagged by the counts)
            }
        }
        // the columns that leave their star, appended warp by warp
        uint32_t incl = nn;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= unsigned(o)) incl += t;
        }
        uint32_t at = 0;
        if (lane == 31 && incl) at = atomicAdd(&b.ctl->nl, incl);
        at = __shfl_sync(0xFFFFFFFFu, at, 31) + incl - nn;
        for (uint32_t i = 0; i < nn; ++i)
            if (at + i < b.mcap) b.list0[at + i] = nonlocal[i];
    }
    ne = __reduce_add_sync(0xFFFFFFFFu, ne);
    pe = __reduce_add_sync(0xFFFFFFFFu, pe);
    pq = __reduce_add_sync(0xFFFFFFFFu, pq);
    nm = __reduce_add_sync(0xFFFFFFFFu, nm);
    if (lane == 0) {
        if (ne) atomicAdd(&b.ctl->neg_e, ne);
        if (pe) atomicAdd(&b.ctl->pos_e, pe);
        if (pq) atomicAdd(&b.ctl->pos_q, pq);
        if (nm) atomicAdd(&b.ctl->m, nm);
    }
}

struct ReduceArgs {
    ItemTable tab;
    H1Bufs b;
    Counters* ctr;
    uint64_t budget_ns;  // wall-clock budget of the rounds
    uint32_t solo_cols;  // see kSoloDefault (0: never alone)
};

// A column's entries: in the pool (off != ~0) or decoded into shared memory.
struct ColSrc {
    uint64_t off;
    const uint64_t* sm;
    uint32_t len;
};

// The warp merges the entries of c and p after their common lowest one into
// out (symmetric difference over F2) and returns how many it wrote.  The
// merged sequence is taken in tiles of kMT positions: the warp stages the
// tile's slices of both columns in shared memory, every lane issuing all of
// its loads before its first store (one round trip per tile instead of one
// per entry), then each lane takes kME positions of the tile, its start found
// by a binary search on the merge path in shared memory.  An entry in both
// columns lands next to its twin (ties put c's first) and both are dropped: a
// lane keeps a c entry unless the next p entry equals it, and a p entry unless
// the last c entry taken equals it.  A first pass counts each lane's
// survivors, a warp prefix sum places them, a second pass writes.
constexpr uint32_t kME = 12;         // merged positions per lane and tile
constexpr uint32_t kMT = 32 * kME;   // merged positions per tile
struct MergeTile {
    uint64_t c[kMT + 1];  // c[it - 1 .. it + kMT) (~0 before c's first entry)
    uint64_t p[kMT];      // p[jt .. jt + kMT)
};

__device__ uint32_t warp_merge(const H1Bufs& b, const ColSrc& c, const ColSrc& p, uint64_t* out, MergeTile& t) {
    const unsigned lane = lane_id();
    const uint32_t nc = c.len - 1u, np = p.len - 1u, total = nc + np;
    auto gc = [&](uint32_t i) { return c.off != ~0ull ? __ldcg(b.pool + c.off + 1 + i) : c.sm[1 + i]; };
    auto gp = [&](uint32_t i) { return p.off != ~0ull ? __ldcg(b.pool + p.off + 1 + i) : p.sm[1 + i]; };
    uint32_t it = 0, jt = 0, written = 0;  // entries of c and p before this tile, entries written
    for (uint32_t dt = 0; dt < total; dt += kMT) {
        const uint32_t tn = min(kMT, total - dt);
        const uint32_t cn = min(tn, nc - it), pn = min(tn, np - jt);  // staged entries of each
        {
            uint64_t vc[kME + 1], vp[kME];
#pragma unroll
            for (uint32_t s = 0; s <= kME; ++s) {
                const uint32_t k = lane + 32u * s;
                vc[s] = k <= cn ? ((it + k == 0u) ? ~0ull : gc(it + k - 1u)) : 0ull;
            }
#pragma unroll
            for (uint32_t s = 0; s < kME; ++s) {
                const uint32_t k = lane + 32u * s;
                vp[s] = k < pn ? gp(jt + k) : 0ull;
            }
#pragma unroll
            for (uint32_t s = 0; s <= kME; ++s)
                if (lane + 32u * s <= cn) t.c[lane + 32u * s] = vc[s];
#pragma unroll
            for (uint32_t s = 0; s < kME; ++s)
                if (lane + 32u * s < pn) t.p[lane + 32u * s] = vp[s];
        }
        __syncwarp();
        const uint32_t d0 = min(tn, lane * kME), d1 = min(tn, d0 + kME);
        // split at d0: the smallest i such that C(i) would not precede P(d0-i-1) (keys descending)
        uint32_t lo = d0 > pn ? d0 - pn : 0u, hi = min(d0, cn);
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (t.c[mid + 1u] >= t.p[d0 - mid - 1u]) lo = mid + 1u;
            else hi = mid;
        }
        const uint32_t i0 = lo, j0 = d0 - lo;
        uint32_t kept = 0, ie = i0, je = j0;
        for (int pass = 0; pass < 2; ++pass) {
            uint64_t* w = nullptr;
            if (pass == 1) {
                uint32_t incl = kept;
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                    if (lane >= unsigned(o)) incl += v;
                }
                w = out + written + (incl - kept);
                written += __shfl_sync(0xFFFFFFFFu, incl, 31);
            }
            uint32_t i = i0, j = j0;
            uint64_t x = i < cn ? t.c[i + 1u] : 0, y = j < pn ? t.p[j] : 0;
            uint64_t prevc = t.c[i];  // the last entry of c taken (~0: none)
            for (uint32_t d = d0; d < d1; ++d) {
                if (j >= pn || (i < cn && x >= y)) {
                    const bool keep = !(j < pn && y == x);
                    if (pass == 0) kept += keep ? 1u : 0u;
                    else if (keep) *w++ = x;
                    prevc = x;
                    ++i;
                    x = i < cn ? t.c[i + 1u] : 0;
                } else {
                    const bool keep = prevc != y;
                    if (pass == 0) kept += keep ? 1u : 0u;
                    else if (keep) *w++ = y;
                    ++j;
                    y = j < pn ? t.p[j] : 0;
                }
            }
            ie = i;
            je = j;
        }
        // the next tile starts where the last lane's range ended (lane 31's
        // range ends at tn: its start is min(tn, kMT - kME))
        it += __shfl_sync(0xFFFFFFFFu, ie, 31);
        jt += __shfl_sync(0xFFFFFFFFu, je, 31);
        __syncwarp();  // the tile is read by every lane before the next one is staged
    }
    return written;
}

// A merge that the first CTA, running the rounds alone, does with all its
// threads (a long one): the same merge path as warp_merge, in tiles of kCT
// positions, kCE per thread, with a CTA-wide prefix sum placing the kept
// entries.  The tile reuses the warps' shared tile space (no warp merge runs
// meanwhile).
constexpr uint32_t kCE = 4;
constexpr uint32_t kCT = kRT * kCE;
constexpr uint32_t kCtaMergeMin = 1024;  // entries from which a lone CTA merges together
struct CtaTile {
    uint64_t c[kCT + 1];
    uint64_t p[kCT];
};
static_assert(sizeof(CtaTile) <= sizeof(MergeTile) * (kRT / 32), "the CTA tile reuses the warps' tiles");
struct MergeJob {
    ColSrc c, p;
    uint64_t base;
    uint32_t q, cap, into;
    uint64_t sc[32], sp[32];  // a source still in its star mask, decoded (its ColSrc points here)
};
constexpr uint32_t kJobs = 16;  // long merges queued per round; beyond, warps merge them

__device__ uint32_t cta_merge(const H1Bufs& b, const ColSrc& c, const ColSrc& p, uint64_t* out, CtaTile& t,
                              uint32_t* sh) {
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t nc = c.len - 1u, np = p.len - 1u, total = nc + np;
    auto gc = [&](uint32_t i) { return c.off != ~0ull ? __ldcg(b.pool + c.off + 1 + i) : c.sm[1 + i]; };
    auto gp = [&](uint32_t i) { return p.off != ~0ull ? __ldcg(b.pool + p.off + 1 + i) : p.sm[1 + i]; };
    uint32_t it = 0, jt = 0, written = 0;
    for (uint32_t dt = 0; dt < total; dt += kCT) {
        const uint32_t tn = min(kCT, total - dt);
        const uint32_t cn = min(tn, nc - it), pn = min(tn, np - jt);
        {
            uint64_t vc[kCE + 1], vp[kCE];
#pragma unroll
            for (uint32_t s = 0; s <= kCE; ++s) {
                const uint32_t k = tid + kRT * s;
                vc[s] = k <= cn ? ((it + k == 0u) ? ~0ull : gc(it + k - 1u)) : 0ull;
            }
#pragma unroll
            for (uint32_t s = 0; s < kCE; ++s) {
                const uint32_t k = tid + kRT * s;
                vp[s] = k < pn ? gp(jt + k) : 0ull;
            }
#pragma unroll
            for (uint32_t s = 0; s <= kCE; ++s)
                if (tid + kRT * s <= cn) t.c[tid + kRT * s] = vc[s];
#pragma unroll
            for (uint32_t s = 0; s < kCE; ++s)
                if (tid + kRT * s < pn) t.p[tid + kRT * s] = vp[s];
        }
        __syncthreads();
        const uint32_t d0 = min(tn, tid * kCE), d1 = min(tn, d0 + kCE);
        uint32_t lo = d0 > pn ? d0 - pn : 0u, hi = min(d0, cn);
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (t.c[mid + 1u] >= t.p[d0 - mid - 1u]) lo = mid + 1u;
            else hi = mid;
        }
        const uint32_t i0 = lo, j0 = d0 - lo;
        uint32_t kept = 0, ie = i0, je = j0, tile_total = 0;
        for (int pass = 0; pass < 2; ++pass) {
            uint64_t* w = nullptr;
            if (pass == 1) {
                // CTA-wide exclusive scan of kept (warp scans, then the warp totals)
                uint32_t incl = kept;
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                    if (lane >= unsigned(o)) incl += v;
                }
                if (lane == 31) sh[warp] = incl;
                __syncthreads();
                if (warp == 0) {
                    const uint32_t v = lane < kRT / 32 ? sh[lane] : 0u;
                    uint32_t x = v;
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, x, o);
                        if (lane >= unsigned(o)) x += u;
                    }
                    if (lane < kRT / 32) sh[lane] = x - v;
                    if (lane == 31) sh[32] = x;
                }
                __syncthreads();
                w = out + written + sh[warp] + (incl - kept);
                tile_total = sh[32];
            }
            uint32_t i = i0, j = j0;
            uint64_t x = i < cn ? t.c[i + 1u] : 0, y = j < pn ? t.p[j] : 0;
            uint64_t prevc = t.c[i];
            for (uint32_t d = d0; d < d1; ++d) {
                if (j >= pn || (i < cn && x >= y)) {
                    const bool keep = !(j < pn && y == x);
                    if (pass == 0) kept += keep ? 1u : 0u;
                    else if (keep) *w++ = x;
                    prevc = x;
                    ++i;
                    x = i < cn ? t.c[i + 1u] : 0;
                } else {
                    const bool keep = prevc != y;
                    if (pass == 0) kept += keep ? 1u : 0u;
                    else if (keep) *w++ = y;
                    ++j;
                    y = j < pn ? t.p[j] : 0;
                }
            }
            ie = i;
            je = j;
        }
        __syncthreads();  // sh[0 .. 32] is read by every thread before it is rewritten
        if (tid == kRT - 1u) {  // its range ends at tn
            sh[33] = ie;
            sh[34] = je;
        }
        __syncthreads();
        it += sh[33];
        jt += sh[34];
        written += tile_total;
        __syncthreads();  // the tile and sh are read by every thread before the next tile
    }
    return written;
}

// Column q lost its row to an older column: add that column (F2: the
// symmetric difference; the common lowest entry cancels).  Columns that no
// addition has reached yet are read from their star masks.  A column that
// has been added to owns two pool regions and is rewritten into the one it
// does not occupy; when the result does not fit, it moves to a fresh pair of
// twice the size, so the pool holds a few times each column's largest size
// rather than every intermediate result.
//
// The addition is done by a whole warp, one warp per losing column
// (warp_merge).  Columns still in their star masks are decoded by the warp
// into shared memory (sc, sp: 30 keys each).
// With jobs set (the first CTA running the rounds alone), a long merge is
// not done here while the queue has room: the warp queues it for the whole
// CTA (cta_merge), with the keys of a source still in its star mask copied
// into the job, and the column's region words are written after it.
__device__ void add_winner_warp(const ReduceArgs& a, uint32_t q, uint32_t r, uint64_t* sc, uint64_t* sp,
                                MergeTile& tile, MergeJob* jobs = nullptr, uint32_t* njobs = nullptr) {
    const H1Bufs& b = a.b;
    const unsigned lane = lane_id();
    auto stop = [&](uint32_t status) {
        if (lane == 0) {
            if (status) set_status(a.ctr, status);
            atomicOr(&b.ctl->stop[r & 1u], 1u);
        }
    };
    if (!CP_IN(q, b.n_ids, a.ctr)) return stop(0);
    const Item* itc;
    int64_t mc;
    const uint64_t kc = column_key(a.tab, q, itc, mc);
    ColSrc c;
    c.off = column_at(b, q);
    c.sm = sc;
    if (c.off != ~0ull) {
        c.len = __ldcg(b.clen + q);
    } else {
        c.len = warp_decode(*itc, mc, __ldcg(b.cmask + q), sc);
    }
    if (c.off != ~0ull && !CP_IN(c.off + c.len, b.pool_cap + 1, a.ctr)) return stop(0);
    const uint64_t low = c.off != ~0ull ? __ldcg(b.pool + c.off) : sc[0];
    const uint32_t eid = edge_id(a.tab, low);
    if (!CP_IN(eid, b.n_ids, a.ctr)) return stop(0);
    const uint64_t kp = __ldcg(b.pivot + eid);
    if (c.len == 0u || kp >= kc) return stop(kStInternal);  // only after an earlier error
    const Item& itp = a.tab.it[item_of_vertex(a.tab, key_vertex(kp))];
    const uint32_t p = cell_id3(itp, kp, true);
    if (!CP_IN(p, b.n_ids, a.ctr)) return stop(0);
    ColSrc pc;
    pc.off = column_at(b, p);
    pc.sm = sp;
    if (pc.off != ~0ull) {
        pc.len = __ldcg(b.clen + p);
    } else {
        pc.len = warp_decode(itp, int64_t(key_vertex(kp)) - itp.voff, __ldcg(b.cmask + p), sp);
    }
    if (pc.off != ~0ull && !CP_IN(pc.off + pc.len, b.pool_cap + 1, a.ctr)) return stop(0);
    const uint64_t need = uint64_t(c.len) + pc.len - 2u;
    if (need == 0u || need > 0x1FFFFFFFull)  // empty: only after an earlier error; 2^29 entries: beyond
        return stop(need ? kStCapacity : kStInternal);  // any volume this library takes
    // the free region of q's pair, or a fresh pair twice the size needed
    uint64_t base = __ldcg(b.coff + q);
    uint32_t cap = base != ~0ull ? (__ldcg(b.ccap + q) & 0x7FFFFFFFu) : 0u;
    uint32_t into = base != ~0ull ? ((__ldcg(b.ccap + q) >> 31) ^ 1u) : 0u;
    if (need > cap) {
        cap = 4u;
        while (cap < need) cap <<= 1;
        cap <<= 1;
        uint64_t got = 0;
        if (lane == 0) got = atomicAdd(&b.ctl->grown, (unsigned long long)(2ull * cap));
        base = __shfl_sync(0xFFFFFFFFu, got, 0);
        if (base + 2ull * cap > b.pool_cap) return stop(kStCapacity);
        into = 0u;
    }
    if (jobs && need >= kCtaMergeMin) {
        uint32_t slot = 0;
        if (lane == 0) slot = atomicAdd(njobs, 1u);
        slot = __shfl_sync(0xFFFFFFFFu, slot, 0);
        if (slot < kJobs) {
            MergeJob& j = jobs[slot];
            if (c.off == ~0ull) j.sc[lane] = sc[lane];
            if (pc.off == ~0ull) j.sp[lane] = sp[lane];
            if (lane == 0) {
                j.c = c;
                j.p = pc;
                j.c.sm = j.sc;
                j.p.sm = j.sp;
                j.base = base;
                j.q = q;
                j.cap = cap;
                j.into = into;
            }
            __syncwarp();
            return;
        }
    }
    const uint32_t k = warp_merge(b, c, pc, b.pool + base + (into ? uint64_t(cap) : 0ull), tile);
    if (lane == 0) {
        atomicAdd(&b.ctl->additions, 1ull);
        atomicAdd(&b.ctl->merged, (unsigned long long)(c.len + pc.len));
        __stcg(b.coff + q, base);
        __stcg(b.ccap + q, cap | (into << 31));
        __stcg(b.clen + q, k);
    }
    if (k == 0) stop(kStInternal);
}

__global__ void __launch_bounds__(kRT) k_h1_reduce(const __grid_constant__ ReduceArgs a) {
    const H1Bufs& b = a.b;
    Counters* ctr = a.ctr;
    H1Ctl* ctl = b.ctl;
    if (ld_acquire_u32(&ctr->status) & kStSkip) return;  // set before the launch: every CTA returns
    if (blockIdx.x == 0 && threadIdx.x == 0 &&
        (ctl->m != b.mcap || ctl->pos_e != b.mcap || ctl->neg_e != b.exp_neg_e || ctl->pos_q != b.exp_pos_q ||
         ctl->nl > b.mcap))
        set_status(ctr, kStInternal);
    __shared__ uint32_t sh_n, sh_stop;
    __shared__ uint64_t sh_col[kRT / 32][2][32];  // per warp: two star columns decoded
    extern __shared__ MergeTile sh_tile[];        // per warp: the staged tile of a merge (kRT / 32)
    __shared__ MergeJob sh_jobs[kJobs];           // the first CTA alone: the round's long merges
    __shared__ uint32_t sh_njobs, sh_scan[35];
    uint32_t epoch = 0;
    const uint64_t t_start = global_timer_ns();  // read by thread 0 of CTA 0 only
    uint64_t t_mode = t_start;   // start of the current mode (thread 0 of CTA 0)
    uint32_t pgen = 0;           // wake-ups of the parked CTAs so far
    __shared__ uint32_t sh_wake[3];
    uint32_t nchg = min(ctl->nl, b.mcap);  // round 0: every column that left its star
    // the whole grid while many columns change; CTA 0 alone while few do (the
    // switches are decided on counts every CTA reads after the same barrier)
    bool solo = false;
    auto barrier = [&]() {
        if (solo) __syncthreads();  // orders the CTA's global writes and atomics too
        else grid_barrier(ctr, gridDim.x, epoch);
    };
    for (uint32_t r = 0;; ++r) {
        const uint32_t nblocks = solo ? 1u : gridDim.x, gstride = nblocks * kRT;
        const uint32_t gtid = blockIdx.x * kRT + threadIdx.x;  // CTA 0 is the one that stays
        uint32_t* work = b.list[r & 1u];
        const uint32_t* chg = r == 0 ? b.list0 : b.list[(r & 1u) ^ 1u];
        uint32_t* wcnt = &ctl->cnt[r % 3u];
        uint64_t tp0 = 0, tp1 = 0, tp2 = 0;
        if (gtid == 0) tp0 = global_timer_ns();
        // ---- bids: the oldest column of each row keeps it
        for (uint32_t i0 = blockIdx.x * kRT; i0 < nchg; i0 += gstride) {
            const uint32_t i = i0 + threadIdx.x;
            uint32_t lose = kNone;
            if (i < nchg) {
                uint32_t q = __ldcg(chg + i);
                if (!CP_IN(q, b.n_ids, ctr)) q = 0;
                const Item* it;
                int64_t m;
                const uint64_t kq = column_key(a.tab, q, it, m);
                const uint64_t low = column_low(b, *it, m, q);
                uint32_t eid = edge_id(a.tab, low);
                if (!CP_IN(eid, b.n_ids, ctr)) eid = 0;
                const unsigned long long old =
                    atomicMin(reinterpret_cast<unsigned long long*>(b.pivot + eid), kq);
                if (old < kq) {
                    lose = q;  // an older column holds the row
                } else if (old != ~0ull) {  // q displaces a younger holder
                    lose = cell_id3(a.tab.it[item_of_vertex(a.tab, key_vertex(old))], old, true);
                }
            }
            const uint32_t pos = warp_append(wcnt, lose != kNone);
            if (lose != kNone && pos < b.mcap) work[pos] = lose;
        }
        if (gtid == 0) tp1 = global_timer_ns();
        barrier();
        // one thread reads the round's outcome for the CTA, so that every CTA
        // takes the same path (the stop word of the previous round is
        // complete; this round's merges write the other one)
        if (threadIdx.x == 0) {
            sh_n = ld_acquire_u32(wcnt);
            sh_stop = (r > 0 ? ld_acquire_u32(&ctl->stop[(r - 1u) & 1u]) : 0u) |
                      (ld_acquire_u32(&ctr->status) & kStTimeout);
        }
        __syncthreads();
        const uint32_t nw = min(sh_n, b.mcap);
        const bool stop = sh_stop != 0u;
        __syncthreads();
        if (nw == 0u || stop || r + 1u >= kMaxRounds) {
            if (gtid == 0) {
                ctl->rounds = r + 1u;
                if (nw != 0u && !stop) set_status(ctr, kStInternal);
                const uint64_t now = global_timer_ns();
                if (solo) ctl->t_solo_ns += now - t_mode;
                else ctl->t_grid_ns += now - t_mode;
                if (solo) {  // the parked CTAs leave too
                    ctl->park_exit = 1u;
                    st_release_u32(&ctl->park_gen, pgen + 1u);
                }
            }
            break;
        }
        if (gtid == 0) {
            ctl->cnt[(r + 1u) % 3u] = 0u;  // the next round's bids (last read two rounds ago)
            ctl->nw_hist[min(31u - __clz(nw), 15u)] += 1u;
            tp2 = global_timer_ns();
            ctl->t_phase_ns[0] += tp1 - tp0;
            ctl->t_phase_ns[1] += tp2 - tp1;
        }
        // ---- every losing column adds the winner of its row
        // (one warp per losing column: long columns are merged 32 lanes wide)
        {
            // the warps take the additions, queueing the long merges of their
            // CTA; then the whole CTA does its queued merges one by one
            if (threadIdx.x == 0) sh_njobs = 0;
            __syncthreads();
            for (uint32_t i = gtid >> 5; i < nw; i += gstride >> 5)
                add_winner_warp(a, __ldcg(work + i), r, sh_col[threadIdx.x >> 5][0], sh_col[threadIdx.x >> 5][1],
                                sh_tile[threadIdx.x >> 5], sh_jobs, &sh_njobs);
            __syncthreads();
            const uint32_t nj = min(sh_njobs, kJobs);
            for (uint32_t jb = 0; jb < nj; ++jb) {
                const MergeJob& j = sh_jobs[jb];
                const uint32_t k = cta_merge(b, j.c, j.p, b.pool + j.base + (j.into ? uint64_t(j.cap) : 0ull),
                                             *reinterpret_cast<CtaTile*>(sh_tile), sh_scan);
                if (threadIdx.x == 0) {
                    atomicAdd(&ctl->additions, 1ull);
                    atomicAdd(&ctl->merged, (unsigned long long)(j.c.len + j.p.len));
                    __stcg(b.coff + j.q, j.base);
                    __stcg(b.ccap + j.q, j.cap | (j.into << 31));
                    __stcg(b.clen + j.q, k);
                    if (k == 0) {
                        set_status(ctr, kStInternal);
                        atomicOr(&ctl->stop[r & 1u], 1u);
                    }
                }
            }
        }
        // the budget: one thread decides, every CTA reads the decision (this
        // round's stop word) after the next barrier, so all leave together
        uint64_t tp3 = 0;
        if (gtid == 0) {
            tp3 = global_timer_ns();
            if (tp3 - t_start > a.budget_ns) {
                set_status(ctr, kStTimeout);
                atomicOr(&ctl->stop[r & 1u], 2u);
            }
        }
        barrier();
        if (gtid == 0) {
            ctl->t_phase_ns[2] += tp3 - tp2;
            ctl->t_phase_ns[3] += global_timer_ns() - tp3;
        }
        nchg = nw;
        if (!solo && nchg <= a.solo_cols) {
            if (gtid == 0) {
                const uint64_t now = global_timer_ns();
                ctl->t_grid_ns += now - t_mode;
                t_mode = now;
                if (ctl->solo_round == 0u) ctl->solo_round = r + 1u;
                ctl->solo_entries += 1u;
            }
            if (blockIdx.x != 0) {
                // parked (nothing of this CTA is in flight) until CTA 0 wakes
                // the grid or ends the rounds; bounded by the rounds' budget
                if (threadIdx.x == 0) {
                    const uint64_t t0 = global_timer_ns();
                    uint32_t g;
                    while ((g = ld_acquire_u32(&ctl->park_gen)) == pgen) {
                        if (global_timer_ns() - t0 > a.budget_ns + kWaitLimitNs) {
                            set_status(ctr, kStTimeout);
                            break;
                        }
                        __nanosleep(1000);
                    }
                    sh_wake[0] = g == pgen ? 1u : ld_acquire_u32(&ctl->park_exit);
                    sh_wake[1] = ctl->park_round;
                    sh_wake[2] = ctl->park_nchg;
                }
                __syncthreads();
                const bool leave = sh_wake[0] != 0u;
                const uint32_t rr = sh_wake[1], nn = sh_wake[2];
                __syncthreads();
                if (leave) return;
                ++pgen;
                r = rr - 1u;  // the loop's increment makes it rr
                nchg = nn;
                continue;
            }
            solo = true;
        } else if (solo && nchg > 2u * a.solo_cols) {
            // wake the grid for round r + 1 (every global write of this CTA
            // is ordered before the release)
            __threadfence();
            __syncthreads();
            if (gtid == 0) {
                const uint64_t now = global_timer_ns();
                ctl->t_solo_ns += now - t_mode;
                t_mode = now;
                ctl->park_round = r + 1u;
                ctl->park_nchg = nchg;
                st_release_u32(&ctl->park_gen, pgen + 1u);
            }
            ++pgen;
            solo = false;
        }
    }
}

// ---- the pairs (lowest entry, square) with nonzero persistence: only the
// columns that left their star (inside a star both cells enter with m)
__global__ void __launch_bounds__(kHT) k_h1_emit(const __grid_constant__ ItemTable tab, H1Bufs b, Counters* ctr,
                                                 cp_pair* pairs, uint32_t cap) {
    if (ld_acquire_u32(&ctr->status) & kStSkip) return;
    const uint32_t M = min(b.ctl->nl, b.mcap);
    for (uint32_t i0 = blockIdx.x * kHT; i0 < M; i0 += gridDim.x * kHT) {
        const uint32_t i = i0 + threadIdx.x;
        bool emit = false;
        cp_pair pr;
        if (i < M) {
            const uint32_t q = b.list0[i];
            const Item* it;
            int64_t m;
            const uint64_t sk = column_key(tab, q, it, m);
            const uint64_t ek = column_low(b, *it, m, q);
            const float fb = ord_float(uint32_t(ek >> 32)), fd = ord_float(uint32_t(sk >> 32));
            if (fb != fd) {  // zero persistence: omitted (Sec. 2.3)
                pr.birth = fb;
                pr.death = fd;
                pr.birth_cell = cell_index(*it, ek);
                pr.death_cell = cell_index(*it, sk);
                pr.birth_pixel = int32_t(int64_t(key_vertex(ek)) - it->voff);
                pr.death_pixel = int32_t(m);
                pr.dim = 1;
                pr.item = it->user;
                emit = true;
            }
        }
        const uint32_t pp = warp_append(&ctr->n_pairs, emit);
        if (emit) {
            if (pp < cap) pairs[pp] = pr;
            else set_status(ctr, kStCapacity);
        }
    }
}

std::atomic<int> g_h1_budget_ms{30000};
std::atomic<int> g_h1_solo_cols{kSoloDefault};

int grid_of(int64_t n) {
    const int64_t blocks = (n + kHT - 1) / kHT;
    const int64_t cap = int64_t(device_sm_count()) * 8;
    return int(blocks < 1 ? 1 : (blocks < cap ? blocks : cap));
}

}  // namespace

void set_h1_budget_ms(int ms) { g_h1_budget_ms.store(ms); }
int get_h1_budget_ms() { return g_h1_budget_ms.load(); }
void set_h1_solo_cols(int n) { g_h1_solo_cols.store(n); }
int get_h1_solo_cols() { return g_h1_solo_cols.load(); }

cudaError_t launch_h1(const ItemTable& tab, const H1Bufs& b, Counters* ctr, cp_pair* pairs, uint32_t pair_cap,
                      cudaStream_t s) {
    if (tab.n3d < 1) return cudaSuccess;
    const int64_t v0 = tab.it[tab.n2d].voff;
    const Item& last = tab.it[tab.n - 1];
    const int64_t v1 = last.voff + int64_t(last.D) * last.H * last.W;
    constexpr size_t kTileBytes = sizeof(MergeTile) * (kRT / 32);
    const int reduce_blocks = device_cached(kCacheH1, [] {
        if (cudaFuncSetAttribute(k_h1_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kTileBytes)) !=
            cudaSuccess)
            return -1;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_h1_reduce, kRT, kTileBytes);
        return per_sm > 0 ? device_sm_count() * per_sm : -1;
    });
    if (reduce_blocks <= 0) return cudaErrorLaunchOutOfResources;
    cudaError_t e = cudaMemsetAsync(b.ctl, 0, sizeof(H1Ctl), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.pivot, 0xFF, sizeof(uint64_t) * size_t(3 * v1), s);
    if (e != cudaSuccess) return e;
    k_h1_direct<<<grid_of(v1 - v0), kHT, 0, s>>>(tab, b, v0, v1);
    k_h1_local<<<grid_of(v1 - v0), kHT, 0, s>>>(tab, b, v0, v1);
    note_launches(2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ReduceArgs ra;
    ra.tab = tab;
    ra.b = b;
    ra.ctr = ctr;
    ra.budget_ns = uint64_t(get_h1_budget_ms()) * 1000000ull;
    ra.solo_cols = uint32_t(get_h1_solo_cols());
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(reduce_blocks);
    cfg.blockDim = dim3(kRT);
    cfg.dynamicSmemBytes = kTileBytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if ((e = cudaMemsetAsync(&ctr->bar_count, 0, sizeof(uint32_t), s)) != cudaSuccess) return e;
    if ((e = cudaLaunchKernelEx(&cfg, k_h1_reduce, ra)) != cudaSuccess) return e;
    k_h1_emit<<<grid_of(b.mcap), kHT, 0, s>>>(tab, b, ctr, pairs, pair_cap);
    note_launches(2);
    return cudaGetLastError();
}

}  // namespace cp
