// K1: fused lookup + local pruning (Sec. 3.2, Sec. 3.3, Sec. 4.1 steps 1-2,
// Sec. 4.2 steps 1-3 before the union-finds).
//
// One CTA per tile of vertices.  The tile and a one-vertex halo are staged
// in shared memory (out-of-image halo = +inf, so such neighbours never
// precede the centre and no bounds test is needed).  Per vertex v:
//   1. 8/26-bit mask of the neighbours that precede v (value, then index);
//   2. collapse to the relevant mask and look it up (2D: direct 256-entry
//      table; 3D: perfect hash of the 15,935 relevant masks);
//   3. write the H0 forest parent of v (first edge of L(v)) or register v as
//      an H0 root (local minimum);
//   4. write the dual forest parent of every top cell of L(v) (the top cell
//      across the facet where it dies locally, or the outside vertex) or
//      register it as a dual root;
//   5. emit the surviving edges and facets as 64-bit order keys.
// Survivors and roots are staged per CTA in shared memory and appended to
// global arrays with one atomic per buffer per flush.
#include "cp_common.cuh"
#include "cp_kernels.h"

namespace cp {

// Lookup tables in global memory, read through the read-only cache (lanes of
// a warp look up different entries, which constant memory would serialise).
__device__ uint64_t g_lut2d[256];
__device__ uint16_t g_disp3d[1 << 12];
// 3D entries as two 32-bit words for cheap decoding:
//   x: direct (3 bits) | h0_surv << 3 (6) | dual_surv << 9 (12) | in_l << 21 (8)
//   y: the eight 4-bit dual codes
__device__ uint2 g_entries3d[1 << 14];  // perfect-hash slots of the 3D table (128 KB)

// slot -> stencil bit tables
__constant__ int8_t c_face_n3[6] = {4, 10, 12, 14, 16, 22};
__constant__ int8_t c_facet_n3[12] = {1, 3, 5, 7, 9, 11, 15, 17, 19, 21, 23, 25};
__constant__ int8_t c_top_n3[8] = {0, 2, 6, 8, 18, 20, 24, 26};
__constant__ int8_t c_face_n2[4] = {1, 3, 5, 7};
__constant__ int8_t c_top_n2[4] = {0, 2, 6, 8};

namespace {

constexpr int kBX = 32, kBY = 8;          // CTA shape
constexpr int kThreads = kBX * kBY;
constexpr int kCapS = 4096;               // staged survivor keys per kind
constexpr int kCapR = 1024;               // staged roots per kind

struct Stage {
    uint64_t s0[kCapS];
    uint64_t st[kCapS];
    uint64_t r0age[kCapR];
    uint64_t rtage[kCapR];
    uint32_t r0node[kCapR];
    uint32_t rtnode[kCapR];
    uint32_t n_s0, n_st, n_r0, n_rt;
    uint32_t base_s0, base_st, base_r0, base_rt;
    unsigned long long gmin;
};

struct Outs {
    uint32_t* uf0;
    uint32_t* uft;
    uint64_t* s0;
    uint64_t* st;
    uint64_t* age0;
    uint64_t* res0;
    uint64_t* aget;
    uint64_t* rest;
    uint32_t cap_s, cap_r0, cap_rt;
    Counters* ctr;
};

// warp-aggregated reservation of `k` slots in a shared-memory buffer
__device__ __forceinline__ uint32_t stage_reserve(uint32_t* counter, uint32_t k) {
    unsigned lane = lane_id();
    uint32_t incl = k;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= unsigned(o)) incl += t;
    }
    uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    uint32_t base = 0;
    if (lane == 31 && total) base = atomicAdd(counter, total);
    base = __shfl_sync(0xFFFFFFFFu, base, 31);
    return base + incl - k;
}

__device__ void flush(Stage& sg, const Outs& o) {
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        sg.base_s0 = sg.n_s0 ? atomicAdd(&o.ctr->n_s0, sg.n_s0) : 0;
        sg.base_st = sg.n_st ? atomicAdd(&o.ctr->n_st, sg.n_st) : 0;
        sg.base_r0 = sg.n_r0 ? atomicAdd(&o.ctr->n_r0, sg.n_r0) : 0;
        sg.base_rt = sg.n_rt ? atomicAdd(&o.ctr->n_rt, sg.n_rt) : 0;
    }
    __syncthreads();
    const int tid = threadIdx.y * kBX + threadIdx.x;
    for (uint32_t i = tid; i < sg.n_s0; i += kThreads) {
        uint32_t g = sg.base_s0 + i;
        if (g < o.cap_s) o.s0[g] = sg.s0[i];
    }
    for (uint32_t i = tid; i < sg.n_st; i += kThreads) {
        uint32_t g = sg.base_st + i;
        if (g < o.cap_s) o.st[g] = sg.st[i];
    }
    for (uint32_t i = tid; i < sg.n_r0; i += kThreads) {
        uint32_t g = sg.base_r0 + i;
        if (g < o.cap_r0) {
            o.age0[g] = sg.r0age[i];
            o.res0[g] = 0;
            o.uf0[sg.r0node[i]] = kTag | g;
        } else {
            o.uf0[sg.r0node[i]] = kTag;  // out of capacity: keep the forest well formed (result flagged invalid)
        }
    }
    for (uint32_t i = tid; i < sg.n_rt; i += kThreads) {
        uint32_t g = sg.base_rt + i;
        if (g < o.cap_rt) {
            o.aget[g] = sg.rtage[i];
            o.rest[g] = 0;
            o.uft[sg.rtnode[i]] = kTag | g;
        } else {
            o.uft[sg.rtnode[i]] = kTag;
        }
    }
    if (tid == 0) {
        bool over = (sg.n_s0 && sg.base_s0 + sg.n_s0 > o.cap_s) || (sg.n_st && sg.base_st + sg.n_st > o.cap_s) ||
                    (sg.n_r0 && sg.base_r0 + sg.n_r0 > o.cap_r0) || (sg.n_rt && sg.base_rt + sg.n_rt > o.cap_rt);
        if (over) set_status(o.ctr, kStCapacity);
    }
    __syncthreads();
    if (tid == 0) sg.n_s0 = sg.n_st = sg.n_r0 = sg.n_rt = 0;
    __syncthreads();
}

// A non-finite pixel flags the call as failed and is read as the largest
// finite float, so the order stays total and every cell still lies in exactly
// one lower star (the forests stay well formed even though the result is
// discarded).  The +inf halo stays above every pixel.
__device__ __forceinline__ float load_finite(const float* p, Counters* ctr) {
    float v = __ldg(p);
    if (!isfinite(v)) {
        set_status(ctr, kStNonfinite);
        v = 3.40282347e38f;
    }
    return v;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(0xFFFFFFFFu, v, o);
        v = t < v ? t : v;
    }
    return v;
}

// Emit everything one vertex contributes, given its lookup entry.
// (z, y, x): local coordinates; vg: global vertex id; valid: vertex exists.
template <int NDIM>
__device__ __forceinline__ void emit_vertex(Stage& sg, const Outs& o, const Item& it, bool valid, int z, int y,
                                            int x, uint32_t vg, uint32_t ord, uint64_t e,
                                            unsigned long long& my_min) {
    // ---- H0 forest parent / root
    int direct = valid ? int(e & 7u) : 0;
    bool root0 = valid && direct == 7;
    if (valid && !root0) {
        int n = NDIM == 3 ? c_face_n3[direct] : c_face_n2[direct];
        int dz, dy, dx;
        stencil_off(NDIM, n, dz, dy, dx);
        o.uf0[vg] = uint32_t(int64_t(vg) + (int64_t(dz) * it.H + dy) * it.W + dx);
    }
    if (root0) {
        unsigned long long k = (unsigned long long)(uint64_t(ord) << 32 | uint32_t(vg - it.voff));
        my_min = k < my_min ? k : my_min;
    }
    uint32_t h0s = valid ? uint32_t((e >> 3) & 0x3Fu) : 0u;
    uint32_t ds = valid ? uint32_t((e >> 41) & 0xFFFu) : 0u;
    // ---- dual forest parents / dual root
    int rt_node = -1;
    uint64_t rt_age = 0;
    if (valid) {
        const int ntops = NDIM == 3 ? 8 : 4;
#pragma unroll
        for (int t = 0; t < ntops; ++t) {
            uint32_t code = uint32_t(e >> (9 + 4 * t)) & 15u;
            if (code == 15u) continue;
            int n = NDIM == 3 ? c_top_n3[t] : c_top_n2[t];
            int dz, dy, dx;
            stencil_off(NDIM, n, dz, dy, dx);
            uint32_t self = top_of_octant(it, z, y, x, dz, dy, dx);
            if (code == 8u) {
                rt_node = int(self);
                rt_age = make_key(ord, vg, NDIM == 3 ? uint32_t(n) : uint32_t(n) << 1);
            } else {
                int n2 = NDIM == 3 ? c_top_n3[code] : c_top_n2[code];
                int ez, ey, ex;
                stencil_off(NDIM, n2, ez, ey, ex);
                o.uft[self] = top_of_octant(it, z, y, x, ez, ey, ex);
            }
        }
    }
    // ---- stage survivors and roots
    uint32_t k0 = __popc(h0s);
    uint32_t kt = NDIM == 3 ? __popc(ds) : __popc(ds & ~h0s);
    uint32_t p0 = stage_reserve(&sg.n_s0, k0);
    uint32_t pt = stage_reserve(&sg.n_st, kt);
    uint32_t pr0 = stage_reserve(&sg.n_r0, root0 ? 1u : 0u);
    uint32_t prt = stage_reserve(&sg.n_rt, rt_node >= 0 ? 1u : 0u);
    const int nf = NDIM == 3 ? 6 : 4;
    for (int s = 0; s < nf; ++s) {
        if (!((h0s >> s) & 1u)) continue;
        int n = NDIM == 3 ? c_face_n3[s] : c_face_n2[s];
        uint32_t low = NDIM == 3 ? uint32_t(n) : (uint32_t(n) << 1) | ((ds >> s) & 1u);
        sg.s0[p0++] = make_key(ord, vg, low);
    }
    if (NDIM == 3) {
        for (int f = 0; f < 12; ++f) {
            if (!((ds >> f) & 1u)) continue;
            sg.st[pt++] = ~make_key(ord, vg, uint32_t(c_facet_n3[f]));
        }
    } else {
        uint32_t m = ds & ~h0s;
        for (int f = 0; f < 4; ++f) {
            if (!((m >> f) & 1u)) continue;
            sg.st[pt++] = ~make_key(ord, vg, uint32_t(c_face_n2[f]) << 1);
        }
    }
    if (root0) {
        sg.r0node[pr0] = vg;
        sg.r0age[pr0] = make_key(ord, vg, 0);
    }
    if (rt_node >= 0) {
        sg.rtnode[prt] = uint32_t(rt_node);
        sg.rtage[prt] = rt_age;
    }
}

__device__ __forceinline__ void finish_min(Stage& sg, const Outs& o, int item, unsigned long long my_min) {
    unsigned long long w = warp_min_u64(my_min);
    if (lane_id() == 0 && w != ~0ull) atomicMin(&sg.gmin, w);
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0 && sg.gmin != ~0ull) atomicMin(&o.ctr->gmin[item], sg.gmin);
}

__device__ __forceinline__ int tile_item(const ItemTable& t, int first, int last, int tile) {
    int lo = first, hi = last;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (t.it[mid].tile0 <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// 3D relevant mask from the raw mask (bit n = 9(dz+1)+3(dy+1)+(dx+1)):
// an edge diagonal needs its two faces, a corner its three edge diagonals.
__device__ __forceinline__ uint32_t collapse3(uint32_t raw) {
    constexpr uint32_t X0 = (1u << 1) | (1u << 4) | (1u << 7) | (1u << 10) | (1u << 13) | (1u << 16) | (1u << 19) |
                            (1u << 22) | (1u << 25);
    constexpr uint32_t Y0 = (7u << 3) | (7u << 12) | (7u << 21);
    constexpr uint32_t Z0 = 0x1FFu << 9;
    constexpr uint32_t FACES = (1u << 4) | (1u << 10) | (1u << 12) | (1u << 14) | (1u << 16) | (1u << 22);
    constexpr uint32_t EDXY = (1u << 9) | (1u << 11) | (1u << 15) | (1u << 17);
    constexpr uint32_t EDXZ = (1u << 3) | (1u << 5) | (1u << 21) | (1u << 23);
    constexpr uint32_t EDYZ = (1u << 1) | (1u << 7) | (1u << 19) | (1u << 25);
    constexpr uint32_t CORN = (1u << 0) | (1u << 2) | (1u << 6) | (1u << 8) | (1u << 18) | (1u << 20) | (1u << 24) |
                              (1u << 26);
    uint32_t f = raw & FACES;
    uint32_t ux = ((f & X0) << 1) | ((f & X0) >> 1);
    uint32_t uy = ((f & Y0) << 3) | ((f & Y0) >> 3);
    uint32_t uz = ((f & Z0) << 9) | ((f & Z0) >> 9);
    uint32_t ed = raw & ((EDXY & ux & uy) | (EDXZ & ux & uz) | (EDYZ & uy & uz));
    uint32_t vx = ((ed & X0) << 1) | ((ed & X0) >> 1);
    uint32_t vy = ((ed & Y0) << 3) | ((ed & Y0) >> 3);
    uint32_t vz = ((ed & Z0) << 9) | ((ed & Z0) >> 9);
    uint32_t co = raw & CORN & vx & vy & vz;
    return f | ed | co;
}

__device__ __forceinline__ uint2 lookup3(uint32_t rel) {
    uint32_t b = (rel * 0x9E3779B1u) >> (32 - 12);
    uint32_t d = __ldg(g_disp3d + b);
    uint32_t s = ((rel ^ (d * 0x27D4EB2Fu)) * 0x85EBCA77u) >> (32 - 14);
    return __ldg(g_entries3d + s);
}

}  // namespace

// ---------------------------------------------------------------- 2D
// Tile: 32 x 32 vertices, CTA 32 x 8, 4 rows per thread.
constexpr int kT2Y = 32;  // largest tile height (the shared tile is sized for it)

__global__ void __launch_bounds__(kThreads) k_prune2d(ItemTable tab, Outs o) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Stage& sg = *reinterpret_cast<Stage*>(smem_raw);
    float* tile = reinterpret_cast<float*>(smem_raw + sizeof(Stage));  // (kT2Y+2) x (32+2)
    const int tid = threadIdx.y * kBX + threadIdx.x;
    const int t = blockIdx.x;
    const int ii = tile_item(tab, 0, tab.n2d - 1, t);
    const Item& it = tab.it[ii];
    const int lt = t - it.tile0;
    const int rows = tab.rows2d;
    const int x0 = (lt % it.tx) * kBX, y0 = (lt / it.tx) * rows;
    __shared__ uint64_t lut[256];
    lut[tid] = g_lut2d[tid];
    if (tid == 0) {
        sg.n_s0 = sg.n_st = sg.n_r0 = sg.n_rt = 0;
        sg.gmin = ~0ull;
    }
    constexpr int SW = kBX + 2;
    for (int i = tid; i < (rows + 2) * SW; i += kThreads) {
        int ly = i / SW, lx = i % SW;
        int gy = y0 + ly - 1, gx = x0 + lx - 1;
        float v = __int_as_float(0x7F800000);  // +inf: never precedes anything
        if (gy >= 0 && gy < it.H && gx >= 0 && gx < it.W) v = load_finite(it.img + int64_t(gy) * it.W + gx, o.ctr);
        tile[i] = v;
    }
    __syncthreads();
    unsigned long long my_min = ~0ull;
    for (int r = 0; r < rows / kBY; ++r) {
        int ly = threadIdx.y + r * kBY, lx = threadIdx.x;
        int y = y0 + ly, x = x0 + lx;
        bool valid = y < it.H && x < it.W;
        const float* c = tile + (ly + 1) * SW + (lx + 1);
        float cv = c[0];
        uint32_t raw = 0;
        if (valid) {
            // bits 0..3: offsets before v in linear order (ties precede); 4..7 after
            raw |= (c[-SW - 1] <= cv) ? 1u : 0u;
            raw |= (c[-SW] <= cv) ? 2u : 0u;
            raw |= (c[-SW + 1] <= cv) ? 4u : 0u;
            raw |= (c[-1] <= cv) ? 8u : 0u;
            raw |= (c[1] < cv) ? 16u : 0u;
            raw |= (c[SW - 1] < cv) ? 32u : 0u;
            raw |= (c[SW] < cv) ? 64u : 0u;
            raw |= (c[SW + 1] < cv) ? 128u : 0u;
        }
        uint64_t e = lut[raw];
        uint32_t vg = uint32_t(it.voff + int64_t(y) * it.W + x);
        emit_vertex<2>(sg, o, it, valid, 0, y, x, vg, ord_bits(cv), e, my_min);
        __syncthreads();
    }
    flush(sg, o);
    finish_min(sg, o, ii, my_min);
}

// ---------------------------------------------------------------- 3D
// A CTA of 9 warps marches through a chunk of planes.  Warp w handles row
// y0-1+w and lane l column x0-1+l: the CTA owns the 31 x 8 vertices with
// w >= 1 and l >= 1; row y0-1 and column x0-1 are a halo whose lookups are
// needed, but whose outputs belong to the neighbouring CTA.
//
// Per plane step z:
//  1. cp.async prefetch of image plane z+kAhead (34 x 11 floats: the CTA's
//     vertices and a one-vertex border) into an 8-slot shared-memory ring;
//  2. the 26-neighbour mask of (z, y, x) from registers (planes z-1, z) and
//     the ring (plane z+1), table lookup, the H0 forest link and the
//     survivors and H0 root of owned vertices; the entry's dual codes go to
//     a 3-plane shared ring;
//  3. one barrier;
//  4. the top cell whose smallest corner is (z-1, y, x): its largest corner
//     m among the 8 corner values (in registers) holds, in its lookup entry,
//     where this top cell dies locally; one coalesced store of its dual
//     forest link (or it becomes a dual root).
// Survivors and roots are staged per warp with ballots and flushed with one
// atomic per buffer when a buffer would overflow and at the end.
constexpr int kW3 = 9;                     // warps per CTA
constexpr int kT3 = kW3 * 32;
constexpr int kOX = 31, kOY = 8;           // owned columns / rows per CTA
constexpr int kZC = 64;                    // default owned planes per task
constexpr int kRW = 34, kRH = kW3 + 2, kRP = kRW * kRH;  // ring plane: cols x0-2.., rows y0-2..
constexpr int kRing = 8, kAhead = 5;       // ring slots, planes in flight
constexpr int kCapW0 = 32 * 5;             // staged H0 keys per warp (one step's maximum)
constexpr int kCapWT = 32 * 7;             // staged dual keys per warp
constexpr int kCapWR = 32;                 // staged roots per warp and kind

struct WarpStage {
    uint64_t s0[kCapW0];
    uint64_t st[kCapWT];
    uint64_t r0age[kCapWR];
    uint64_t rtage[kCapWR];
    uint32_t r0node[kCapWR];
    uint32_t rtnode[kCapWR];
};

struct Smem3 {
    float ring[kRing][kRP];
    uint32_t codes[3][kW3][32];
    WarpStage ws[kW3];
};

struct WarpCounts {
    uint32_t s0, st, r0, rt;
};

__device__ __forceinline__ void warp_flush(WarpStage& ws, WarpCounts& c, const Outs& o) {
    __syncwarp();
    const unsigned lane = lane_id();
    uint32_t b0 = 0, bt = 0, br0 = 0, brt = 0;
    if (lane == 0) {
        if (c.s0) b0 = atomicAdd(&o.ctr->n_s0, c.s0);
        if (c.st) bt = atomicAdd(&o.ctr->n_st, c.st);
        if (c.r0) br0 = atomicAdd(&o.ctr->n_r0, c.r0);
        if (c.rt) brt = atomicAdd(&o.ctr->n_rt, c.rt);
        bool over = (c.s0 && b0 + c.s0 > o.cap_s) || (c.st && bt + c.st > o.cap_s) ||
                    (c.r0 && br0 + c.r0 > o.cap_r0) || (c.rt && brt + c.rt > o.cap_rt);
        if (over) set_status(o.ctr, kStCapacity);
    }
    b0 = __shfl_sync(0xFFFFFFFFu, b0, 0);
    bt = __shfl_sync(0xFFFFFFFFu, bt, 0);
    br0 = __shfl_sync(0xFFFFFFFFu, br0, 0);
    brt = __shfl_sync(0xFFFFFFFFu, brt, 0);
    for (uint32_t i = lane; i < c.s0; i += 32)
        if (b0 + i < o.cap_s) o.s0[b0 + i] = ws.s0[i];
    for (uint32_t i = lane; i < c.st; i += 32)
        if (bt + i < o.cap_s) o.st[bt + i] = ws.st[i];
    for (uint32_t i = lane; i < c.r0; i += 32) {
        uint32_t g = br0 + i;
        if (g < o.cap_r0) {
            o.age0[g] = ws.r0age[i];
            o.res0[g] = 0;
            o.uf0[ws.r0node[i]] = kTag | g;
        } else {
            o.uf0[ws.r0node[i]] = kTag;  // out of capacity: keep the forest well formed (result flagged invalid)
        }
    }
    for (uint32_t i = lane; i < c.rt; i += 32) {
        uint32_t g = brt + i;
        if (g < o.cap_rt) {
            o.aget[g] = ws.rtage[i];
            o.rest[g] = 0;
            o.uft[ws.rtnode[i]] = kTag | g;
        } else {
            o.uft[ws.rtnode[i]] = kTag;
        }
    }
    c.s0 = c.st = c.r0 = c.rt = 0;
    __syncwarp();
}

// lower-than bit: all ones when the neighbour precedes the centre
__device__ __forceinline__ uint32_t set_le(float a, float b) {
    uint32_t r;
    asm("set.le.u32.f32 %0, %1, %2;" : "=r"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ uint32_t set_lt(float a, float b) {
    uint32_t r;
    asm("set.lt.u32.f32 %0, %1, %2;" : "=r"(r) : "f"(a), "f"(b));
    return r;
}

struct Nbr {
    float v[3][3];  // [row y-1, y, y+1][col x-1, x, x+1] of one plane
};

__device__ __forceinline__ void read_nbr(const float* plane, int ly, int lx, Nbr& P) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) P.v[r][c] = plane[(ly + r) * kRW + (lx + c)];
}

// raw mask: bit n = 9a + 3b + c set when the neighbour at plane a, row b,
// column c precedes the centre (ties: earlier linear index first)
__device__ __forceinline__ uint32_t mask26(const Nbr& A, const Nbr& B, const Nbr& C) {
    const float cv = B.v[1][1];
    uint32_t raw = 0;
#pragma unroll
    for (int n = 26; n >= 0; --n) {
        if (n == 13) continue;
        const int a = n / 9, b = (n / 3) % 3, c = n % 3;
        const Nbr& P = a == 0 ? A : (a == 1 ? B : C);
        const uint32_t t = n < 13 ? set_le(P.v[b][c], cv) : set_lt(P.v[b][c], cv);
        raw = (raw << 1) - t;  // append one bit (t is 0 or all ones)
        if (n == 14) raw <<= 1;  // leave bit 13 (the centre) clear
    }
    return raw;
}

// ---- image plane ring, filled with cp.async
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    const uint32_t d = uint32_t(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Ring positions of this thread (at most two), fixed for a task.
struct RingPos {
    uint32_t off0, off1;  // offset of the pixel in a plane
    bool in0, in1;        // inside the image (x, y)
    bool has1;            // second position exists
};

__device__ __forceinline__ void ring_positions(const Item& it, int x0, int y0, RingPos& rp) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int i = tid + k * kT3;
        const int ly = i / kRW, lx = i - ly * kRW;
        const int gy = y0 - 2 + ly, gx = x0 - 2 + lx;
        const bool in = i < kRP && unsigned(gy) < unsigned(it.H) && unsigned(gx) < unsigned(it.W);
        const uint32_t off = in ? uint32_t(gy) * uint32_t(it.W) + uint32_t(gx) : 0u;
        if (k == 0) {
            rp.off0 = off;
            rp.in0 = in;
        } else {
            rp.off1 = off;
            rp.in1 = in;
            rp.has1 = i < kRP;
        }
    }
}

// Out-of-image positions read +inf (never precede anything): set once per
// task in every slot; the copies below only fill in-image positions.
__device__ __forceinline__ void ring_init(Smem3& sm, const RingPos& rp) {
    const float inf = __int_as_float(0x7F800000);
    const int tid = threadIdx.x;
#pragma unroll
    for (int s = 0; s < kRing; ++s) {
        if (!rp.in0) sm.ring[s][tid] = inf;
        if (rp.has1 && !rp.in1) sm.ring[s][tid + kT3] = inf;
    }
}

__device__ __forceinline__ void issue_plane(Smem3& sm, const Item& it, int z, const RingPos& rp, uint32_t HW) {
    float* plane = sm.ring[(z + kRing) & (kRing - 1)];
    const int tid = threadIdx.x;
    if (unsigned(z) < unsigned(it.D)) {
        const float* base = it.img + uint32_t(z) * HW;
        if (rp.in0) cp_async4(plane + tid, base + rp.off0);
        if (rp.in1) cp_async4(plane + tid + kT3, base + rp.off1);
    } else {  // a plane outside the volume: every position +inf
        const float inf = __int_as_float(0x7F800000);
        if (rp.in0) plane[tid] = inf;
        if (rp.in1) plane[tid + kT3] = inf;
    }
    cp_async_commit();
}

struct Col {
    int x, y;
    uint32_t W, H, D, HW, W1, HW1, voff, toff, OUT;
    bool in_xy;      // (x, y) inside the image
    bool owned_xy;   // and owned by this CTA
    bool cube_xy;    // (x, y) is the smallest corner of a top cell written by this thread
    uint32_t bxy;    // boundary bits (2: y==0, 3: y==H-1, 4: x==0, 5: x==W-1)
};

__device__ __forceinline__ uint32_t age_slot(uint32_t t) {
    return 18u * ((t >> 2) & 1u) + 6u * ((t >> 1) & 1u) + 2u * (t & 1u);
}

__global__ void __launch_bounds__(kT3, 4) k_prune3d(ItemTable tab, Outs o) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem3& sm = *reinterpret_cast<Smem3*>(smem_raw);
    const int warp = threadIdx.x >> 5;
    const int lane = int(lane_id());
    const unsigned lt = (1u << lane) - 1u;
    WarpStage& ws = sm.ws[warp];
    WarpCounts cnt = {0, 0, 0, 0};
    for (int task = blockIdx.x; task < tab.tiles3d; task += gridDim.x) {
        const int ii = tile_item(tab, tab.n2d, tab.n - 1, task);
        const Item& it = tab.it[ii];
        const int ltask = task - it.tile0;
        // task order: x segment fastest, then y segment, then z chunk
        const int xs = ltask % it.tx;
        const int rest = ltask / it.tx;
        const int ys = rest % it.ty;
        const int zc = rest / it.ty;
        const int x0 = xs * kOX, y0 = ys * kOY;
        Col cc;
        cc.x = x0 - 1 + lane;
        cc.y = y0 - 1 + warp;
        cc.W = uint32_t(it.W);
        cc.H = uint32_t(it.H);
        cc.D = uint32_t(it.D);
        cc.HW = cc.H * cc.W;
        cc.W1 = cc.W - 1u;
        cc.HW1 = (cc.H - 1u) * cc.W1;
        cc.voff = uint32_t(it.voff);
        cc.toff = uint32_t(it.toff);
        cc.OUT = uint32_t(it.toff + it.T);
        cc.in_xy = cc.x >= 0 && cc.y >= 0 && cc.x < it.W && cc.y < it.H;
        cc.owned_xy = cc.in_xy && lane >= 1 && warp >= 1;
        cc.cube_xy = cc.x >= 0 && cc.y >= 0 && cc.x < it.W - 1 && cc.y < it.H - 1 && lane <= 30 && warp <= 7;
        cc.bxy = (cc.y == 0 ? 4u : 0u) | (cc.y == it.H - 1 ? 8u : 0u) | (cc.x == 0 ? 16u : 0u) |
                 (cc.x == it.W - 1 ? 32u : 0u);
        const int z0 = zc * tab.zchunk3d;
        const int z1 = min(it.D, z0 + tab.zchunk3d);  // owned planes [z0, z1)
        const int zlast = min(z1, it.D - 1);       // entries computed for planes [z0, zlast]
        RingPos rp;
        ring_positions(it, x0, y0, rp);
        unsigned long long my_min = ~0ull;
        uint32_t far = 0;
        __syncthreads();  // the rings may still be read by the previous task
        ring_init(sm, rp);
#pragma unroll
        for (int k = -1; k < kAhead; ++k) issue_plane(sm, it, z0 + k, rp, cc.HW);
        cp_async_wait<kAhead - 2>();  // planes z0-1 .. z0+1 have landed
        __syncthreads();
        Nbr A, B, C;
        read_nbr(sm.ring[(z0 - 1 + kRing) & (kRing - 1)], warp, lane, A);
        read_nbr(sm.ring[z0 & (kRing - 1)], warp, lane, B);
        for (int z = z0; z <= zlast; ++z) {
            issue_plane(sm, it, z + kAhead, rp, cc.HW);
            read_nbr(sm.ring[(z + 1) & (kRing - 1)], warp, lane, C);
            // ---- lookup of (z, y, x)
            const float cv = B.v[1][1];
            const uint32_t raw = mask26(A, B, C);
            const uint2 e = lookup3(collapse3(raw));
            sm.codes[z % 3][warp][lane] = e.y;
            const bool owned = cc.owned_xy && z < z1;
            const uint32_t ord = ord_bits(cv);
            const uint32_t vl = (uint32_t(z) * cc.H + uint32_t(cc.y)) * cc.W + uint32_t(cc.x);
            const uint32_t vg = cc.voff + vl;
            const int direct = int(e.x & 7u);
            bool root0 = false;
            if (owned) {
                if (!(fabsf(cv) <= 3.40282347e38f)) set_status(o.ctr, kStNonfinite);
                if (direct == 7) {
                    root0 = true;
                    far = vg;
                    const unsigned long long k = (unsigned long long)(uint64_t(ord) << 32 | vl);
                    my_min = k < my_min ? k : my_min;
                } else {
                    // face slots: (-1,0,0) (0,-1,0) (0,0,-1) (0,0,1) (0,1,0) (1,0,0); a z-1 link
                    // continues the chain that the z-1 neighbour (same thread, previous
                    // step) started
                    const uint32_t mag = (direct == 0 || direct == 5) ? cc.HW : ((direct == 1 || direct == 4) ? cc.W : 1u);
                    const uint32_t u = direct < 3 ? vg - mag : vg + mag;
                    far = (direct == 0 && z > z0) ? far : u;
                    o.uf0[vg] = far;
                }
            }
            const uint32_t h0s = owned ? (e.x >> 3) & 0x3Fu : 0u;
            const uint32_t ds = owned ? (e.x >> 9) & 0xFFFu : 0u;
            cp_async_wait<kAhead - 2>();  // plane z+2 has landed (for the next step)
            __syncthreads();              // codes of plane z and image plane z+2 visible
            // ---- the top cell with smallest corner (z-1, y, x)
            bool rootT = false;
            uint32_t rt_node = 0;
            uint64_t rt_age = 0;
            if (cc.cube_xy && z > z0) {
                // largest of the 8 corners under (value, linear index), in index order
                const float cvals[8] = {A.v[1][1], A.v[1][2], A.v[2][1], A.v[2][2],
                                        B.v[1][1], B.v[1][2], B.v[2][1], B.v[2][2]};
                int k = 0;
                float best = cvals[0];
#pragma unroll
                for (int j = 1; j < 8; ++j) {
                    const bool ge = cvals[j] >= best;
                    best = ge ? cvals[j] : best;
                    k = ge ? j : k;
                }
                const int dz = k >> 2, dy = (k >> 1) & 1, dx = k & 1;
                const uint32_t word = sm.codes[(z - 1 + dz) % 3][warp + dy][lane + dx];
                const uint32_t t = uint32_t(7 - k);  // octant of the top cell as seen from m
                const uint32_t code = (word >> (4u * t)) & 15u;
                const uint32_t self = cc.toff + (uint32_t(z - 1) * (cc.H - 1u) + uint32_t(cc.y)) * cc.W1 + uint32_t(cc.x);
                const int mz = z - 1 + dz, my = cc.y + dy, mx = cc.x + dx;
                if (code == 8u) {
                    rootT = true;
                    rt_node = self;
                    const uint32_t mg = cc.voff + (uint32_t(mz) * cc.H + uint32_t(my)) * cc.W + uint32_t(mx);
                    rt_age = make_key(ord_bits(best), mg, age_slot(t));
                } else if (code < 8u) {
                    // the top cell across: octant `code` of m, smallest corner m - (negative axes)
                    const int tz = mz - int(((code >> 2) & 1u) ^ 1u);
                    const int ty = my - int(((code >> 1) & 1u) ^ 1u);
                    const int tx = mx - int((code & 1u) ^ 1u);
                    const bool out = unsigned(tz) >= cc.D - 1u || unsigned(ty) >= cc.H - 1u || unsigned(tx) >= cc.W1;
                    o.uft[self] = out ? cc.OUT : cc.toff + (uint32_t(tz) * (cc.H - 1u) + uint32_t(ty)) * cc.W1 + uint32_t(tx);
                } else {
                    o.uft[self] = kTag;  // only reachable with non-finite input (flagged): keep the forest well formed
                }
            }
            // ---- stage survivors and roots (rare in smooth fields)
            if (__any_sync(0xFFFFFFFFu, root0 || rootT || (h0s | ds) != 0u)) {
                const unsigned m_r0 = __ballot_sync(0xFFFFFFFFu, root0);
                const unsigned m_rt = __ballot_sync(0xFFFFFFFFu, rootT);
                const uint32_t or0 = __reduce_or_sync(0xFFFFFFFFu, h0s);
                const uint32_t ort = __reduce_or_sync(0xFFFFFFFFu, ds);
                const uint32_t n0 = __reduce_add_sync(0xFFFFFFFFu, uint32_t(__popc(h0s)));  // <= 32 * 5
                const uint32_t nt = __reduce_add_sync(0xFFFFFFFFu, uint32_t(__popc(ds)));   // <= 32 * 7
                if (cnt.s0 + n0 > uint32_t(kCapW0) || cnt.st + nt > uint32_t(kCapWT) ||
                    cnt.r0 + __popc(m_r0) > uint32_t(kCapWR) || cnt.rt + __popc(m_rt) > uint32_t(kCapWR))
                    warp_flush(ws, cnt, o);
                if (m_r0) {
                    if (root0) {
                        const uint32_t p = cnt.r0 + __popc(m_r0 & lt);
                        ws.r0node[p] = vg;
                        ws.r0age[p] = make_key(ord, vg, 0);
                    }
                    cnt.r0 += __popc(m_r0);
                }
                if (m_rt) {
                    if (rootT) {
                        const uint32_t p = cnt.rt + __popc(m_rt & lt);
                        ws.rtnode[p] = rt_node;
                        ws.rtage[p] = rt_age;
                    }
                    cnt.rt += __popc(m_rt);
                }
                uint32_t bits = or0;
                while (bits) {
                    const int s = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const bool mine = (h0s >> s) & 1u;
                    const unsigned m = __ballot_sync(0xFFFFFFFFu, mine);
                    if (mine) {
                        const uint32_t n = s == 0 ? 4u : (s == 1 ? 10u : (s == 2 ? 12u : (s == 3 ? 14u : (s == 4 ? 16u : 22u))));
                        ws.s0[cnt.s0 + __popc(m & lt)] = make_key(ord, vg, n);
                    }
                    cnt.s0 += __popc(m);
                }
                bits = ort;
                while (bits) {
                    const int f = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const bool mine = (ds >> f) & 1u;
                    const unsigned m = __ballot_sync(0xFFFFFFFFu, mine);
                    if (mine) {
                        // facet slots 0..11 -> stencil bits 1,3,5,7,9,11,15,17,19,21,23,25
                        const uint32_t n = f < 6 ? uint32_t(2 * f + 1) : uint32_t(2 * f + 3);
                        ws.st[cnt.st + __popc(m & lt)] = ~make_key(ord, vg, n);
                    }
                    cnt.st += __popc(m);
                }
                __syncwarp();
            }
            A = B;
            B = C;
        }
        cp_async_wait<0>();
        const unsigned long long w = warp_min_u64(my_min);
        if (lane == 0 && w != ~0ull) atomicMin(&o.ctr->gmin[ii], w);
    }
    if (__any_sync(0xFFFFFFFFu, (cnt.s0 | cnt.st | cnt.r0 | cnt.rt) != 0)) warp_flush(ws, cnt, o);
}

// ---------------------------------------------------------------- host side
size_t prune_smem2d() { return sizeof(Stage) + sizeof(float) * (kT2Y + 2) * (kBX + 2); }
size_t prune_smem3d() { return sizeof(Smem3); }
int prune_tile_x() { return kBX; }
int prune_tile_x3d() { return kOX; }
int g_rows2d = kT2Y, g_zchunk3d = kZC, g_ctas3d = 0;  // tuning (cp_set_tuning)
int prune_tile_y2d() { return g_rows2d; }
int prune_tile_y3d() { return kOY; }
int prune_tile_z3d() { return g_zchunk3d; }

int set_tuning(int key, int value) {
    switch (key) {
        case 1:  // planes per 3D pruning task
            if (value < 4 || value > 4096) return -1;
            g_zchunk3d = value;
            return 0;
        case 2:  // 3D pruning CTAs per SM (0: as many as fit)
            if (value < 0 || value > 8) return -1;
            g_ctas3d = value;
            return 0;
        case 3:  // rows per 2D pruning tile
            if (value != 8 && value != 16 && value != 24 && value != 32) return -1;
            g_rows2d = value;
            return 0;
        default:
            return -1;
    }
}

int get_tuning(int key) {
    return key == 1 ? g_zchunk3d : key == 2 ? g_ctas3d : key == 3 ? g_rows2d : -1;
}

cudaError_t upload_luts(const uint64_t* lut2d, const uint16_t* disp3d, const uint64_t* entries3d) {
    cudaError_t e = cudaMemcpyToSymbol(g_lut2d, lut2d, sizeof(uint64_t) * 256);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyToSymbol(g_disp3d, disp3d, sizeof(uint16_t) * (1 << 12));
    if (e != cudaSuccess) return e;
    static uint2 packed[1 << 14];
    for (int i = 0; i < (1 << 14); ++i) {
        const uint64_t v = entries3d[i];
        const uint32_t direct = uint32_t(v & 7u), h0s = uint32_t((v >> 3) & 0x3Fu);
        const uint32_t ds = uint32_t((v >> 41) & 0xFFFu), in_l = uint32_t((v >> 53) & 0xFFu);
        packed[i].x = direct | (h0s << 3) | (ds << 9) | (in_l << 21);
        packed[i].y = uint32_t((v >> 9) & 0xFFFFFFFFu);
    }
    return cudaMemcpyToSymbol(g_entries3d, packed, sizeof(packed));
}

cudaError_t launch_prune(const ItemTable& tab, const PruneOuts& po, cudaStream_t s) {
    Outs o;
    o.uf0 = po.uf0;
    o.uft = po.uft;
    o.s0 = po.s0;
    o.st = po.st;
    o.age0 = po.age0;
    o.res0 = po.res0;
    o.aget = po.aget;
    o.rest = po.rest;
    o.cap_s = po.cap_s;
    o.cap_r0 = po.cap_r0;
    o.cap_rt = po.cap_rt;
    o.ctr = po.ctr;
    static bool attr_set = false;
    static int blocks3d = 0;
    if (!attr_set) {
        cudaFuncSetAttribute(k_prune2d, cudaFuncAttributeMaxDynamicSharedMemorySize, int(prune_smem2d()));
        cudaFuncSetAttribute(k_prune3d, cudaFuncAttributeMaxDynamicSharedMemorySize, int(prune_smem3d()));
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_prune3d, kT3, prune_smem3d());
        blocks3d = device_sm_count() * (per_sm > 0 ? per_sm : 1);
        attr_set = true;
    }
    if (tab.tiles2d > 0) {
        k_prune2d<<<tab.tiles2d, dim3(kBX, kBY), prune_smem2d(), s>>>(tab, o);
        note_launches(1);
    }
    if (tab.tiles3d > 0) {
        int cap = blocks3d;
        if (g_ctas3d > 0) cap = device_sm_count() * g_ctas3d < blocks3d ? device_sm_count() * g_ctas3d : blocks3d;
        int grid = tab.tiles3d < cap ? tab.tiles3d : cap;
        k_prune3d<<<grid, kT3, prune_smem3d(), s>>>(tab, o);
        note_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace cp
