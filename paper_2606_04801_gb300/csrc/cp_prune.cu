// K1: fused lookup + local pruning (Sec. 3.2, Sec. 3.3, Sec. 4.1 steps 1-2,
// Sec. 4.2 steps 1-3 before the union-finds).
//
// Warps march through the image row by row (2D) or plane by plane (3D) with
// the neighbourhood of the current vertex in registers and the rows / planes
// ahead prefetched into shared memory with cp.async (out-of-image positions
// read +inf, so such neighbours never precede the centre).  Per vertex v:
//   1. 8/26-bit mask of the neighbours that precede v (value, then index);
//   2. collapse to the relevant mask and look it up (2D: direct 256-entry
//      table; 3D: perfect hash of the 15,935 relevant masks);
//   3. write the H0 forest parent of v (first edge of L(v), chained through
//      the previous step's vertex when that edge points back along the
//      marching axis) or register v as an H0 root (local minimum);
//   4. for the top cell whose smallest corner is one step behind v, find its
//      largest corner m (the vertex whose lower star holds it) and write its
//      dual forest parent from m's entry: the top cell across the facet where
//      it dies locally, the outside vertex, or register it as a dual root;
//   5. emit the surviving edges and facets as 64-bit order keys.
// Survivors and roots are staged per warp with ballots and appended to the
// global arrays with one atomic per buffer per flush.
#include "cp_common.cuh"
#include "cp_kernels.h"
#include "cp_mask3.cuh"

#include <type_traits>

namespace cp {

// Lookup tables in global memory, read through the read-only cache (lanes of
// a warp look up different entries, which constant memory would serialise).
__device__ uint2 g_lut2d[256];  // same two-word entry layout as the 3D table
__device__ uint16_t g_disp3d[1 << 12];
// The 3D table in three parts, each indexed by the perfect-hash slot of the
// relevant mask (the H0 direct link is not stored: it is the lowest face bit
// of the relevant mask):
//   g_codes3d: eight 4-bit fields, field t for top-cell slot t of L(v):
//              0 = not in L(v); 1 + c = linked locally to top-cell slot c of
//              v (it dies at zero persistence); 9 = survives locally
//   g_sbits3d: one bit per slot: the class has H0 or dual survivors
//   g_surv3d:  h0_surv | dual_surv << 6, read for survivor vertices only
// The hot part (codes, 64 KB) stays in L1 far better than full entries would.
__device__ uint32_t g_codes3d[1 << 14];
__device__ uint32_t g_sbits3d[1 << 9];
__device__ uint32_t g_surv3d[1 << 14];

namespace {

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
    uint32_t n_uf0, n_uft;  // forest sizes (bounds-checked build)
};

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(0xFFFFFFFFu, v, o);
        v = t < v ? t : v;
    }
    return v;
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

// Perfect hash of the 15,935 relevant masks (device layout, cp_mask3.cuh):
// bucket -> displacement (a copy of the 8 KB displacement table in shared
// memory) -> slot.
__device__ __forceinline__ uint32_t hash_slot3(uint32_t rel, const uint16_t* disp) {
    const uint32_t b = (rel * 0x9E3779B1u) >> (32 - 12);
    const uint32_t d = disp[b];
    return ((rel ^ (d * 0x27D4EB2Fu)) * 0x85EBCA77u) >> (32 - 14);
}

}  // namespace

// ---------------------------------------------------------------- 3D
// A CTA of 9 warps marches through a chunk of planes.  Warp w handles row
// y0-1+w and lane l column x0-1+l: the CTA owns the 31 x 8 vertices with
// w >= 1 and l >= 1; row y0-1 and column x0-1 are a halo whose lookups are
// needed, but whose outputs belong to the neighbouring CTA.
//
// Per plane step z:
//  1. one thread issues the TMA copy of image plane z+kAhead (a 40 x 11 box:
//     the CTA's vertices and a one-vertex border) into an 8-slot shared ring
//     (items without a tensor map: every thread's cp.async copies);
//  2. the 26-neighbour mask of (z, y, x) from registers (planes z-1, z) and
//     the ring (plane z+1), built in the lattice layout of cp_mask3.cuh and
//     collapsed there, the perfect-hash lookup, the H0 forest link and the
//     survivor bits of owned vertices; the entry's code fields for the top
//     cells above and below the vertex go to a 3-slot column-word ring;
//  3. one barrier;
//  4. the top cell whose smallest corner is (z-1, y, x): of its 8 corners
//     exactly the largest holds it, so the OR of the 4 columns' words has
//     one field set, which gives the top cell across the facet where it
//     dies locally (or marks it a dual root); one coalesced store of its
//     dual forest link.
// The first three and the last few steps of a task take every boundary
// check; the interior steps are a second instantiation of the step without
// them.
// Survivors and roots are staged per warp with ballots and flushed with one
// atomic per buffer when a buffer would overflow and at the end.
constexpr int kW3 = 9;                     // warps per CTA
constexpr int kT3 = kW3 * 32;
constexpr int kOX = 31, kOY = 8;           // owned columns / rows per CTA
constexpr int kZC = 64;                    // default owned planes per task
constexpr int kRW = 34, kRH = kW3 + 2, kRP = kRW * kRH;  // plane tile: cols x0-2 .. x0+31, rows y0-2 ..
constexpr int kRS = 40;                    // ring row stride in floats (a TMA box row: x from a multiple of 4)
constexpr int kSlot = 448;                 // ring slot in floats: kRH rows of kRS, padded to 128 bytes
constexpr int kRing = 8, kAhead = 5;       // ring slots, planes in flight
// staging per warp: flushed before a 32-lane slot would overflow it (small,
// so that shared memory leaves L1 room for the lookup table)
constexpr int kCapW0 = 64;                 // staged H0 keys per warp
constexpr int kCapWT = 64;                 // staged dual keys per warp
constexpr int kCapWR = 32;                 // staged roots per warp and kind

struct WarpStage {
    uint64_t s0[kCapW0];
    uint64_t st[kCapWT];
    uint64_t r0age[kCapWR];
    uint64_t rtage[kCapWR];
    uint32_t r0node[kCapWR];
    uint32_t rtnode[kCapWR];
};

// Dual link of a top cell, by (slot t of the top cell in its largest corner's
// lower star, that corner's 4-bit code field v): x = offset of the linked top
// cell in the item's top-cell index space; y = the moves (bit 0 -z, 1 -y,
// 2 -x, 3 +x, 4 +y, 5 +z) and flags
constexpr uint32_t kMvChain = 1u << 6;    // the only move is -z (the chain of this thread's column)
constexpr uint32_t kMvRoot = 1u << 7;     // survives locally: a dual root
constexpr uint32_t kMvInvalid = 1u << 8;  // no corner holds the top cell (non-finite input only)

struct Smem3 {
    float ring[kRing][kSlot];  // first: slots 128-byte aligned (TMA destinations)
    uint64_t bar[kRing];       // mbarrier of each slot (TMA completion)
    const CUtensorMap* tma_map;  // the current task's plane source (read by the issuing thread only)
    int tma_xs, tma_ys;
    // the current task's constants, read where used (fewer live registers)
    uint32_t t_HW, t_HW1, t_OUT;
    int t_z0, t_z1;
    int2 tlink[8 * 16];        // dual links by (t, v), for the current item
    int32_t h0link[64];        // H0 link offset by the face bits of the mask (their lowest: z-, y-, x-, x+, y+, z+), for the current item
    uint16_t disp[1 << 12];    // displacement table of the 3D perfect hash
    uint32_t sbits[1 << 9];    // survivor bit of each slot
    // per column and plane step: the code fields of the top cells on the +z
    // side of the column's vertex at z-1 and on the -z side of its vertex at z
    uint32_t q[3][kW3 + 1][32];
    unsigned long long tmin[kT3];  // each thread's smallest H0 root key in the current task (rarely touched)
    WarpStage ws[kW3];
};

struct WarpCounts {
    uint32_t s0, st, r0, rt;
};

template <class WS>
__device__ __forceinline__ void warp_flush(WS& ws, WarpCounts& c, const Outs& o) {
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
            if (CP_IN(ws.r0node[i], o.n_uf0, o.ctr)) o.uf0[ws.r0node[i]] = kTag | g;
        } else if (CP_IN(ws.r0node[i], o.n_uf0, o.ctr)) {
            o.uf0[ws.r0node[i]] = kTag;  // out of capacity: keep the forest well formed (result flagged invalid)
        }
    }
    for (uint32_t i = lane; i < c.rt; i += 32) {
        uint32_t g = brt + i;
        if (g < o.cap_rt) {
            o.aget[g] = ws.rtage[i];
            o.rest[g] = 0;
            if (CP_IN(ws.rtnode[i], o.n_uft, o.ctr)) o.uft[ws.rtnode[i]] = kTag | g;
        } else if (CP_IN(ws.rtnode[i], o.n_uft, o.ctr)) {
            o.uft[ws.rtnode[i]] = kTag;
        }
    }
    c.s0 = c.st = c.r0 = c.rt = 0;
    __syncwarp();
}

// raw |= kBit when the neighbour value u precedes the centre value c (kLe:
// the neighbour comes earlier in linear order, so it also precedes on a tie;
// NaN, the out-of-image fill, never precedes): a compare into a predicate and
// a predicated OR, two instructions per bit
template <uint32_t kBit, bool kLe>
__device__ __forceinline__ void or_if_precedes(uint32_t& raw, float u, float c) {
    if constexpr (kLe)
        asm("{\n\t.reg .pred p;\n\tsetp.le.f32 p, %1, %2;\n\t@p or.b32 %0, %0, %3;\n\t}"
            : "+r"(raw) : "f"(u), "f"(c), "n"(kBit));
    else
        asm("{\n\t.reg .pred p;\n\tsetp.lt.f32 p, %1, %2;\n\t@p or.b32 %0, %0, %3;\n\t}"
            : "+r"(raw) : "f"(u), "f"(c), "n"(kBit));
}

struct Nbr {
    float v[3][3];  // [row y-1, y, y+1][col x-1, x, x+1] of one plane
};

__device__ __forceinline__ void read_nbr(const float* plane, int ly, int lx, Nbr& P) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) P.v[r][c] = plane[(ly + r) * kRS + (lx + c)];
}

template <int n>
__device__ __forceinline__ void mask_bit(uint32_t& raw, const Nbr& A, const Nbr& B, const Nbr& C, float cv) {
    constexpr int a = n / 9, b = (n / 3) % 3, c = n % 3;
    const Nbr& P = a == 0 ? A : (a == 1 ? B : C);
    or_if_precedes<(1u << mask3_pos(n)), (n < 13)>(raw, P.v[b][c], cv);
}

// raw mask in the device layout (cp_mask3.cuh): the bit of canonical
// neighbour n = 9a + 3b + c set when the neighbour at plane a, row b, column
// c precedes the centre (ties: earlier linear index first)
__device__ __forceinline__ uint32_t mask26(const Nbr& A, const Nbr& B, const Nbr& C) {
    const float cv = B.v[1][1];
    uint32_t raw = 0;
    mask_bit<0>(raw, A, B, C, cv);
    mask_bit<1>(raw, A, B, C, cv);
    mask_bit<2>(raw, A, B, C, cv);
    mask_bit<3>(raw, A, B, C, cv);
    mask_bit<4>(raw, A, B, C, cv);
    mask_bit<5>(raw, A, B, C, cv);
    mask_bit<6>(raw, A, B, C, cv);
    mask_bit<7>(raw, A, B, C, cv);
    mask_bit<8>(raw, A, B, C, cv);
    mask_bit<9>(raw, A, B, C, cv);
    mask_bit<10>(raw, A, B, C, cv);
    mask_bit<11>(raw, A, B, C, cv);
    mask_bit<12>(raw, A, B, C, cv);
    mask_bit<14>(raw, A, B, C, cv);
    mask_bit<15>(raw, A, B, C, cv);
    mask_bit<16>(raw, A, B, C, cv);
    mask_bit<17>(raw, A, B, C, cv);
    mask_bit<18>(raw, A, B, C, cv);
    mask_bit<19>(raw, A, B, C, cv);
    mask_bit<20>(raw, A, B, C, cv);
    mask_bit<21>(raw, A, B, C, cv);
    mask_bit<22>(raw, A, B, C, cv);
    mask_bit<23>(raw, A, B, C, cv);
    mask_bit<24>(raw, A, B, C, cv);
    mask_bit<25>(raw, A, B, C, cv);
    mask_bit<26>(raw, A, B, C, cv);
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

// ---- image plane ring, filled by TMA (one tensor copy per plane, completing
// on the slot's mbarrier; out-of-image positions read NaN, which never
// precedes anything, like +inf) or, for items without a tensor map, by
// cp.async (out-of-image positions set to +inf once per task)
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for a slot's copy; a copy that never lands flags the call.
__device__ __forceinline__ void mbar_wait(uint64_t* bar, uint32_t parity, Counters* ctr) {
    if (mbar_try_wait(bar, parity)) return;
    const uint64_t t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_timer_ns() - t0 > kWaitLimitNs) {
            set_status(ctr, kStTimeout);
            return;
        }
    }
}
__device__ __forceinline__ void tma_load_plane(float* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Plane tile positions of this thread for the cp.async path (at most two),
// fixed for a task.
struct RingPos {
    uint32_t off0, off1;  // offset of the pixel in a plane
    uint32_t dst0, dst1;  // position in a ring slot
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
        const uint32_t dst = uint32_t(ly * kRS + lx);
        if (k == 0) {
            rp.off0 = off;
            rp.dst0 = dst;
            rp.in0 = in;
        } else {
            rp.off1 = off;
            rp.dst1 = dst;
            rp.in1 = in;
            rp.has1 = i < kRP;
        }
    }
}

__device__ __forceinline__ void ring_init(Smem3& sm, const RingPos& rp) {
    const float inf = __int_as_float(0x7F800000);
#pragma unroll
    for (int s = 0; s < kRing; ++s) {
        if (!rp.in0) sm.ring[s][rp.dst0] = inf;
        if (rp.has1 && !rp.in1) sm.ring[s][rp.dst1] = inf;
    }
}

// Where a task's planes come from.
struct PlaneSrc {
    const CUtensorMap* map;  // nullptr: cp.async path
    int xs, ys;              // TMA box origin: x rounded down to a multiple of 4, y0 - 2
    int zneed;               // last plane the task reads (TMA path loads no plane beyond it)
};

// kCheck false: the caller knows that plane z lies inside the volume and
// within the task's reads (an interior plane step)
template <bool kTma, bool kCheck>
__device__ __forceinline__ void issue_plane(Smem3& sm, const Item& it, int z, const RingPos& rp, uint32_t HW,
                                            const PlaneSrc& ps) {
    const int slot = (z + kRing) & (kRing - 1);
    float* plane = sm.ring[slot];
    const float inf = __int_as_float(0x7F800000);
    if constexpr (kTma) {
        if (kCheck && z > ps.zneed) return;
        if (!kCheck || unsigned(z) < unsigned(it.D)) {
            if (threadIdx.x == 0) {
                // earlier generic-proxy accesses of the slot come before the copy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(&sm.bar[slot], uint32_t(kRH * kRS * sizeof(float)));
                tma_load_plane(plane, sm.tma_map, &sm.bar[slot], sm.tma_xs, sm.tma_ys, z);
            }
        } else {  // a plane outside the volume: every position +inf
            for (int i = threadIdx.x; i < kRH * kRS; i += kT3) plane[i] = inf;
        }
        return;
    }
    if (!kCheck || unsigned(z) < unsigned(it.D)) {
        const float* base = it.img + uint32_t(z) * HW;
        if (rp.in0) cp_async4(plane + rp.dst0, base + rp.off0);
        if (rp.in1) cp_async4(plane + rp.dst1, base + rp.off1);
    } else {  // a plane outside the volume: every position +inf
        if (rp.in0) plane[rp.dst0] = inf;
        if (rp.in1) plane[rp.dst1] = inf;
    }
    cp_async_commit();
}

// Before reading plane z: wait for its TMA copy (cp.async planes are covered
// by the wait_group and the barrier of the previous step).
template <bool kTma, bool kCheck>
__device__ __forceinline__ void wait_plane(Smem3& sm, const Item& it, int z, uint32_t& par, Counters* ctr) {
    if (!kTma || (kCheck && unsigned(z) >= unsigned(it.D))) return;
    const int slot = z & (kRing - 1);
    mbar_wait(&sm.bar[slot], (par >> slot) & 1u, ctr);
    par ^= 1u << slot;
}

struct Col {
    int x, y;
    uint32_t W, H, D, HW, W1, HW1, voff, toff, OUT;
    bool in_xy;      // (x, y) inside the image
    bool owned_xy;   // and owned by this CTA
    bool cube_xy;    // (x, y) is the smallest corner of a top cell written by this thread
    uint32_t bmv;    // moves that leave the image from this column's top cell (-y, -x, +x, +y)
};

__device__ __forceinline__ uint32_t age_slot(uint32_t t) {
    return 18u * ((t >> 2) & 1u) + 6u * ((t >> 1) & 1u) + 2u * (t & 1u);
}

// One task of the 3D pruning pass: a 31 x 8 column block of one item over a
// chunk of planes (kTma: planes by TMA, else by cp.async; the two paths are
// separate instantiations so that each keeps only its own state live).
template <bool kTma>
__device__ __forceinline__ void prune_task3d(Smem3& sm, const ItemTable& tab, const Outs& o, int ii, int ltask,
                                             int warp, int lane, unsigned lt, WarpStage& ws, WarpCounts& cnt,
                                             const CUtensorMap* map, uint32_t& par) {
    const Item& it = tab.it[ii];
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
    cc.cube_xy = cc.x >= 0 && cc.y >= 0 && cc.x < it.W - 1 && cc.y < it.H - 1 && lane <= 30 && warp <= kW3 - 2;
    cc.bmv = (cc.y == 0 ? 2u : 0u) | (cc.x == 0 ? 4u : 0u) | (cc.x == it.W - 2 ? 8u : 0u) | (cc.y == it.H - 2 ? 16u : 0u);
    const int z0 = zc * tab.zchunk3d;
    const int z1 = min(it.D, z0 + tab.zchunk3d);  // owned planes [z0, z1)
    const int zlast = min(z1, it.D - 1);       // entries computed for planes [z0, zlast]
    RingPos rp;
    PlaneSrc src;
    src.map = map;
    src.xs = (x0 - 2) & ~3;
    src.ys = y0 - 2;
    src.zneed = zlast + 1;
    if constexpr (!kTma) ring_positions(it, x0, y0, rp);
    const int xo = kTma ? (x0 - 2) - src.xs : 0;  // column x0-2 within a slot row
    if (kTma && threadIdx.x == 0) {
        sm.tma_map = map;
        sm.tma_xs = src.xs;
        sm.tma_ys = src.ys;
    }
    if (kTma && threadIdx.x == 0) atomicAdd(&o.ctr->tma_tasks, 1u);
    // global vertex index and top-cell index of this column in plane 0
    const uint32_t colv = cc.voff + uint32_t(cc.y) * cc.W + uint32_t(cc.x);
    const uint32_t colt = cc.toff + uint32_t(cc.y) * cc.W1 + uint32_t(cc.x);
    uint32_t far = 0, far_t = 0;  // last H0 link / dual link written by this thread
    uint32_t cprev = 0;           // code fields of this column's vertex one plane behind
    bool nonfinite = false;       // an owned value is NaN or infinite (checked once per task)
    __syncthreads();  // the rings, link tables and task constants may still be read by the previous task
    if (threadIdx.x == 0) {
        sm.t_HW = cc.HW;
        sm.t_HW1 = cc.HW1;
        sm.t_OUT = cc.OUT;
        sm.t_z0 = z0;
        sm.t_z1 = z1;
    }
    __syncthreads();  // the task constants are read from here on
    sm.tmin[threadIdx.x] = ~0ull;
    if constexpr (!kTma) ring_init(sm, rp);
    if (threadIdx.x < 8 * 16) {
        // top cell in slot t of its largest corner m, linked to slot c of m: the
        // smallest corners differ by (bit of c) - (bit of t) along each axis
        const int t = threadIdx.x >> 4, v = threadIdx.x & 15;
        int2 d;
        d.x = 0;
        if (v >= 1 && v <= 8) {
            const int c = v - 1;
            const int dz = ((c >> 2) & 1) - ((t >> 2) & 1), dy = ((c >> 1) & 1) - ((t >> 1) & 1), dx = (c & 1) - (t & 1);
            d.x = dz * int((cc.H - 1u) * cc.W1) + dy * int(cc.W1) + dx;
            uint32_t mv = (dz < 0 ? 1u : 0u) | (dy < 0 ? 2u : 0u) | (dx < 0 ? 4u : 0u) | (dx > 0 ? 8u : 0u) |
                          (dy > 0 ? 16u : 0u) | (dz > 0 ? 32u : 0u);
            d.y = int(mv == 1u ? mv | kMvChain : mv);
        } else {
            d.y = int(v == 9 ? kMvRoot : kMvInvalid);
        }
        sm.tlink[threadIdx.x] = d;
    } else if (threadIdx.x < 8 * 16 + 64) {
        const int f = threadIdx.x - 8 * 16, s = __ffs(f) - 1;  // f == 0 (a root): unused
        const int hw = int(cc.HW), w = int(cc.W);
        sm.h0link[f] = s == 0 ? -hw : (s == 1 ? -w : (s == 2 ? -1 : (s == 3 ? 1 : (s == 4 ? w : (s == 5 ? hw : 0)))));
    }
#pragma unroll
    for (int k = -1; k < kAhead; ++k) issue_plane<kTma, true>(sm, it, z0 + k, rp, cc.HW, src);
    cp_async_wait<kAhead - 2>();  // planes z0-1 .. z0+1 have landed
    __syncthreads();
    Nbr A, B, C;
    wait_plane<kTma, true>(sm, it, z0 - 1, par, o.ctr);
    read_nbr(sm.ring[(z0 - 1 + kRing) & (kRing - 1)] + xo, warp, lane, A);
    wait_plane<kTma, true>(sm, it, z0, par, o.ctr);
    read_nbr(sm.ring[z0 & (kRing - 1)] + xo, warp, lane, B);
    // One plane step: A (plane z-1) and B (plane z) in registers, C receives
    // plane z+1.
    // interior: a std::integral_constant; true for a step with z >= z0 + 2 and
    // z + kAhead <= zlast, where no boundary plane or end-of-task case arises
    auto step = [&](const Nbr& A, const Nbr& B, Nbr& C, const int z, const int qs, auto interior) {
        constexpr bool kIn = decltype(interior)::value;
        issue_plane<kTma, !kIn>(sm, it, z + kAhead, rp, cc.HW, src);
        wait_plane<kTma, !kIn>(sm, it, z + 1, par, o.ctr);
        read_nbr(sm.ring[(z + 1) & (kRing - 1)] + xo, warp, lane, C);
        // ---- lookup of (z, y, x)
        const float cv = B.v[1][1];
        const uint32_t rel = collapse3_lattice(mask26(A, B, C));
        const uint32_t slot = hash_slot3(rel, sm.disp);
        const uint32_t codes = __ldg(g_codes3d + slot);
        // top cells on the +z side of (z-1, y, x) are slots 4..7 of that vertex,
        // those on the -z side of (z, y, x) slots 0..3 of this one
        const uint32_t q = (cprev & 0xFFFF0000u) | (codes & 0x0000FFFFu);
        sm.q[qs][warp][lane] = q;
        cprev = codes;
        const bool owned = cc.owned_xy && (kIn || z < sm.t_z1);
        const uint32_t ord = ord_bits(cv);
        const uint32_t vg = colv + uint32_t(z) * sm.t_HW;
        const uint32_t f0 = rel & kM3Faces;  // the first edge of L(v) is its lowest face bit
        // H0: a local minimum becomes a root (registered in the staging block
        // below); otherwise the link along the first edge, where a link to
        // (z-1, y, x) (face bit 0, the lowest) continues the chain that the
        // z-1 neighbour (same thread, previous step) started
        const bool root0 = owned && f0 == 0u;
        nonfinite |= owned && !(fabsf(cv) <= 3.40282347e38f);
        const uint32_t u = vg + uint32_t(sm.h0link[f0]);  // (f0 == 0: unused)
        if (owned) far = root0 ? vg : (((f0 & 1u) && (kIn || z > sm.t_z0)) ? far : u);
        if (owned && !root0 && CP_IN(vg, o.n_uf0, o.ctr)) o.uf0[vg] = far;
        // survivor fields (owned survivor vertices only; rare)
        const bool sbit = owned && ((sm.sbits[slot >> 5] >> (slot & 31u)) & 1u);
        const uint32_t sv = sbit ? __ldg(g_surv3d + slot) : 0u;
        // ---- the top cell with smallest corner (z-1, y, x): exactly one of its
        // 8 corners (the largest) holds it in its lower star; OR the corners'
        // fields for it (slot 7-k of corner k = 4dz + 2dy + dx), this row's two
        // columns now, the next row's after the barrier
        constexpr uint32_t kM73 = 0xF000F000u, kM62 = 0x0F000F00u, kM51 = 0x00F000F0u, kM40 = 0x000F000Fu;
        const uint32_t acc_row = (q & kM73) | (__shfl_down_sync(0xFFFFFFFFu, q, 1) & kM62);
        cp_async_wait<kAhead - 2>();  // plane z+2 has landed (for the next step)
        __syncthreads();              // column words of plane step z and image plane z+2 visible
        const uint32_t q10 = sm.q[qs][warp + 1][lane];
        const uint32_t q11 = __shfl_down_sync(0xFFFFFFFFu, q10, 1);
        // the field that is set is the one of the largest corner m; with
        // non-finite input none may be, and any field then reads "invalid"
        const bool cube = cc.cube_xy && (kIn || z > z0);
        const uint32_t acc = acc_row | (q10 & kM51) | (q11 & kM40);
        const uint32_t fs = uint32_t(31 - __clz(acc)) & 28u;  // 4 t: the field that is set
        const int2 lk = sm.tlink[(fs << 2) | ((acc >> fs) & 15u)];
        const uint32_t bits = uint32_t(lk.y);
        const uint32_t self = colt + uint32_t(z - 1) * sm.t_HW1;
        const bool rootT = cube && (bits & kMvRoot);  // registered in the staging block below
        {
            const uint32_t bnd = kIn ? cc.bmv : (cc.bmv | (z == 1 ? 1u : 0u) | (uint32_t(z) == cc.D - 1u ? 32u : 0u));
            // a link to (z-2, y, x) continues the chain that this thread wrote for
            // that top cell in the previous step; an invalid entry (non-finite
            // input only, flagged) writes a root tag to keep the forest well formed
            const bool chain = (bits & kMvChain) && (kIn || z - 1 > sm.t_z0);
            const uint32_t tgt = (bits & kMvInvalid) ? kTag : ((bits & bnd) ? sm.t_OUT : self + uint32_t(lk.x));
            if (cube) far_t = rootT ? self : (chain ? far_t : tgt);
            if (cube && !rootT && CP_IN(self, o.n_uft, o.ctr)) o.uft[self] = far_t;
        }
        // ---- stage survivors and roots (rare in smooth fields)
        if (__any_sync(0xFFFFFFFFu, root0 || rootT || sv != 0u)) {
            const uint32_t h0s = sv & 0x3Fu, ds = sv >> 6;
            const unsigned m_r0 = __ballot_sync(0xFFFFFFFFu, root0);
            const unsigned m_rt = __ballot_sync(0xFFFFFFFFu, rootT);
            const uint32_t or0 = __reduce_or_sync(0xFFFFFFFFu, h0s);
            const uint32_t ort = __reduce_or_sync(0xFFFFFFFFu, ds);
            if (cnt.r0 + __popc(m_r0) > uint32_t(kCapWR) || cnt.rt + __popc(m_rt) > uint32_t(kCapWR))
                warp_flush(ws, cnt, o);
            if (m_r0) {
                if (root0) {
                    const uint32_t p = cnt.r0 + __popc(m_r0 & lt);
                    ws.r0node[p] = vg;
                    ws.r0age[p] = make_key(ord, vg, 0);
                    const unsigned long long k = (unsigned long long)(uint64_t(ord) << 32 | (vg - uint32_t(it.voff)));
                    if (k < sm.tmin[threadIdx.x]) sm.tmin[threadIdx.x] = k;
                }
                cnt.r0 += __popc(m_r0);
            }
            if (m_rt) {
                if (rootT) {
                    // the age of a dual root: the key of the top cell, whose
                    // largest corner m is corner k = 7 - t of the cube
                    const uint32_t t = fs >> 2, k = 7u - t;
                    const uint32_t dz = k >> 2, dy = (k >> 1) & 1u, dx = k & 1u;
                    const Nbr& P = dz ? B : A;
                    const float mv = dy ? (dx ? P.v[2][2] : P.v[2][1]) : (dx ? P.v[1][2] : P.v[1][1]);
                    const uint32_t mg = colv + (uint32_t(z - 1) + dz) * cc.HW + dy * uint32_t(it.W) + dx;
                    const uint32_t p = cnt.rt + __popc(m_rt & lt);
                    ws.rtnode[p] = self;
                    ws.rtage[p] = make_key(ord_bits(mv), mg, age_slot(t));
                }
                cnt.rt += __popc(m_rt);
            }
            uint32_t bits = or0;
            while (bits) {
                const int s = __ffs(bits) - 1;
                bits &= bits - 1;
                const bool mine = (h0s >> s) & 1u;
                const unsigned m = __ballot_sync(0xFFFFFFFFu, mine);
                if (cnt.s0 + __popc(m) > uint32_t(kCapW0)) warp_flush(ws, cnt, o);
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
                if (cnt.st + __popc(m) > uint32_t(kCapWT)) warp_flush(ws, cnt, o);
                if (mine) {
                    // facet slots 0..11 -> stencil bits 1,3,5,7,9,11,15,17,19,21,23,25
                    const uint32_t n = f < 6 ? uint32_t(2 * f + 1) : uint32_t(2 * f + 3);
                    ws.st[cnt.st + __popc(m & lt)] = ~make_key(ord, vg, n);
                }
                cnt.st += __popc(m);
            }
            __syncwarp();
        }
    };
    // The first three planes and the last few take every check, one at a time
    // with the register planes copied along; the interior planes go three at
    // a time with the planes and column-word slots rotated, nothing copied.
    const std::integral_constant<bool, false> kEdge;
    const std::integral_constant<bool, true> kInner;
    int z = z0, qs = 0;
    for (; z <= zlast && z < z0 + 3; ++z) {
        step(A, B, C, z, qs, kEdge);
        A = B;
        B = C;
        qs = qs == 2 ? 0 : qs + 1;
    }
    for (; z + 2 + kAhead <= zlast; z += 3) {
        step(A, B, C, z, 0, kInner);
        step(B, C, A, z + 1, 1, kInner);
        step(C, A, B, z + 2, 2, kInner);
    }
    for (; z <= zlast; ++z) {
        step(A, B, C, z, qs, kEdge);
        A = B;
        B = C;
        qs = qs == 2 ? 0 : qs + 1;
    }
    cp_async_wait<0>();
    if (__any_sync(0xFFFFFFFFu, nonfinite) && lane == 0) set_status(o.ctr, kStNonfinite);
    const unsigned long long w = warp_min_u64(sm.tmin[threadIdx.x]);
    if (lane == 0 && w != ~0ull) atomicMin(&o.ctr->gmin[ii], w);
}

__global__ void __launch_bounds__(kT3, 4) k_prune3d(ItemTable tab, Outs o, const __grid_constant__ TmaMaps maps) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem3& sm = *reinterpret_cast<Smem3*>(smem_raw);
    const int warp = threadIdx.x >> 5;
    const int lane = int(lane_id());
    const unsigned lt = (1u << lane) - 1u;
    for (int i = threadIdx.x; i < (1 << 12); i += kT3) sm.disp[i] = g_disp3d[i];
    for (int i = threadIdx.x; i < (1 << 9); i += kT3) sm.sbits[i] = g_sbits3d[i];
    if (threadIdx.x == 0) {
        for (int s = 0; s < kRing; ++s) mbar_init(&sm.bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // TMA destinations must be 128-byte aligned; otherwise every item takes the cp.async path
    const bool tma_ok = (smem_u32(sm.ring) & 127u) == 0;
    uint32_t par = 0;  // phase parity of each slot's mbarrier (every thread waits on every TMA plane)
    WarpStage& ws = sm.ws[warp];
    WarpCounts cnt = {0, 0, 0, 0};
    for (int task = blockIdx.x; task < tab.tiles3d; task += gridDim.x) {
        const int ii = tile_item(tab, tab.n2d, tab.n - 1, task);
        const Item& it = tab.it[ii];
        const int ltask = task - it.tile0;
        if (tma_ok && it.tma >= 0)
            prune_task3d<true>(sm, tab, o, ii, ltask, warp, lane, lt, ws, cnt, &maps.m[it.tma], par);
        else
            prune_task3d<false>(sm, tab, o, ii, ltask, warp, lane, lt, ws, cnt, nullptr, par);
    }
    if (__any_sync(0xFFFFFFFFu, (cnt.s0 | cnt.st | cnt.r0 | cnt.rt) != 0)) warp_flush(ws, cnt, o);
}

// ---------------------------------------------------------------- 2D
// Each warp marches down a strip of one image on its own (no block
// barriers): lane l handles column x0-1+l; lanes 1..31 own their columns (31
// per strip), lane 0 is a halo whose lookup codes the top cells of column
// x0-1 need.  The task owns rows [y0, y1) and computes lookups for rows
// [y0, min(y1, H-1)].
//
// Per row step y:
//  1. cp.async prefetch of row y+kAhead2 (columns x0-2 .. x0+31) into the
//     warp's 8-row shared-memory ring; out-of-image positions read +inf;
//  2. the 8-neighbour mask of (y, x) from registers (rows y-1, y) and the
//     ring (row y+1), direct table lookup, the H0 forest link (an up link
//     continues the chain of (y-1, x), the same lane's previous step) and
//     the survivors and H0 root of owned vertices;
//  3. the top cell whose smallest corner is (y-1, x): its largest corner m
//     among the 4 corner values holds, in its entry, where the top cell dies
//     locally; the codes of rows y-1 and y of column x+1 come by shuffle, so
//     each lane stores one coalesced dual forest link (or a dual root).
constexpr int kW2 = 8;                   // warps per CTA (independent tasks)
constexpr int kOX2 = 31;                 // owned columns per strip
constexpr int kRW2 = 34;                 // ring row: columns x0-2 .. x0+31
constexpr int kRing2 = 8, kAhead2 = 5;   // ring rows, rows in flight
constexpr int kCap2 = 32 * 4;            // staged keys per warp and kind (one step's maximum)

struct WarpStage2 {
    uint64_t s0[kCap2];
    uint64_t st[kCap2];
    uint64_t r0age[kCapWR];
    uint64_t rtage[kCapWR];
    uint32_t r0node[kCapWR];
    uint32_t rtnode[kCapWR];
};

struct Smem2 {
    uint2 lut[256];
    float ring[kW2][kRing2][kRW2];
    WarpStage2 ws[kW2];
};

struct Row {
    float l, c, r;  // columns x-1, x, x+1
};

__device__ __forceinline__ void read_row(const float* slot, int lane, Row& R) {
    R.l = slot[lane];
    R.c = slot[lane + 1];
    R.r = slot[lane + 2];
}

struct RowPos {
    const float* img;
    uint32_t W, H;
    int gx0, gx1;     // image columns copied by this lane
    int idx1;         // ring position of the second column
    bool in0, in1;    // inside the image
};

// kCheck false: the caller knows that row y lies inside the image
template <bool kCheck = true>
__device__ __forceinline__ void issue_row(float (*ring)[kRW2], const RowPos& p, int lane, int y) {
    float* slot = ring[(y + kRing2) & (kRing2 - 1)];
    if (!kCheck || unsigned(y) < p.H) {
        const float* base = p.img + uint32_t(y) * p.W;
        if (p.in0) cp_async4(slot + lane + 1, base + p.gx0);
        if (p.in1) cp_async4(slot + p.idx1, base + p.gx1);
    } else {  // a row outside the image: every position +inf
        const float inf = __int_as_float(0x7F800000);
        if (p.in0) slot[lane + 1] = inf;
        if (p.in1) slot[p.idx1] = inf;
    }
    cp_async_commit();
}

__global__ void __launch_bounds__(kW2 * 32) k_prune2d(ItemTable tab, Outs o) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem2& sm = *reinterpret_cast<Smem2*>(smem_raw);
    const int warp = threadIdx.x >> 5;
    const int lane = int(lane_id());
    const unsigned lt = (1u << lane) - 1u;
    for (int i = threadIdx.x; i < 256; i += kW2 * 32) sm.lut[i] = g_lut2d[i];
    __syncthreads();
    WarpStage2& ws = sm.ws[warp];
    float(*ring)[kRW2] = sm.ring[warp];
    WarpCounts cnt = {0, 0, 0, 0};
    const float inf = __int_as_float(0x7F800000);
    for (int task = blockIdx.x * kW2 + warp; task < tab.tiles2d; task += gridDim.x * kW2) {
        const int ii = tile_item(tab, 0, tab.n2d - 1, task);
        const Item& it = tab.it[ii];
        const int ltask = task - it.tile0;
        const int x0 = (ltask % it.tx) * kOX2, y0 = (ltask / it.tx) * tab.rows2d;
        const int y1 = min(it.H, y0 + tab.rows2d);  // owned rows [y0, y1)
        const int ylast = min(y1, it.H - 1);        // lookups for rows [y0, ylast]
        const int x = x0 - 1 + lane;
        const uint32_t W = uint32_t(it.W), H = uint32_t(it.H), W1 = W - 1u;
        const uint32_t voff = uint32_t(it.voff), toff = uint32_t(it.toff), OUT = uint32_t(it.toff + it.T);
        const bool owned_x = lane >= 1 && x < it.W;
        const bool cube_x = lane <= 30 && x >= 0 && x < it.W - 1;
        RowPos rp;
        rp.img = it.img;
        rp.W = W;
        rp.H = H;
        rp.gx0 = x;
        rp.in0 = unsigned(x) < W;
        rp.gx1 = lane == 0 ? x0 - 2 : x0 + 31;
        rp.idx1 = lane == 0 ? 0 : kRW2 - 1;
        rp.in1 = (lane == 0 || lane == 31) && unsigned(rp.gx1) < W;
        const bool has1 = lane == 0 || lane == 31;
        __syncwarp();  // the ring may still be read by the previous task
#pragma unroll
        for (int s = 0; s < kRing2; ++s) {
            if (!rp.in0) ring[s][lane + 1] = inf;
            if (has1 && !rp.in1) ring[s][rp.idx1] = inf;
        }
#pragma unroll
        for (int k = -1; k < kAhead2; ++k) issue_row(ring, rp, lane, y0 + k);
        cp_async_wait<kAhead2 - 2>();  // rows y0-1 .. y0+1 have landed
        __syncwarp();
        Row A, B, C;
        read_row(ring[(y0 - 1 + kRing2) & (kRing2 - 1)], lane, A);
        read_row(ring[y0 & (kRing2 - 1)], lane, B);
        unsigned long long my_min = ~0ull;
        uint32_t far = 0, far_t = 0, cprev = 0;  // last H0 link / dual link written by this lane
        bool nonfinite = false;                   // an owned value is NaN or infinite (checked once per task)
        // interior: a std::integral_constant; true for a row with y >= y0 + 2 and
        // y + kAhead2 <= ylast, where no boundary row or end-of-task case arises
        auto step = [&](const int y, auto interior) {
            constexpr bool kIn = decltype(interior)::value;
            issue_row<!kIn>(ring, rp, lane, y + kAhead2);
            read_row(ring[(y + 1) & (kRing2 - 1)], lane, C);
            // ---- lookup of (y, x): bit i of the mask is stencil offset n = i (i < 4) or
            // i + 1 (i >= 4); offsets before the centre in linear order precede on ties
            const float cv = B.c;
            uint32_t raw = 0;
            or_if_precedes<1u << 0, true>(raw, A.l, cv);
            or_if_precedes<1u << 1, true>(raw, A.c, cv);
            or_if_precedes<1u << 2, true>(raw, A.r, cv);
            or_if_precedes<1u << 3, true>(raw, B.l, cv);
            or_if_precedes<1u << 4, false>(raw, B.r, cv);
            or_if_precedes<1u << 5, false>(raw, C.l, cv);
            or_if_precedes<1u << 6, false>(raw, C.c, cv);
            or_if_precedes<1u << 7, false>(raw, C.r, cv);
            const uint2 e = sm.lut[raw];
            const bool owned = owned_x && (kIn || y < y1);
            const uint32_t ord = ord_bits(cv);
            const uint32_t vl = uint32_t(y) * W + uint32_t(x);
            const uint32_t vg = voff + vl;
            const uint32_t direct = e.x & 7u;
            // H0: a local minimum becomes a root (registered in the staging block
            // below); otherwise the link along the first edge (face slots: up,
            // left, right, down), where a link up continues the chain that this
            // lane started one row before
            const bool root0 = owned && direct == 7u;
            nonfinite |= owned && !(fabsf(cv) <= 3.40282347e38f);
            {
                const uint32_t mag = (direct == 0u || direct == 3u) ? W : 1u;
                const uint32_t u = direct < 2u ? vg - mag : vg + mag;
                if (owned) far = root0 ? vg : ((direct == 0u && (kIn || y > y0)) ? far : u);
                if (owned && !root0 && CP_IN(vg, o.n_uf0, o.ctr)) o.uf0[vg] = far;
            }
            const uint32_t h0s = owned ? (e.x >> 3) & 0xFu : 0u;
            const uint32_t ds = owned ? (e.x >> 9) & 0xFu : 0u;
            // cross-pruning: dual survivors that are also H0 survivors wait for the
            // H0 union-find (flag bit of the H0 key); otherwise every dual survivor
            // goes to the dual list now (one that kills an H0 class closes a dual
            // cycle there: a no-op)
            const uint32_t flg = tab.cross2d ? ds : 0u;
            const uint32_t dn = tab.cross2d ? ds & ~h0s : ds;
            // ---- the top cell with smallest corner (y-1, x): its largest corner m
            // (value, then linear index) holds it; m's code field for it says where
            // it dies locally (8: a dual root, registered in the staging block
            // below; 15: not held, non-finite input only)
            const uint32_t cprev_r = __shfl_down_sync(0xFFFFFFFFu, cprev, 1);
            const uint32_t ccur_r = __shfl_down_sync(0xFFFFFFFFu, e.y, 1);
            const bool cube = cube_x && (kIn || y > y0);
            const float cvals[4] = {A.c, A.r, B.c, B.r};
            int k = 0;
            float best = cvals[0];
#pragma unroll
            for (int j = 1; j < 4; ++j) {
                const bool ge = cvals[j] >= best;
                best = ge ? cvals[j] : best;
                k = ge ? j : k;
            }
            const uint32_t word = k == 0 ? cprev : (k == 1 ? cprev_r : (k == 2 ? e.y : ccur_r));
            const uint32_t t = uint32_t(3 - k);  // quadrant of the top cell as seen from m
            const uint32_t code = (word >> (4u * t)) & 15u;
            const uint32_t self = toff + uint32_t(y - 1) * W1 + uint32_t(x);
            const bool rootT = cube && code == 8u;
            {
                // the top cell across: quadrant `code` of m, smallest corner m - (negative axes)
                const int my = y - 1 + (k >> 1), mx = x + (k & 1);
                const int ty = my - int(((code >> 1) & 1u) ^ 1u);
                const int tx = mx - int((code & 1u) ^ 1u);
                const bool out = unsigned(ty) >= H - 1u || unsigned(tx) >= W1;
                // a link to (y-2, x) continues the chain that this lane wrote for that top
                // cell in the previous step; a code of 15 writes a root tag to keep the
                // forest well formed
                const bool chain = ty == y - 2 && tx == x && (kIn || y - 1 > y0);
                const uint32_t tgt = code < 4u ? (out ? OUT : toff + uint32_t(ty) * W1 + uint32_t(tx)) : kTag;
                if (cube) far_t = rootT ? self : ((code < 4u && chain) ? far_t : tgt);
                if (cube && !rootT && CP_IN(self, o.n_uft, o.ctr)) o.uft[self] = far_t;
            }
            cprev = e.y;
            // ---- stage survivors and roots
            if (__any_sync(0xFFFFFFFFu, root0 || rootT || (h0s | dn) != 0u)) {
                const unsigned m_r0 = __ballot_sync(0xFFFFFFFFu, root0);
                const unsigned m_rt = __ballot_sync(0xFFFFFFFFu, rootT);
                const uint32_t or0 = __reduce_or_sync(0xFFFFFFFFu, h0s);
                const uint32_t ort = __reduce_or_sync(0xFFFFFFFFu, dn);
                const uint32_t n0 = __reduce_add_sync(0xFFFFFFFFu, uint32_t(__popc(h0s)));  // <= 32 * 4
                const uint32_t nt = __reduce_add_sync(0xFFFFFFFFu, uint32_t(__popc(dn)));   // <= 32 * 4
                if (cnt.s0 + n0 > uint32_t(kCap2) || cnt.st + nt > uint32_t(kCap2) ||
                    cnt.r0 + __popc(m_r0) > uint32_t(kCapWR) || cnt.rt + __popc(m_rt) > uint32_t(kCapWR))
                    warp_flush(ws, cnt, o);
                if (m_r0) {
                    if (root0) {
                        const uint32_t p = cnt.r0 + __popc(m_r0 & lt);
                        ws.r0node[p] = vg;
                        ws.r0age[p] = make_key(ord, vg, 0);
                        const unsigned long long kk = (unsigned long long)(uint64_t(ord) << 32 | vl);
                        my_min = kk < my_min ? kk : my_min;
                    }
                    cnt.r0 += __popc(m_r0);
                }
                if (m_rt) {
                    if (rootT) {
                        const uint32_t my = uint32_t(y - 1 + (k >> 1)), mx = uint32_t(x + (k & 1));
                        const uint32_t mg = voff + my * W + mx;
                        const uint32_t p = cnt.rt + __popc(m_rt & lt);
                        ws.rtnode[p] = self;
                        ws.rtage[p] = make_key(ord_bits(best), mg, (6u * (t >> 1) + 2u * (t & 1u)) << 1);
                    }
                    cnt.rt += __popc(m_rt);
                }
                uint32_t bits = or0;
                while (bits) {
                    const int s = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const bool mine = (h0s >> s) & 1u;
                    const unsigned m = __ballot_sync(0xFFFFFFFFu, mine);
                    if (mine)  // face slot s is stencil offset 2s+1; low bit: the dual waits for it
                        ws.s0[cnt.s0 + __popc(m & lt)] = make_key(ord, vg, (uint32_t(2 * s + 1) << 1) | ((flg >> s) & 1u));
                    cnt.s0 += __popc(m);
                }
                bits = ort;
                while (bits) {
                    const int f = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const bool mine = (dn >> f) & 1u;
                    const unsigned m = __ballot_sync(0xFFFFFFFFu, mine);
                    if (mine) ws.st[cnt.st + __popc(m & lt)] = ~make_key(ord, vg, uint32_t(2 * f + 1) << 1);
                    cnt.st += __popc(m);
                }
                __syncwarp();
            }
            cp_async_wait<kAhead2 - 2>();  // row y+2 has landed (for the next step)
            __syncwarp();
            A = B;
            B = C;
        };
        // the first two rows and the last few take every check; the interior rows
        // are a second instantiation of the step without them
        int y = y0;
        for (; y <= ylast && y < y0 + 2; ++y) step(y, std::false_type());
        for (; y + kAhead2 <= ylast; ++y) step(y, std::true_type());
        for (; y <= ylast; ++y) step(y, std::false_type());
        if (__any_sync(0xFFFFFFFFu, nonfinite) && lane == 0) set_status(o.ctr, kStNonfinite);
        cp_async_wait<0>();
        const unsigned long long w = warp_min_u64(my_min);
        if (lane == 0 && w != ~0ull) atomicMin(&o.ctr->gmin[ii], w);
    }
    if (__any_sync(0xFFFFFFFFu, (cnt.s0 | cnt.st | cnt.r0 | cnt.rt) != 0)) warp_flush(ws, cnt, o);
}

// ---------------------------------------------------------------- host side
size_t prune_smem2d() { return sizeof(Smem2); }
size_t prune_smem3d() { return sizeof(Smem3); }

bool encode_plane_map(CUtensorMap* map, const float* img, int64_t D, int64_t H, int64_t W) {
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static const Encode encode = []() -> Encode {  // looked up once (thread-safe initialisation)
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<Encode>(fn);
        return nullptr;
    }();
    // row stride a multiple of 16 bytes, 16-byte aligned base, a plane at least one box
    if (!encode || !img || (W & 3) != 0 || (reinterpret_cast<uintptr_t>(img) & 15u) != 0 || W < kRS || H < kRH || D < 2)
        return false;
    const cuuint64_t dim[3] = {cuuint64_t(W), cuuint64_t(H), cuuint64_t(D)};
    const cuuint64_t stride[2] = {cuuint64_t(W) * 4u, cuuint64_t(W) * cuuint64_t(H) * 4u};
    const cuuint32_t box[3] = {cuuint32_t(kRS), cuuint32_t(kRH), 1u};
    const cuuint32_t estride[3] = {1u, 1u, 1u};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(img), dim, stride, box, estride,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NAN_REQUEST_ZERO_FMA) == CUDA_SUCCESS;
}
int prune_tile_x() { return kOX2; }
int prune_tile_x3d() { return kOX; }
int g_rows2d = 64, g_zchunk3d = kZC, g_ctas3d = 0, g_cross2d = 0, g_uf_variant = 0;  // tuning (cp_set_tuning)
int prune_tile_y2d() { return g_rows2d; }
int prune_tile_y3d() { return kOY; }
int prune_tile_z3d() { return g_zchunk3d; }
int prune_cross2d() { return g_cross2d; }
int uf_variant() { return g_uf_variant; }

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
        case 3:  // rows per 2D pruning task
            if (value < 4 || value > 4096) return -1;
            g_rows2d = value;
            return 0;
        case 5:  // 2D items: sequential cross-pruning (1) or H0 and the dual at once (0)
            if (value != 0 && value != 1) return -1;
            g_cross2d = value;
            return 0;
        case 7:  // union-find design: reservation rounds (0) or Borůvka's forest first (1)
            if (value != 0 && value != 1) return -1;
            g_uf_variant = value;
            return 0;
        default:
            return -1;
    }
}

int get_tuning(int key) {
    return key == 1 ? g_zchunk3d
           : key == 2 ? g_ctas3d
           : key == 3 ? g_rows2d
           : key == 5 ? g_cross2d
           : key == 7 ? g_uf_variant
                      : -1;
}

// Table entry as two 32-bit words:
//   x: direct (3 bits) | h0_surv << 3 (6) | dual_surv << 9 (12) | in_l << 21 (8)
//   y: the eight 4-bit dual codes
static uint2 pack_entry(uint64_t v) {
    const uint32_t direct = uint32_t(v & 7u), h0s = uint32_t((v >> 3) & 0x3Fu);
    const uint32_t ds = uint32_t((v >> 41) & 0xFFFu), in_l = uint32_t((v >> 53) & 0xFFu);
    uint2 r;
    r.x = direct | (h0s << 3) | (ds << 9) | (in_l << 21);
    r.y = uint32_t((v >> 9) & 0xFFFFFFFFu);
    return r;
}

cudaError_t upload_luts(const uint64_t* lut2d, const uint16_t* disp3d, const uint64_t* entries3d,
                        const uint32_t* keys3d) {
    uint2 p2[256];
    for (int i = 0; i < 256; ++i) p2[i] = pack_entry(lut2d[i]);
    cudaError_t e = cudaMemcpyToSymbol(g_lut2d, p2, sizeof(p2));
    if (e != cudaSuccess) return e;
    e = cudaMemcpyToSymbol(g_disp3d, disp3d, sizeof(uint16_t) * (1 << 12));
    if (e != cudaSuccess) return e;
    // 3D: the device form of each slot's entry (see g_codes3d)
    static uint32_t codes[1 << 14], surv[1 << 14], sbits[1 << 9];
    constexpr uint32_t kFaceBits[6] = {4, 10, 12, 14, 16, 22};
    for (int i = 0; i < (1 << 9); ++i) sbits[i] = 0;
    for (int i = 0; i < (1 << 14); ++i) {
        const uint64_t v = entries3d[i];
        codes[i] = surv[i] = 0;
        if (keys3d[i] == 0xFFFFFFFFu) continue;  // empty slot
        const uint32_t rel = keys3d[i];
        // the kernel takes the direct edge as the lowest face bit of the mask
        uint32_t direct = 7;
        for (int s = 0; s < 6 && direct == 7; ++s)
            if ((rel >> kFaceBits[s]) & 1u) direct = uint32_t(s);
        if (direct != uint32_t(v & 7u)) return cudaErrorInvalidValue;
        uint32_t c = 0;
        for (int t = 0; t < 8; ++t) {
            const uint32_t code = uint32_t((v >> (9 + 4 * t)) & 0xFu);
            uint32_t f;
            if (code == 15u) f = 0;            // not in L(v)
            else if (code == 8u) f = 9;        // survives locally
            else if (code < 8u && code != uint32_t(t)) f = code + 1u;
            else return cudaErrorInvalidValue;
            c |= f << (4 * t);
        }
        codes[i] = c;
        const uint32_t h0s = uint32_t((v >> 3) & 0x3Fu), ds = uint32_t((v >> 41) & 0xFFFu);
        surv[i] = h0s | (ds << 6);
        if (surv[i]) sbits[i >> 5] |= 1u << (i & 31);
    }
    e = cudaMemcpyToSymbol(g_codes3d, codes, sizeof(codes));
    if (e != cudaSuccess) return e;
    e = cudaMemcpyToSymbol(g_surv3d, surv, sizeof(surv));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(g_sbits3d, sbits, sizeof(sbits));
}

cudaError_t launch_prune(const ItemTable& tab, const PruneOuts& po, const TmaMaps& maps, cudaStream_t s) {
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
    o.n_uf0 = po.n_uf0;
    o.n_uft = po.n_uft;
    const int blocks3d = device_cached(kCachePrune3d, [] {
        cudaFuncSetAttribute(k_prune3d, cudaFuncAttributeMaxDynamicSharedMemorySize, int(prune_smem3d()));
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_prune3d, kT3, prune_smem3d());
        return device_sm_count() * (per_sm > 0 ? per_sm : 1);
    });
    const int blocks2d = device_cached(kCachePrune2d, [] {
        cudaFuncSetAttribute(k_prune2d, cudaFuncAttributeMaxDynamicSharedMemorySize, int(prune_smem2d()));
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_prune2d, kW2 * 32, prune_smem2d());
        return device_sm_count() * (per_sm > 0 ? per_sm : 1);
    });
    if (tab.tiles2d > 0) {
        const int need2 = (tab.tiles2d + kW2 - 1) / kW2;
        k_prune2d<<<need2 < blocks2d ? need2 : blocks2d, kW2 * 32, prune_smem2d(), s>>>(tab, o);
        note_launches(1);
    }
    if (tab.tiles3d > 0) {
        int cap = blocks3d;
        if (g_ctas3d > 0) cap = device_sm_count() * g_ctas3d < blocks3d ? device_sm_count() * g_ctas3d : blocks3d;
        int grid = tab.tiles3d < cap ? tab.tiles3d : cap;
        k_prune3d<<<grid, kT3, prune_smem3d(), s>>>(tab, o, maps);
        note_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace cp
