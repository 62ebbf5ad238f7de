// K3: elder-rule union-find over the sorted survivors, H0 (Sec. 4.1 step 3,
// Sec. 4.2 step 2) and the dual graph (Sec. 3.1, Appendix A; Sec. 4.1 step 5,
// Sec. 4.2 step 3), plus the 2D cross-pruning of Sec. 3.2 / Sec. 4.1 step 4.
//
// Sequential union-find processes the sorted survivors one at a time; the
// pairs depend on that order.  Here every unresolved survivor is processed
// in rounds ("deterministic reservations"): in a round each survivor i finds
// the roots of its two endpoints; equal roots mean a positive cell (done);
// otherwise it writes the stamp (round, i) into the reservation word of both
// roots with an atomic max that favours the smallest i.  Survivor i then
// commits (links its younger root under the older one and reports the pair)
// only if it holds the reservation of the root that dies.  That root is then
// touched by no earlier unresolved survivor, so its class is exactly what the
// sequential run would see when it reaches i, and the other class's root at
// that time can only be older: the pair is the sequential one.  Linking early
// changes nothing that an earlier survivor observes (roots keep their age).
// The smallest unresolved i always commits, so the rounds end; results are
// identical to the sequential order whatever the thread schedule.
//
// The H0 forest and the dual forest written by the pruning pass are the
// initial parent arrays; roots carry a tag and a root id, which indexes the
// age and reservation arrays.  The first round's root walks (the long ones,
// through the large forests) run in their own launch and hand over root ids;
// from then on the union-find lives in root-id space: a root that dies gets
// the dead mark and its parent's root id in its reservation word, so the
// finds of later rounds read only the compact per-root arrays (which stay in
// L2).  The rounds run as one persistent cooperative kernel with a grid
// barrier between phases.  A commit only marks the root and notes its id in
// a per-survivor log; the pairs are written from the log in one parallel pass
// after the last round.
#include "cp_common.cuh"
#include "cp_grid.cuh"
#include "cp_kernels.h"
#include "cp_pairs.cuh"

namespace cp {
namespace {

constexpr int kT = 1024;  // one large CTA per SM keeps grid barriers cheap
constexpr uint32_t kInvalid = 0xFFFFFFFFu;

struct UfKernelArgs {
    ItemTable tab;
    UfParams p[2];
    int nprob;
};

// Roots of a and b, walking both paths in lockstep (two independent loads in
// flight per thread).  The walks only read: the active survivors carry their
// roots from round to round, so nothing needs compressing, and random partial
// writes into the large forest array would cost read-modify-write traffic.
// Paths end at roots (the forests are acyclic); the wall-clock bound only
// guards against a corrupted forest (the walk then stops and reports false).
// (Bounds-checked build: a parent outside the forest ends the walk, flagged.)
__device__ __forceinline__ bool walk(const uint32_t* uf, uint32_t n_nodes, Counters* ctr, uint32_t& a, uint32_t& pa,
                                     uint32_t& b, uint32_t& pb, uint32_t& hops) {
    uint64_t t0 = 0;
    (void)n_nodes;
    (void)ctr;
    while (!(pa & kTag) || !(pb & kTag)) {
        ++hops;
        if (!(pa & kTag)) {
            a = pa;
            pa = CP_IN(a, n_nodes, ctr) ? __ldcg(uf + a) : kTag;
        }
        if (!(pb & kTag)) {
            b = pb;
            pb = CP_IN(b, n_nodes, ctr) ? __ldcg(uf + b) : kTag;
        }
        if ((hops & 1023u) == 0) {
            const uint64_t now = global_timer_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > kWaitLimitNs) return false;
        }
    }
    return true;
}

__device__ __forceinline__ bool find_two(const uint32_t* uf, uint32_t n_nodes, Counters* ctr, uint32_t a, uint32_t b,
                                         uint32_t& rida, uint32_t& ridb, uint32_t& ra, uint32_t& rb, uint32_t& hops) {
    uint32_t pa = CP_IN(a, n_nodes, ctr) ? __ldcg(uf + a) : kTag, pb = CP_IN(b, n_nodes, ctr) ? __ldcg(uf + b) : kTag;
    const bool ok = walk(uf, n_nodes, ctr, a, pa, b, pb, hops);
    ra = a;
    rb = b;
    rida = pa & ~kTag;
    ridb = pb & ~kTag;
    return ok;
}


// Current root id of a class given a root id it once had.
// (Bounds-checked build: an id outside the root ids becomes 0, flagged.)
__device__ __forceinline__ bool find_rid(const uint64_t* res, uint32_t n_rids, Counters* ctr, uint32_t& rid,
                                         uint32_t& hops) {
    (void)n_rids;
    (void)ctr;
    if (!CP_IN(rid, n_rids, ctr)) rid = 0;
    uint64_t w = __ldcg(res + rid);
    uint64_t t0 = 0;
    while ((w & kDead) == kDead) {
        rid = uint32_t(w);
        if (!CP_IN(rid, n_rids, ctr)) {
            rid = 0;
            return true;
        }
        w = __ldcg(res + rid);
        if ((++hops & 1023u) == 0) {
            const uint64_t now = global_timer_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > kWaitLimitNs) return false;
        }
    }
    return true;
}

// The result is not needed: the atomic goes out as a reduction, and the
// thread does not wait for it (the grid barrier orders it before the checks).
__device__ __forceinline__ void reserve(uint64_t* res, uint32_t rid, uint64_t stamp) {
    atomicMax(reinterpret_cast<unsigned long long*>(res + rid), (unsigned long long)stamp);
}

// Endpoints of survivor key k (H0: the edge's two vertices; dual: the two top
// cells on either side of the facet, or the item's outside vertex).
__device__ __forceinline__ void endpoints(const ItemTable& tab, uint64_t k, int dual, uint32_t& a, uint32_t& b,
                                          int& item) {
    uint32_t vg = key_vertex(k);
    item = item_of_vertex(tab, vg);
    const Item& it = tab.it[item];
    int n = int(key_n(k, it.ndim));
    int dz, dy, dx;
    stencil_off(it.ndim, n, dz, dy, dx);
    if (!dual) {
        a = vg;
        b = uint32_t(int64_t(vg) + (int64_t(dz) * it.H + dy) * it.W + dx);
        return;
    }
    const uint32_t local = vg - uint32_t(it.voff), W = uint32_t(it.W), H = uint32_t(it.H);
    const uint32_t row = local / W;
    const int x = int(local - row * W), y = int(row % H), z = int(row / H);
    // the facet's zero coordinate (on one of the item's axes) picks the side
    int sz0 = dz, sy0 = dy, sx0 = dx, sz1 = dz, sy1 = dy, sx1 = dx;
    if (it.ndim == 3 && dz == 0) {
        sz0 = -1;
        sz1 = 1;
    } else if (dy == 0) {
        sy0 = -1;
        sy1 = 1;
    } else {
        sx0 = -1;
        sx1 = 1;
    }
    a = top_of_octant(it, z, y, x, sz0, sy0, sx0);
    b = top_of_octant(it, z, y, x, sz1, sy1, sx1);
}

// The pair of a committed survivor (see commit_pair).
__device__ __forceinline__ void emit_pair(const UfParams& p, const ItemTable& tab, uint64_t key, int item,
                                          uint32_t yrid, bool* emitted, cp_pair& out) {
    *emitted = commit_pair(tab, p.age, p.dual, key, item, yrid, out);
}

__device__ __forceinline__ bool side_by_side(const UfKernelArgs& args, uint32_t n0, uint32_t n1) {
    return uint64_t(n0) + n1 <= args.p[0].scratch_cap;
}

constexpr int kR = 4;  // active items per thread whose phase-A results stay in registers

// 2D cross-pruning: a positive edge of H0 whose key carries the dual flag is
// a merging facet of the dual graph (only the H0 problem of a call with 2D
// items has that list, and it runs alone).
__device__ __forceinline__ void cross_prune(const ItemTable& tab, const UfParams& p, uint32_t i) {
    if (p.dual || !p.dual_keys) return;
    const uint64_t key = p.keys[i];
    if (tab.it[item_of_vertex(tab, key_vertex(key))].ndim == 2 && (key & 1u)) {
        const uint32_t pos = atomicAdd(p.d_ndual, 1u);
        if (pos < p.dual_cap) p.dual_keys[pos] = ~(key & ~1ull);
        else set_status(p.ctr, kStCapacity);
    }
}

// The first round's root walks, the long ones (later rounds start from root
// ids carried over).  They run before the sort, over the survivors in the
// order the pruning pass wrote them -- tile by tile, so neighbouring
// survivors walk through the same parts of the forest and share its sectors
// in L2 -- and the sort carries each survivor's position as its payload.  A
// separate, non-cooperative launch: warps take 32 survivors at a time from a
// counter, so a warp held up by a long path delays no other warp.
constexpr int kFT = 256;
constexpr int kRootsPerLane = 1;  // survivors per lane (more paths in lockstep measured slower: the walks are
                                  // bound by random DRAM accesses, and lockstep waste grows)

__global__ void __launch_bounds__(kFT) k_roots(const __grid_constant__ RootArgs r) {
    Counters* ctr = r.ctr;
    if (ld_acquire_u32(&ctr->status) & (kStTimeout | kStNonfinite)) return;
    const uint32_t n = min(*r.d_n, r.cap);
    const unsigned lane = lane_id();
    uint32_t hops = 0;
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&ctr->find_ctr, 32u * kRootsPerLane);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (base >= n) break;
        // the endpoints of this lane's survivors and their first parents (all loads in flight together)
        uint32_t node[2 * kRootsPerLane], par[2 * kRootsPerLane];
#pragma unroll
        for (int s = 0; s < kRootsPerLane; ++s) {
            const uint32_t i = base + 32u * s + lane;
            node[2 * s] = node[2 * s + 1] = 0;
            if (i < n) {
                uint64_t key = r.keys[i];
                if (r.dual) key = ~key;
                int item;
                endpoints(r.tab, key, r.dual, node[2 * s], node[2 * s + 1], item);
            }
        }
#pragma unroll
        for (int k = 0; k < 2 * kRootsPerLane; ++k)
            par[k] = base + 32u * (k >> 1) + lane < n && CP_IN(node[k], r.n_nodes, ctr) ? __ldcg(r.uf + node[k]) : kTag;
        // walk all paths one hop per step until every one has reached its root
        uint64_t t0 = 0;
        uint32_t steps = 0;
        for (;;) {
            bool more = false;
#pragma unroll
            for (int k = 0; k < 2 * kRootsPerLane; ++k) {
                if (!(par[k] & kTag)) {
                    node[k] = par[k];
                    par[k] = CP_IN(node[k], r.n_nodes, ctr) ? __ldcg(r.uf + node[k]) : kTag;
                    more = true;
                }
            }
            if (!more) break;
            ++hops;
            if ((++steps & 1023u) == 0) {
                const uint64_t now = global_timer_ns();
                if (t0 == 0) t0 = now;
                else if (now - t0 > kWaitLimitNs) {  // only a corrupted forest gets here
                    set_status(ctr, kStTimeout);
#pragma unroll
                    for (int k = 0; k < 2 * kRootsPerLane; ++k) par[k] = kTag;
                    break;
                }
            }
        }
#pragma unroll
        for (int s = 0; s < kRootsPerLane; ++s) {
            const uint32_t i = base + 32u * s + lane;
            if (i < n) {
                __stcg(r.ra + i, par[2 * s] & ~kTag);
                __stcg(r.rb + i, par[2 * s + 1] & ~kTag);
                __stcg(r.pos + i, i);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) hops += __shfl_xor_sync(0xFFFFFFFFu, hops, o);
    if (lane == 0 && hops) atomicAdd(&ctr->trace_hops[r.dual][0], (unsigned long long)hops);
}

// Both lists' first-round walks in one launch (volumes): warps take 32
// survivors at a time from one counter running over the H0 list and then the
// dual list, so the long walks of one list overlap those of the other instead
// of following them.  Each lane walks its own list's forest.
__global__ void __launch_bounds__(kFT) k_roots2(const __grid_constant__ RootArgs r0,
                                                const __grid_constant__ RootArgs r1) {
    Counters* ctr = r0.ctr;
    if (ld_acquire_u32(&ctr->status) & (kStTimeout | kStNonfinite)) return;
    const uint32_t n0 = min(*r0.d_n, r0.cap), n1 = min(*r1.d_n, r1.cap);
    const uint32_t n = n0 + n1;
    const unsigned lane = lane_id();
    uint32_t hops[2] = {0, 0};
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&ctr->find_ctr, 32u);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (base >= n) break;
        const uint32_t g = base + lane;
        const bool live = g < n;
        const int l = g >= n0 ? 1 : 0;  // this lane's list
        const RootArgs& r = l ? r1 : r0;
        const uint32_t i = l ? g - n0 : g;
        uint32_t node[2] = {0, 0}, par[2] = {kTag, kTag};
        if (live) {
            uint64_t key = r.keys[i];
            if (r.dual) key = ~key;
            int item;
            endpoints(r0.tab, key, r.dual, node[0], node[1], item);
            par[0] = CP_IN(node[0], r.n_nodes, ctr) ? __ldcg(r.uf + node[0]) : kTag;
            par[1] = CP_IN(node[1], r.n_nodes, ctr) ? __ldcg(r.uf + node[1]) : kTag;
        }
        uint64_t t0 = 0;
        uint32_t steps = 0;
        for (;;) {
            bool more = false;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (!(par[k] & kTag)) {
                    node[k] = par[k];
                    par[k] = CP_IN(node[k], r.n_nodes, ctr) ? __ldcg(r.uf + node[k]) : kTag;
                    more = true;
                }
            }
            if (!more) break;
            ++hops[l];
            if ((++steps & 1023u) == 0) {
                const uint64_t now = global_timer_ns();
                if (t0 == 0) t0 = now;
                else if (now - t0 > kWaitLimitNs) {  // only a corrupted forest gets here
                    set_status(ctr, kStTimeout);
                    par[0] = par[1] = kTag;
                    break;
                }
            }
        }
        if (live) {
            __stcg(r.ra + i, par[0] & ~kTag);
            __stcg(r.rb + i, par[1] & ~kTag);
            __stcg(r.pos + i, i);
        }
    }
    for (int l = 0; l < 2; ++l) {
        uint32_t h = hops[l];
        for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xFFFFFFFFu, h, o);
        const int d = (l ? r1 : r0).dual;
        if (lane == 0 && h) atomicAdd(&ctr->trace_hops[d][0], (unsigned long long)h);
    }
}

// The first active list of a problem from the sorted positions: slot off + j
// gets sorted survivor j and the root ids of its endpoints.  The dual list of
// a call without 2D items sits after the H0 list (off = the H0 count) when
// both fit the scratch; otherwise the union-find walks it itself.
__global__ void __launch_bounds__(kFT) k_place_roots(const __grid_constant__ RootArgs r) {
    // k_roots skipped the walks (the payload was never written): nothing to place
    if (ld_acquire_u32(&r.ctr->status) & (kStTimeout | kStNonfinite)) return;
    const uint32_t n = min(*r.d_n, r.cap);
    uint32_t off = 0;
    if (r.d_n_before) {
        off = min(*r.d_n_before, r.cap);
        if (uint64_t(off) + n > r.scratch_cap) return;
    }
    for (uint32_t j = blockIdx.x * kFT + threadIdx.x; j < n; j += gridDim.x * kFT) {
        uint32_t i = __ldcg(r.sorted_pos + j);
        if (i >= n) {  // never: the payload is a permutation of 0 .. n-1
            set_status(r.ctr, kStInternal);
            i = 0;
        }
        __stcg(r.act + off + j, j);
        __stcg(r.na + off + j, __ldcg(r.ra + i));
        __stcg(r.nb + off + j, __ldcg(r.rb + i));
    }
}

// Root ids of the two endpoints of a survivor that starts here (the first
// round of a problem whose walks did not run before the sort): a walk
// through the forest.
__device__ __forceinline__ void fresh_roots(const UfKernelArgs& args, const UfParams& p, uint32_t i, uint32_t& ra,
                                            uint32_t& rb, uint32_t& hops) {
    uint64_t key = p.keys[i];
    if (p.dual) key = ~key;
    uint32_t a, b, va, vb;
    int item;
    endpoints(args.tab, key, p.dual, a, b, item);
    if (!find_two(p.uf, p.n_nodes, p.ctr, a, b, ra, rb, va, vb, hops)) {
        set_status(p.ctr, kStTimeout);
        rb = ra;
    }
}

// Phase A of one active item whose results go through memory (the items of a
// thread beyond the first kR).
__device__ __forceinline__ void phase_a_mem(const UfKernelArgs& args, int q, uint32_t jj, uint32_t slot, bool fresh,
                                            int cur, uint32_t round, uint32_t& hops) {
    const UfParams& p = args.p[q];
    uint32_t i, a, b;
    if (round == 1) __stcg(p.log + slot, ~0ull);  // no commit yet
    if (fresh) {
        i = jj;
        fresh_roots(args, p, i, a, b, hops);
    } else {
        i = __ldcg(p.act[cur] + slot);
        a = __ldcg(p.na[cur] + slot);
        b = __ldcg(p.nb[cur] + slot);
    }
    if (!find_rid(p.res, p.n_rids, p.ctr, a, hops) || !find_rid(p.res, p.n_rids, p.ctr, b, hops)) {
        set_status(p.ctr, kStTimeout);
        b = a;
    }
    if (a == b) {
        __stcg(p.ynode + slot, kInvalid);
        cross_prune(args.tab, p, i);
        return;
    }
    const uint64_t aa = p.age[a], ab = p.age[b];
    const bool a_young = p.dual ? (aa < ab) : (aa > ab);
    const uint64_t stamp = (uint64_t(round) << 32) | (0xFFFFFFFFu - i);
    if (aa != ~0ull) reserve(p.res, a, stamp);  // the outside vertex never dies
    if (ab != ~0ull) reserve(p.res, b, stamp);
    __stcg(p.ynode + slot, a_young ? a : b);
    __stcg(p.onode + slot, a_young ? b : a);
}

// The rounds of one or two problems (H0 and the dual of a call without 2D
// items, whose lists do not depend on each other) in lockstep: one round
// covers the active survivors of both, so the grid barriers and the memory
// latency of a round are paid once for the two.  Problem q's entries of the
// shared scratch lists and of the commit log start at 0 and base1.  The
// first kR items of each thread keep their phase-A results in registers, and
// their loads are issued together.
__device__ void uf_rounds(const UfKernelArgs& args, uint32_t n0, uint32_t n1, uint32_t base1, unsigned live,
                          unsigned prefound, uint32_t& epoch) {
    const ItemTable& tab = args.tab;
    Counters* ctr = args.p[0].ctr;
    const uint32_t nblocks = gridDim.x;
    const uint32_t gstride = nblocks * kT;
    const uint32_t gtid = blockIdx.x * kT + threadIdx.x;
    const unsigned lane = lane_id();
    const uint32_t ninit[2] = {n0, n1};
    uint32_t n[2] = {n0, n1};
    uint32_t rounds[2] = {0u, 0u};
    int cur = 0;
    uint32_t round = 1;
    for (;; ++round) {
        if (gtid == 0 && round <= uint32_t(kTraceRounds)) {
            const uint64_t now = global_timer_ns();
            for (int q = 0; q < 2; ++q) {
                if (!((live >> q) & 1u)) continue;
                const int d = args.p[q].dual;
                ctr->trace_active[d][round - 1] = n[q];
                ctr->trace_t[d][round - 1] = now;
            }
        }
        if (n[0] + n[1] == 0) break;
        if (n[0]) rounds[0] = round;
        if (n[1]) rounds[1] = round;
        if (gtid == 0) ctr->act_count[0][round % 3] = ctr->act_count[1][round % 3] = 0;
        const uint32_t ntot = n[0] + n[1];
        uint32_t hops0 = 0, hops1 = 0;
        // ---- phase A: find roots, resolve positives, reserve
        uint32_t ri[kR], ry[kR], ro[kR];  // survivor index, young and old root ids
        unsigned pend = 0, isq1 = 0;  // bit k: item k waits for its check / belongs to problem 1
        {
            uint32_t a[kR], b[kR];
            uint64_t wa[kR], wb[kR];
            unsigned has = 0;
#pragma unroll
            for (int k = 0; k < kR; ++k) {
                const uint32_t j = gtid + uint32_t(k) * gstride;
                ri[k] = ry[k] = ro[k] = 0;
                a[k] = b[k] = 0;
                if (j < ntot) {
                    const int q = j >= n[0] ? 1 : 0;
                    const UfParams& p = args.p[q];
                    const uint32_t jj = j - (q ? n[0] : 0u);
                    const uint32_t slot = (q ? base1 : 0u) + jj;
                    has |= 1u << k;
                    if (q) isq1 |= 1u << k;
                    if (round == 1) __stcg(p.log + slot, ~0ull);  // no commit yet
                    if (round == 1 && !((prefound >> q) & 1u)) {
                        ri[k] = jj;
                        uint32_t h = 0;
                        fresh_roots(args, p, jj, a[k], b[k], h);
                        if (q) hops1 += h;
                        else hops0 += h;
                    } else {
                        ri[k] = __ldcg(p.act[cur] + slot);
                        a[k] = __ldcg(p.na[cur] + slot);
                        b[k] = __ldcg(p.nb[cur] + slot);
                    }
                }
            }
            // reservation words of the carried roots (loads of the kR items in flight together)
#pragma unroll
            for (int k = 0; k < kR; ++k) {
                const UfParams& pk = args.p[(isq1 >> k) & 1u];
                const uint64_t* res = pk.res;
                const bool h = (has >> k) & 1u;
                if (h && !CP_IN(a[k], pk.n_rids, ctr)) a[k] = 0;
                if (h && !CP_IN(b[k], pk.n_rids, ctr)) b[k] = 0;
                wa[k] = h ? __ldcg(res + a[k]) : 0ull;
                wb[k] = h ? __ldcg(res + b[k]) : 0ull;
            }
#pragma unroll
            for (int k = 0; k < kR; ++k) {
                if ((wa[k] & kDead) != kDead && (wb[k] & kDead) != kDead) continue;  // both still roots
                // a carried root has died: follow the dead marks to the current roots
                const int q = (isq1 >> k) & 1u;
                const uint64_t* res = args.p[q].res;
                uint32_t h = 0;
                if ((wa[k] & kDead) == kDead) {
                    a[k] = uint32_t(wa[k]);
                    if (!find_rid(res, args.p[q].n_rids, ctr, a[k], h)) set_status(ctr, kStTimeout);
                    ++h;
                }
                if ((wb[k] & kDead) == kDead) {
                    b[k] = uint32_t(wb[k]);
                    if (!find_rid(res, args.p[q].n_rids, ctr, b[k], h)) set_status(ctr, kStTimeout);
                    ++h;
                }
                if (q) hops1 += h;
                else hops0 += h;
            }
            uint64_t aa[kR], ab[kR];
#pragma unroll
            for (int k = 0; k < kR; ++k) {
                aa[k] = ab[k] = 0;
                if (((has >> k) & 1u) && a[k] != b[k]) {
                    const uint64_t* age = ((isq1 >> k) & 1u) ? args.p[1].age : args.p[0].age;
                    aa[k] = age[a[k]];
                    ab[k] = age[b[k]];
                }
            }
#pragma unroll
            for (int k = 0; k < kR; ++k) {
                if (!((has >> k) & 1u)) continue;
                const int q = (isq1 >> k) & 1u;
                const UfParams& p = args.p[q];
                if (a[k] == b[k]) {
                    cross_prune(tab, p, ri[k]);
                    continue;
                }
                // H0: the root with the larger key (later vertex) dies; dual: the smaller key dies
                const bool a_young = p.dual ? (aa[k] < ab[k]) : (aa[k] > ab[k]);
                const uint64_t stamp = (uint64_t(round) << 32) | (0xFFFFFFFFu - ri[k]);
                if (aa[k] != ~0ull) reserve(p.res, a[k], stamp);  // the outside vertex never dies
                if (ab[k] != ~0ull) reserve(p.res, b[k], stamp);
                ry[k] = a_young ? a[k] : b[k];
                ro[k] = a_young ? b[k] : a[k];
                pend |= 1u << k;
            }
        }
        // items beyond kR per thread: state through memory
        for (uint32_t j0 = blockIdx.x * kT + kR * gstride; j0 < ntot; j0 += gstride) {
            const uint32_t j = j0 + threadIdx.x;
            if (j >= ntot) continue;
            const int q = j >= n[0] ? 1 : 0;
            const uint32_t jj = j - (q ? n[0] : 0u);
            uint32_t h = 0;
            phase_a_mem(args, q, jj, (q ? base1 : 0u) + jj, round == 1 && !((prefound >> q) & 1u), cur, round, h);
            if (q) hops1 += h;
            else hops0 += h;
        }
        if (round <= uint32_t(kTraceRounds)) {
            for (int q = 0; q < 2; ++q) {
                uint32_t h = q ? hops1 : hops0;
                for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xFFFFFFFFu, h, o);
                if (lane == 0 && h) atomicAdd(&ctr->trace_hops[args.p[q].dual][round - 1], (unsigned long long)h);
            }
        }
        grid_barrier(ctr, nblocks, epoch);
        if (gtid == 0 && round <= uint32_t(kTraceRounds))
            for (int q = 0; q < 2; ++q)
                if ((live >> q) & 1u) ctr->trace_ta[args.p[q].dual][round - 1] = global_timer_ns();
        // ---- phase B: commit the survivors that hold the reservation of their dying root
        {
            uint64_t rv[kR];
#pragma unroll
            for (int k = 0; k < kR; ++k) {
                const uint64_t* res = ((isq1 >> k) & 1u) ? args.p[1].res : args.p[0].res;
                rv[k] = ((pend >> k) & 1u) ? __ldcg(res + ry[k]) : 0ull;
            }
            unsigned keep = 0;
#pragma unroll
            for (int k = 0; k < kR; ++k) {
                if (!((pend >> k) & 1u)) continue;
                const int q = (isq1 >> k) & 1u;
                const UfParams& p = args.p[q];
                const uint64_t stamp = (uint64_t(round) << 32) | (0xFFFFFFFFu - ri[k]);
                if (rv[k] == stamp) {
                    __stcg(p.res + ry[k], kDead | ro[k]);  // the young class joins the old one
                    __stcg(p.log + (q ? base1 : 0u) + ri[k], uint64_t(ry[k]));
                } else {
                    keep |= 1u << k;
                }
            }
            // one atomic per warp and problem for the next round's slots
            uint32_t c0 = __popc(keep & ~isq1), c1 = __popc(keep & isq1);
            uint32_t s0 = c0, s1 = c1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t0 = __shfl_up_sync(0xFFFFFFFFu, s0, o), t1 = __shfl_up_sync(0xFFFFFFFFu, s1, o);
                if (lane >= unsigned(o)) {
                    s0 += t0;
                    s1 += t1;
                }
            }
            uint32_t b0 = 0, b1 = 0;
            if (lane == 31) {
                if (s0) b0 = atomicAdd(&ctr->act_count[0][round % 3], s0);
                if (s1) b1 = atomicAdd(&ctr->act_count[1][round % 3], s1);
            }
            b0 = __shfl_sync(0xFFFFFFFFu, b0, 31) + s0 - c0;
            b1 = __shfl_sync(0xFFFFFFFFu, b1, 31) + s1 - c1;
#pragma unroll
            for (int k = 0; k < kR; ++k) {
                if (!((keep >> k) & 1u)) continue;
                const int q = (isq1 >> k) & 1u;
                const UfParams& p = args.p[q];
                const uint32_t at = q ? base1 + b1++ : b0++;
                p.act[cur ^ 1][at] = ri[k];
                p.na[cur ^ 1][at] = ry[k];
                p.nb[cur ^ 1][at] = ro[k];
            }
        }
        for (uint32_t j0 = blockIdx.x * kT + kR * gstride; j0 < ntot; j0 += gstride) {
            const uint32_t j = j0 + threadIdx.x;
            const int q = j >= n[0] ? 1 : 0;
            const UfParams& p = args.p[q];
            const uint32_t jj = j - (q ? n[0] : 0u);
            const uint32_t slot = (q ? base1 : 0u) + jj;
            bool keep = false;
            uint32_t i = 0, y = 0;
            if (j < ntot) {
                y = __ldcg(p.ynode + slot);
                if (y != kInvalid) {
                    i = (round == 1 && !((prefound >> q) & 1u)) ? jj : __ldcg(p.act[cur] + slot);
                    const uint64_t stamp = (uint64_t(round) << 32) | (0xFFFFFFFFu - i);
                    if (__ldcg(p.res + y) == stamp) {
                        __stcg(p.res + y, kDead | __ldcg(p.onode + slot));
                        __stcg(p.log + (q ? base1 : 0u) + i, uint64_t(y));
                    } else {
                        keep = true;
                    }
                }
            }
            const uint32_t pos0 = warp_append(&ctr->act_count[0][round % 3], keep && q == 0);
            const uint32_t pos1 = warp_append(&ctr->act_count[1][round % 3], keep && q == 1);
            if (keep) {
                const uint32_t at = (q ? base1 + pos1 : pos0);
                p.act[cur ^ 1][at] = i;
                p.na[cur ^ 1][at] = y;
                p.nb[cur ^ 1][at] = __ldcg(p.onode + slot);
            }
        }
        grid_barrier(ctr, nblocks, epoch);
        // one thread reads the next round's counts and the status for the CTA,
        // so that every thread of the CTA takes the same path even after a
        // bounded wait has given up
        __shared__ uint32_t sh_n[2], sh_stop;
        if (threadIdx.x == 0) {
            sh_n[0] = ld_acquire_u32(&ctr->act_count[0][round % 3]);
            sh_n[1] = ld_acquire_u32(&ctr->act_count[1][round % 3]);
            sh_stop = ld_acquire_u32(&ctr->status) & kStTimeout;
        }
        __syncthreads();
        n[0] = sh_n[0];
        n[1] = sh_n[1];
        const bool stop = sh_stop != 0;
        __syncthreads();  // sh_* are rewritten in the next round
        cur ^= 1;
        if (stop) break;
        if (round > 0x7FFFFFF0u) {
            if (gtid == 0) set_status(ctr, kStInternal);
            break;
        }
    }
    if (gtid == 0)
        for (int q = 0; q < 2; ++q) {
            if (!((live >> q) & 1u)) continue;
            if (args.p[q].dual) ctr->roundst = rounds[q];
            else ctr->rounds0 = rounds[q];
        }
    // ---- the pairs, from the commit log (the last round's commits are ordered
    // before this by its final grid barrier)
    for (int q = 0; q < 2; ++q) {
        if (!((live >> q) & 1u)) continue;
        const UfParams& p = args.p[q];
        if (!p.pairs) continue;  // the commit log is the result (the first stage of a slab split)
        const uint64_t* log = p.log + (q ? base1 : 0u);
        for (uint32_t i0 = blockIdx.x * kT; i0 < ninit[q]; i0 += gstride) {
            const uint32_t i = i0 + threadIdx.x;
            bool emit = false;
            cp_pair pr;
            if (i < ninit[q]) {
                const uint64_t e = __ldcg(log + i);
                if (e != ~0ull) {
                    uint64_t key = p.keys[i];
                    if (p.dual) key = ~key;
                    const int item = item_of_vertex(tab, key_vertex(key));
                    if (p.h1flags && tab.it[item].ndim == 3) {
                        const uint32_t id = cell_id3(tab.it[item], key, p.dual != 0);
                        atomicOr(p.h1flags + (id >> 5), 1u << (id & 31u));
                    }
                    emit_pair(p, tab, key, item, uint32_t(e), &emit, pr);
                }
            }
            const uint32_t pp = warp_append(&ctr->n_pairs, emit);
            if (emit) {
                if (pp < p.pair_cap) p.pairs[pp] = pr;
                else set_status(ctr, kStCapacity);
            }
        }
    }
}

__global__ void __launch_bounds__(kT) k_uf(const __grid_constant__ UfKernelArgs args) {
    Counters* ctr = args.p[0].ctr;
    // a bounded wait that gave up earlier leaves the sorted keys unreliable;
    // non-finite input leaves the forests unreliable: the call fails anyway
    if (ld_acquire_u32(&ctr->status) & (kStTimeout | kStNonfinite)) return;
    const uint32_t n0 = min(*args.p[0].d_nkeys, args.p[0].cap_keys);
    uint32_t epoch = 0;  // grid barriers passed in this launch
    // k_roots / k_place_roots have walked the first round's paths of problem
    // 0, and of problem 1 when the two lists sit side by side
    if (args.nprob == 1) {
        uf_rounds(args, n0, 0u, 0u, 1u, 1u, epoch);
        return;
    }
    const uint32_t n1 = min(*args.p[1].d_nkeys, args.p[1].cap_keys);
    if (side_by_side(args, n0, n1)) {
        uf_rounds(args, n0, n1, n0, 3u, 3u, epoch);
    } else {  // one after the other, each with the whole scratch and log
        uf_rounds(args, n0, 0u, 0u, 1u, 1u, epoch);
        grid_barrier(ctr, gridDim.x, epoch);  // problem 0's log is read before problem 1 rewrites it
        uf_rounds(args, 0u, n1, 0u, 2u, 0u, epoch);
    }
}

int find_blocks() {
    return device_cached(kCacheRoots, [] {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_roots, kFT, 0);
        return device_sm_count() * (per_sm > 0 ? per_sm : 1);
    });
}

}  // namespace

cudaError_t launch_uf(const ItemTable& tab, const UfParams* p, int nprob, cudaStream_t s) {
    if (nprob < 1 || nprob > 2) return cudaErrorInvalidValue;
    const int uf_blocks = device_cached(kCacheUf, [] {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_uf, kT, 0);
        return per_sm > 0 ? device_sm_count() * per_sm : -1;
    });
    if (uf_blocks <= 0) return cudaErrorLaunchOutOfResources;
    UfKernelArgs args;
    args.tab = tab;
    args.p[0] = p[0];
    args.p[1] = p[nprob - 1];
    args.nprob = nprob;
    // cooperative launch (all CTAs co-resident, as the grid barrier needs);
    // launched through cudaLaunchKernelEx so that it can also be captured
    // into a CUDA graph
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(uf_blocks);
    cfg.blockDim = dim3(kT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaMemsetAsync(&p[0].ctr->bar_count, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    note_launches(1);
    return cudaLaunchKernelEx(&cfg, k_uf, args);
}

cudaError_t launch_roots(const RootArgs& r, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(&r.ctr->find_ctr, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_roots<<<find_blocks(), kFT, 0, s>>>(r);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_roots2(const RootArgs& r0, const RootArgs& r1, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(&r0.ctr->find_ctr, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_roots2<<<find_blocks(), kFT, 0, s>>>(r0, r1);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_place_roots(const RootArgs& r, cudaStream_t s) {
    k_place_roots<<<device_sm_count() * 4, kFT, 0, s>>>(r);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace cp
