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
// age and reservation arrays.  The union-find runs as one persistent
// cooperative kernel with a grid barrier between phases.
#include "cp_common.cuh"
#include "cp_kernels.h"

namespace cp {
namespace {

constexpr int kT = 1024;  // one large CTA per SM keeps grid barriers cheap
constexpr uint32_t kInvalid = 0xFFFFFFFFu;

struct UfKernelArgs {
    ItemTable tab;
    UfParams p;
};

// Roots of a and b, walking both paths in lockstep (two independent loads in
// flight per thread).  The walks only read: the active survivors carry their
// roots from round to round, so nothing needs compressing, and random partial
// writes into the large forest array would cost read-modify-write traffic.
__device__ __forceinline__ void find_two(const uint32_t* uf, uint32_t a, uint32_t b, uint32_t& rida, uint32_t& ridb,
                                         uint32_t& ra, uint32_t& rb, uint32_t& hops) {
    uint32_t pa = __ldcg(uf + a), pb = __ldcg(uf + b);
    while (!(pa & kTag) || !(pb & kTag)) {
        ++hops;
        if (!(pa & kTag)) {
            a = pa;
            pa = __ldcg(uf + a);
        }
        if (!(pb & kTag)) {
            b = pb;
            pb = __ldcg(uf + b);
        }
    }
    ra = a;
    rb = b;
    rida = pa & ~kTag;
    ridb = pb & ~kTag;
}

__device__ __forceinline__ void reserve(uint64_t* res, uint32_t rid, uint64_t stamp) {
    uint64_t cur = __ldcg(res + rid);
    if (cur < stamp) atomicMax(reinterpret_cast<unsigned long long*>(res + rid), (unsigned long long)stamp);
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).
__device__ void grid_barrier(Counters* ctr, uint32_t nblocks) {
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t gen = ld_acquire_u32(&ctr->bar_gen);
        __threadfence();
        uint32_t arrived = atomicAdd(&ctr->bar_count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&ctr->bar_count, 0u);
            __threadfence();
            atomicAdd(&ctr->bar_gen, 1u);
        } else {
            bounded_wait_ne(&ctr->bar_gen, gen, ctr, kWaitLimitNs);
        }
        __threadfence();
    }
    __syncthreads();
}

// warp-aggregated append of one element per active lane
__device__ __forceinline__ uint32_t warp_append(uint32_t* counter, bool want) {
    unsigned m = __ballot_sync(0xFFFFFFFFu, want);
    if (!m) return 0;
    int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (int(lane_id()) == leader) base = atomicAdd(counter, uint32_t(__popc(m)));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    return base + __popc(m & ((1u << lane_id()) - 1u));
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
    int64_t local = int64_t(vg) - it.voff;
    int x = int(local % it.W), y = int((local / it.W) % it.H), z = int(local / (int64_t(it.W) * it.H));
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

__device__ __forceinline__ void emit_pair(const UfParams& p, const ItemTable& tab, uint64_t key, int item,
                                          uint32_t young, uint32_t yrid, bool* emitted, cp_pair& out) {
    const Item& it = tab.it[item];
    uint64_t age = p.age[yrid];
    uint32_t vg = key_vertex(key);
    int n = int(key_n(key, it.ndim));
    int dz, dy, dx;
    stencil_off(it.ndim, n, dz, dy, dx);
    int64_t lv = int64_t(vg) - it.voff;
    int x = int(lv % it.W), y = int((lv / it.W) % it.H), z = int(lv / (int64_t(it.W) * it.H));
    float fv = ord_float(uint32_t(key >> 32));
    float fy = ord_float(uint32_t(age >> 32));
    if (!p.dual) {
        // H0: birth at the dying root vertex, death at the edge (value of its higher endpoint v)
        out.birth = fy;
        out.death = fv;
        int64_t ly = int64_t(young) - it.voff;
        int yx = int(ly % it.W), yy = int((ly / it.W) % it.H), yz = int(ly / (int64_t(it.W) * it.H));
        out.birth_cell = int32_t(doubled_index(it, yz, yy, yx, 0, 0, 0));
        out.death_cell = int32_t(doubled_index(it, z, y, x, dz, dy, dx));
        out.birth_pixel = int32_t(ly);
        out.death_pixel = int32_t(lv);
        out.dim = 0;
    } else {
        // top dimension: birth at the facet, death at the dying top cell
        uint32_t mg = key_vertex(age);
        int nt = int(key_n(age, it.ndim));
        int tz, ty, tx;
        stencil_off(it.ndim, nt, tz, ty, tx);
        int64_t lm = int64_t(mg) - it.voff;
        int mx = int(lm % it.W), my = int((lm / it.W) % it.H), mz = int(lm / (int64_t(it.W) * it.H));
        out.birth = fv;
        out.death = fy;
        out.birth_cell = int32_t(doubled_index(it, z, y, x, dz, dy, dx));
        out.death_cell = int32_t(doubled_index(it, mz, my, mx, tz, ty, tx));
        out.birth_pixel = int32_t(lv);
        out.death_pixel = int32_t(lm);
        out.dim = it.ndim - 1;
    }
    out.item = it.user;
    *emitted = out.birth != out.death;  // zero persistence: omitted (Sec. 2.3)
}

__global__ void __launch_bounds__(kT) k_uf(UfKernelArgs args) {
    const ItemTable& tab = args.tab;
    const UfParams& p = args.p;
    Counters* ctr = p.ctr;
    const uint32_t nblocks = gridDim.x;
    const uint32_t gtid = blockIdx.x * kT + threadIdx.x;
    const uint32_t gstride = nblocks * kT;
    // a bounded wait that gave up earlier leaves the sorted keys unreliable
    // non-finite input leaves the forests unreliable: the call fails anyway
    if (ld_acquire_u32(&ctr->status) & (kStTimeout | kStNonfinite)) return;
    uint32_t n = min(*p.d_nkeys, p.cap_keys);
    int cur = 0;
    uint32_t round = 1;
    for (;; ++round) {
        if (gtid == 0 && round <= uint32_t(kTraceRounds)) {
            ctr->trace_active[p.dual][round - 1] = n;
            ctr->trace_t[p.dual][round - 1] = global_timer_ns();
        }
        if (n == 0) break;
        if (gtid == 0) ctr->act_count[round % 3] = 0;
        // ---- phase A: find roots, resolve positives, reserve
        uint32_t hops = 0;
        for (uint32_t j0 = blockIdx.x * kT; j0 < n; j0 += gstride) {
            uint32_t j = j0 + threadIdx.x;
            bool active = j < n;
            bool cross = false;
            uint64_t ckey = 0;
            if (active) {
                uint32_t i, a, b;
                int item = 0;
                if (round == 1) {
                    i = j;
                    uint64_t key = p.keys[i];
                    if (p.dual) key = ~key;
                    endpoints(tab, key, p.dual, a, b, item);
                } else {
                    i = __ldcg(p.act[cur] + j);
                    a = __ldcg(p.na[cur] + j);
                    b = __ldcg(p.nb[cur] + j);
                }
                uint32_t ra, ra_id, rb, rb_id;
                find_two(p.uf, a, b, ra_id, rb_id, ra, rb, hops);
                if (ra == rb) {
                    __stcg(p.ynode + j, kInvalid);
                    // 2D cross-pruning: a positive edge of H0 is a merging facet of the dual
                    if (!p.dual && p.dual_keys) {
                        uint64_t key = p.keys[i];
                        if (tab.it[item_of_vertex(tab, key_vertex(key))].ndim == 2 && (key & 1u)) {
                            cross = true;
                            ckey = ~(key & ~1ull);
                        }
                    }
                } else {
                    uint64_t aa = p.age[ra_id], ab = p.age[rb_id];
                    // H0: the root with the larger key (later vertex) dies; dual: the smaller key dies
                    bool a_young = p.dual ? (aa < ab) : (aa > ab);
                    uint32_t y = a_young ? ra : rb, o = a_young ? rb : ra;
                    uint32_t yr = a_young ? ra_id : rb_id;
                    uint64_t stamp = (uint64_t(round) << 32) | (0xFFFFFFFFu - i);
                    if (aa != ~0ull) reserve(p.res, ra_id, stamp);  // the outside vertex never dies
                    if (ab != ~0ull) reserve(p.res, rb_id, stamp);
                    __stcg(p.ynode + j, y);
                    __stcg(p.onode + j, o);
                    __stcg(p.yrid + j, yr);
                }
                (void)item;
            }
            uint32_t pos = warp_append(p.d_ndual, cross);
            if (cross) {
                if (pos < p.dual_cap) p.dual_keys[pos] = ckey;
                else set_status(ctr, kStCapacity);
            }
        }
        if (round <= uint32_t(kTraceRounds)) {
            uint32_t h = hops;
            for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xFFFFFFFFu, h, o);
            if (lane_id() == 0 && h) atomicAdd(&ctr->trace_hops[p.dual][round - 1], (unsigned long long)h);
        }
        grid_barrier(ctr, nblocks);
        if (gtid == 0 && round <= uint32_t(kTraceRounds)) ctr->trace_ta[p.dual][round - 1] = global_timer_ns();
        // ---- phase B: commit the survivors that hold the reservation of their dying root
        uint32_t* next = p.act[cur ^ 1];
        for (uint32_t j0 = blockIdx.x * kT; j0 < n; j0 += gstride) {
            uint32_t j = j0 + threadIdx.x;
            bool keep = false, emit = false;
            uint32_t i = 0;
            cp_pair pr;
            if (j < n) {
                uint32_t y = __ldcg(p.ynode + j);
                if (y != kInvalid) {
                    i = round == 1 ? j : __ldcg(p.act[cur] + j);
                    uint32_t yr = __ldcg(p.yrid + j);
                    uint64_t stamp = (uint64_t(round) << 32) | (0xFFFFFFFFu - i);
                    if (__ldcg(p.res + yr) == stamp) {
                        __stcg(p.uf + y, __ldcg(p.onode + j));
                        uint64_t key = p.keys[i];
                        if (p.dual) key = ~key;
                        uint32_t vg = key_vertex(key);
                        int item = item_of_vertex(tab, vg);
                        emit_pair(p, tab, key, item, y, yr, &emit, pr);
                    } else {
                        keep = true;
                    }
                }
            }
            uint32_t pos = warp_append(&ctr->act_count[round % 3], keep);
            if (keep) {
                next[pos] = i;
                p.na[cur ^ 1][pos] = __ldcg(p.ynode + j);
                p.nb[cur ^ 1][pos] = __ldcg(p.onode + j);
            }
            uint32_t pp = warp_append(&ctr->n_pairs, emit);
            if (emit) {
                if (pp < p.pair_cap) p.pairs[pp] = pr;
                else set_status(ctr, kStCapacity);
            }
        }
        grid_barrier(ctr, nblocks);
        n = ld_acquire_u32(&ctr->act_count[round % 3]);
        cur ^= 1;
        if (ld_acquire_u32(&ctr->status) & kStTimeout) break;
        if (round > 0x7FFFFFF0u) {
            if (gtid == 0) set_status(ctr, kStInternal);
            break;
        }
    }
    if (gtid == 0) {
        if (p.dual) ctr->roundst = round - 1;
        else ctr->rounds0 = round - 1;
    }
}

int g_uf_blocks = 0;

}  // namespace

cudaError_t launch_uf(const ItemTable& tab, const UfParams& p, cudaStream_t s) {
    if (g_uf_blocks == 0) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_uf, kT, 0);
        if (per_sm <= 0) return cudaErrorLaunchOutOfResources;
        g_uf_blocks = device_sm_count() * per_sm;
    }
    UfKernelArgs args;
    args.tab = tab;
    args.p = p;
    // cooperative launch (all CTAs co-resident, as the grid barrier needs);
    // launched through cudaLaunchKernelEx so that it can also be captured
    // into a CUDA graph
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g_uf_blocks);
    cfg.blockDim = dim3(kT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    note_launches(1);
    return cudaLaunchKernelEx(&cfg, k_uf, args);
}

}  // namespace cp
