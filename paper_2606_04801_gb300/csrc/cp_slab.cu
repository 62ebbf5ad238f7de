// Slab decomposition of the two union-finds (the parallelisation across
// devices that Sec. 6 leaves to future work), on one GPU.
//
// Each root class of the pruned forests belongs to one slab: the slab of the
// vertex its age key names (volumes are cut along z, images along y, into S
// slabs of near-equal extent; the outside vertex belongs to slab 0).  A
// survivor is internal when both endpoint classes lie in one slab, crossing
// otherwise.  Stage 1 runs the elder-rule union-find over the internal
// survivors only: their root classes are disjoint between slabs, so this one
// launch is S independent union-finds (no reservation word is shared by two
// slabs, and each slab's rounds go exactly as they would alone).  Stage 2 runs
// the union-find over what stage 1 hands on and the crossing survivors, in
// filtration order, and writes the remaining pairs.
//
// What stage 1 hands on.  A class of a slab is a boundary class once one of
// its roots is an endpoint of a crossing survivor.  A stage 1 commit whose
// dying class is not a boundary class at that time is final: no survivor
// leads out of that class, so the whole image's union-find sees exactly it
// then, and sees the surviving class inside a class at least as old; the
// same class dies with the same pair.  Stage 1 writes that pair, and nothing
// of the dead class is needed again.  Every other commit goes to stage 2 with
// its endpoints replaced by the two classes' roots at its time (their oldest
// members), since stage 2 does not see the final commits that built those
// classes.  Stage 2 then sees, for every class of the whole image that spans
// slabs, its slab classes' roots joined through the commits and crossing
// survivors in filtration order: its commits and pairs are the whole image's.
// (Without the reduction, stage 1 hands on every commit: a survivor that its
// slab does not commit closes a cycle of earlier survivors, so the whole
// image's union-find, Kruskal's minimum spanning forest with distinct keys,
// does not commit it either.)
//
// A dying class's members at its death all lie in its root's subtree of
// stage 1's links, so "met a crossing survivor" is tested by an upward
// propagation of the endpoint marks through those links.  The subtree can be
// larger: a commit of a later survivor in the same round may link a class
// under a root that an earlier survivor of that round has just killed.  The
// test then errs towards handing a commit on, which is always exact.  For the
// same reason the root a commit records as its surviving side may have died
// earlier in the filtration; the surviving class's root at the commit's time
// is found by following the links whose commits came before it.
//
// The lists are compacted stably (filtration order kept) by a count pass, one
// scan over the per-block counts and a scatter pass.
#include "cp_common.cuh"
#include "cp_grid.cuh"
#include "cp_kernels.h"
#include "cp_pairs.cuh"

namespace cp {
namespace {

constexpr int kST = 1024;                   // threads per CTA
constexpr int kPer = 4;                     // elements per thread in a virtual block
constexpr uint32_t kVB = uint32_t(kST) * kPer;  // elements per virtual block

enum : uint8_t { kFlagInternal = 1, kFlagCrossing = 2, kFlagCommitted = 3 };

// The slab of a root class: of the vertex that its age key names.
__device__ __forceinline__ uint32_t slab_of_root(const ItemTable& tab, const uint64_t* age, uint32_t rid,
                                                 uint32_t n_rids, Counters* ctr, int S) {
    if (!CP_IN(rid, n_rids, ctr)) return 0;
    const uint64_t a = age[rid];
    if (a == ~0ull) return 0;  // an outside vertex
    const uint32_t v = key_vertex(a);
    const Item& it = tab.it[item_of_vertex(tab, v)];
    const int64_t local = int64_t(v) - it.voff;
    const int64_t c = it.ndim == 3 ? local / (int64_t(it.H) * it.W) : local / it.W;
    const int64_t ext = it.ndim == 3 ? it.D : it.H;
    return uint32_t(c * S / ext);
}

// Counts of the two lists (side by side: list 1 starts at slot n0).
__device__ __forceinline__ void list_counts(const SlabArgs& a, uint32_t& n0, uint32_t& n1) {
    n0 = min(*a.d_n[0], a.cap);
    n1 = min(*a.d_n[1], a.cap);
}

// Virtual block vb of the concatenated lists: its list, its first slot in the
// concatenation, and its element range [lo, hi) within its list.
__device__ __forceinline__ void vblock(uint32_t vb, uint32_t n0, uint32_t n1, int& q, uint32_t& jbase, uint32_t& lo,
                                       uint32_t& hi) {
    const uint32_t b0 = (n0 + kVB - 1) / kVB;
    if (vb < b0) {
        q = 0;
        jbase = 0;
        lo = vb * kVB;
        hi = min(n0, lo + kVB);
    } else {
        q = 1;
        jbase = n0;
        lo = (vb - b0) * kVB;
        hi = min(n1, lo + kVB);
    }
}

__device__ __forceinline__ uint32_t n_vblocks(uint32_t n0, uint32_t n1) {
    return (n0 + kVB - 1) / kVB + (n1 + kVB - 1) / kVB;
}

__device__ __forceinline__ bool selected(uint8_t f, int sel) {
    return sel == 0 ? f == kFlagInternal : f >= kFlagCrossing;
}

// Exclusive rank of this thread's predicate among the CTA's threads (thread
// order) and the CTA's total.  Uses sh[0 .. 32].
__device__ __forceinline__ uint32_t cta_rank(bool p, uint32_t* sh, uint32_t& total) {
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const unsigned m = __ballot_sync(0xFFFFFFFFu, p);
    if (lane == 0) sh[warp] = __popc(m);
    __syncthreads();
    if (warp == 0) {
        const uint32_t c = lane < (kST >> 5) ? sh[lane] : 0u;
        uint32_t s = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, s, o);
            if (lane >= unsigned(o)) s += t;
        }
        if (lane < (kST >> 5)) sh[lane] = s - c;
        if (lane == 31) sh[32] = s;
    }
    __syncthreads();
    const uint32_t r = sh[warp] + __popc(m & ((1u << lane) - 1u));
    total = sh[32];
    __syncthreads();  // sh is rewritten by the next call
    return r;
}

// Root counts of the two lists (registered by the pruning pass).
__device__ __forceinline__ void root_counts(const SlabArgs& a, uint32_t& r0, uint32_t& r1) {
    r0 = min(a.ctr->n_r0, a.n_rids[0]);
    r1 = min(a.ctr->n_rt, a.n_rids[1]);
}

__global__ void __launch_bounds__(kST) k_slab_clear(const __grid_constant__ SlabArgs a) {
    uint32_t r0, r1;
    root_counts(a, r0, r1);
    const uint32_t stride = gridDim.x * kST;
    for (uint32_t i = blockIdx.x * kST + threadIdx.x; i < r0; i += stride) a.sub[0][i] = 0;
    for (uint32_t i = blockIdx.x * kST + threadIdx.x; i < r1; i += stride) a.sub[1][i] = 0;
}

// Flags every slot of both lists internal or crossing; marks the endpoint
// classes of the crossing survivors.
__global__ void __launch_bounds__(kST) k_slab_classify(const __grid_constant__ SlabArgs a) {
    Counters* ctr = a.ctr;
    if (ld_acquire_u32(&ctr->status) & (kStTimeout | kStNonfinite)) return;
    uint32_t n0, n1;
    list_counts(a, n0, n1);
    if (uint64_t(n0) + n1 > a.cap) {  // the dual list was not placed after the H0 list
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(ctr, kStCapacity);
        return;
    }
    const uint32_t n = n0 + n1;
    for (uint32_t j0 = blockIdx.x * kST; j0 < n; j0 += gridDim.x * kST) {
        const uint32_t j = j0 + threadIdx.x;
        bool cross = false;
        int q = 0;
        if (j < n) {
            q = j >= n0 ? 1 : 0;
            const uint32_t ra = __ldcg(a.na + j), rb = __ldcg(a.nb + j);
            const uint32_t sa = slab_of_root(a.tab, a.age[q], ra, a.n_rids[q], ctr, a.S);
            const uint32_t sb = slab_of_root(a.tab, a.age[q], rb, a.n_rids[q], ctr, a.S);
            cross = sa != sb;
            a.flag[j] = cross ? kFlagCrossing : kFlagInternal;
            if (cross && CP_IN(ra, a.n_rids[q], ctr) && CP_IN(rb, a.n_rids[q], ctr)) {
                atomicOr(a.sub[q] + ra, 1u);
                atomicOr(a.sub[q] + rb, 1u);
            }
        }
        warp_append(&a.sc->n_cross[0], cross && q == 0);
        warp_append(&a.sc->n_cross[1], cross && q == 1);
    }
}

// Per virtual block: how many of its slots the compaction selects.
__global__ void __launch_bounds__(kST) k_compact_count(const __grid_constant__ SlabArgs a, int sel) {
    if (ld_acquire_u32(&a.ctr->status) & (kStTimeout | kStNonfinite | kStCapacity)) return;
    uint32_t n0, n1;
    list_counts(a, n0, n1);
    const uint32_t nvb = n_vblocks(n0, n1);
    for (uint32_t vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
        int q;
        uint32_t jbase, lo, hi;
        vblock(vb, n0, n1, q, jbase, lo, hi);
        uint32_t cnt = 0;
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            const uint32_t l = lo + uint32_t(r) * kST + threadIdx.x;
            cnt += __syncthreads_count(l < hi && selected(a.flag[jbase + l], sel));
        }
        if (threadIdx.x == 0) a.vcnt[vb] = cnt;
    }
}

// One CTA: the per-block counts become exclusive offsets within each list;
// n_out[q] receives list q's selected total.
__global__ void __launch_bounds__(kST) k_compact_scan(const __grid_constant__ SlabArgs a, uint32_t* n_out) {
    if (ld_acquire_u32(&a.ctr->status) & (kStTimeout | kStNonfinite | kStCapacity)) {
        if (threadIdx.x == 0) n_out[0] = n_out[1] = 0;
        return;
    }
    __shared__ uint32_t sh[33];
    uint32_t n0, n1;
    list_counts(a, n0, n1);
    const uint32_t b0 = (n0 + kVB - 1) / kVB, b1 = (n1 + kVB - 1) / kVB;
    for (int q = 0; q < 2; ++q) {
        const uint32_t first = q ? b0 : 0u, count = q ? b1 : b0;
        uint32_t carry = 0;
        for (uint32_t c0 = 0; c0 < count; c0 += kST) {
            const uint32_t i = c0 + threadIdx.x;
            const uint32_t v = i < count ? a.vcnt[first + i] : 0u;
            // exclusive scan of v over the CTA (warp scans, then the warp totals)
            const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
            uint32_t s = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, s, o);
                if (lane >= unsigned(o)) s += t;
            }
            if (lane == 31) sh[warp] = s;
            __syncthreads();
            if (warp == 0) {
                const uint32_t w = lane < (kST >> 5) ? sh[lane] : 0u;
                uint32_t ws = w;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, ws, o);
                    if (lane >= unsigned(o)) ws += t;
                }
                if (lane < (kST >> 5)) sh[lane] = ws - w;
                if (lane == 31) sh[32] = ws;
            }
            __syncthreads();
            if (i < count) a.vcnt[first + i] = carry + sh[warp] + s - v;
            carry += sh[32];
            __syncthreads();
        }
        if (threadIdx.x == 0) n_out[q] = carry;
    }
}

// The selected slots, in their order, to the output lists: keys of list q to
// ko[q][k]; survivor index, root ids (and the slot, if map is set) to the
// side-by-side active lists at (q ? n_out[0] : 0) + k.
__global__ void __launch_bounds__(kST) k_compact_scatter(const __grid_constant__ SlabArgs a, int sel,
                                                         const uint32_t* n_out) {
    if (ld_acquire_u32(&a.ctr->status) & (kStTimeout | kStNonfinite | kStCapacity)) return;
    __shared__ uint32_t sh[33];
    uint32_t n0, n1;
    list_counts(a, n0, n1);
    const uint32_t nvb = n_vblocks(n0, n1);
    const uint32_t base1 = n_out[0];
    for (uint32_t vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
        int q;
        uint32_t jbase, lo, hi;
        vblock(vb, n0, n1, q, jbase, lo, hi);
        uint32_t k = a.vcnt[vb];
        const uint32_t off = q ? base1 : 0u;
        for (int r = 0; r < kPer; ++r) {
            const uint32_t l = lo + uint32_t(r) * kST + threadIdx.x;
            const bool p = l < hi && selected(a.flag[jbase + l], sel);
            uint32_t total;
            const uint32_t rank = cta_rank(p, sh, total);
            if (p) {
                const uint32_t kk = k + rank;
                a.ko[q][kk] = __ldcg(a.keys[q] + l);
                a.act[off + kk] = kk;
                a.oa[off + kk] = __ldcg(a.na + jbase + l);
                a.ob[off + kk] = __ldcg(a.nb + jbase + l);
                if (a.map) a.map[off + kk] = jbase + l;
            }
            k += total;
        }
    }
}

// After stage 1: bit 1 on every root whose subtree of stage 1's links holds
// an endpoint of a crossing survivor (walks up from each marked root; a walk
// stops where another has passed).
__global__ void __launch_bounds__(kST) k_slab_up(const __grid_constant__ SlabArgs a) {
    Counters* ctr = a.ctr;
    if (ld_acquire_u32(&ctr->status) & (kStTimeout | kStNonfinite | kStCapacity)) return;
    uint32_t r0, r1;
    root_counts(a, r0, r1);
    for (uint32_t g = blockIdx.x * kST + threadIdx.x; g < r0 + r1; g += gridDim.x * kST) {
        const int q = g >= r0 ? 1 : 0;
        uint32_t x = q ? g - r0 : g;
        if (!(__ldcg(a.sub[q] + x) & 1u)) continue;
        const uint64_t t0 = global_timer_ns();
        for (uint32_t hops = 1;; ++hops) {
            if (atomicOr(a.sub[q] + x, 2u) & 2u) break;
            const uint64_t w = __ldcg(a.res[q] + x);
            if ((w & kDead) != kDead) break;  // a root of stage 1's result
            x = uint32_t(w);
            if (!CP_IN(x, a.n_rids[q], ctr)) break;
            if ((hops & 1023u) == 0 && global_timer_ns() - t0 > kWaitLimitNs) {  // only corrupted links get here
                set_status(ctr, kStTimeout);
                break;
            }
        }
    }
}

// After stage 1: the commit index of every root that stage 1 killed.
__global__ void __launch_bounds__(kST) k_slab_died(const __grid_constant__ SlabArgs a) {
    Counters* ctr = a.ctr;
    if (ld_acquire_u32(&ctr->status) & (kStTimeout | kStNonfinite | kStCapacity)) return;
    const uint32_t ni0 = a.sc->n_in[0], n = ni0 + a.sc->n_in[1];
    for (uint32_t k = blockIdx.x * kST + threadIdx.x; k < n; k += gridDim.x * kST) {
        const uint64_t e = __ldcg(a.log + k);
        const int q = k >= ni0 ? 1 : 0;
        if (e != ~0ull && CP_IN(uint32_t(e), a.n_rids[q], ctr)) a.died[q][uint32_t(e)] = q ? k - ni0 : k;
    }
}

// After stage 1: each commit either writes its pair (its dying class met no
// crossing survivor) or is flagged for stage 2 with its classes' roots.
__global__ void __launch_bounds__(kST) k_slab_mark(const __grid_constant__ SlabArgs a) {
    Counters* ctr = a.ctr;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.sc->rounds_slab[0] = ctr->rounds0;
        a.sc->rounds_slab[1] = ctr->roundst;
    }
    if (ld_acquire_u32(&ctr->status) & (kStTimeout | kStNonfinite | kStCapacity)) return;
    const uint32_t ni0 = a.sc->n_in[0], n = ni0 + a.sc->n_in[1];
    for (uint32_t k0 = blockIdx.x * kST; k0 < n; k0 += gridDim.x * kST) {
        const uint32_t k = k0 + threadIdx.x;
        const int q = k >= ni0 ? 1 : 0;
        bool sent = false, emit = false, fin = false;
        cp_pair pr;
        if (k < n) {
            const uint64_t e = __ldcg(a.log + k);
            if (e != ~0ull) {
                const uint32_t y = uint32_t(e), j = __ldcg(a.map + k);
                if (CP_IN(y, a.n_rids[q], ctr) && CP_IN(j, a.cap, ctr)) {
                    const uint32_t kl = q ? k - ni0 : k;
                    if (__ldcg(a.sub[q] + y) & 2u) {
                        // the surviving class's root at this commit: past the
                        // links whose commits came earlier
                        uint32_t o = uint32_t(__ldcg(a.res[q] + y));
                        for (uint32_t hops = 0; hops < a.n_rids[q]; ++hops) {
                            if (!CP_IN(o, a.n_rids[q], ctr)) break;
                            const uint64_t w = __ldcg(a.res[q] + o);
                            if ((w & kDead) != kDead || __ldcg(a.died[q] + o) >= kl) break;
                            o = uint32_t(w);
                        }
                        a.flag[j] = kFlagCommitted;
                        a.na[j] = y;
                        a.nb[j] = o;
                        sent = true;
                    } else {
                        uint64_t key = __ldcg(a.ko[q] + kl);
                        if (q) key = ~key;
                        const int item = item_of_vertex(a.tab, key_vertex(key));
                        emit = commit_pair(a.tab, a.age[q], q, key, item, y, pr);
                        fin = true;
                    }
                }
            }
        }
        warp_append(&a.sc->n_sent[0], sent && q == 0);
        warp_append(&a.sc->n_sent[1], sent && q == 1);
        warp_append(&a.sc->n_final[0], fin && q == 0);
        warp_append(&a.sc->n_final[1], fin && q == 1);
        const uint32_t pp = warp_append(&ctr->n_pairs, emit);
        if (emit) {
            if (pp < a.pair_cap) a.pairs[pp] = pr;
            else set_status(ctr, kStCapacity);
        }
    }
}

// Between the stages: every registered root is a root again.
__global__ void __launch_bounds__(kST) k_slab_reset(const __grid_constant__ SlabArgs a) {
    Counters* ctr = a.ctr;
    const uint32_t r0 = min(ctr->n_r0, a.n_rids[0]), rt = min(ctr->n_rt, a.n_rids[1]);
    const uint32_t stride = gridDim.x * kST;
    for (uint32_t i = blockIdx.x * kST + threadIdx.x; i < r0; i += stride) a.res[0][i] = 0;
    for (uint32_t i = blockIdx.x * kST + threadIdx.x; i < rt; i += stride) a.res[1][i] = 0;
}

int slab_blocks() { return device_sm_count() * 2; }

}  // namespace

uint32_t slab_vblocks_cap(uint32_t cap) { return 2 * ((cap + kVB - 1) / kVB) + 2; }

cudaError_t launch_slab_classify(const SlabArgs& a, cudaStream_t s) {
    k_slab_clear<<<slab_blocks(), kST, 0, s>>>(a);
    k_slab_classify<<<slab_blocks(), kST, 0, s>>>(a);
    note_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_slab_compact(const SlabArgs& a, int sel, uint32_t* n_out, cudaStream_t s) {
    k_compact_count<<<slab_blocks(), kST, 0, s>>>(a, sel);
    k_compact_scan<<<1, kST, 0, s>>>(a, n_out);
    k_compact_scatter<<<slab_blocks(), kST, 0, s>>>(a, sel, n_out);
    note_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_slab_mark(const SlabArgs& a, cudaStream_t s) {
    k_slab_up<<<slab_blocks(), kST, 0, s>>>(a);
    k_slab_died<<<slab_blocks(), kST, 0, s>>>(a);
    k_slab_mark<<<slab_blocks(), kST, 0, s>>>(a);
    k_slab_reset<<<slab_blocks(), kST, 0, s>>>(a);
    note_launches(4);
    return cudaGetLastError();
}

}  // namespace cp
