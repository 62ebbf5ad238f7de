// K2: LSD radix sort of 64-bit keys (optional 32-bit payload), 8-bit
// digits, one kernel per digit pass with decoupled look-back ("onesweep").
//
// The filtration order of the survivors (Sec. 2.3) is a total order on
// their 64-bit keys, so sorting the keys orders the union-find input
// (ascending for H0; the dual keys are stored complemented, so ascending
// order of the stored words is the reversed filtration order, Sec. 3.1).
//
// The number of keys lives on the device; every kernel runs a fixed grid and
// takes tiles from a ticket counter, so no host round trip is needed.  Tiles
// are ranked in ticket order, which makes the look-back wait only on tiles
// that already run: every wait ends.  Each wait is still bounded in wall
// time and reports kStTimeout when it gives up.
#include "cp_common.cuh"
#include "cp_kernels.h"

namespace cp {
namespace {

constexpr int kT = 256;                 // threads per CTA
constexpr int kWarps = kT / 32;
constexpr int kKPT = kSortTile / kT;    // keys per thread (8)
constexpr uint32_t kFlagAgg = 1u, kFlagIncl = 2u;
constexpr int kLook = 16;               // look-back window: predecessor tiles read together

// Digit histograms of every pass, for one or two key lists, from one read;
// also clears the look-back words the passes will use.
struct HistArgs {
    const uint64_t* keys[2];
    const uint32_t* d_count[2];
    uint32_t cap[2];
    uint32_t* hist[2];        // npasses x 256 per list
    uint64_t* status[2];      // look-back words: the ones this sort will use are cleared here
    int nl, first_byte, npasses;
};

__global__ void __launch_bounds__(kT) k_hist(const __grid_constant__ HistArgs a) {
    __shared__ uint32_t h[8][256];
    for (int l = 0; l < a.nl; ++l) {
        for (int i = threadIdx.x; i < 8 * 256; i += kT) (&h[0][0])[i] = 0;
        __syncthreads();
        const uint32_t n = min(*a.d_count[l], a.cap[l]);
        const uint64_t* keys = a.keys[l];
        const uint32_t nwords = (n + kSortTile - 1) / kSortTile * 256u;
        for (uint32_t i = blockIdx.x * kT + threadIdx.x; i < nwords; i += gridDim.x * kT) a.status[l][i] = 0ull;
        for (uint32_t i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT) {
            const uint64_t k = keys[i];
            for (int p = 0; p < a.npasses; ++p) atomicAdd(&h[p][(k >> (8 * (a.first_byte + p))) & 255u], 1u);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < a.npasses * 256; i += kT) {
            const uint32_t v = (&h[0][0])[i];
            if (v) atomicAdd(a.hist[l] + i, v);
        }
        __syncthreads();
    }
}

// exclusive scan of each pass's 256 digit counts (in place): one warp per
// (list, pass), 8 digits per lane, with shuffles (no block barriers)
__global__ void __launch_bounds__(512) k_hist_scan(uint32_t* hist0, uint32_t* hist1, int npasses, int nl) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w >= npasses * nl) return;
    uint32_t* h = (w >= npasses ? hist1 : hist0) + (w % npasses) * 256 + lane * 8;
    uint32_t v[8], sum = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        v[k] = h[k];
        sum += v[k];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    uint32_t run = incl - sum;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        h[k] = run;
        run += v[k];
    }
}

__device__ __forceinline__ uint64_t pack_status(uint32_t epoch, uint32_t flag, uint32_t count) {
    return (uint64_t(epoch) << 34) | (uint64_t(flag) << 32) | count;
}

struct SortSmem {
    uint32_t whist[kWarps][256];   // per-warp digit counts, then warp offsets
    uint32_t excl[256];            // tile-local exclusive offset per digit
    uint32_t glob[256];            // global offset of the tile's first key of each digit
    uint32_t scan[256];
    uint64_t stage[kSortTile];
    uint32_t vstage[kSortTile];
    uint32_t tile;
};

// One digit pass over one or two key lists: tickets [0, tiles of list 0) are
// list 0's tiles, the next ones list 1's, so a pass over both lists is one
// launch (a pass is latency-bound at these sizes).
struct SortList {
    const uint64_t* src;
    uint64_t* dst;
    const uint32_t* vsrc;   // payload (nullptr: keys only)
    uint32_t* vdst;
    const uint32_t* d_count;
    uint32_t cap;
    const uint32_t* digit_off;  // this pass's exclusive digit offsets
    uint64_t* status;           // look-back words of this list
};
struct SweepArgs {
    SortList l[2];
    int nl;
    uint32_t* tile_ctr;
    int shift;
    uint32_t epoch;
    Counters* ctr;
};

__global__ void __launch_bounds__(kT) k_onesweep(const __grid_constant__ SweepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem& sm = *reinterpret_cast<SortSmem*>(smem_raw);
    const uint32_t n0 = min(*a.l[0].d_count, a.l[0].cap);
    const uint32_t n1 = a.nl > 1 ? min(*a.l[1].d_count, a.l[1].cap) : 0u;
    const uint32_t nt0 = (n0 + kSortTile - 1) / kSortTile, nt1 = (n1 + kSortTile - 1) / kSortTile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int shift = a.shift;
    const uint32_t epoch = a.epoch;
    for (;;) {
        if (threadIdx.x == 0) sm.tile = atomicAdd(a.tile_ctr, 1u);
        for (int i = threadIdx.x; i < kWarps * 256; i += kT) (&sm.whist[0][0])[i] = 0;
        __syncthreads();
        const uint32_t ticket = sm.tile;
        if (ticket >= nt0 + nt1) break;
        const int li = ticket >= nt0 ? 1 : 0;
        const SortList& L = a.l[li];
        const uint32_t tile = li ? ticket - nt0 : ticket;
        const uint32_t n = li ? n1 : n0;
        const uint64_t* __restrict__ src = L.src;
        uint64_t* __restrict__ dst = L.dst;
        const uint32_t* __restrict__ vsrc = L.vsrc;
        uint32_t* __restrict__ vdst = L.vdst;
        uint64_t* status = L.status;
        const uint32_t* __restrict__ digit_off = L.digit_off;
        Counters* ctr = a.ctr;
        const bool has_vals = vsrc != nullptr;
        const uint32_t base = tile * kSortTile;
        uint64_t key[kKPT];
        uint32_t val[kKPT];
        uint32_t rank[kKPT];
#pragma unroll
        for (int r = 0; r < kKPT; ++r) {
            uint32_t idx = base + warp * (32 * kKPT) + r * 32 + lane;
            key[r] = idx < n ? src[idx] : ~0ull;
            val[r] = (has_vals && idx < n) ? vsrc[idx] : 0u;
        }
        // stable warp-local ranking, 32 keys at a time in input order
#pragma unroll
        for (int r = 0; r < kKPT; ++r) {
            uint32_t idx = base + warp * (32 * kKPT) + r * 32 + lane;
            uint32_t d = idx < n ? uint32_t(key[r] >> shift) & 255u : 256u;
            unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
            int leader = __ffs(peers) - 1;
            uint32_t b = 0;
            if (lane == leader && d < 256u) {
                b = sm.whist[warp][d];
                sm.whist[warp][d] = b + __popc(peers);
            }
            b = __shfl_sync(0xFFFFFFFFu, b, leader);
            rank[r] = b + __popc(peers & lt_mask);
            __syncwarp();
        }
        __syncthreads();
        // per digit: warp offsets and the tile count
        const uint32_t d = threadIdx.x;
        uint32_t cnt = 0;
        for (int w = 0; w < kWarps; ++w) {
            uint32_t c = sm.whist[w][d];
            sm.whist[w][d] = cnt;
            cnt += c;
        }
        // publish this tile's aggregate, then look back
        uint64_t* my = status + size_t(tile) * 256 + d;
        st_release_u64(my, pack_status(epoch, kFlagAgg, cnt));
        // Look back over windows of kLook predecessors whose status words are
        // read together (relaxed loads: the counts are in the words themselves,
        // nothing else is read through them), summing aggregates until an
        // inclusive prefix: a round trip per window, not per tile.
        uint32_t prefix = 0;
        bool timed_out = false;
        uint64_t t0 = 0;
        for (int64_t j = int64_t(tile) - 1; j >= 0 && !timed_out; j -= kLook) {
            uint64_t w[kLook];
#pragma unroll
            for (int k = 0; k < kLook; ++k)
                w[k] = j - k >= 0 ? ld_relaxed_u64(status + size_t(j - k) * 256 + d) : 0ull;
            bool done = false;
#pragma unroll
            for (int k = 0; k < kLook; ++k) {
                if (!done && !timed_out && j - k >= 0) {
                    uint64_t v = w[k];
                    // a predecessor that has not published yet (this epoch): wait for it
                    while (uint32_t(v >> 34) != epoch || ((v >> 32) & 3u) == 0u) {
                        if (t0 == 0) t0 = global_timer_ns();
                        else if (global_timer_ns() - t0 > kWaitLimitNs) {
                            timed_out = true;
                            break;
                        }
                        __nanosleep(32);
                        v = ld_relaxed_u64(status + size_t(j - k) * 256 + d);
                    }
                    if (!timed_out) {
                        prefix += uint32_t(v);
                        done = ((v >> 32) & 3u) == kFlagIncl;
                    }
                }
            }
            if (done) break;
        }
        if (timed_out) set_status(ctr, kStTimeout);
        st_release_u64(my, pack_status(epoch, kFlagIncl, prefix + cnt));
        sm.glob[d] = digit_off[d] + prefix;
        // tile-local exclusive scan over digits
        sm.scan[d] = cnt;
        __syncthreads();
        for (int o = 1; o < 256; o <<= 1) {
            uint32_t t = d >= unsigned(o) ? sm.scan[d - o] : 0u;
            __syncthreads();
            sm.scan[d] += t;
            __syncthreads();
        }
        sm.excl[d] = sm.scan[d] - cnt;
        __syncthreads();
        // place keys in tile-local sorted order
#pragma unroll
        for (int r = 0; r < kKPT; ++r) {
            uint32_t idx = base + warp * (32 * kKPT) + r * 32 + lane;
            if (idx < n) {
                uint32_t dd = uint32_t(key[r] >> shift) & 255u;
                uint32_t pos = sm.excl[dd] + sm.whist[warp][dd] + rank[r];
                if (CP_IN(pos, kSortTile, ctr)) {
                    sm.stage[pos] = key[r];
                    if (has_vals) sm.vstage[pos] = val[r];
                }
            }
        }
        __syncthreads();
        const uint32_t nv = min(uint32_t(kSortTile), n - base);
        for (uint32_t i = threadIdx.x; i < nv; i += kT) {
            uint64_t k = sm.stage[i];
            uint32_t dd = uint32_t(k >> shift) & 255u;
            uint32_t out = sm.glob[dd] + (i - sm.excl[dd]);
            if (out < n) {  // always true unless a bounded wait gave up
                dst[out] = k;
                if (has_vals) vdst[out] = sm.vstage[i];
            }
        }
        __syncthreads();
    }
}

}  // namespace

size_t sort_status_words(uint32_t cap) { return size_t((cap + kSortTile - 1) / kSortTile + 1) * 256; }

cudaError_t sort_keys_multi(const SortBufs* b, int nl, int first_byte, int npasses, uint32_t epoch, cudaStream_t s) {
    if (nl < 1 || nl > 2 || npasses <= 0 || (npasses & 1) || first_byte + npasses > 8) return cudaErrorInvalidValue;
    const size_t smem = sizeof(SortSmem);
    const int sort_blocks = device_cached(kCacheSort, [] {
        cudaFuncSetAttribute(k_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sizeof(SortSmem)));
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_onesweep, kT, sizeof(SortSmem));
        return device_sm_count() * (per_sm > 0 ? per_sm : 1);
    });
    HistArgs h;
    uint32_t max_tiles = 0;
    for (int l = 0; l < 2; ++l) {
        const SortBufs& q = b[l < nl ? l : 0];
        h.keys[l] = q.keys;
        h.d_count[l] = q.d_count;
        h.cap[l] = q.cap;
        h.hist[l] = q.hist;
        h.status[l] = q.status;
    }
    h.nl = nl;
    h.first_byte = first_byte;
    h.npasses = npasses;
    for (int l = 0; l < nl; ++l) {
        cudaError_t e = cudaMemsetAsync(b[l].hist, 0, sizeof(uint32_t) * 8 * 256, s);
        if (e != cudaSuccess) return e;
        max_tiles += (b[l].cap + kSortTile - 1) / kSortTile;
    }
    k_hist<<<device_sm_count() * 2, kT, 0, s>>>(h);
    k_hist_scan<<<1, 512, 0, s>>>(b[0].hist, nl > 1 ? b[1].hist : b[0].hist, npasses, nl);
    note_launches(2 + npasses);
    const int grid = int(max_tiles < uint32_t(sort_blocks) ? (max_tiles ? max_tiles : 1) : sort_blocks);
    for (int p = 0; p < npasses; ++p) {
        SweepArgs a;
        for (int l = 0; l < 2; ++l) {
            const SortBufs& q = b[l < nl ? l : 0];
            a.l[l].src = (p & 1) ? q.keys_alt : q.keys;
            a.l[l].dst = (p & 1) ? q.keys : q.keys_alt;
            a.l[l].vsrc = q.vals ? ((p & 1) ? q.vals_alt : q.vals) : nullptr;
            a.l[l].vdst = q.vals ? ((p & 1) ? q.vals : q.vals_alt) : nullptr;
            a.l[l].d_count = q.d_count;
            a.l[l].cap = q.cap;
            a.l[l].digit_off = q.hist + p * 256;
            a.l[l].status = q.status;
        }
        a.nl = nl;
        a.tile_ctr = b[0].tile_ctr + p;
        a.shift = 8 * (first_byte + p);
        a.epoch = epoch + uint32_t(p);
        a.ctr = b[0].ctr;
        k_onesweep<<<grid, kT, smem, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t sort_keys(const SortBufs& b, int first_byte, int npasses, uint32_t epoch, cudaStream_t s) {
    return sort_keys_multi(&b, 1, first_byte, npasses, epoch, s);
}

}  // namespace cp
