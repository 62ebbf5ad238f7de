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
constexpr int kKPT = kSortTile / kT;    // keys per thread (16)
constexpr uint32_t kFlagAgg = 1u, kFlagIncl = 2u;
constexpr int kLook = 16;               // look-back window: predecessor tiles read together

__global__ void __launch_bounds__(kT) k_hist(const uint64_t* __restrict__ keys, const uint32_t* d_count, uint32_t cap,
                                             uint32_t* __restrict__ hist, int first_byte, int npasses) {
    __shared__ uint32_t h[8][256];
    for (int i = threadIdx.x; i < 8 * 256; i += kT) (&h[0][0])[i] = 0;
    __syncthreads();
    uint32_t n = min(*d_count, cap);
    for (uint32_t i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT) {
        uint64_t k = keys[i];
        for (int p = 0; p < npasses; ++p) atomicAdd(&h[p][(k >> (8 * (first_byte + p))) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npasses * 256; i += kT) {
        uint32_t v = (&h[0][0])[i];
        if (v) atomicAdd(hist + i, v);
    }
}

// exclusive scan of each pass's 256 digit counts (in place): warp p scans
// pass p, 8 digits per lane, with shuffles (no block barriers)
__global__ void __launch_bounds__(kT) k_hist_scan(uint32_t* hist, int npasses) {
    const int p = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (p >= npasses) return;
    uint32_t* h = hist + p * 256 + lane * 8;
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

__global__ void __launch_bounds__(kT) k_onesweep(const uint64_t* __restrict__ src, uint64_t* __restrict__ dst,
                                                 const uint32_t* __restrict__ vsrc, uint32_t* __restrict__ vdst,
                                                 const uint32_t* d_count, uint32_t cap,
                                                 const uint32_t* __restrict__ digit_off, uint64_t* status,
                                                 uint32_t* tile_ctr, int shift, uint32_t epoch, Counters* ctr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem& sm = *reinterpret_cast<SortSmem*>(smem_raw);
    const uint32_t n = min(*d_count, cap);
    const uint32_t ntiles = (n + kSortTile - 1) / kSortTile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const bool has_vals = vsrc != nullptr;
    for (;;) {
        if (threadIdx.x == 0) sm.tile = atomicAdd(tile_ctr, 1u);
        for (int i = threadIdx.x; i < kWarps * 256; i += kT) (&sm.whist[0][0])[i] = 0;
        __syncthreads();
        const uint32_t tile = sm.tile;
        if (tile >= ntiles) break;
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
                sm.stage[pos] = key[r];
                if (has_vals) sm.vstage[pos] = val[r];
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

int g_sort_blocks = 0;

}  // namespace

size_t sort_status_words(uint32_t cap) { return size_t((cap + kSortTile - 1) / kSortTile + 1) * 256; }

cudaError_t sort_keys(const SortBufs& b, int first_byte, int npasses, uint32_t epoch, cudaStream_t s) {
    if (npasses <= 0 || (npasses & 1) || first_byte + npasses > 8) return cudaErrorInvalidValue;
    const size_t smem = sizeof(SortSmem);
    if (g_sort_blocks == 0) {
        cudaFuncSetAttribute(k_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_onesweep, kT, smem);
        g_sort_blocks = device_sm_count() * (per_sm > 0 ? per_sm : 1);
    }
    cudaError_t e = cudaMemsetAsync(b.hist, 0, sizeof(uint32_t) * 8 * 256, s);
    if (e != cudaSuccess) return e;
    uint32_t max_tiles = (b.cap + kSortTile - 1) / kSortTile;
    int hist_blocks = device_sm_count() * 2;
    k_hist<<<hist_blocks, kT, 0, s>>>(b.keys, b.d_count, b.cap, b.hist, first_byte, npasses);
    k_hist_scan<<<1, kT, 0, s>>>(b.hist, npasses);
    note_launches(2 + npasses);
    int grid = int(max_tiles < uint32_t(g_sort_blocks) ? (max_tiles ? max_tiles : 1) : g_sort_blocks);
    for (int p = 0; p < npasses; ++p) {
        const uint64_t* src = (p & 1) ? b.keys_alt : b.keys;
        uint64_t* dst = (p & 1) ? b.keys : b.keys_alt;
        const uint32_t* vs = b.vals ? ((p & 1) ? b.vals_alt : b.vals) : nullptr;
        uint32_t* vd = b.vals ? ((p & 1) ? b.vals : b.vals_alt) : nullptr;
        k_onesweep<<<grid, kT, smem, s>>>(src, dst, vs, vd, b.d_count, b.cap, b.hist + p * 256, b.status,
                                          b.tile_ctr + p, 8 * (first_byte + p), epoch + uint32_t(p), b.ctr);
    }
    return cudaGetLastError();
}

}  // namespace cp
