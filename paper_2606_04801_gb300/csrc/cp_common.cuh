// Internal definitions shared by the sm_103a kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/cubical_persistence.h"

namespace cp {

// ---------------------------------------------------------------- limits
constexpr int kVBits = 27;                        // global vertex id bits in a key
constexpr uint64_t kVMask = (1ull << kVBits) - 1;
constexpr uint32_t kTag = 0x80000000u;            // union-find word: root tag | root id
constexpr int kMaxItems = CP_MAX_ITEMS;

// status bits (device word)
constexpr uint32_t kStNonfinite = 1u << 0;
constexpr uint32_t kStCapacity = 1u << 1;
constexpr uint32_t kStTimeout = 1u << 2;
constexpr uint32_t kStInternal = 1u << 3;
constexpr uint32_t kStBounds = 1u << 4;   // bounds-checked build: a data-dependent index was out of range

// ---------------------------------------------------------------- items
// One image or volume of a call.  2D items have D = 1.  Vertices of item i
// have global ids voff + local id; its top cells have global ids toff + local
// id (local id of the top cell whose smallest corner is (z, y, x) is
// (z*(H-1) + y)*(W-1) + x, z = 0 in 2D), and its outside vertex is toff + T.
struct Item {
    const float* img;
    int32_t ndim, D, H, W;
    int64_t voff, toff, T;
    int32_t tile0;            // first pruning tile of the item (per kind)
    int32_t tx, ty, tz;       // pruning tiles along x, y, z
    int32_t user;             // the caller's index of the item
    int32_t tma;              // 3D: index of the item's plane tensor map (TMA loads), or -1
};

struct ItemTable {
    int32_t n;
    int32_t n2d, n3d;         // items 0..n2d-1 are 2D, n2d..n-1 are 3D
    int32_t tiles2d, tiles3d; // total pruning tiles of each kind
    int32_t rows2d;           // vertex rows per 2D pruning task (4 .. 4096)
    int32_t zchunk3d;         // planes per 3D pruning task
    int32_t cross2d;          // 2D items: 1 = the dual list waits for H0 (cross-pruning), 0 = both at once
    Item it[kMaxItems];
};

// ---------------------------------------------------------------- counters
// Lives at the start of the workspace.  Zeroed at the start of every call.
struct Counters {
    uint32_t status;
    uint32_t n_s0;            // H0 survivors appended
    uint32_t n_st;            // dual survivors appended
    uint32_t n_r0;            // H0 roots registered
    uint32_t n_rt;            // dual roots registered
    uint32_t n_pairs;         // pairs appended by the union-finds
    uint32_t rounds0, roundst;
    uint32_t bar_count, bar_gen;
    uint32_t act_count[2][3]; // active survivors of the next round (H0 / dual list), rotating
    uint32_t sort_tile[64];   // tile tickets of the sort passes of one call
    uint32_t find_ctr;        // work counter of the first union-find round's root walks
    uint32_t tma_tasks;       // 3D pruning tasks whose planes came by TMA (a check that the path runs)
    uint32_t t_keep;          // T-filtration calls: pairs kept after the mapping (the output count)
    uint32_t mst_rounds;      // Borůvka rounds (the spanning-forest union-find variant), else 0
    unsigned long long gmin[kMaxItems];  // (ord bits << 32 | local vertex) of each item's minimum
    int64_t out_count;
    // union-find trace: active survivors and device time at the start of each
    // of the first kTraceRounds rounds (H0, dual)
    uint32_t trace_active[2][48];
    unsigned long long trace_t[2][48];
    unsigned long long trace_ta[2][48];   // end of phase A
    unsigned long long trace_hops[2][48]; // parent hops walked in phase A
};
constexpr int kTraceRounds = 48;

// ---------------------------------------------------------------- order keys
// Order-preserving bits of a finite float: a < b as floats <=> ord(a) < ord(b)
// as unsigned integers; -0.0 and +0.0 map to the same value.
__host__ __device__ __forceinline__ uint32_t ord_bits(float f) {
    uint32_t b;
#ifdef __CUDA_ARCH__
    b = __float_as_uint(f);
#else
    __builtin_memcpy(&b, &f, 4);
#endif
    if ((b << 1) == 0) b = 0;
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__host__ __device__ __forceinline__ float ord_float(uint32_t u) {
    uint32_t b = (u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u;
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float f;
    __builtin_memcpy(&f, &b, 4);
    return f;
#endif
}

// Survivor / age key: ord(f(v)) << 32 | v << 5 | low.  `low` orders the cells
// of one lower star (second-order tie-break): the stencil bit n in 3D, n << 1
// in 2D (| 1 on an H0 survivor whose dual status waits for the H0 union-find,
// under cross-pruning).
__host__ __device__ __forceinline__ uint64_t make_key(uint32_t ord, uint64_t v, uint32_t low) {
    return (uint64_t(ord) << 32) | (v << 5) | low;
}
__host__ __device__ __forceinline__ uint32_t key_vertex(uint64_t k) { return uint32_t((k >> 5) & kVMask); }
__host__ __device__ __forceinline__ uint32_t key_low(uint64_t k) { return uint32_t(k & 31u); }
__host__ __device__ __forceinline__ uint32_t key_n(uint64_t k, int ndim) {
    return ndim == 3 ? key_low(k) : (key_low(k) >> 1);
}

// Offset (dz, dy, dx) of stencil bit n.
__host__ __device__ __forceinline__ void stencil_off(int ndim, int n, int& dz, int& dy, int& dx) {
    if (ndim == 3) {
        dz = n / 9 - 1;
        dy = (n / 3) % 3 - 1;
        dx = n % 3 - 1;
    } else {
        dz = 0;
        dy = n / 3 - 1;
        dx = n % 3 - 1;
    }
}

__host__ __device__ __forceinline__ int item_of_vertex(const ItemTable& t, uint32_t v) {
    int lo = 0, hi = t.n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (t.it[mid].voff <= int64_t(v)) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Doubled-grid index of the cell spanned by local vertex (z, y, x) and
// offset (dz, dy, dx) in {-1, 0, 1}^3.
__host__ __device__ __forceinline__ int64_t doubled_index(const Item& it, int z, int y, int x, int dz, int dy,
                                                          int dx) {
    int64_t GH = 2 * it.H - 1, GW = 2 * it.W - 1;
    return (int64_t(2 * z + dz) * GH + (2 * y + dy)) * GW + (2 * x + dx);
}

// Top cell (global id, or the item's outside vertex) in octant (sz, sy, sx)
// (each +-1; sz ignored in 2D) of local vertex (z, y, x).
__host__ __device__ __forceinline__ uint32_t top_of_octant(const Item& it, int z, int y, int x, int sz, int sy,
                                                           int sx) {
    int cz = it.ndim == 3 ? z + (sz < 0 ? -1 : 0) : 0;
    int cy = y + (sy < 0 ? -1 : 0);
    int cx = x + (sx < 0 ? -1 : 0);
    bool out = cy < 0 || cy >= it.H - 1 || cx < 0 || cx >= it.W - 1 ||
               (it.ndim == 3 && (cz < 0 || cz >= it.D - 1));
    if (out) return uint32_t(it.toff + it.T);
    return uint32_t(it.toff + (int64_t(cz) * (it.H - 1) + cy) * (it.W - 1) + cx);
}

// ---------------------------------------------------------------- device utils
#ifdef __CUDACC__
__device__ __forceinline__ void set_status(Counters* c, uint32_t bit) { atomicOr(&c->status, bit); }

// CP_IN(i, n, ctr): in the bounds-checked build (-DCP_CHECKED), true when the
// data-dependent index i lies in [0, n), else the call is flagged
// (kStBounds) and the caller skips the access; in the normal build, true.
#ifdef CP_CHECKED
__device__ __forceinline__ bool cp_in_checked(uint64_t i, uint64_t n, Counters* c) {
    if (i < n) return true;
    set_status(c, kStBounds);
    return false;
}
#define CP_IN(i, n, ctr) ::cp::cp_in_checked(uint64_t(i), uint64_t(n), (ctr))
#else
#define CP_IN(i, n, ctr) true
#endif

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
// Relaxed (unordered) load at GPU scope: several can be in flight at once.
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_u64(uint64_t* p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Bounded waits give up after this many nanoseconds of wall time and set
// kStTimeout; the work that depended on them is then invalid but every
// thread still terminates.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Waits until *p != v, for at most limit_ns of wall time.  Returns false
// (and sets kStTimeout) when it gave up; the caller then carries on, its
// result flagged invalid, so every thread terminates.
__device__ __forceinline__ bool bounded_wait_ne(const uint32_t* p, uint32_t v, Counters* ctr, uint64_t limit_ns) {
    const uint64_t t0 = global_timer_ns();
    while (ld_acquire_u32(p) == v) {
        if (global_timer_ns() - t0 > limit_ns) {
            set_status(ctr, kStTimeout);
            return false;
        }
        __nanosleep(20);
    }
    return true;
}
#endif

}  // namespace cp
