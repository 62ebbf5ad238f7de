// Device helpers shared by the kernels that run in rounds over the whole
// grid (the union-finds and the H1 reduction).
#pragma once
#include "cp_common.cuh"

namespace cp {

// Id of an edge or a square of a 3D item from its key (the cell spanned by
// the key's vertex m and stencil offset n): 3 * (global id of its lowest
// corner) + axis, the axis being the edge's direction or the square's normal
// (0: x, 1: y, 2: z).  Edges and squares have separate id spaces.
__host__ __device__ __forceinline__ uint32_t cell_id3(const Item& it, uint64_t key, bool square) {
    int dz, dy, dx;
    stencil_off(3, int(key_low(key)), dz, dy, dx);
    const int64_t corner = int64_t(key_vertex(key)) + (dz < 0 ? -int64_t(it.H) * it.W : 0) +
                           (dy < 0 ? -int64_t(it.W) : 0) + (dx < 0 ? -1 : 0);
    const int axis = square ? (dx == 0 ? 0 : (dy == 0 ? 1 : 2)) : (dx != 0 ? 0 : (dy != 0 ? 1 : 2));
    return uint32_t(3 * corner + axis);
}

// Union-find reservation word of a root that has died: this mark in the
// high half (above every reservation stamp, whose high half is the round)
// and the root id it was linked under in the low half.
constexpr uint64_t kDead = 0xFFFFFFFF00000000ull;

#ifdef __CUDACC__
// Grid-wide barrier for a cooperative launch (all CTAs co-resident): a
// monotonic arrival counter (zeroed before the launch).  Barrier number e of
// the launch is passed when the counter reaches e * nblocks, so it completes
// as soon as the last CTA's arrival lands.  The wait is bounded.
__device__ inline void grid_barrier(Counters* ctr, uint32_t nblocks, uint32_t& epoch) {
    __syncthreads();
    ++epoch;
    if (threadIdx.x == 0) {
        const uint32_t target = epoch * nblocks;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&ctr->bar_count) : "memory");
        if (ld_acquire_u32(&ctr->bar_count) < target) {
            const uint64_t t0 = global_timer_ns();
            while (ld_acquire_u32(&ctr->bar_count) < target) {
                if (global_timer_ns() - t0 > kWaitLimitNs) {
                    set_status(ctr, kStTimeout);
                    break;
                }
            }
        }
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
#endif

}  // namespace cp
