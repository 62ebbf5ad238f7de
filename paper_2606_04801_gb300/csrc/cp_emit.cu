// K4: pair emission (outside vertices, essential class, canonical order) and
// K5: the backward scatter.
#include "cp_common.cuh"
#include "cp_kernels.h"

namespace cp {
namespace {

constexpr int kT = 256;

// One outside vertex per item: the oldest dual vertex (Sec. 3.1), never
// paired (Appendix A.4); it takes dual root id = item index.
__global__ void k_init(ItemTable tab, Counters* ctr, uint32_t* uft, uint64_t* aget, uint64_t* rest) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < tab.n) {
        const Item& it = tab.it[i];
        uft[it.toff + it.T] = kTag | uint32_t(i);
        aget[i] = ~0ull;
        rest[i] = 0;
        ctr->gmin[i] = ~0ull;
    }
    if (i == 0) ctr->n_rt = uint32_t(tab.n);
}

// The essential H0 class of each item: born at its minimum, never dies.
__global__ void k_essential(ItemTable tab, Counters* ctr, cp_pair* pairs, uint32_t cap) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= tab.n) return;
    const Item& it = tab.it[i];
    unsigned long long g = ctr->gmin[i];
    if (g == ~0ull) {
        set_status(ctr, kStInternal);
        return;
    }
    uint32_t v = uint32_t(g & 0xFFFFFFFFu);
    int x = int(v % uint32_t(it.W)), y = int((v / uint32_t(it.W)) % uint32_t(it.H)), z = int(v / uint32_t(it.W * it.H));
    cp_pair p;
    p.birth = ord_float(uint32_t(g >> 32));
    p.death = __int_as_float(0x7F800000);
    p.birth_cell = int32_t(doubled_index(it, z, y, x, 0, 0, 0));
    p.death_cell = -1;
    p.birth_pixel = int32_t(v);
    p.death_pixel = -1;
    p.dim = 0;
    p.item = it.user;
    uint32_t pos = atomicAdd(&ctr->n_pairs, 1u);
    if (pos < cap) pairs[pos] = p;
    else set_status(ctr, kStCapacity);
}

// Canonical order: (item, dim, birth cell).
// Sort key of the canonical output order (item, dim, birth cell), packed in
// as few bits as the call needs: birth cells take cell_bits bits.
__global__ void k_pair_keys(const cp_pair* __restrict__ pairs, const uint32_t* d_n, uint32_t cap,
                            uint64_t* __restrict__ keys, uint32_t* __restrict__ vals, int cell_bits,
                            int dim_bits) {
    uint32_t n = min(*d_n, cap);
    for (uint32_t i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT) {
        const cp_pair& p = pairs[i];
        const uint32_t dc = dim_bits == 1 ? (p.dim > 0 ? 1u : 0u) : uint32_t(p.dim);
        keys[i] = (uint64_t(uint32_t(p.item)) << (cell_bits + dim_bits)) | (uint64_t(dc) << cell_bits) |
                  uint32_t(p.birth_cell);
        vals[i] = i;
    }
}

__global__ void k_gather(const cp_pair* __restrict__ pairs, const uint32_t* __restrict__ vals, const uint32_t* d_n,
                         uint32_t cap, cp_pair* __restrict__ out, int64_t out_cap, int64_t* d_out_count,
                         Counters* ctr) {
    uint32_t n = min(*d_n, cap);
    int64_t m = int64_t(n) < out_cap ? int64_t(n) : out_cap;
    for (int64_t j = int64_t(blockIdx.x) * kT + threadIdx.x; j < m; j += int64_t(gridDim.x) * kT) {
        uint32_t v = vals[j];
        if (v < n) out[j] = pairs[v];  // always true unless a bounded wait gave up
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctr->out_count = int64_t(n);
        if (d_out_count) *d_out_count = int64_t(n);
        if (int64_t(n) > out_cap) set_status(ctr, kStCapacity);
    }
}

__global__ void k_scatter(const cp_pair* __restrict__ pairs, int64_t n, const float* __restrict__ gb,
                          const float* __restrict__ gd, const int64_t* __restrict__ offs, double* acc,
                          int64_t n_pixels) {
    for (int64_t i = int64_t(blockIdx.x) * kT + threadIdx.x; i < n; i += int64_t(gridDim.x) * kT) {
        const cp_pair& p = pairs[i];
        int64_t off = offs ? offs[p.item] : 0;
        if (p.birth_pixel >= 0) {
            int64_t q = off + p.birth_pixel;
            if (q < n_pixels) atomicAdd(acc + q, double(gb[i]));
        }
        if (p.death_pixel >= 0) {
            int64_t q = off + p.death_pixel;
            if (q < n_pixels) atomicAdd(acc + q, double(gd[i]));
        }
    }
}

// Total-persistence loss of the pairs above a persistence threshold and its
// gradient: dL/ddeath = 2 (d - b), dL/dbirth = -2 (d - b).  The loss is summed
// in a fixed order (per-block partials, then one ordered pass), so it is
// identical from run to run.
constexpr int kLossBlocks = 256;

__global__ void __launch_bounds__(kT) k_loss_scatter(const cp_pair* __restrict__ pairs, int64_t n,
                                                     const int64_t* d_n, float tau,
                                                     const int64_t* __restrict__ offs, double* acc, int64_t n_pixels,
                                                     double* partials) {
    __shared__ double red[kT / 32];
    double local = 0.0;
    if (d_n) n = *d_n < n ? *d_n : n;
    for (int64_t i = int64_t(blockIdx.x) * kT + threadIdx.x; i < n; i += int64_t(gridDim.x) * kT) {
        const cp_pair& p = pairs[i];
        if (p.death_pixel < 0) continue;
        double pers = double(p.death) - double(p.birth);
        if (!(pers > double(tau))) continue;
        local += pers * pers;
        int64_t off = offs ? offs[p.item] : 0;
        int64_t qd = off + p.death_pixel, qb = off + p.birth_pixel;
        if (qd < n_pixels) atomicAdd(acc + qd, 2.0 * pers);
        if (qb >= 0 && qb < n_pixels) atomicAdd(acc + qb, -2.0 * pers);
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xFFFFFFFFu, local, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kT / 32; ++w) t += red[w];
        partials[blockIdx.x] = t;
    }
}

__global__ void k_loss_sum(const double* partials, int n, double* loss) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < n; ++i) t += partials[i];
        *loss = t;
    }
}

// Sparse accumulation: only the birth and death pixels of the pairs carry
// gradient, so the accumulators of those pixels alone are cleared, filled and
// rounded; the output is zeroed as a whole first.
__global__ void k_touch_clear(const cp_pair* __restrict__ pairs, int64_t n, const int64_t* d_n,
                              const int64_t* __restrict__ offs, double* acc, int64_t n_pixels) {
    if (d_n) n = *d_n < n ? *d_n : n;
    for (int64_t i = int64_t(blockIdx.x) * kT + threadIdx.x; i < n; i += int64_t(gridDim.x) * kT) {
        const cp_pair& p = pairs[i];
        int64_t off = offs ? offs[p.item] : 0;
        int64_t qb = off + p.birth_pixel, qd = off + p.death_pixel;
        if (p.birth_pixel >= 0 && qb < n_pixels) acc[qb] = 0.0;
        if (p.death_pixel >= 0 && qd < n_pixels) acc[qd] = 0.0;
    }
}

__global__ void k_touch_round(const cp_pair* __restrict__ pairs, int64_t n, const int64_t* d_n,
                              const int64_t* __restrict__ offs, const double* __restrict__ acc,
                              float* __restrict__ grad, int64_t n_pixels) {
    if (d_n) n = *d_n < n ? *d_n : n;
    for (int64_t i = int64_t(blockIdx.x) * kT + threadIdx.x; i < n; i += int64_t(gridDim.x) * kT) {
        const cp_pair& p = pairs[i];
        int64_t off = offs ? offs[p.item] : 0;
        int64_t qb = off + p.birth_pixel, qd = off + p.death_pixel;
        if (p.birth_pixel >= 0 && qb < n_pixels) grad[qb] = float(acc[qb]);
        if (p.death_pixel >= 0 && qd < n_pixels) grad[qd] = float(acc[qd]);
    }
}

int grid_for(int64_t n) {
    int64_t b = (n + kT - 1) / kT;
    int64_t cap = int64_t(device_sm_count()) * 8;
    return int(b < 1 ? 1 : (b > cap ? cap : b));
}

// Test of the bounded-wait path: waits on a word that nothing sets.
__global__ void k_wait_flag(Counters* ctr, const uint32_t* flag, uint64_t limit_ns) {
    if (threadIdx.x == 0) bounded_wait_ne(flag, 0u, ctr, limit_ns);
}

}  // namespace

cudaError_t launch_wait_test(Counters* ctr, const uint32_t* flag, uint64_t limit_ns, cudaStream_t s) {
    k_wait_flag<<<1, 32, 0, s>>>(ctr, flag, limit_ns);
    note_launches(1);
    return cudaGetLastError();
}

int loss_partials() { return kLossBlocks; }

cudaError_t launch_loss_backward(const cp_pair* pairs, int64_t n, const int64_t* d_n, float tau, const int64_t* offs,
                                 double* acc, double* partials, int nparts, double* d_loss, float* grad,
                                 int64_t n_pixels, cudaStream_t s) {
    if (nparts < kLossBlocks) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * size_t(n_pixels), s);
    if (e != cudaSuccess) return e;
    k_touch_clear<<<grid_for(n), kT, 0, s>>>(pairs, n, d_n, offs, acc, n_pixels);
    k_loss_scatter<<<kLossBlocks, kT, 0, s>>>(pairs, n, d_n, tau, offs, acc, n_pixels, partials);
    k_loss_sum<<<1, 32, 0, s>>>(partials, kLossBlocks, d_loss);
    k_touch_round<<<grid_for(n), kT, 0, s>>>(pairs, n, d_n, offs, acc, grad, n_pixels);
    note_launches(4);
    return cudaGetLastError();
}

cudaError_t launch_init(const ItemTable& tab, Counters* ctr, uint32_t* uft, uint64_t* aget, uint64_t* rest,
                        cudaStream_t s) {
    k_init<<<1, kMaxItems, 0, s>>>(tab, ctr, uft, aget, rest);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_essential(const ItemTable& tab, Counters* ctr, cp_pair* pairs, uint32_t cap, cudaStream_t s) {
    k_essential<<<1, kMaxItems, 0, s>>>(tab, ctr, pairs, cap);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pair_keys(const cp_pair* pairs, const uint32_t* d_n, uint32_t cap, uint64_t* keys, uint32_t* vals,
                             int cell_bits, int dim_bits, cudaStream_t s) {
    k_pair_keys<<<grid_for(cap), kT, 0, s>>>(pairs, d_n, cap, keys, vals, cell_bits, dim_bits);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gather(const cp_pair* pairs, const uint32_t* vals, const uint32_t* d_n, uint32_t cap,
                          cp_pair* out, int64_t out_cap, int64_t* d_out_count, Counters* ctr, cudaStream_t s) {
    k_gather<<<grid_for(cap), kT, 0, s>>>(pairs, vals, d_n, cap, out, out_cap, d_out_count, ctr);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_backward(const cp_pair* pairs, int64_t n, const float* gb, const float* gd, const int64_t* offs,
                            double* acc, float* grad, int64_t n_pixels, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * size_t(n_pixels), s);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        k_touch_clear<<<grid_for(n), kT, 0, s>>>(pairs, n, nullptr, offs, acc, n_pixels);
        k_scatter<<<grid_for(n), kT, 0, s>>>(pairs, n, gb, gd, offs, acc, n_pixels);
        k_touch_round<<<grid_for(n), kT, 0, s>>>(pairs, n, nullptr, offs, acc, grad, n_pixels);
        note_launches(3);
    }
    return cudaGetLastError();
}

}  // namespace cp
