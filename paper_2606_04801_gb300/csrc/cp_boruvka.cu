// The other union-find design: Borůvka's minimum spanning forest, then the
// elder-rule pairing of its edges alone (a merge tree built in filtration
// order).
//
// With distinct keys the survivors that the sequential elder-rule
// union-find commits are exactly the minimum spanning forest of the survivor
// graph (Kruskal's algorithm), and a survivor that does not commit changes
// nothing; so the union-find over the forest's edges alone gives the same
// pairs (Sec. 4.1 step 3, Sec. 4.2 steps 2-3).  Borůvka finds that forest in
// rounds: every component takes the survivor of smallest sorted index (the
// smallest key) that leaves it, hooks itself along it (of two components
// that take the same survivor the one with the larger id hooks), and the
// hooks are flattened, until no survivor leaves a component.  The dual list
// runs in descending filtration order, which its sorted index already is.
//
// One cooperative launch carries both lists through the rounds (four grid
// barriers per round), in root-id space (the first round's root walks ran
// before the sort).  The forest's edges are then compacted in order and
// paired by the union-find (cp_uf.cu).
#include "cp_common.cuh"
#include "cp_grid.cuh"
#include "cp_kernels.h"

namespace cp {
namespace {

constexpr int kBT = 1024;
constexpr uint32_t kNoEdge = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t find_comp(uint32_t* comp, uint32_t x, Counters* ctr, uint32_t n) {
    uint32_t r = x;
    for (uint32_t hops = 0; hops < n; ++hops) {
        const uint32_t c = __ldcg(comp + r);
        if (c == r) break;
        if (!CP_IN(c, n, ctr)) break;
        r = c;
    }
    return r;
}

__global__ void __launch_bounds__(kBT) k_boruvka(const __grid_constant__ BoruvkaArgs a) {
    Counters* ctr = a.ctr;
    if (ld_acquire_u32(&ctr->status) & (kStTimeout | kStNonfinite)) return;
    const uint32_t n0 = min(*a.d_n[0], a.cap), n1 = min(*a.d_n[1], a.cap);
    const uint32_t r0 = min(ctr->n_r0, a.n_rids[0]), r1 = min(ctr->n_rt, a.n_rids[1]);
    const uint32_t gstride = gridDim.x * kBT, gtid = blockIdx.x * kBT + threadIdx.x;
    uint32_t epoch = 0;
    if (uint64_t(n0) + n1 > a.cap) {  // the dual list was not placed after the H0 list
        if (gtid == 0) set_status(ctr, kStCapacity);
        return;
    }
    // every root its own component; no edge taken yet; every slot active
    for (uint32_t g = gtid; g < r0 + r1; g += gstride) {
        const int q = g >= r0 ? 1 : 0;
        const uint32_t x = q ? g - r0 : g;
        a.comp[q][x] = x;
        a.best[q][x] = kNoEdge;
    }
    uint32_t n = n0 + n1;
    for (uint32_t j = gtid; j < n; j += gstride) {
        a.act[0][j] = j;
        a.flag[j] = 2;  // not (yet) a forest edge
    }
    if (gtid == 0) ctr->act_count[0][0] = ctr->act_count[0][1] = ctr->act_count[0][2] = 0;
    grid_barrier(ctr, gridDim.x, epoch);
    uint32_t rounds = 0;
    for (uint32_t round = 0; n > 0; ++round) {
        const uint32_t* in = a.act[round & 1u];
        uint32_t* out = a.act[(round & 1u) ^ 1u];
        uint32_t* cnt = &ctr->act_count[0][round % 3u];
        if (gtid == 0) ctr->act_count[0][(round + 1u) % 3u] = 0;
        ++rounds;
        // ---- each active survivor that leaves its component bids for the
        // components at both ends
        for (uint32_t k = gtid; k < n; k += gstride) {
            const uint32_t j = __ldcg(in + k);
            const int q = j >= n0 ? 1 : 0;
            const uint32_t i = q ? j - n0 : j, nr = q ? r1 : r0;
            const uint32_t ca = find_comp(a.comp[q], __ldcg(a.na + j), ctr, nr);
            const uint32_t cb = find_comp(a.comp[q], __ldcg(a.nb + j), ctr, nr);
            if (ca != cb) {
                atomicMin(a.best[q] + ca, i);
                atomicMin(a.best[q] + cb, i);
            }
        }
        grid_barrier(ctr, gridDim.x, epoch);
        // ---- the survivors that some component took are forest edges; each
        // component hooks along its own (of a pair that took the same edge,
        // the larger id); the others stay active.  Only representatives'
        // comp words are written, and only here.
        for (uint32_t k0 = blockIdx.x * kBT; k0 < n; k0 += gstride) {
            const uint32_t k = k0 + threadIdx.x;
            bool keep = false;
            uint32_t j = 0;
            if (k < n) {
                j = __ldcg(in + k);
                const int q = j >= n0 ? 1 : 0;
                const uint32_t i = q ? j - n0 : j, nr = q ? r1 : r0;
                const uint32_t ca = find_comp(a.comp[q], __ldcg(a.na + j), ctr, nr);
                const uint32_t cb = find_comp(a.comp[q], __ldcg(a.nb + j), ctr, nr);
                if (ca != cb) {
                    const bool ta = __ldcg(a.best[q] + ca) == i, tb = __ldcg(a.best[q] + cb) == i;
                    if (ta || tb) {
                        a.flag[j] = 1;
                        if (ta && (!tb || ca > cb)) a.hook[q][ca] = cb;
                        if (tb && (!ta || cb > ca)) a.hook[q][cb] = ca;
                    } else {
                        keep = true;
                    }
                }
            }
            const uint32_t pos = warp_append(cnt, keep);
            if (keep) out[pos] = j;
        }
        grid_barrier(ctr, gridDim.x, epoch);
        // ---- apply the hooks, then flatten (each root id to its
        // representative) and clear the bids
        for (uint32_t g = gtid; g < r0 + r1; g += gstride) {
            const int q = g >= r0 ? 1 : 0;
            const uint32_t x = q ? g - r0 : g;
            const uint32_t h = __ldcg(a.hook[q] + x);
            if (h != kNoEdge) {
                a.comp[q][x] = h;
                a.hook[q][x] = kNoEdge;
            }
            a.best[q][x] = kNoEdge;
        }
        grid_barrier(ctr, gridDim.x, epoch);
        for (uint32_t g = gtid; g < r0 + r1; g += gstride) {
            const int q = g >= r0 ? 1 : 0;
            const uint32_t x = q ? g - r0 : g;
            a.comp[q][x] = find_comp(a.comp[q], x, ctr, q ? r1 : r0);
        }
        grid_barrier(ctr, gridDim.x, epoch);
        __shared__ uint32_t sh_n, sh_stop;
        if (threadIdx.x == 0) {
            sh_n = ld_acquire_u32(cnt);
            sh_stop = ld_acquire_u32(&ctr->status) & kStTimeout;
        }
        __syncthreads();
        n = sh_n;
        const bool stop = sh_stop != 0u;
        __syncthreads();
        if (stop) break;
        if (round > 64u) {  // log2 of the root count bounds the rounds
            if (gtid == 0) set_status(ctr, kStInternal);
            break;
        }
    }
    if (gtid == 0) *a.d_rounds = rounds;
}

}  // namespace

cudaError_t launch_boruvka(const BoruvkaArgs& a, cudaStream_t s) {
    const int blocks = device_cached(kCacheBoruvka, [] {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_boruvka, kBT, 0);
        return per_sm > 0 ? device_sm_count() * per_sm : -1;
    });
    if (blocks <= 0) return cudaErrorLaunchOutOfResources;
    // hooks start empty; the kernel leaves them empty
    cudaError_t e = cudaMemsetAsync(a.hook[0], 0xFF, sizeof(uint32_t) * a.n_rids[0], s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.hook[1], 0xFF, sizeof(uint32_t) * a.n_rids[1], s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&a.ctr->bar_count, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kBT);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    note_launches(1);
    return cudaLaunchKernelEx(&cfg, k_boruvka, a);
}

}  // namespace cp
