// K1: fused lookup + local pruning (Sec. 3.2, Sec. 3.3, Sec. 4.1 steps 1-2,
// Sec. 4.2 steps 1-3 before the union-finds).
//
// One CTA per tile of vertices.  The tile and a one-vertex halo are staged
// in shared memory (out-of-image halo = +inf, so such neighbours never
// precede the centre and no bounds test is needed).  Per vertex v:
//   1. 8/26-bit mask of the neighbours that precede v (value, then index);
//   2. collapse to the relevant mask and look it up (2D: direct 256-entry
//      table; 3D: perfect hash of the 15,935 relevant masks);
//   3. write the H0 forest parent of v (first edge of L(v)) or register v as
//      an H0 root (local minimum);
//   4. write the dual forest parent of every top cell of L(v) (the top cell
//      across the facet where it dies locally, or the outside vertex) or
//      register it as a dual root;
//   5. emit the surviving edges and facets as 64-bit order keys.
// Survivors and roots are staged per CTA in shared memory and appended to
// global arrays with one atomic per buffer per flush.
#include "cp_common.cuh"
#include "cp_kernels.h"

namespace cp {

__constant__ uint64_t c_lut2d[256];
__constant__ uint16_t c_disp3d[1 << 12];
__device__ uint64_t g_entries3d[1 << 14];  // perfect-hash slots of the 3D table (128 KB)

// slot -> stencil bit tables
__constant__ int8_t c_face_n3[6] = {4, 10, 12, 14, 16, 22};
__constant__ int8_t c_facet_n3[12] = {1, 3, 5, 7, 9, 11, 15, 17, 19, 21, 23, 25};
__constant__ int8_t c_top_n3[8] = {0, 2, 6, 8, 18, 20, 24, 26};
__constant__ int8_t c_face_n2[4] = {1, 3, 5, 7};
__constant__ int8_t c_top_n2[4] = {0, 2, 6, 8};

namespace {

constexpr int kBX = 32, kBY = 8;          // CTA shape
constexpr int kThreads = kBX * kBY;
constexpr int kCapS = 4096;               // staged survivor keys per kind
constexpr int kCapR = 1024;               // staged roots per kind

struct Stage {
    uint64_t s0[kCapS];
    uint64_t st[kCapS];
    uint64_t r0age[kCapR];
    uint64_t rtage[kCapR];
    uint32_t r0node[kCapR];
    uint32_t rtnode[kCapR];
    uint32_t n_s0, n_st, n_r0, n_rt;
    uint32_t base_s0, base_st, base_r0, base_rt;
    unsigned long long gmin;
};

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
};

// warp-aggregated reservation of `k` slots in a shared-memory buffer
__device__ __forceinline__ uint32_t stage_reserve(uint32_t* counter, uint32_t k) {
    unsigned lane = lane_id();
    uint32_t incl = k;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= unsigned(o)) incl += t;
    }
    uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    uint32_t base = 0;
    if (lane == 31 && total) base = atomicAdd(counter, total);
    base = __shfl_sync(0xFFFFFFFFu, base, 31);
    return base + incl - k;
}

__device__ void flush(Stage& sg, const Outs& o) {
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        sg.base_s0 = sg.n_s0 ? atomicAdd(&o.ctr->n_s0, sg.n_s0) : 0;
        sg.base_st = sg.n_st ? atomicAdd(&o.ctr->n_st, sg.n_st) : 0;
        sg.base_r0 = sg.n_r0 ? atomicAdd(&o.ctr->n_r0, sg.n_r0) : 0;
        sg.base_rt = sg.n_rt ? atomicAdd(&o.ctr->n_rt, sg.n_rt) : 0;
    }
    __syncthreads();
    const int tid = threadIdx.y * kBX + threadIdx.x;
    for (uint32_t i = tid; i < sg.n_s0; i += kThreads) {
        uint32_t g = sg.base_s0 + i;
        if (g < o.cap_s) o.s0[g] = sg.s0[i];
    }
    for (uint32_t i = tid; i < sg.n_st; i += kThreads) {
        uint32_t g = sg.base_st + i;
        if (g < o.cap_s) o.st[g] = sg.st[i];
    }
    for (uint32_t i = tid; i < sg.n_r0; i += kThreads) {
        uint32_t g = sg.base_r0 + i;
        if (g < o.cap_r0) {
            o.age0[g] = sg.r0age[i];
            o.res0[g] = 0;
            o.uf0[sg.r0node[i]] = kTag | g;
        } else {
            o.uf0[sg.r0node[i]] = kTag;  // out of capacity: keep the forest well formed (result flagged invalid)
        }
    }
    for (uint32_t i = tid; i < sg.n_rt; i += kThreads) {
        uint32_t g = sg.base_rt + i;
        if (g < o.cap_rt) {
            o.aget[g] = sg.rtage[i];
            o.rest[g] = 0;
            o.uft[sg.rtnode[i]] = kTag | g;
        } else {
            o.uft[sg.rtnode[i]] = kTag;
        }
    }
    if (tid == 0) {
        bool over = (sg.n_s0 && sg.base_s0 + sg.n_s0 > o.cap_s) || (sg.n_st && sg.base_st + sg.n_st > o.cap_s) ||
                    (sg.n_r0 && sg.base_r0 + sg.n_r0 > o.cap_r0) || (sg.n_rt && sg.base_rt + sg.n_rt > o.cap_rt);
        if (over) set_status(o.ctr, kStCapacity);
    }
    __syncthreads();
    if (tid == 0) sg.n_s0 = sg.n_st = sg.n_r0 = sg.n_rt = 0;
    __syncthreads();
}

// A non-finite pixel flags the call as failed and is read as the largest
// finite float, so the order stays total and every cell still lies in exactly
// one lower star (the forests stay well formed even though the result is
// discarded).  The +inf halo stays above every pixel.
__device__ __forceinline__ float load_finite(const float* p, Counters* ctr) {
    float v = __ldg(p);
    if (!isfinite(v)) {
        set_status(ctr, kStNonfinite);
        v = 3.40282347e38f;
    }
    return v;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(0xFFFFFFFFu, v, o);
        v = t < v ? t : v;
    }
    return v;
}

// Emit everything one vertex contributes, given its lookup entry.
// (z, y, x): local coordinates; vg: global vertex id; valid: vertex exists.
template <int NDIM>
__device__ __forceinline__ void emit_vertex(Stage& sg, const Outs& o, const Item& it, bool valid, int z, int y,
                                            int x, uint32_t vg, uint32_t ord, uint64_t e,
                                            unsigned long long& my_min) {
    // ---- H0 forest parent / root
    int direct = valid ? int(e & 7u) : 0;
    bool root0 = valid && direct == 7;
    if (valid && !root0) {
        int n = NDIM == 3 ? c_face_n3[direct] : c_face_n2[direct];
        int dz, dy, dx;
        stencil_off(NDIM, n, dz, dy, dx);
        o.uf0[vg] = uint32_t(int64_t(vg) + (int64_t(dz) * it.H + dy) * it.W + dx);
    }
    if (root0) {
        unsigned long long k = (unsigned long long)(uint64_t(ord) << 32 | uint32_t(vg - it.voff));
        my_min = k < my_min ? k : my_min;
    }
    uint32_t h0s = valid ? uint32_t((e >> 3) & 0x3Fu) : 0u;
    uint32_t ds = valid ? uint32_t((e >> 41) & 0xFFFu) : 0u;
    // ---- dual forest parents / dual root
    int rt_node = -1;
    uint64_t rt_age = 0;
    if (valid) {
        const int ntops = NDIM == 3 ? 8 : 4;
#pragma unroll
        for (int t = 0; t < ntops; ++t) {
            uint32_t code = uint32_t(e >> (9 + 4 * t)) & 15u;
            if (code == 15u) continue;
            int n = NDIM == 3 ? c_top_n3[t] : c_top_n2[t];
            int dz, dy, dx;
            stencil_off(NDIM, n, dz, dy, dx);
            uint32_t self = top_of_octant(it, z, y, x, dz, dy, dx);
            if (code == 8u) {
                rt_node = int(self);
                rt_age = make_key(ord, vg, NDIM == 3 ? uint32_t(n) : uint32_t(n) << 1);
            } else {
                int n2 = NDIM == 3 ? c_top_n3[code] : c_top_n2[code];
                int ez, ey, ex;
                stencil_off(NDIM, n2, ez, ey, ex);
                o.uft[self] = top_of_octant(it, z, y, x, ez, ey, ex);
            }
        }
    }
    // ---- stage survivors and roots
    uint32_t k0 = __popc(h0s);
    uint32_t kt = NDIM == 3 ? __popc(ds) : __popc(ds & ~h0s);
    uint32_t p0 = stage_reserve(&sg.n_s0, k0);
    uint32_t pt = stage_reserve(&sg.n_st, kt);
    uint32_t pr0 = stage_reserve(&sg.n_r0, root0 ? 1u : 0u);
    uint32_t prt = stage_reserve(&sg.n_rt, rt_node >= 0 ? 1u : 0u);
    const int nf = NDIM == 3 ? 6 : 4;
    for (int s = 0; s < nf; ++s) {
        if (!((h0s >> s) & 1u)) continue;
        int n = NDIM == 3 ? c_face_n3[s] : c_face_n2[s];
        uint32_t low = NDIM == 3 ? uint32_t(n) : (uint32_t(n) << 1) | ((ds >> s) & 1u);
        sg.s0[p0++] = make_key(ord, vg, low);
    }
    if (NDIM == 3) {
        for (int f = 0; f < 12; ++f) {
            if (!((ds >> f) & 1u)) continue;
            sg.st[pt++] = ~make_key(ord, vg, uint32_t(c_facet_n3[f]));
        }
    } else {
        uint32_t m = ds & ~h0s;
        for (int f = 0; f < 4; ++f) {
            if (!((m >> f) & 1u)) continue;
            sg.st[pt++] = ~make_key(ord, vg, uint32_t(c_face_n2[f]) << 1);
        }
    }
    if (root0) {
        sg.r0node[pr0] = vg;
        sg.r0age[pr0] = make_key(ord, vg, 0);
    }
    if (rt_node >= 0) {
        sg.rtnode[prt] = uint32_t(rt_node);
        sg.rtage[prt] = rt_age;
    }
}

__device__ __forceinline__ void finish_min(Stage& sg, const Outs& o, int item, unsigned long long my_min) {
    unsigned long long w = warp_min_u64(my_min);
    if (lane_id() == 0 && w != ~0ull) atomicMin(&sg.gmin, w);
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0 && sg.gmin != ~0ull) atomicMin(&o.ctr->gmin[item], sg.gmin);
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

// 3D relevant mask from the raw mask (bit n = 9(dz+1)+3(dy+1)+(dx+1)):
// an edge diagonal needs its two faces, a corner its three edge diagonals.
__device__ __forceinline__ uint32_t collapse3(uint32_t raw) {
    constexpr uint32_t X0 = (1u << 1) | (1u << 4) | (1u << 7) | (1u << 10) | (1u << 13) | (1u << 16) | (1u << 19) |
                            (1u << 22) | (1u << 25);
    constexpr uint32_t Y0 = (7u << 3) | (7u << 12) | (7u << 21);
    constexpr uint32_t Z0 = 0x1FFu << 9;
    constexpr uint32_t FACES = (1u << 4) | (1u << 10) | (1u << 12) | (1u << 14) | (1u << 16) | (1u << 22);
    constexpr uint32_t EDXY = (1u << 9) | (1u << 11) | (1u << 15) | (1u << 17);
    constexpr uint32_t EDXZ = (1u << 3) | (1u << 5) | (1u << 21) | (1u << 23);
    constexpr uint32_t EDYZ = (1u << 1) | (1u << 7) | (1u << 19) | (1u << 25);
    constexpr uint32_t CORN = (1u << 0) | (1u << 2) | (1u << 6) | (1u << 8) | (1u << 18) | (1u << 20) | (1u << 24) |
                              (1u << 26);
    uint32_t f = raw & FACES;
    uint32_t ux = ((f & X0) << 1) | ((f & X0) >> 1);
    uint32_t uy = ((f & Y0) << 3) | ((f & Y0) >> 3);
    uint32_t uz = ((f & Z0) << 9) | ((f & Z0) >> 9);
    uint32_t ed = raw & ((EDXY & ux & uy) | (EDXZ & ux & uz) | (EDYZ & uy & uz));
    uint32_t vx = ((ed & X0) << 1) | ((ed & X0) >> 1);
    uint32_t vy = ((ed & Y0) << 3) | ((ed & Y0) >> 3);
    uint32_t vz = ((ed & Z0) << 9) | ((ed & Z0) >> 9);
    uint32_t co = raw & CORN & vx & vy & vz;
    return f | ed | co;
}

__device__ __forceinline__ uint64_t lookup3(uint32_t rel) {
    uint32_t b = (rel * 0x9E3779B1u) >> (32 - 12);
    uint32_t d = c_disp3d[b];
    uint32_t s = ((rel ^ (d * 0x27D4EB2Fu)) * 0x85EBCA77u) >> (32 - 14);
    return __ldg(g_entries3d + s);
}

}  // namespace

// ---------------------------------------------------------------- 2D
// Tile: 32 x 32 vertices, CTA 32 x 8, 4 rows per thread.
constexpr int kT2Y = 32;

__global__ void __launch_bounds__(kThreads) k_prune2d(ItemTable tab, Outs o) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Stage& sg = *reinterpret_cast<Stage*>(smem_raw);
    float* tile = reinterpret_cast<float*>(smem_raw + sizeof(Stage));  // (kT2Y+2) x (32+2)
    const int tid = threadIdx.y * kBX + threadIdx.x;
    const int t = blockIdx.x;
    const int ii = tile_item(tab, 0, tab.n2d - 1, t);
    const Item& it = tab.it[ii];
    const int lt = t - it.tile0;
    const int x0 = (lt % it.tx) * kBX, y0 = (lt / it.tx) * kT2Y;
    if (tid == 0) {
        sg.n_s0 = sg.n_st = sg.n_r0 = sg.n_rt = 0;
        sg.gmin = ~0ull;
    }
    constexpr int SW = kBX + 2;
    for (int i = tid; i < (kT2Y + 2) * SW; i += kThreads) {
        int ly = i / SW, lx = i % SW;
        int gy = y0 + ly - 1, gx = x0 + lx - 1;
        float v = __int_as_float(0x7F800000);  // +inf: never precedes anything
        if (gy >= 0 && gy < it.H && gx >= 0 && gx < it.W) v = load_finite(it.img + int64_t(gy) * it.W + gx, o.ctr);
        tile[i] = v;
    }
    __syncthreads();
    unsigned long long my_min = ~0ull;
    for (int r = 0; r < kT2Y / kBY; ++r) {
        int ly = threadIdx.y + r * kBY, lx = threadIdx.x;
        int y = y0 + ly, x = x0 + lx;
        bool valid = y < it.H && x < it.W;
        const float* c = tile + (ly + 1) * SW + (lx + 1);
        float cv = c[0];
        uint32_t raw = 0;
        if (valid) {
            // bits 0..3: offsets before v in linear order (ties precede); 4..7 after
            raw |= (c[-SW - 1] <= cv) ? 1u : 0u;
            raw |= (c[-SW] <= cv) ? 2u : 0u;
            raw |= (c[-SW + 1] <= cv) ? 4u : 0u;
            raw |= (c[-1] <= cv) ? 8u : 0u;
            raw |= (c[1] < cv) ? 16u : 0u;
            raw |= (c[SW - 1] < cv) ? 32u : 0u;
            raw |= (c[SW] < cv) ? 64u : 0u;
            raw |= (c[SW + 1] < cv) ? 128u : 0u;
        }
        uint64_t e = c_lut2d[raw];
        uint32_t vg = uint32_t(it.voff + int64_t(y) * it.W + x);
        emit_vertex<2>(sg, o, it, valid, 0, y, x, vg, ord_bits(cv), e, my_min);
        __syncthreads();
    }
    flush(sg, o);
    finish_min(sg, o, ii, my_min);
}

// ---------------------------------------------------------------- 3D
// Tile: 32 x 8 x kT3Z vertices (x, y, z), CTA 32 x 8, one z column per thread.
constexpr int kT3Z = 8;

__global__ void __launch_bounds__(kThreads) k_prune3d(ItemTable tab, Outs o) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Stage& sg = *reinterpret_cast<Stage*>(smem_raw);
    float* tile = reinterpret_cast<float*>(smem_raw + sizeof(Stage));  // (kT3Z+2) x 10 x 34
    const int tid = threadIdx.y * kBX + threadIdx.x;
    const int t = blockIdx.x;
    const int ii = tile_item(tab, tab.n2d, tab.n - 1, t);
    const Item& it = tab.it[ii];
    const int lt = t - it.tile0;
    const int x0 = (lt % it.tx) * kBX;
    const int y0 = ((lt / it.tx) % it.ty) * kBY;
    const int z0 = (lt / (it.tx * it.ty)) * kT3Z;
    if (tid == 0) {
        sg.n_s0 = sg.n_st = sg.n_r0 = sg.n_rt = 0;
        sg.gmin = ~0ull;
    }
    constexpr int SW = kBX + 2, SH = kBY + 2, SP = SW * SH;
    for (int i = tid; i < (kT3Z + 2) * SP; i += kThreads) {
        int lz = i / SP, rem = i % SP, ly = rem / SW, lx = rem % SW;
        int gz = z0 + lz - 1, gy = y0 + ly - 1, gx = x0 + lx - 1;
        float v = __int_as_float(0x7F800000);
        if (gz >= 0 && gz < it.D && gy >= 0 && gy < it.H && gx >= 0 && gx < it.W)
            v = load_finite(it.img + (int64_t(gz) * it.H + gy) * it.W + gx, o.ctr);
        tile[i] = v;
    }
    __syncthreads();
    unsigned long long my_min = ~0ull;
    const int lx = threadIdx.x, ly = threadIdx.y;
    const int x = x0 + lx, y = y0 + ly;
    for (int lz = 0; lz < kT3Z; ++lz) {
        // keep room in the stage buffers for one more plane of vertices
        if (sg.n_s0 > uint32_t(kCapS - 5 * kThreads) || sg.n_st > uint32_t(kCapS - 7 * kThreads) ||
            sg.n_r0 > uint32_t(kCapR - kThreads) || sg.n_rt > uint32_t(kCapR - kThreads))
            flush(sg, o);
        int z = z0 + lz;
        bool valid = z < it.D && y < it.H && x < it.W;
        const float* c = tile + ((lz + 1) * SH + (ly + 1)) * SW + (lx + 1);
        float cv = c[0];
        uint32_t raw = 0;
        if (valid) {
#pragma unroll
            for (int n = 0; n < 27; ++n) {
                if (n == 13) continue;
                const int dz = n / 9 - 1, dy = (n / 3) % 3 - 1, dx = n % 3 - 1;
                float nv = c[(dz * SH + dy) * SW + dx];
                bool lower = n < 13 ? (nv <= cv) : (nv < cv);
                raw |= lower ? (1u << n) : 0u;
            }
        }
        uint64_t e = lookup3(collapse3(raw));
        uint32_t vg = uint32_t(it.voff + (int64_t(z) * it.H + y) * it.W + x);
        emit_vertex<3>(sg, o, it, valid, z, y, x, vg, ord_bits(cv), e, my_min);
        __syncthreads();
    }
    flush(sg, o);
    finish_min(sg, o, ii, my_min);
}

// ---------------------------------------------------------------- host side
size_t prune_smem2d() { return sizeof(Stage) + sizeof(float) * (kT2Y + 2) * (kBX + 2); }
size_t prune_smem3d() { return sizeof(Stage) + sizeof(float) * (kT3Z + 2) * (kBY + 2) * (kBX + 2); }
int prune_tile_x() { return kBX; }
int prune_tile_y2d() { return kT2Y; }
int prune_tile_y3d() { return kBY; }
int prune_tile_z3d() { return kT3Z; }

cudaError_t upload_luts(const uint64_t* lut2d, const uint16_t* disp3d, const uint64_t* entries3d) {
    cudaError_t e = cudaMemcpyToSymbol(c_lut2d, lut2d, sizeof(uint64_t) * 256);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyToSymbol(c_disp3d, disp3d, sizeof(uint16_t) * (1 << 12));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(g_entries3d, entries3d, sizeof(uint64_t) * (1 << 14));
}

cudaError_t launch_prune(const ItemTable& tab, const PruneOuts& po, cudaStream_t s) {
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
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_prune2d, cudaFuncAttributeMaxDynamicSharedMemorySize, int(prune_smem2d()));
        cudaFuncSetAttribute(k_prune3d, cudaFuncAttributeMaxDynamicSharedMemorySize, int(prune_smem3d()));
        attr_set = true;
    }
    if (tab.tiles2d > 0) {
        k_prune2d<<<tab.tiles2d, dim3(kBX, kBY), prune_smem2d(), s>>>(tab, o);
        note_launches(1);
    }
    if (tab.tiles3d > 0) {
        k_prune3d<<<tab.tiles3d, dim3(kBX, kBY), prune_smem3d(), s>>>(tab, o);
        note_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace cp
