// T-filtration by duality.
//
// Under the T-construction (Sec. 2.2) the pixel values sit on the top cells
// of the lattice complex and every other cell takes the smallest value of the
// top cells that contain it.  The paper leaves this filtration to future work
// (Sec. 6), noting that its duality argument carries over.  This file computes
// it with the V-filtration pipeline, through the duality between the
// T-complex of an image I and the V-complex of
//     J = -I, flipped along every axis, padded with a one-voxel frame whose
//         value lies below every value of -I.
// A T-cell of dimension k is dual to a V-cell of J of dimension d-k (a T top
// cell to a J vertex, a T vertex to a J top cell); f_T(s) = -f_V(s*), and with
// the flip, increasing order in one complex is decreasing order in the other,
// ties included (the top cell a T-cell enters with is the vertex of J that
// its dual cell enters with; the doubled-grid indices reverse).  So:
//   - the T-filtration's H0 union-find (Kruskal over T-edges) is the dual
//     union-find of the V top dimension on J (J top cells = T vertices,
//     J facets = T edges); its last merge, into the outside through a frame
//     facet, is the T essential class;
//   - the T top-dimension dual union-find (T top cells + outside) is the V
//     H0 union-find on J (J vertices = T top cells, the frame = the outside);
//     the frame's own class is the V essential class and is dropped.
// A V pair (b, d) becomes the T pair (-d, -b) with its cells and pixels
// exchanged and mapped back: doubled coordinate a of J becomes 2n+1-a of the
// T grid, vertex coordinate c of J becomes pixel n-c of I.
//
// Kernels: J itself (with a check that every pixel lies below the largest
// finite float, so that the frame comes first), and the in-place mapping of
// the V pairs before the canonical output sort.
#include "cp_common.cuh"
#include "cp_kernels.h"

namespace cp {
namespace {

constexpr int kTT = 256;
// The frame value: below every value of -I as long as every pixel is below
// the largest finite float (a pixel at that float, or above it, is flagged).
constexpr float kFrame = -3.40282347e38f;

// J four rows at a time, item blockIdx.y (the rows' divisions once per group;
// consecutive threads write consecutive x and read consecutive, reversed,
// pixels of the mirrored rows of the image; four loads in flight per thread).
constexpr int kTRows = 4;

__global__ void __launch_bounds__(kTT) k_t_build(const __grid_constant__ TItems t, uint32_t* bad) {
    const int item = blockIdx.y;
    const TDims& d = t.d[item];
    const float* __restrict__ img = t.img[item];
    float* __restrict__ J = t.J[item];
    const int64_t Dj = d.ndim == 3 ? d.D + 2 : 1, Hj = d.H + 2, Wj = d.W + 2;
    const int64_t rows = Dj * Hj;
    bool flag = false;
    for (int64_t r0 = int64_t(blockIdx.x) * kTRows; r0 < rows; r0 += int64_t(gridDim.x) * kTRows) {
        const float* in[kTRows];
        bool live[kTRows];  // an image row (else a frame row, or past the end)
#pragma unroll
        for (int k = 0; k < kTRows; ++k) {
            const int64_t r = r0 + k;
            const int64_t z = r / Hj, y = r - z * Hj;
            live[k] = r < rows && y != 0 && y != Hj - 1 && (d.ndim != 3 || (z != 0 && z != Dj - 1));
            const int64_t iz = d.ndim == 3 ? d.D - z : 0;
            in[k] = img + (iz * d.H + (d.H - y)) * d.W;  // dereferenced only when live
        }
        for (int64_t x = threadIdx.x; x < Wj; x += kTT) {
            const bool inner = x > 0 && x < Wj - 1;
            float a[kTRows];
#pragma unroll
            for (int k = 0; k < kTRows; ++k) a[k] = (live[k] && inner) ? __ldg(in[k] + (d.W - x)) : 0.0f;
#pragma unroll
            for (int k = 0; k < kTRows; ++k) {
                if (r0 + k >= rows) break;
                float v = kFrame;
                if (live[k] && inner) {
                    flag |= !(a[k] < 3.40282347e38f);  // NaN, +inf, the largest float: the frame would not lie below
                    v = -a[k];
                }
                J[(r0 + k) * Wj + x] = v;
            }
        }
    }
    if (__any_sync(0xFFFFFFFFu, flag) && (threadIdx.x & 31u) == 0) atomicOr(bad, 1u);
}

// After the pruning pass: every frame vertex of J points straight at J's
// vertex 0, the frame's root.  The frame is one tree of equal values in which
// the pruning pass links each vertex to an earlier neighbour; its chains
// along y and x run the whole length of a face, and every walk from a basin
// that drains to the border would otherwise follow them.  Vertex 0 is an
// ancestor of every frame vertex (every frame vertex but 0 has an earlier
// neighbour in the frame, and equal values order by index), so the shortcut
// changes no root.  Item blockIdx.y.
__global__ void __launch_bounds__(kTT) k_t_flatten(uint32_t* __restrict__ uf0, const __grid_constant__ TItems t) {
    const int item = blockIdx.y;
    const TDims& d = t.d[item];
    uint32_t* __restrict__ uf = uf0 + t.voff[item];
    const uint32_t root = uint32_t(t.voff[item]);
    const int64_t Dj = d.ndim == 3 ? d.D + 2 : 1, Hj = d.H + 2, Wj = d.W + 2;
    // whole frame rows, one block per row: both y faces of every plane, and
    // the two z faces (3D)
    const int64_t zf = d.ndim == 3 ? 2 * Hj : 0;  // rows of the two z faces
    const int64_t nrows = zf + 2 * (d.ndim == 3 ? Dj - 2 : 1);
    for (int64_t f = blockIdx.x; f < nrows; f += gridDim.x) {
        int64_t z, y;
        if (f < zf) {
            z = f < Hj ? 0 : Dj - 1;
            y = f % Hj;
        } else {
            const int64_t g = f - zf;
            z = d.ndim == 3 ? 1 + g / 2 : 0;
            y = (g & 1) ? Hj - 1 : 0;
        }
        uint32_t* row = uf + (z * Hj + y) * Wj;
        for (int64_t x = threadIdx.x; x < Wj; x += kTT)
            if (z != 0 || y != 0 || x != 0) row[x] = root;
    }
    // the two x faces of the other rows
    const int64_t zi = d.ndim == 3 ? Dj - 2 : 1, yi = Hj - 2;
    const int64_t nside = 2 * zi * yi;
    for (int64_t k = int64_t(blockIdx.x) * kTT + threadIdx.x; k < nside; k += int64_t(gridDim.x) * kTT) {
        const int64_t q = k >> 1;
        const int64_t z = d.ndim == 3 ? 1 + q / yi : 0, y = 1 + q % yi;
        uf[(z * Hj + y) * Wj + ((k & 1) ? Wj - 1 : 0)] = root;
    }
}

// Doubled-grid index in J -> doubled-grid index in the T-complex of I.
__device__ __forceinline__ int32_t t_cell(const TDims& t, int32_t vc) {
    if (vc < 0) return -1;
    const int64_t GWv = 2 * (t.W + 2) - 1, GHv = 2 * (t.H + 2) - 1;
    const int64_t X = vc % GWv, Y = (vc / GWv) % GHv, Z = vc / (GWv * GHv);
    const int64_t GWt = 2 * t.W + 1, GHt = 2 * t.H + 1, GDt = t.ndim == 3 ? 2 * t.D + 1 : 1;
    const int64_t tx = GWt - X, ty = GHt - Y, tz = t.ndim == 3 ? GDt - Z : 0;
    if (tx < 0 || tx >= GWt || ty < 0 || ty >= GHt || tz < 0 || tz >= GDt) return -1;  // a frame cell
    return int32_t((tz * GHt + ty) * GWt + tx);
}

// Vertex of J -> pixel of I.
__device__ __forceinline__ int32_t t_pixel(const TDims& t, int32_t vp) {
    if (vp < 0) return -1;
    const int64_t Wj = t.W + 2, Hj = t.H + 2;
    const int64_t x = vp % Wj, y = (vp / Wj) % Hj, z = vp / (Wj * Hj);
    const int64_t iz = t.ndim == 3 ? t.D - z : 0;
    return int32_t((iz * t.H + (t.H - y)) * t.W + (t.W - x));
}

__device__ __forceinline__ float neg_canon(float v) {
    const float r = -v;
    return r == 0.0f ? 0.0f : r;  // -0.0 reads as +0.0
}

__global__ void __launch_bounds__(kTT) k_t_map(cp_pair* __restrict__ pairs, const uint32_t* d_n, uint32_t cap,
                                               const __grid_constant__ TItems ti, const uint32_t* bad,
                                               Counters* ctr) {
    const uint32_t n = min(*d_n, cap);
    for (uint32_t i = blockIdx.x * kTT + threadIdx.x; i < n; i += gridDim.x * kTT) {
        const cp_pair p = pairs[i];
        const TDims& t = ti.d[(p.item >= 0 && p.item < ti.n) ? p.item : 0];
        const int top = t.ndim - 1;
        cp_pair q;
        q.item = p.item;
        if (p.dim == 0 && p.death_cell < 0) {
            // an item's frame class (the outside of its T-complex): dropped; its
            // item index one past the last sorts it after every kept pair,
            // outside the kept count
            q = p;
            q.item = ti.n;
            q.dim = 0;
            q.birth_cell = 0;
        } else if (p.dim == top && p.birth == kFrame) {
            // the last merge into the outside, through a frame facet: the T
            // essential class, born at the T vertex dual to the dying top cell
            q.dim = 0;
            q.birth = neg_canon(p.death);
            q.death = __int_as_float(0x7F800000);
            q.birth_cell = t_cell(t, p.death_cell);
            q.death_cell = -1;
            q.birth_pixel = t_pixel(t, p.death_pixel);
            q.death_pixel = -1;
        } else {
            q.dim = p.dim == 0 ? top : 0;
            q.birth = neg_canon(p.death);
            q.death = neg_canon(p.birth);
            q.birth_cell = t_cell(t, p.death_cell);
            q.death_cell = t_cell(t, p.birth_cell);
            q.birth_pixel = t_pixel(t, p.death_pixel);
            q.death_pixel = t_pixel(t, p.birth_pixel);
        }
        pairs[i] = q;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctr->t_keep = n > uint32_t(ti.n) ? n - uint32_t(ti.n) : 0u;  // one frame class per item
        if (*bad) set_status(ctr, kStNonfinite);
    }
}

int grid_of(int64_t n) {
    const int64_t b = (n + kTT - 1) / kTT;
    const int64_t cap = int64_t(device_sm_count()) * 8;
    return int(b < 1 ? 1 : (b < cap ? b : cap));
}

}  // namespace

cudaError_t launch_t_build(const TItems& t, uint32_t* bad, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    if (t.n < 1 || t.n > kMaxItems) return cudaErrorInvalidValue;
    const int gx = (device_sm_count() * 16 + t.n - 1) / t.n;
    k_t_build<<<dim3(gx, t.n), kTT, 0, s>>>(t, bad);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_t_flatten(uint32_t* uf0, const TItems& t, cudaStream_t s) {
    if (t.n < 1 || t.n > kMaxItems) return cudaErrorInvalidValue;
    const int gx = (device_sm_count() * 8 + t.n - 1) / t.n;
    k_t_flatten<<<dim3(gx, t.n), kTT, 0, s>>>(uf0, t);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_t_map(cp_pair* pairs, const uint32_t* d_n, uint32_t cap, const TItems& t, const uint32_t* bad,
                         Counters* ctr, cudaStream_t s) {
    k_t_map<<<grid_of(cap), kTT, 0, s>>>(pairs, d_n, cap, t, bad, ctr);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace cp
