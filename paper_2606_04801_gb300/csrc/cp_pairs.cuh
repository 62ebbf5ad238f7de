// The pair that a union-find commit writes (shared by the union-find and
// the slab split's first stage).
#pragma once
#include "cp_common.cuh"

namespace cp {

// The pair of a committed survivor with key `key` (the key itself, not its
// complement) of item `item`, whose dying class has root id yrid with age
// key age[yrid] (the root vertex; for the dual the vertex whose lower star
// holds the dying top cell).  Returns false for a zero-persistence pair,
// which is omitted (Sec. 2.3).
__device__ __forceinline__ bool commit_pair(const ItemTable& tab, const uint64_t* age, int dual, uint64_t key,
                                            int item, uint32_t yrid, cp_pair& out) {
    const Item& it = tab.it[item];
    uint64_t a = age[yrid];
    const uint32_t young = key_vertex(a);
    uint32_t vg = key_vertex(key);
    int n = int(key_n(key, it.ndim));
    int dz, dy, dx;
    stencil_off(it.ndim, n, dz, dy, dx);
    int64_t lv = int64_t(vg) - it.voff;
    int x = int(lv % it.W), y = int((lv / it.W) % it.H), z = int(lv / (int64_t(it.W) * it.H));
    float fv = ord_float(uint32_t(key >> 32));
    float fy = ord_float(uint32_t(a >> 32));
    if (!dual) {
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
        uint32_t mg = key_vertex(a);
        int nt = int(key_n(a, it.ndim));
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
    return out.birth != out.death;
}

}  // namespace cp
