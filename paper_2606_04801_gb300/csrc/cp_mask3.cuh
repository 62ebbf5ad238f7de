// Device form of the 3D lower-neighbour mask (Sec. 3.3): the bit layout the
// pruning kernel builds its 26 comparisons into, and the collapse to the
// relevant mask in that layout.  Host code uses the same functions to hash
// the lookup table's keys and to check the layout against the definition.
//
// The canonical numbering of a neighbour at offset (dz, dy, dx) is
// n = 9(dz+1) + 3(dy+1) + (dx+1).  The device layout places the bits on a
// lattice with steps Dx = 1, Dy = 3, Dz = 5 (writing [s] for 1 when the
// coordinate s is +1, else 0):
//   faces    z-, y-, x-, x+, y+, z+      bits 0..5 (the canonical order, so
//                                        the lowest face bit is the first
//                                        edge of the lower star)
//   xy edges (dx, dy, 0)   kM3XY + [dx] Dx + [dy] Dy   (bits 6, 7, 9, 10)
//   xz edges (dx, 0, dz)   kM3XZ + [dx] Dx + [dz] Dz   (12, 13, 17, 18)
//   yz edges (0, dy, dz)   kM3YZ + [dy] Dy + [dz] Dz   (11, 14, 16, 19)
//   corners  (dx, dy, dz)  kM3CO + [dx] Dx + [dy] Dy + [dz] Dz
//                                                      (20, 21, 23..26, 28, 29)
// A face, an edge and a corner differing by one coordinate's sign then sit a
// fixed distance apart for every position, so one multiplication copies
// every face bit of an axis onto the edges it bounds, and every edge bit of a
// plane onto the corners it bounds.  The collapse keeps an edge whose two
// faces precede v and a corner whose three edges are kept:
//   edge  (dx, dy, 0) kept = raw(edge) & face x(dx) & face y(dy)  (likewise xz, yz)
//   corner kept = raw(corner) & the three kept edges below it
// which is the sub-offset rule of the definition (every nonzero sub-offset
// of a kept offset precedes v).
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define CP_HD __host__ __device__
#else
#define CP_HD
#endif

namespace cp {

constexpr int kM3Dx = 1, kM3Dy = 3, kM3Dz = 5;
constexpr int kM3XY = 6, kM3XZ = 12, kM3YZ = 11, kM3CO = 20;
constexpr uint32_t kM3Faces = 0x3Fu;

// bit of the device layout for canonical neighbour n (n != 13)
CP_HD constexpr int mask3_pos(int n) {
    const int dz = n / 9 - 1, dy = (n / 3) % 3 - 1, dx = n % 3 - 1;
    const int px = dx > 0 ? kM3Dx : 0, py = dy > 0 ? kM3Dy : 0, pz = dz > 0 ? kM3Dz : 0;
    const int nz = (dz != 0) + (dy != 0) + (dx != 0);
    if (nz == 1) return dz < 0 ? 0 : dy < 0 ? 1 : dx < 0 ? 2 : dx > 0 ? 3 : dy > 0 ? 4 : 5;  // faces
    if (nz == 3) return kM3CO + px + py + pz;
    if (dz == 0) return kM3XY + px + py;
    if (dy == 0) return kM3XZ + px + pz;
    return kM3YZ + py + pz;
}

// canonical mask -> device layout
CP_HD inline uint32_t mask3_from_canonical(uint32_t raw) {
    uint32_t m = 0;
    for (int n = 0; n < 27; ++n)
        if (n != 13 && ((raw >> n) & 1u)) m |= 1u << mask3_pos(n);
    return m;
}

// Relevant mask of a device-layout raw mask, in the device layout.
CP_HD inline uint32_t collapse3_lattice(uint32_t raw) {
    // faces of each axis copied onto the edges they bound: from face x- (bit
    // 2) to xy (dx-, dy-/+) and xz (dx-, dz-/+); x+ lands Dx further
    constexpr uint32_t kX = (1u << (kM3XY - 2)) | (1u << (kM3XY - 2 + kM3Dy)) | (1u << (kM3XZ - 2)) |
                            (1u << (kM3XZ - 2 + kM3Dz));
    // from face y- (bit 1) to xy (dx-/+, dy-) and yz (dy-, dz-/+)
    constexpr uint32_t kY = (1u << (kM3XY - 1)) | (1u << (kM3XY - 1 + kM3Dx)) | (1u << (kM3YZ - 1)) |
                            (1u << (kM3YZ - 1 + kM3Dz));
    // from face z- (bit 0) to xz (dx-/+, dz-) and yz (dy-/+, dz-)
    constexpr uint32_t kZ = (1u << kM3XZ) | (1u << (kM3XZ + kM3Dx)) | (1u << kM3YZ) | (1u << (kM3YZ + kM3Dy));
    // kept edges of each plane copied onto the corners they bound
    constexpr uint32_t kCxy = (1u << (kM3CO - kM3XY)) | (1u << (kM3CO - kM3XY + kM3Dz));
    constexpr uint32_t kCxz = (1u << (kM3CO - kM3XZ)) | (1u << (kM3CO - kM3XZ + kM3Dy));
    constexpr uint32_t kCyz = (1u << (kM3CO - kM3YZ)) | (1u << (kM3CO - kM3YZ + kM3Dx));
    const uint32_t rx = (raw & 0x0Cu) * kX;  // faces x-, x+
    const uint32_t ry = (raw & 0x12u) * kY;  // faces y-, y+
    const uint32_t rz = (raw & 0x21u) * kZ;  // faces z-, z+
    const uint32_t exy = raw & rx & ry;      // rx lands on xy and xz edges only, ry on xy and yz
    const uint32_t exz = raw & rx & rz;
    const uint32_t eyz = raw & ry & rz;
    const uint32_t co = raw & (exy * kCxy) & (exz * kCxz) & (eyz * kCyz);
    return (raw & kM3Faces) | exy | exz | eyz | co;
}

}  // namespace cp
