// Neighbourhood lookup table for the V-filtration lower star (Sec. 3.3).
//
// A vertex v is looked up by the set of its neighbours (vertices sharing a
// top cell with v: 8 in 2D, 26 in 3D) that precede it in the semi-refined
// order.  A neighbour at offset o matters only when every neighbour whose
// offset is a nonzero sub-offset of o precedes v as well (the collapse of
// Sec. 3.3); the collapsed set ("relevant mask") determines the lower star
// L(v) and everything the pruning needs.  There are 47 relevant masks in 2D
// and 15,935 in 3D (the 3D count is the one printed in Sec. 3.3).
//
// Neighbour offsets are numbered n = 9(dz+1) + 3(dy+1) + (dx+1) in 3D and
// n = 3(dy+1) + (dx+1) in 2D; the centre (13, resp. 4) is unused.  The cell
// of L(v) spanned by v and v+o sits at doubled coordinates 2v+o, so ordering
// the cells of one lower star by doubled-grid index orders them by n.
//
// Entry layout (one per relevant mask):
//   bits  0.. 2  direct    : face slot of the first edge of L(v) (the edge that
//                            kills v at zero persistence), 7 = v is a local min
//   bits  3.. 8  h0_surv   : face slots whose edge is the first edge of a local
//                            group other than the direct one (H0 survivors)
//   bits  9..40  dual      : per top-cell slot, 4 bits: 0..7 slot of the top
//                            cell across the facet at which this top cell dies
//                            locally, 8 = survives locally (dual root),
//                            15 = not in L(v)
//   bits 41..52  dual_surv : facet slots of L(v) left for the dual union-find
//   bits 53..60  in_l      : top-cell slots that belong to L(v) (dual code != 15)
// 2D uses the same fields with 4 face slots, 4 facet slots (the same edges)
// and 4 top-cell slots.
//
// Slots: faces, facets and top cells of L(v) are numbered by ascending n.
#pragma once
#include <cstdint>
#include <vector>

namespace cp {

struct LutEntry {
    uint64_t bits;
};

inline int lut_direct(uint64_t e) { return int(e & 7u); }
inline uint32_t lut_h0_surv(uint64_t e) { return uint32_t((e >> 3) & 0x3Fu); }
inline uint32_t lut_dual(uint64_t e, int t) { return uint32_t((e >> (9 + 4 * t)) & 0xFu); }
inline uint32_t lut_dual_surv(uint64_t e) { return uint32_t((e >> 41) & 0xFFFu); }
inline uint32_t lut_in_l(uint64_t e) { return uint32_t((e >> 53) & 0xFFu); }

// Offsets and slot tables for one dimension.
struct Stencil {
    int ndim;
    int nbits;                  // 9 (2D) or 27 (3D) bit positions, centre unused
    int center;                 // 4 or 13
    int off[27][3];             // (dz, dy, dx) of bit n (dz = 0 in 2D)
    int nfaces, nfacets, ntops;
    int face_n[6];              // bit n of face slot s
    int facet_n[12];            // bit n of facet slot s
    int top_n[8];               // bit n of top-cell slot s
    int facet_tops[12][2];      // top-cell slots on the two sides of facet slot s
    uint32_t sub[27];           // mask of nonzero sub-offsets of n (including n)
};

const Stencil& stencil(int ndim);

// Relevant (collapsed) mask of a raw lower-neighbour mask.
uint32_t collapse(const Stencil& st, uint32_t raw);

// Number of raw 3D masks (all 2^26) whose collapse in the pruning kernel's
// bit layout (cp_mask3.cuh) differs from the definition above, carried into
// that layout; 0 when the layout is right.
uint64_t check_mask3_layout();

// Lookup entry of a relevant mask.
uint64_t classify(const Stencil& st, uint32_t rel);

// All relevant masks, ascending.
std::vector<uint32_t> relevant_masks(const Stencil& st);

// Perfect hash of the 15,935 relevant 3D masks into a table of 2^kLog2Slots
// entries: bucket = (m * kH1) >> (32 - kLog2Buckets), slot =
// ((m ^ disp[bucket] * kD) * kH2) >> (32 - kLog2Slots), with m the relevant
// mask in the pruning kernel's bit layout (cp_mask3.cuh).
constexpr int kLog2Buckets = 12;
constexpr int kLog2Slots = 14;
constexpr uint32_t kH1 = 0x9E3779B1u;
constexpr uint32_t kH2 = 0x85EBCA77u;
constexpr uint32_t kD = 0x27D4EB2Fu;

struct Lut3D {
    std::vector<uint16_t> disp;   // 2^kLog2Buckets
    std::vector<uint64_t> entry;  // 2^kLog2Slots
    std::vector<uint32_t> key;    // 2^kLog2Slots (0xFFFFFFFF = empty), host-side checks only
    int nclasses;
};

// Builds the 3D table; returns false if no perfect hash was found.
bool build_lut3d(Lut3D& out);

// 2D table indexed directly by the 8-bit raw mask (bits 0..3 = n 0..3,
// bits 4..7 = n 5..8); entries already collapsed.
void build_lut2d(std::vector<uint64_t>& out, int* nclasses);

}  // namespace cp
