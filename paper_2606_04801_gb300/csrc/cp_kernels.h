// Host-side interface between the C-ABI layer and the kernels.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "cp_common.cuh"

namespace cp {

// ---- K1 pruning
struct PruneOuts {
    uint32_t* uf0;   // H0 forest over global vertices
    uint32_t* uft;   // dual forest over global top cells (+ one outside vertex per item)
    uint64_t* s0;    // H0 survivor keys
    uint64_t* st;    // dual survivor keys (complemented: ascending sort = descending order)
    uint64_t* age0;  // age of each H0 root id
    uint64_t* res0;  // reservation word of each H0 root id
    uint64_t* aget;  // age of each dual root id
    uint64_t* rest;  // reservation word of each dual root id
    uint32_t cap_s, cap_r0, cap_rt;
    Counters* ctr;
    uint32_t n_uf0, n_uft;  // forest sizes (for the bounds-checked build)
};
size_t prune_smem2d();
size_t prune_smem3d();
int prune_tile_x();
int prune_tile_x3d();
int prune_tile_y2d();
int prune_tile_y3d();
int prune_tile_z3d();
int prune_cross2d();
int set_tuning(int key, int value);
int get_tuning(int key);
cudaError_t upload_luts(const uint64_t* lut2d, const uint16_t* disp3d, const uint64_t* entries3d,
                        const uint32_t* keys3d);
// Tensor maps for TMA loads of 3D planes (one per item that qualifies: width a
// multiple of 4, 16-byte aligned image, at least 40 x 11 per plane); the other
// items load their planes with cp.async.
constexpr int kMaxTma = 64;
struct TmaMaps {
    CUtensorMap m[kMaxTma];
};
// Encodes the plane map of a D x H x W float volume; false if it cannot be used.
bool encode_plane_map(CUtensorMap* map, const float* img, int64_t D, int64_t H, int64_t W);
cudaError_t launch_prune(const ItemTable& tab, const PruneOuts& po, const TmaMaps& maps, cudaStream_t s);

// ---- K2 radix sort (LSD, 8-bit digits, decoupled look-back)
struct SortBufs {
    uint64_t* keys;       // in/out (result lands here: the pass count is even)
    uint64_t* keys_alt;
    uint32_t* vals;       // optional payload (nullptr = keys only)
    uint32_t* vals_alt;
    const uint32_t* d_count;  // number of keys, on the device
    uint32_t cap;             // capacity of the key arrays
    uint32_t* hist;           // 8 x 256 scratch
    uint64_t* status;         // sort_status_words(cap) scratch (cleared by the sort itself)
    uint32_t* tile_ctr;       // one ticket counter per pass, zeroed once per call
    Counters* ctr;
};
size_t sort_status_words(uint32_t cap);
constexpr int kSortTile = 2048;
// Sorts bytes [first_byte, first_byte + npasses) of each key, npasses even.
cudaError_t sort_keys(const SortBufs& b, int first_byte, int npasses, uint32_t epoch, cudaStream_t s);
// The same over two lists at once (one launch per pass; separate buffers,
// histograms and status words; the tile tickets of b[0]).
cudaError_t sort_keys_multi(const SortBufs* b, int nl, int first_byte, int npasses, uint32_t epoch, cudaStream_t s);

// ---- K3 union-find (deterministic reservations)
struct UfParams {
    const uint64_t* keys;     // sorted survivor keys
    const uint32_t* d_nkeys;
    uint32_t cap_keys;
    uint32_t* uf;
    const uint64_t* age;
    uint64_t* res;
    uint32_t* act[2];         // survivor index of each active slot (ping-pong)
    uint32_t* na[2];          // a root id of the first endpoint's class, per active slot
    uint32_t* nb[2];          // a root id of the second endpoint's class
    uint32_t* ynode;          // young / old root id between the phases (slots past the registers)
    uint32_t* onode;
    uint32_t scratch_cap;     // entries of act / na / nb / ynode / onode and of log
    uint64_t* log;            // per survivor: young root << 32 | its age id, or ~0 (no commit)
    cp_pair* pairs;           // nullptr: commits are logged, no pairs written
    uint32_t pair_cap;
    uint64_t* dual_keys;      // H0 of 2D items: positive edges that the dual needs (cross-pruning)
    uint32_t* d_ndual;
    uint32_t dual_cap;
    Counters* ctr;
    int dual;                 // 0: H0 (ascending, larger age dies); 1: dual (smaller age dies)
    // H1 of volumes: bit cell_id3 of every committed survivor of a 3D item
    // (H0: a negative edge; dual: a square that creates a 2-cycle), or nullptr
    uint32_t* h1flags = nullptr;
    uint32_t n_nodes = 0;     // forest entries, and root ids (age / res entries):
    uint32_t n_rids = 0;      // bounds of the bounds-checked build
};
// First-round root walks, before the sort (k_roots: ra / rb / pos per unsorted
// survivor), and the first active list from the sorted positions
// (k_place_roots).
struct RootArgs {
    ItemTable tab;
    const uint64_t* keys;        // unsorted survivor keys (k_roots)
    const uint32_t* d_n;
    uint32_t cap;
    const uint32_t* uf;
    int dual;
    uint32_t* ra;                // root id of each survivor's endpoints, by unsorted position
    uint32_t* rb;
    uint32_t* pos;               // sort payload: the unsorted position
    const uint32_t* sorted_pos;  // k_place_roots: the payload after the sort
    const uint32_t* d_n_before;  // dual list after the H0 list: the H0 count (else nullptr)
    uint32_t scratch_cap;
    uint32_t* act;               // first active list (ping-pong buffer 0)
    uint32_t* na;
    uint32_t* nb;
    Counters* ctr;
    uint32_t n_nodes;            // forest entries (bounds-checked build)
};
cudaError_t launch_roots(const RootArgs& r, cudaStream_t s);
// Both lists' first-round walks in one launch (one work counter over both).
cudaError_t launch_roots2(const RootArgs& r0, const RootArgs& r1, cudaStream_t s);
cudaError_t launch_place_roots(const RootArgs& r, cudaStream_t s);

// One problem, or two (H0 and dual of a call without 2D items) carried through
// the same rounds.  Two problems share the scratch lists (the pointers of p[0])
// side by side when both fit, else they run one after the other.
cudaError_t launch_uf(const ItemTable& tab, const UfParams* p, int nprob, cudaStream_t s);

// ---- slab decomposition of the union-finds (cp_slab.cu)
struct SlabCtr {
    uint32_t n_in[2];        // stage 1 survivors (both endpoint classes in one slab), per list
    uint32_t n_cross[2];     // survivors whose endpoint classes lie in two slabs
    uint32_t n_sent[2];      // stage 1 commits handed to stage 2
    uint32_t n_merge[2];     // stage 2 survivors (sent + crossing)
    uint32_t rounds_slab[2]; // rounds of stage 1
    uint32_t n_final[2];     // stage 1 commits whose pairs stage 1 wrote (their dying class met no crossing survivor)
};
// The Borůvka variant's counts share this block: n_in = forest edges per list.
struct SlabArgs {
    ItemTable tab;
    int S;                       // slabs per item
    const uint32_t* d_n[2];      // survivors of the H0 and dual lists (device counts)
    uint32_t cap;                // scratch capacity (the two lists side by side)
    const uint64_t* keys[2];     // the sorted lists
    const uint64_t* age[2];      // age of each root id, per list
    uint32_t n_rids[2];          // root ids per list
    uint64_t* res[2];            // reservation word of each root id, per list
    uint32_t* na;                // root ids of both endpoints of every slot (list 1 after list 0); a commit
    uint32_t* nb;                // that stage 1 sends on gets the two classes' roots at its time instead
    uint32_t* sub[2];            // per root id: bit 0 an endpoint of a crossing survivor, bit 1 its
                                 // subtree of stage 1's links holds such a root
    uint32_t* died[2];           // per root id that stage 1 killed: the index of the commit
    uint8_t* flag;               // per slot: 1 internal, 2 crossing, 3 committed in stage 1 and sent on
    uint32_t* vcnt;              // per virtual block of the compaction: count, then offset
    SlabCtr* sc;
    Counters* ctr;
    uint64_t* ko[2];             // compaction output: the selected keys of each list
    uint32_t* act;               // and the active lists (survivor index, root ids), side by side
    uint32_t* oa;
    uint32_t* ob;
    uint32_t* map;               // stage 1 only: the slot each selected survivor came from
    const uint64_t* log;         // stage 1's commit log (read by the marking pass)
    cp_pair* pairs;              // the final commits' pairs are appended here
    uint32_t pair_cap;
};
// ---- Borůvka's minimum spanning forest of both survivor lists (cp_boruvka.cu)
struct BoruvkaArgs {
    const uint32_t* d_n[2];      // survivors of the H0 and dual lists (device counts)
    uint32_t cap;                // scratch capacity (the two lists side by side)
    uint32_t n_rids[2];          // root ids per list
    const uint32_t* na;          // root ids of both endpoints of every slot (list 1 after list 0)
    const uint32_t* nb;
    uint32_t* comp[2];           // per root id: its component's representative
    uint32_t* best[2];           // per representative: the smallest sorted index leaving it
    uint32_t* hook[2];           // per representative: the component it hooks to this round
    uint32_t* act[2];            // active slots (ping-pong, cap entries each)
    uint8_t* flag;               // per slot: 1 a forest edge, 2 not
    uint32_t* d_rounds;          // rounds run
    Counters* ctr;
};
cudaError_t launch_boruvka(const BoruvkaArgs& a, cudaStream_t s);
int uf_variant();  // 0: reservation rounds over every survivor; 1: Borůvka, then rounds over its forest

// Entries of SlabArgs::vcnt for a scratch capacity.
uint32_t slab_vblocks_cap(uint32_t cap);
// Flags each slot internal or crossing (kStCapacity if the lists are not
// side by side) and marks the crossing survivors' endpoint classes.
cudaError_t launch_slab_classify(const SlabArgs& a, cudaStream_t s);
// Stable compaction of the slots selected by sel (0: flag 1, the slab
// split's internal survivors or the Borůvka forest's edges; 1: flag 2 or 3,
// the slab split's crossing and handed-on survivors) to ko / act / oa / ob
// (/ map); n_out[q] receives list q's count.
cudaError_t launch_slab_compact(const SlabArgs& a, int sel, uint32_t* n_out, cudaStream_t s);
// After stage 1: marks the classes that met a crossing survivor, writes the
// pairs of the commits whose dying class did not and flags the others (with
// their classes' roots) for stage 2, then clears the reservation words.
cudaError_t launch_slab_mark(const SlabArgs& a, cudaStream_t s);

// ---- H1 of volumes (cp_h1.cu): column reduction of the square-edge boundary
// matrix restricted to the squares that do not create 2-cycles and the edges
// that do not merge components; first inside each lower star, then across
// stars.
struct H1Ctl {
    uint32_t m;                   // columns (squares not paired in H2)
    uint32_t nl;                  // columns whose lowest entry leaves their lower star
    uint32_t cnt[3];              // work-list counters of the reduction rounds (rotating)
    uint32_t neg_e, pos_q, pos_e; // checks: marked edges, marked squares, unmarked edges
    uint32_t rounds;              // reduction rounds run
    uint32_t stop[2];             // a round's merges hit an error (read one round later, by parity)
    uint32_t solo_round;          // the round from which the first CTA ran the rounds alone (0: never)
    unsigned long long grown;     // pool entries taken by merged columns
    unsigned long long t_grid_ns, t_solo_ns;  // wall time of the rounds on the whole grid / in one CTA
    unsigned long long t_phase_ns[4];  // thread 0 of CTA 0, summed over rounds: its bids, the wait after
                                       // them, its merges, the wait after them
    unsigned long long additions, merged;  // column additions, and the entries they read
    uint32_t park_gen, park_exit, park_round, park_nchg;  // the first CTA wakes the parked ones
    uint32_t solo_entries;        // times the first CTA went on alone
    uint32_t nw_hist[16];         // rounds by losing columns: bucket floor(log2(count)), capped at 15
};
struct H1Bufs {
    uint32_t* neg_e;         // bitmap over edge ids (cell_id3): edge kills an H0 class
    uint32_t* pos_q;         // bitmap over square ids: square creates a 2-cycle
    size_t map_words;        // words per bitmap
    H1Ctl* ctl;
    uint32_t* cmask;         // per square id: its column inside its lower star (30 edge slots), 0: no column
    uint64_t* coff;          // per square id: pool offset of its column once it has been added to, or ~0
    uint32_t* clen;          // per square id: entries of that pool column
    uint32_t* ccap;          // per square id: capacity of the two pool regions at coff (each), and in
                             // bit 31 which of the two holds the column
    uint32_t* list0;         // the columns whose lowest entry leaves their star (square ids)
    uint32_t* list[2];       // columns changed in a round (ping-pong)
    uint64_t* pivot;         // per edge id: key of the oldest column whose lowest entry it is, or ~0
    uint64_t* pool;          // explicit columns (edge keys, descending)
    uint64_t pool_cap;
    uint32_t mcap;           // columns expected: sum over 3D items of E - N + 1
    uint32_t exp_neg_e;      // sum over 3D items of N - 1
    uint32_t exp_pos_q;      // sum over 3D items of (D-1)(H-1)(W-1)
    uint32_t n_ids = 0;      // edge / square ids (entries of the per-id arrays; bounds-checked build)
};
// After the union-finds have marked their committed survivors in the two
// bitmaps (zeroed before them): marks what the lower stars settle, reduces
// every lower star's columns, reduces the columns that leave their star in
// rounds, and appends the H1 pairs (zero persistence omitted) to pairs.
cudaError_t launch_h1(const ItemTable& tab, const H1Bufs& b, Counters* ctr, cp_pair* pairs, uint32_t pair_cap,
                      cudaStream_t s);
// Wall-clock budget of the cross-star rounds (one non-preemptible launch):
// once it is spent, the rounds stop at the next round boundary and the call
// returns CP_ERR_TIMEOUT.
void set_h1_budget_ms(int ms);
int get_h1_budget_ms();
// Columns entering a round at or below which the first CTA runs the
// cross-star rounds alone (0: never).
void set_h1_solo_cols(int n);
int get_h1_solo_cols();

// ---- K4 emission, K5 backward
cudaError_t launch_init(const ItemTable& tab, Counters* ctr, uint32_t* uft, uint64_t* aget, uint64_t* rest,
                        cudaStream_t s);
// T-filtration by duality (cp_tfilt.cu), per item by the caller's index.
struct TDims {
    int ndim;
    int64_t D, H, W;  // the image's extents (D = 1 in 2D)
};
struct TItems {
    int n;
    TDims d[kMaxItems];
    const float* img[kMaxItems];  // the image
    float* J[kMaxItems];          // its dual image: extents +2 along each image axis
    int64_t voff[kMaxItems];      // J's first vertex in the call's vertex space
};
// J <- -image flipped along every axis, inside a one-voxel frame at -FLT_MAX;
// *bad <- 1 if a pixel is not below FLT_MAX (the frame would not come first).
cudaError_t launch_t_build(const TItems& t, uint32_t* bad, cudaStream_t s);
// After the pruning pass: every frame vertex's H0 link points at the item's
// vertex 0.
cudaError_t launch_t_flatten(uint32_t* uf0, const TItems& t, cudaStream_t s);
// V pairs of J -> T pairs of the images, in place; each item's frame class
// gets item index n (it sorts after every kept pair), ctr->t_keep the count
// without them, and a set *bad flags the call as non-finite.
cudaError_t launch_t_map(cp_pair* pairs, const uint32_t* d_n, uint32_t cap, const TItems& t, const uint32_t* bad,
                         Counters* ctr, cudaStream_t s);
cudaError_t launch_essential(const ItemTable& tab, Counters* ctr, cp_pair* pairs, uint32_t pair_cap, cudaStream_t s);
// dim_bits 1: dimension 0 or top; 2: dimension 0, 1 or 2 (calls with H1)
cudaError_t launch_pair_keys(const cp_pair* pairs, const uint32_t* d_n, uint32_t cap, uint64_t* keys, uint32_t* vals,
                             int cell_bits, int dim_bits, cudaStream_t s);
cudaError_t launch_gather(const cp_pair* pairs, const uint32_t* vals, const uint32_t* d_n, uint32_t cap,
                          cp_pair* out, int64_t out_cap, int64_t* d_out_count, Counters* ctr, cudaStream_t s);
cudaError_t launch_backward(const cp_pair* pairs, int64_t n, const float* gb, const float* gd, const int64_t* offs,
                            double* acc, float* grad, int64_t n_pixels, cudaStream_t s);

int device_sm_count();
// init() run once per device and slot (thread-safe), its result cached: the
// launch set-up of a kernel (attributes, occupancy-derived grid size).
enum { kCachePrune3d, kCachePrune2d, kCacheSort, kCacheUf, kCacheRoots, kCacheH1, kCacheBoruvka, kCacheSlots };
int device_cached(int slot, int (*init)());

// Kernel launches made by the library (for the benchmark's launch count).
void note_launches(int n);

// Loss sum(death - birth)^2 over finite pairs with death - birth > tau, and
// its gradient scattered to the pixels (double-precision accumulators).
cudaError_t launch_loss_backward(const cp_pair* pairs, int64_t n, const int64_t* d_n, float tau, const int64_t* offs,
                                 double* acc, double* partials, int nparts, double* d_loss, float* grad,
                                 int64_t n_pixels, cudaStream_t s);
int loss_partials();
cudaError_t launch_wait_test(Counters* ctr, const uint32_t* flag, uint64_t limit_ns, cudaStream_t s);

}  // namespace cp
