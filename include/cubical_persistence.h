/*
 * C-ABI of the GB300 (sm_103a) library for V-filtration cubical persistence
 * over F2 on float32 2D images and 3D volumes: the H0 pairs and the
 * top-dimension pairs (H1 in 2D, H2 in 3D), after local pruning through the
 * neighbourhood lookup table.  Method: arXiv 2606.04801, Sec. 2-4 and
 * Appendix A (H0 by elder-rule union-find on vertices and edges, Sec. 4.1
 * step 3 / Sec. 4.2 step 2; top dimension by union-find on the dual graph of
 * top cells plus one outside vertex, Sec. 3.1 and Appendix A; pruning,
 * Sec. 3.2; lookup table, Sec. 3.3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Images are C-order float32: (H, W) in 2D, (D, H, W) in 3D.  Every axis
 *    must be at least 2 long, every value finite.  -0.0 is read as +0.0.
 *  - Pixels are ordered by (value, linear index) (first-order tie-break);
 *    cells of one lower star by (dimension, doubled-grid index)
 *    (second-order tie-break).
 *  - A cell is named by its index in the doubled grid of its item: the cell
 *    with doubled coordinates (Z, Y, X) (Z = 0 in 2D) has index
 *    (Z*(2H-1) + Y)*(2W-1) + X; its dimension is the number of odd
 *    coordinates.  A pixel is named by its linear index in its item.
 *  - Limits per call: at most CP_MAX_ITEMS items; at most 2^27 pixels in
 *    total over all items; every doubled grid below 2^31 cells.
 *  - Memory: the caller owns every buffer and the stream.  Pointers marked
 *    d_ are device pointers, h_ host pointers.  The library allocates no
 *    device memory; it needs one caller-provided workspace whose size the
 *    *_workspace_size functions return.  Nothing is printed, nothing aborts.
 *  - Synchronisation: the work is enqueued on `stream`.  When h_out_count is
 *    non-NULL the call waits for the stream once, to read the pair count and
 *    the status word back; with h_out_count == NULL it returns right after
 *    enqueueing, d_out_count (if non-NULL) receives the count on the device,
 *    and cubical_persistence_stats() reads the status later.
 *  - Return value: CP_OK (0) or a negative CP_ERR_* code.
 */
#ifndef CUBICAL_PERSISTENCE_H
#define CUBICAL_PERSISTENCE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CP_MAX_ITEMS 128

enum {
    CP_OK = 0,
    CP_ERR_ARG = -1,       /* null pointer, axis < 2, too many pixels or items, bad sizes */
    CP_ERR_NONFINITE = -2, /* NaN or +-inf in an input image */
    CP_ERR_CAPACITY = -3,  /* an output or workspace capacity was too small; counts are still reported */
    CP_ERR_CUDA = -4,      /* a CUDA runtime call failed */
    CP_ERR_TIMEOUT = -5,   /* a bounded device-side wait gave up */
    CP_ERR_INTERNAL = -6   /* an internal consistency check failed */
};

/*
 * One persistence pair (32 bytes).
 *  birth, death   : values copied from the input (-0.0 reported as +0.0);
 *                   death = +inf for the essential H0 class.
 *  birth_cell     : doubled-grid index of the positive cell (a vertex for
 *                   H0, a facet for the top dimension).
 *  death_cell     : doubled-grid index of the negative cell (an edge for H0,
 *                   a top cell for the top dimension); -1 if essential.
 *  birth_pixel,
 *  death_pixel    : the pixel that gives the cell its value (its largest
 *                   vertex under (value, index)); -1 if essential.
 *  dim            : 0, or the top homology dimension (1 in 2D, 2 in 3D).
 *  item           : index of the item in a batched call (0 otherwise).
 * Only pairs with birth != death are reported (Sec. 2.3), sorted by
 * (item, dim, birth_cell).
 */
typedef struct cp_pair {
    float birth, death;
    int32_t birth_cell, death_cell;
    int32_t birth_pixel, death_pixel;
    int32_t dim, item;
} cp_pair;

/* Per-call counters, filled by cubical_persistence_stats(). */
typedef struct cp_stats {
    int64_t n_pixels;
    int64_t h0_survivors;     /* edges left for the H0 union-find after pruning */
    int64_t top_survivors;    /* facets left for the dual union-find after pruning */
    int64_t h0_roots;         /* local minima (roots of the H0 forest) */
    int64_t top_roots;        /* top cells left as roots of the dual forest */
    int64_t h0_rounds;        /* rounds of the H0 union-find */
    int64_t top_rounds;       /* rounds of the dual union-find */
    int64_t pairs;            /* reported pairs (nonzero persistence + essential) */
    uint32_t status;          /* raw device status bits */
    uint32_t mst_rounds;      /* Borůvka rounds (CP_TUNE_UF_VARIANT = 1), else 0 */
} cp_stats;

/* ---------------------------------------------------------------- info */

/* Library version (major*10000 + minor*100 + patch). */
int cp_version(void);

/* Human-readable name of a CP_* code; never NULL. */
const char *cp_error_string(int code);

/*
 * Number of relevant neighbourhood configurations of the lookup table
 * (Sec. 3.3): 47 for ndim = 2, 15,935 for ndim = 3; -1 for another ndim.
 * Host only; needs no GPU.
 */
int cp_lut_num_classes(int ndim);

/*
 * Lookup-table entry of a raw lower-neighbour mask (host only, for tests).
 * raw: bit n set when the neighbour at offset n precedes the vertex, with
 * n = 9(dz+1)+3(dy+1)+(dx+1) in 3D (bit 13 ignored) and n = 3(dy+1)+(dx+1)
 * in 2D (bit 4 ignored).  *relevant receives the collapsed mask, *entry the
 * 64-bit entry (layout documented in the library source).  Returns CP_OK or
 * CP_ERR_ARG.
 */
int cp_lut_lookup(int ndim, uint32_t raw, uint32_t *relevant, uint64_t *entry);

/*
 * Self-check of the 3D pruning kernel's mask form (host only, for tests):
 * the kernel builds the 26 neighbour comparisons into its own bit layout
 * and collapses them there with a few multiplications and masks (Sec. 3.3's
 * rule that an offset matters only when every nonzero sub-offset precedes).
 * This runs that collapse on the host for all 2^26 raw masks and compares it
 * with the definition; *n_mismatch receives the number of masks that
 * differ (0 when the layout is right).  Takes a few seconds.  Returns CP_OK,
 * or CP_ERR_ARG for a null pointer.
 */
int cp_lut_check_layout(uint64_t *n_mismatch);

/* ---------------------------------------------------------------- forward */

/*
 * Workspace bytes for one image (ndim 2 or 3, dims as for the image).
 * max_survivors bounds the edges (and, separately, the facets and the roots)
 * that survive pruning; 0 picks the default N/2 + 65536, which covers
 * i.i.d. noise and smoother inputs.  Adversarial inputs (checkerboards) may
 * need up to 2.5 N in 3D; a call that runs out returns CP_ERR_CAPACITY with
 * the required counts in cubical_persistence_stats().  Returns 0 on bad
 * arguments.
 */
size_t cubical_persistence_workspace_size(int ndim, const int64_t *dims, int64_t max_survivors);

/*
 * Persistence pairs of one 2D image (dims = {H, W}) (Sec. 4.1: lookup ->
 * local pruning -> H0 union-find -> cross-pruning -> H1 dual union-find).
 *  d_image     : device, H*W float32, read only.
 *  d_out_pairs : device, capacity entries, written with the sorted pairs.
 *  capacity    : entries available in d_out_pairs; H*W + (H-1)(W-1) + 1
 *                always suffices.
 *  h_out_count : host, optional: receives the number of pairs (may exceed
 *                capacity: then CP_ERR_CAPACITY and the first `capacity`
 *                pairs are not guaranteed).  Makes the call synchronous.
 *  d_out_count : device, optional int64: receives the count on the device.
 *  d_workspace : device, ws_bytes >= cubical_persistence_workspace_size().
 *  stream      : a cudaStream_t (NULL = legacy default stream).
 */
int cubical_persistence_2d(const float *d_image, const int64_t dims[2], cp_pair *d_out_pairs, int64_t capacity,
                           int64_t *h_out_count, int64_t *d_out_count, void *d_workspace, size_t ws_bytes,
                           int64_t max_survivors, void *stream);

/*
 * Persistence pairs of one 3D volume (dims = {D, H, W}) (Sec. 4.2 steps 1-3:
 * lookup -> H0 prune + union-find -> H2 prune + dual union-find).
 * Arguments as for cubical_persistence_2d; capacity D*H*W +
 * (D-1)(H-1)(W-1) + 1 always suffices.
 */
int cubical_persistence_3d(const float *d_image, const int64_t dims[3], cp_pair *d_out_pairs, int64_t capacity,
                           int64_t *h_out_count, int64_t *d_out_count, void *d_workspace, size_t ws_bytes,
                           int64_t max_survivors, void *stream);

/*
 * Slab split of the two union-finds (the parallelisation across devices that
 * Sec. 6 leaves to future work), run on one GPU.  The image is cut into
 * n_slabs slabs along its slowest axis (z for a volume, y for an image;
 * element c of that axis lies in slab c * n_slabs / extent).  After the
 * pruning pass, each root class of the pruned forests belongs to the slab of
 * the vertex its age key names (the outside vertex to slab 0), and a surviving
 * edge (facet) is internal when both endpoint classes lie in one slab,
 * crossing otherwise.
 *  Stage 1: the elder-rule union-find of every slab over its internal
 *  survivors (one launch; the slabs share no class).  A commit whose dying
 *  class has met no crossing survivor (no root of that class is an endpoint
 *  of one) writes its pair here: the whole image's union-find kills the same
 *  class then.  Every other commit is handed to stage 2 with its endpoints
 *  replaced by the two classes' roots at its time.
 *  Stage 2: one union-find over the handed-on commits and the crossing
 *  survivors, in filtration order; it writes the other pairs.
 * The result equals cubical_persistence_2d / _3d on the same image, pair for
 * pair.  Across devices, stage 2's input is what the slabs would exchange
 * (the boundary part of each slab's merge forest plus the crossing
 * survivors); h_stats reports its size.
 *  n_slabs  : 1 .. 65536 (more slabs than planes leaves some empty).
 *  h_stats  : host, optional: the split's counts (makes the call
 *             synchronous).
 *  d_workspace : ws_bytes >= cubical_persistence_slabs_workspace_size()
 *             with the same n_slabs.
 * Other arguments, ownership and errors as for cubical_persistence_2d /
 * _3d.  CP_ERR_ARG also when cross-pruning of images is switched on
 * (CP_TUNE_CROSS_PRUNE_2D = 1): both survivor lists must be ready before the
 * union-finds.  CP_ERR_CAPACITY when the two survivor lists together exceed
 * max_survivors.
 */
typedef struct cp_slab_stats {
    int64_t survivors[2];    /* [0] H0 edges, [1] dual facets, after pruning */
    int64_t internal[2];     /* survivors whose endpoint classes lie in one slab */
    int64_t crossing[2];     /* survivors whose endpoint classes lie in two slabs */
    int64_t committed[2];    /* internal survivors that their slab's union-find committed */
    int64_t final_pairs[2];  /* of those, the ones whose pairs stage 1 wrote (zero persistence included) */
    int64_t merged[2];       /* survivors of stage 2: committed - final_pairs + crossing */
    int64_t rounds_slab[2];  /* rounds of stage 1 (its slowest slab) */
    int64_t rounds_merge[2]; /* rounds of stage 2 */
} cp_slab_stats;
size_t cubical_persistence_slabs_workspace_size(int ndim, const int64_t *dims, int n_slabs, int64_t max_survivors);
int cubical_persistence_slabs(int ndim, const float *d_image, const int64_t *dims, int n_slabs, cp_pair *d_out_pairs,
                              int64_t capacity, int64_t *h_out_count, int64_t *d_out_count, void *d_workspace,
                              size_t ws_bytes, int64_t max_survivors, void *stream, cp_slab_stats *h_stats);

/*
 * T-filtration (the T-construction of Sec. 2.2; the paper leaves it to future
 * work in Sec. 6): the pixel values sit on the top cells of the lattice
 * complex [0,H]x[0,W] (x[0,D]), and every other cell takes the smallest value
 * of the top cells that contain it.  Refined order: a cell enters with the
 * top cell of smallest (value, linear pixel index) that contains it, then by
 * dimension, then by index in the T doubled grid, whose extents are 2n+1 per
 * axis (lattice points at even, pixels at odd coordinates; the cell with
 * doubled coordinates (Z, Y, X) has index (Z*(2H+1) + Y)*(2W+1) + X, Z = 0
 * in 2D).  Pairs: H0 (essential class: the oldest vertex, death +inf, death
 * cell -1) and the top dimension (H1 in 2D, H2 in 3D); pixels are the top
 * cells the birth and death cells enter with, so the backward entries apply
 * unchanged.
 * Computed by duality with the V pipeline on J = -image, flipped along every
 * axis, inside a one-voxel frame below every value: T-H0 is the V top
 * dimension of J, the T top dimension is V-H0 of J.
 *  - dims: every extent >= 1; (D+2)(H+2)(W+2) (3D) or (H+2)(W+2) (2D) at
 *    most 2^27.
 *  - Every pixel must be below the largest finite float (the frame sits at
 *    -FLT_MAX and must come first): otherwise CP_ERR_NONFINITE, as for NaN
 *    and +-inf.
 *  - capacity: D*H*W + (D+1)(H+1)(W+1) always suffices.
 *  - d_workspace: ws_bytes >= cubical_persistence_t_workspace_size(); it
 *    holds the V workspace of J (so cubical_persistence_stats() reads this
 *    call's counters from it), then J.
 * Other arguments, ownership and errors as for cubical_persistence_2d.
 */
size_t cubical_persistence_t_workspace_size(int ndim, const int64_t *dims, int64_t max_survivors);
int cubical_persistence_t_2d(const float *d_image, const int64_t dims[2], cp_pair *d_out_pairs, int64_t capacity,
                             int64_t *h_out_count, int64_t *d_out_count, void *d_workspace, size_t ws_bytes,
                             int64_t max_survivors, void *stream);
int cubical_persistence_t_3d(const float *d_image, const int64_t dims[3], cp_pair *d_out_pairs, int64_t capacity,
                             int64_t *h_out_count, int64_t *d_out_count, void *d_workspace, size_t ws_bytes,
                             int64_t max_survivors, void *stream);
/*
 * Batched T-filtration: n_items images and volumes (arguments laid out as
 * for cubical_persistence_batched, every extent >= 1, each padded item within
 * 2^27 vertices) in one pass; pairs carry their item index, cells and pixels
 * are item-local (T doubled grid).  Workspace:
 * cubical_persistence_t_batched_workspace_size().
 */
size_t cubical_persistence_t_batched_workspace_size(int n_items, const int32_t *ndims, const int64_t *dims,
                                                    int64_t max_survivors);
int cubical_persistence_t_batched(int n_items, const float *const *h_images, const int32_t *ndims,
                                  const int64_t *dims, cp_pair *d_out_pairs, int64_t capacity, int64_t *h_out_count,
                                  int64_t *d_out_count, void *d_workspace, size_t ws_bytes, int64_t max_survivors,
                                  void *stream);

/*
 * Batched form: n_items independent images and volumes of any sizes in one
 * pass (one lookup pass, one sort and one union-find per dimension for the
 * whole batch; unions never cross items).
 *  h_images : host array of n_items device pointers.
 *  ndims    : host array, 2 or 3 per item.
 *  dims     : host array of 3*n_items extents: (D, H, W) per item, D ignored
 *             (set to 1) for 2D items.
 * Pairs carry their item index and item-local cells and pixels.  The other
 * arguments are as for the single-image calls.
 */
size_t cubical_persistence_batched_workspace_size(int n_items, const int32_t *ndims, const int64_t *dims,
                                                  int64_t max_survivors);
int cubical_persistence_batched(int n_items, const float *const *h_images, const int32_t *ndims,
                                const int64_t *dims, cp_pair *d_out_pairs, int64_t capacity, int64_t *h_out_count,
                                int64_t *d_out_count, void *d_workspace, size_t ws_bytes, int64_t max_survivors,
                                void *stream);

/*
 * The whole diagram of volumes: the pairs of cubical_persistence_3d /
 * _batched plus the H1 pairs of every 3D item (dim 1; zero persistence
 * omitted; birth cell an edge, death cell a square, pixels their largest
 * vertices).  Sec. 4.2 (3D steps 4-5) computes the middle dimension of a
 * volume by an F2 matrix reduction over the cells that H0 and H2 leave
 * unpaired; here it is the column reduction (Sec. 2.1) of the boundary
 * matrix of the squares not paired in H2 over the edges not paired in H0,
 * in the refined order of
 * Sec. 2.3, on the device: first inside each lower star (a star's cells are
 * consecutive in that order), then, for the columns whose lowest entry
 * leaves their star, in parallel rounds.  2D items get their plain diagram.
 * Output order (item, dim, birth cell) as for the other calls.
 *  pool_entries : device pool entries (8 bytes each) for the columns that
 *                 additions across stars create (each addition writes
 *                 its result anew); 0 picks 4 per column + 2^20.  A call
 *                 that runs out returns
 *                 CP_ERR_CAPACITY (repeat with a larger pool).
 *  capacity     : E + (D-1)(H-1)(W-1) + 1 always suffices for a volume
 *                 (E = its edges).
 *  d_workspace  : ws_bytes >= cubical_persistence_full_workspace_size() /
 *                 cubical_persistence_full_batched_workspace_size().
 * Other arguments, ownership and errors as for cubical_persistence_3d and
 * cubical_persistence_batched.  CP_ERR_INTERNAL reports a failed count
 * check (merging edges N - 1, squares paired in H2 (D-1)(H-1)(W-1), one
 * column per unpaired edge).
 */
size_t cubical_persistence_full_workspace_size(int ndim, const int64_t *dims, int64_t max_survivors,
                                               int64_t pool_entries);
int cubical_persistence_full_3d(const float *d_image, const int64_t dims[3], cp_pair *d_out_pairs, int64_t capacity,
                                int64_t *h_out_count, int64_t *d_out_count, void *d_workspace, size_t ws_bytes,
                                int64_t max_survivors, int64_t pool_entries, void *stream);
size_t cubical_persistence_full_batched_workspace_size(int n_items, const int32_t *ndims, const int64_t *dims,
                                                       int64_t max_survivors, int64_t pool_entries);
int cubical_persistence_full_batched(int n_items, const float *const *h_images, const int32_t *ndims,
                                     const int64_t *dims, cp_pair *d_out_pairs, int64_t capacity,
                                     int64_t *h_out_count, int64_t *d_out_count, void *d_workspace, size_t ws_bytes,
                                     int64_t max_survivors, int64_t pool_entries, void *stream);
/*
 * The H1 stage of the last full call on this workspace (same item, size
 * and pool arguments as that call; waits for `stream`): h_info[0] columns,
 * [1] reduction rounds, [2] pool entries used, [3] pool entries available;
 * with cap >= 10 also [4] edges paired in H0, [5] squares paired in H2,
 * [6] edges not paired in H0, [7] and [8] the byte offsets of the two
 * bitmaps of those edges and squares (bit 3 * lowest corner + axis) in the
 * workspace, [9] columns whose lowest entry left their lower star; with
 * cap >= 13 also [10] the first round that the first CTA ran alone while
 * the others waited (0: never), [11] and [12] the wall time in ns of the
 * rounds on the whole grid and in that CTA alone; [13 + k] (k < 16, as far as cap allows) the
 * rounds in which 2^k .. 2^(k+1) - 1 columns added (k = 15: 2^15 or more);
 * [29 .. 32] thread 0 of the first CTA's time in ns, summed over the
 * rounds: its bids, the wait after them, its additions, the wait after them;
 * [33] column additions, [34] the entries those additions read, [35] times
 * the first CTA went on alone (cap >= 36 for [33 .. 35]).
 * cap >= 4.
 */
int cubical_persistence_full_info(const void *d_workspace, int n_items, const int32_t *ndims, const int64_t *dims,
                                  int64_t max_survivors, int64_t pool_entries, int64_t *h_info, int cap,
                                  void *stream);

/*
 * Counters and status of the last call that used this workspace (waits for
 * `stream`).  Returns the CP_* code the call would report.
 */
int cubical_persistence_stats(const void *d_workspace, cp_stats *h_stats, void *stream);

/* ---------------------------------------------------------------- backward */

/*
 * Gradient of a loss L(birth, death) with respect to the image pixels.
 * Each birth (death) value is a copy of one pixel, its birth_pixel
 * (death_pixel), so dL/dx[p] is the sum of dL/dbirth over the pairs born at
 * p plus the sum of dL/ddeath over the pairs that die at p.  Essential
 * deaths (death_pixel = -1) contribute nothing.
 *  d_pairs        : device, n_pairs pairs as returned by a forward call.
 *  d_grad_birth,
 *  d_grad_death   : device, n_pairs float32 each (dL/dbirth, dL/ddeath).
 *  d_item_offsets : device, int64 per item: offset of the item's first pixel
 *                   in d_grad_image (NULL for a single image).
 *  d_grad_image   : device, n_pixels float32, overwritten (zeros where no
 *                   pair lands).
 *  d_workspace    : device, cubical_persistence_backward_workspace_size()
 *                   bytes (double-precision accumulators).
 * Sums are accumulated in double precision and rounded once to float32.
 */
size_t cubical_persistence_backward_workspace_size(int64_t n_pixels);
int cubical_persistence_backward(const cp_pair *d_pairs, int64_t n_pairs, const float *d_grad_birth,
                                 const float *d_grad_death, const int64_t *d_item_offsets, float *d_grad_image,
                                 int64_t n_pixels, void *d_workspace, size_t ws_bytes, void *stream);

/*
 * Fused loss and backward for the total-persistence loss
 *   L = sum over finite pairs with death - birth > min_persistence
 *       of (death - birth)^2,
 * with dL/ddeath = 2 (death - birth) and dL/dbirth = -2 (death - birth)
 * scattered to the death and birth pixels as in cubical_persistence_backward.
 *  n_pairs   : number of pairs in d_pairs, or an upper bound when d_n_pairs
 *              is given;
 *  d_n_pairs : device, optional int64: the actual count (as written by a
 *              forward call's d_out_count), read on the device so that a
 *              forward + backward sequence needs no host round trip (and
 *              can be captured in a CUDA graph);
 *  d_loss    : device, one double, receives L (summed in a fixed order, so
 *              it is the same on every run).
 * Other arguments as for cubical_persistence_backward; the workspace size is
 * cubical_persistence_loss_backward_workspace_size(n_pixels).
 */
size_t cubical_persistence_loss_backward_workspace_size(int64_t n_pixels);
int cubical_persistence_loss_backward(const cp_pair *d_pairs, int64_t n_pairs, const int64_t *d_n_pairs,
                                      float min_persistence, double *d_loss, const int64_t *d_item_offsets,
                                      float *d_grad_image, int64_t n_pixels, void *d_workspace, size_t ws_bytes,
                                      void *stream);

/*
 * Backward scatter that allocates nothing (the paper has no counterpart: it
 * is a convenience of this library).  For callers that cannot allocate
 * device memory, such as code inside another framework's hooks without
 * access to its allocator, or deployments whose device memory is reserved
 * up front by another component, this computes exactly what
 * cubical_persistence_backward
 * computes, but keeps its double-precision accumulators in a fixed array
 * inside the library's device image instead of a caller-provided workspace.
 *  - The array holds cubical_persistence_backward_noalloc_max_pixels()
 *    (= 4,194,304) doubles, 32 MiB; every GPU that loads the library keeps it
 *    until the process exits.  n_pixels above that maximum returns
 *    CP_ERR_CAPACITY without touching the GPU.
 *  - The first call on a device looks the array's device address up
 *    (cudaGetSymbolAddress, with that device current); make that first call
 *    before any stream capture on that device.  The address is cached per
 *    device ordinal: a cudaDeviceReset of that device after its first call
 *    here is not supported.
 *  - Every call shares the one array: each call clears the part it uses
 *    before accumulating, so consecutive calls are independent, but calls
 *    whose work overlaps on the GPU (unordered streams) race on it.
 *  - It calls no allocating function.  Other arguments as for
 *    cubical_persistence_backward.
 */
int64_t cubical_persistence_backward_noalloc_max_pixels(void);
int cubical_persistence_backward_noalloc(const cp_pair *d_pairs, int64_t n_pairs, const float *d_grad_birth,
                                         const float *d_grad_death, const int64_t *d_item_offsets,
                                         float *d_grad_image, int64_t n_pixels, void *stream);

/* ---------------------------------------------------------------- instrumentation */

/*
 * Union-find trace of the last forward call that used this workspace (waits
 * for `stream`): for round i (up to min(cap, 48) rounds, plus the final
 * empty one), h_active[i] = survivors still unresolved at its start and
 * h_us[i] = microseconds since the start of round 0.  dual = 0 for H0, 1 for
 * the top dimension.  Returns the number of entries or a CP_ERR_* code.
 */
int cubical_persistence_uf_trace(const void *d_workspace, int dual, uint32_t *h_active, double *h_us, int cap,
                                 void *stream);
/* As above, plus (if non-NULL) the end of each round's find phase in
 * microseconds since the start of round 0, and the parent hops walked in it. */
int cubical_persistence_uf_trace2(const void *d_workspace, int dual, uint32_t *h_active, double *h_us,
                                  double *h_us_phase_a, uint64_t *h_hops, int cap, void *stream);

/*
 * Debugging and stage tests (not part of the method): run only the lookup +
 * pruning pass (K1) of a batched call, leaving in the workspace the H0
 * forest, the dual forest, the survivor keys and the roots; and report where
 * they are.  cubical_persistence_debug_layout writes 12 values: byte offsets
 * of the counters, H0 forest (uint32 per vertex), dual forest (uint32 per top
 * cell plus one outside vertex per item), H0 survivor keys (uint64), dual
 * survivor keys (uint64, stored complemented), H0 root ages, dual root ages;
 * then the total vertices, total top-cell slots, survivor capacity, H0 root
 * capacity and dual root capacity.  Forest words with the top bit set are
 * roots (low bits: root id).  Survivor and root counts are the 2nd to 5th
 * uint32 of the counters.  With cap >= 13 a 13th value follows: the byte
 * offset of a uint32 counting the 3D pruning tasks whose image planes were
 * loaded by TMA (the others use cp.async).  Returns the number of values
 * written (12 or 13) or a CP_ERR_* code.
 */
int cubical_persistence_debug_prune(int n_items, const float *const *h_images, const int32_t *ndims,
                                    const int64_t *dims, void *d_workspace, size_t ws_bytes, int64_t max_survivors,
                                    void *stream);
int cubical_persistence_debug_layout(int n_items, const int32_t *ndims, const int64_t *dims, int64_t max_survivors,
                                     int64_t *h_offsets, int cap);

/*
 * Failure-path test: a kernel waits, through the library's bounded-wait
 * routine (every device-side wait gives up the same way, after 2 s in
 * production), on a workspace word that nothing sets, and gives up after
 * limit_us microseconds (1 .. 2,000,000).  Needs a workspace of at
 * least 4 KiB.  Returns CP_ERR_TIMEOUT when the wait gave up as designed
 * (the CUDA context stays usable), another code otherwise.  Waits for
 * `stream`.
 */
int cubical_persistence_debug_wait_timeout(void *d_workspace, size_t ws_bytes, int64_t limit_us, void *stream);

/*
 * Tuning of the pruning pass (process-wide; read by the following calls;
 * results never depend on it).  Keys:
 *   CP_TUNE_ZCHUNK_3D    planes per 3D pruning task (4..4096, default 64)
 *   CP_TUNE_CTAS_PER_SM  3D pruning CTAs per SM (0 = as many as fit, default)
 *   CP_TUNE_ROWS_2D      rows per 2D pruning task (4 .. 4096; default 64)
 *   CP_TUNE_CROSS_PRUNE_2D  1: the top dimension of 2D images waits for H0
 *                        and takes only the edges H0 leaves positive (the
 *                        cross-pruning of Sec. 3.2, Sec. 4.1 step 4: two sorts
 *                        and two union-find launches in sequence); 0 (default):
 *                        both dimensions run at once (one sort and one
 *                        union-find launch), the dual list keeping the edges
 *                        the table cannot settle, which the dual union-find
 *                        then finds closing dual cycles.  Same pairs.
 *   CP_TUNE_H1_BUDGET_MS wall-clock budget in milliseconds of the cross-star
 *                        reduction rounds of the _full calls (0 .. 3,600,000;
 *                        default 30,000).  Those rounds run in one
 *                        non-preemptible cooperative launch; once the budget
 *                        is spent, every block leaves at the next round
 *                        boundary and the call returns CP_ERR_TIMEOUT (no
 *                        H1 pairs).  0 stops after the first round.
 *   CP_TUNE_H1_SOLO      the cross-star rounds: once at most this many
 *                        columns enter a round, the first CTA runs the rounds
 *                        alone while the others wait, until more than twice
 *                        as many enter one (0 .. 1024; 0: every round on the
 *                        whole grid; default 16).  Same pairs.
 *   CP_TUNE_UF_VARIANT   0 (default): the elder-rule union-find runs in
 *                        reservation rounds over every survivor; 1: Borůvka's
 *                        minimum spanning forest of the survivor graph first
 *                        (the survivors the union-find commits), then the
 *                        rounds over the forest's edges alone.  Same pairs.
 *                        Calls with H1 or with cross-pruning of images keep
 *                        0.  Read when the workspace is sized: set it before
 *                        the _workspace_size call.
 * cp_set_tuning returns CP_OK or CP_ERR_ARG; cp_get_tuning the value or -1.
 * The autotuner in the Python package picks these per GPU and shape.
 */
#define CP_TUNE_ZCHUNK_3D 1
#define CP_TUNE_CTAS_PER_SM 2
#define CP_TUNE_ROWS_2D 3
#define CP_TUNE_H1_BUDGET_MS 4
#define CP_TUNE_CROSS_PRUNE_2D 5
#define CP_TUNE_H1_SOLO 6
#define CP_TUNE_UF_VARIANT 7
int cp_set_tuning(int key, int value);
int cp_get_tuning(int key);

/* Kernel launches the library has made since it was loaded. */
long long cp_launch_count(void);

/*
 * cp_profile(1) makes every following forward call record CUDA events on its
 * stream between its stages; cp_stage_times() then waits for the last call
 * and writes the six stage durations in milliseconds (prune, sort H0,
 * union-find H0, sort dual, union-find dual, emit) into ms[0..5] and returns
 * 6 (or a negative CP_ERR_* code; cap must be >= 6).  Each sort stage
 * includes the first-round root walks of its list.  In a call with volumes
 * only, both lists are walked and sorted together and both union-finds run in
 * one launch: ms[1] and ms[2] hold those joint times and ms[3], ms[4] are 0.
 * In a cubical_persistence_slabs call, ms[2] holds stage 1 (the split and the
 * slabs' union-finds) and ms[4] stage 2 (marking, compaction and the merge
 * union-find).  cp_profile(0) stops recording.  Not thread-safe across concurrent calls.
 */
int cp_profile(int enable);
int cp_stage_times(float *ms, int cap);

#ifdef __cplusplus
}
#endif

#endif /* CUBICAL_PERSISTENCE_H */
