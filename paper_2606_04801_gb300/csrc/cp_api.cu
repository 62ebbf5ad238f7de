// C-ABI entry points: argument checks, workspace layout, lookup-table set-up
// and the enqueueing of the pipeline
//   init -> K1 prune -> K2 sort (H0) -> K3 H0 union-find (+ 2D cross-pruning)
//        -> K2 sort (dual) -> K3 dual union-find -> essential pairs
//        [-> H1 of the volumes: columns, sort, reduction, pairs]
//        -> K2 sort (pairs, canonical order) -> gather.
#include <algorithm>
#include <atomic>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "cp_common.cuh"
#include "cp_kernels.h"
#include "cp_lut.h"

namespace cp {

namespace {

std::mutex g_mu;
bool g_lut_built = false;
std::vector<uint64_t> g_lut2d;
Lut3D g_lut3d;
int g_lut2d_classes = 0;
uint64_t g_dev_ready = 0;  // bit d set once device d holds the tables
std::atomic<long long> g_launches{0};

// Optional stage timing: CUDA events recorded on the call's stream between
// stages (prune | sort H0 | union-find H0 | sort dual | union-find dual | emit).
constexpr int kStages = 6;
bool g_profile = false;
cudaEvent_t g_ev[kStages + 1];
bool g_ev_made = false;
bool g_ev_joint = false;  // the last profiled call ran both union-finds in one launch

void mark(int i, cudaStream_t s) {
    if (g_profile && g_ev_made) cudaEventRecord(g_ev[i], s);
}

// NVTX ranges on the host timeline of a forward call: one enclosing range and
// one per stage, marking when each stage is enqueued (a profiler that records
// NVTX, such as ncu with --nvtx, can filter or group the kernels by them).
struct StageRanges {
    int depth = 0;
    StageRanges() {
        nvtxRangePushA("cp.forward");
        depth = 1;
    }
    void next(const char* name) {
        if (depth == 2) nvtxRangePop();
        nvtxRangePushA(name);
        depth = 2;
    }
    ~StageRanges() {
        while (depth-- > 0) nvtxRangePop();
    }
};

bool build_host_luts() {
    if (g_lut_built) return true;
    build_lut2d(g_lut2d, &g_lut2d_classes);
    if (!build_lut3d(g_lut3d)) return false;
    g_lut_built = true;
    return true;
}

int ensure_device_tables() {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!build_host_luts()) return CP_ERR_INTERNAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CP_ERR_CUDA;
    if (dev < 64 && (g_dev_ready >> dev) & 1u) return CP_OK;
    const cudaError_t ue = upload_luts(g_lut2d.data(), g_lut3d.disp.data(), g_lut3d.entry.data(), g_lut3d.key.data());
    if (ue == cudaErrorInvalidValue) return CP_ERR_INTERNAL;  // the table failed its consistency checks
    if (ue != cudaSuccess) return CP_ERR_CUDA;
    if (dev < 64) g_dev_ready |= 1ull << dev;
    return CP_OK;
}

struct Plan {
    ItemTable tab;
    TmaMaps tma;  // plane tensor maps of the 3D items that take TMA loads
    int64_t ntot = 0, ttot = 0;
    uint32_t cap_s = 0, cap_r0 = 0, cap_rt = 0, cap_p = 0, cap_big = 0;
    // byte offsets into the workspace
    size_t o_ctr, o_uf0, o_uft, o_s0, o_st, o_salt, o_age0, o_res0, o_aget, o_rest;
    size_t o_act0, o_act1, o_yn, o_on, o_na0, o_na1, o_nb0, o_nb1, o_pairs, o_pvals, o_pvalt, o_hist, o_status;
    size_t o_hist2, o_status2;
    // H1 of the volumes (calls that ask for it): see H1Bufs
    bool h1 = false;
    uint32_t h1_mcap = 0, h1_neg = 0, h1_posq = 0;
    uint64_t h1_pool = 0;
    size_t h1_words = 0;
    size_t o_h1_neg, o_h1_pos, o_h1_ctl, o_h1_cmask, o_h1_coff, o_h1_clen, o_h1_ccap, o_h1_list0, o_h1_l0, o_h1_l1,
        o_h1_piv, o_h1_pool;
    // slab split of the union-finds (calls that ask for it): slabs per item
    // and the buffers of cp_slab.cu
    int slabs = 0;
    bool split_bufs = false;  // the compaction buffers below are laid out
    size_t o_sl_ctr, o_sl_flag, o_sl_vcnt, o_sl_k0, o_sl_k1, o_sl_act, o_sl_a, o_sl_b, o_sl_map, o_sl_sub0,
        o_sl_sub1, o_sl_died0, o_sl_died1;
    // the Borůvka variant of the union-finds (CP_TUNE_UF_VARIANT = 1)
    bool boruvka = false;
    size_t o_bv_comp0, o_bv_comp1, o_bv_best0, o_bv_best1, o_bv_hook0, o_bv_hook1, o_bv_act0, o_bv_act1;
    size_t bytes = 0;
};

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }
void plan_boruvka(Plan& P);

// h1: also lay out the H1 stage of the 3D items, with h1_pool pool entries
// for the columns that additions create (0: 4 per column + 2^20).
int make_plan(int n_items, const int32_t* ndims, const int64_t* dims, const float* const* imgs,
              int64_t max_survivors, Plan& P, bool h1 = false, int64_t h1_pool = 0) {
    if (n_items <= 0 || n_items > kMaxItems || !ndims || !dims) return CP_ERR_ARG;
    std::memset(&P.tab, 0, sizeof(P.tab));
    P.tab.n = n_items;
    // table order: 2D items first, then 3D items, each in the caller's order
    std::vector<int> order;
    for (int k = 0; k < 2; ++k)
        for (int i = 0; i < n_items; ++i)
            if (ndims[i] == (k == 0 ? 2 : 3)) order.push_back(i);
    if (int(order.size()) != n_items) return CP_ERR_ARG;
    int64_t voff = 0, toff = 0, edges = 0, facets = 0;
    int64_t h1_cols = 0, h1_neg = 0, h1_posq = 0;  // 3D items: sums of E - N + 1, N - 1, (D-1)(H-1)(W-1)
    int32_t t2 = 0, t3 = 0;
    for (int j = 0; j < n_items; ++j) {
        int i = order[j];
        Item& it = P.tab.it[j];
        it.ndim = ndims[i];
        it.D = it.ndim == 3 ? int32_t(dims[3 * i]) : 1;
        it.H = int32_t(dims[3 * i + 1]);
        it.W = int32_t(dims[3 * i + 2]);
        int64_t D = it.ndim == 3 ? dims[3 * i] : 1, H = dims[3 * i + 1], W = dims[3 * i + 2];
        if (H < 2 || W < 2 || (it.ndim == 3 && D < 2)) return CP_ERR_ARG;
        if (H > (1 << 27) || W > (1 << 27) || D > (1 << 27)) return CP_ERR_ARG;
        int64_t N = D * H * W;
        int64_t G = (2 * D - 1) * (2 * H - 1) * (2 * W - 1);
        if (N > (int64_t(1) << kVBits) || G >= (int64_t(1) << 31)) return CP_ERR_ARG;
        it.img = imgs ? imgs[i] : nullptr;
        if (imgs && !imgs[i]) return CP_ERR_ARG;
        it.voff = voff;
        it.toff = toff;
        it.T = (it.ndim == 3 ? D - 1 : 1) * (H - 1) * (W - 1);
        it.user = i;
        it.tma = -1;
        voff += N;
        toff += it.T + 1;
        if (it.ndim == 2) {
            it.tx = int32_t((W + prune_tile_x() - 1) / prune_tile_x());
            it.ty = int32_t((H + prune_tile_y2d() - 1) / prune_tile_y2d());
            it.tz = 1;
            it.tile0 = t2;
            t2 += it.tx * it.ty;
            P.tab.n2d++;
            edges += H * (W - 1) + (H - 1) * W;
            facets += H * (W - 1) + (H - 1) * W;
        } else {
            it.tx = int32_t((W + prune_tile_x3d() - 1) / prune_tile_x3d());
            it.ty = int32_t((H + prune_tile_y3d() - 1) / prune_tile_y3d());
            it.tz = int32_t((D + prune_tile_z3d() - 1) / prune_tile_z3d());
            it.tile0 = t3;
            t3 += it.tx * it.ty * it.tz;
            P.tab.n3d++;
            edges += D * H * (W - 1) + D * (H - 1) * W + (D - 1) * H * W;
            facets += D * (H - 1) * (W - 1) + (D - 1) * H * (W - 1) + (D - 1) * (H - 1) * W;
            h1_cols += D * H * (W - 1) + D * (H - 1) * W + (D - 1) * H * W - N + 1;
            h1_neg += N - 1;
            h1_posq += it.T;
        }
        if (voff > (int64_t(1) << kVBits) || toff > (int64_t(1) << kVBits) + kMaxItems) return CP_ERR_ARG;
    }
    P.tab.tiles2d = t2;
    P.tab.tiles3d = t3;
    int ntma = 0;
    for (int j = 0; j < n_items && imgs; ++j) {
        Item& it = P.tab.it[j];
        if (it.ndim == 3 && ntma < kMaxTma && encode_plane_map(&P.tma.m[ntma], it.img, it.D, it.H, it.W))
            it.tma = ntma++;
    }
    P.tab.rows2d = prune_tile_y2d();
    P.tab.zchunk3d = prune_tile_z3d();
    P.tab.cross2d = prune_cross2d();
    P.ntot = voff;
    P.ttot = toff;
    int64_t ms = max_survivors > 0 ? max_survivors : voff / 2 + 65536;
    ms = std::min<int64_t>(ms, std::max(edges, facets) + 1);
    ms = std::min<int64_t>(ms, int64_t(0x7FFFFFFF));
    P.cap_s = uint32_t(ms);
    P.cap_r0 = uint32_t(std::min<int64_t>(ms / 2 + n_items + 1024, voff + 1));
    P.cap_rt = uint32_t(std::min<int64_t>(ms / 2 + n_items + 1024, toff + 1));
    P.cap_p = P.cap_r0 + P.cap_rt;
    P.h1 = h1 && h1_cols > 0;
    if (P.h1) {
        if (h1_pool < 0 || int64_t(P.cap_p) + h1_cols > int64_t(0xFFFFFFFF) - 65536) return CP_ERR_ARG;
        P.h1_mcap = uint32_t(h1_cols);
        P.h1_neg = uint32_t(h1_neg);
        P.h1_posq = uint32_t(h1_posq);
        P.h1_pool = uint64_t(h1_pool > 0 ? h1_pool : 4 * h1_cols + (int64_t(1) << 20));
        P.cap_p += P.h1_mcap;  // H1 pairs (the nonzero ones are far fewer)
    }
    P.cap_big = std::max(P.cap_s, P.cap_p);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    P.o_ctr = take(sizeof(Counters));
    P.o_uf0 = take(sizeof(uint32_t) * size_t(P.ntot));
    P.o_uft = take(sizeof(uint32_t) * size_t(P.ttot));
    P.o_s0 = take(sizeof(uint64_t) * P.cap_big);
    P.o_st = take(sizeof(uint64_t) * P.cap_s);
    P.o_salt = take(sizeof(uint64_t) * P.cap_big);
    P.o_age0 = take(sizeof(uint64_t) * P.cap_r0);
    P.o_res0 = take(sizeof(uint64_t) * P.cap_r0);
    P.o_aget = take(sizeof(uint64_t) * P.cap_rt);
    P.o_rest = take(sizeof(uint64_t) * P.cap_rt);
    P.o_act0 = take(sizeof(uint32_t) * P.cap_big);
    P.o_act1 = take(sizeof(uint32_t) * P.cap_big);
    P.o_yn = take(sizeof(uint32_t) * P.cap_s);
    P.o_on = take(sizeof(uint32_t) * P.cap_s);
    P.o_na0 = take(sizeof(uint32_t) * P.cap_s);
    P.o_na1 = take(sizeof(uint32_t) * P.cap_s);
    P.o_nb0 = take(sizeof(uint32_t) * P.cap_s);
    P.o_nb1 = take(sizeof(uint32_t) * P.cap_s);
    // the pairs buffer also holds the dual list's sort scratch (key ping-pong,
    // endpoint root ids, payload) while both survivor lists are sorted together
    P.o_pairs = take(std::max(sizeof(cp_pair) * size_t(P.cap_p), size_t(8 + 4 + 4 + 4) * P.cap_s + 1024));
    P.o_pvals = P.o_act0;  // the active lists are dead once both union-finds are done
    P.o_pvalt = P.o_act1;
    P.o_hist = take(sizeof(uint32_t) * 8 * 256);
    P.o_status = take(sizeof(uint64_t) * sort_status_words(P.cap_big));
    P.o_hist2 = take(sizeof(uint32_t) * 8 * 256);
    P.o_status2 = take(sizeof(uint64_t) * sort_status_words(P.cap_s));
    if (P.h1) {
        const size_t m = P.h1_mcap;
        P.h1_words = (3 * size_t(P.ntot) + 31) / 32;
        P.o_h1_neg = take(sizeof(uint32_t) * P.h1_words);
        P.o_h1_pos = take(sizeof(uint32_t) * P.h1_words);
        const size_t ids = 3 * size_t(P.ntot);  // edge and square ids
        P.o_h1_ctl = take(sizeof(H1Ctl));
        P.o_h1_cmask = take(sizeof(uint32_t) * ids);
        P.o_h1_coff = take(sizeof(uint64_t) * ids);
        P.o_h1_clen = take(sizeof(uint32_t) * ids);
        P.o_h1_ccap = take(sizeof(uint32_t) * ids);
        P.o_h1_list0 = take(sizeof(uint32_t) * m);
        P.o_h1_l0 = take(sizeof(uint32_t) * m);
        P.o_h1_l1 = take(sizeof(uint32_t) * m);
        P.o_h1_piv = take(sizeof(uint64_t) * ids);
        P.o_h1_pool = take(sizeof(uint64_t) * P.h1_pool);
    }
    P.bytes = o;
    if (uf_variant() == 1) plan_boruvka(P);
    return CP_OK;
}

// Appends the slab split's buffers to a plan: S slabs per item (each item
// cut along its slowest axis).  Both survivor lists must sit side by side in
// the scratch lists, so 2D items with cross-pruning are refused.
// The stable compactions' buffers (shared by the slab split and the
// Borůvka variant).
void plan_split_buffers(Plan& P) {
    if (P.split_bufs) return;
    size_t o = P.bytes;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    P.split_bufs = true;
    P.o_sl_ctr = take(sizeof(SlabCtr));
    P.o_sl_flag = take(size_t(P.cap_s));
    P.o_sl_vcnt = take(sizeof(uint32_t) * slab_vblocks_cap(P.cap_s));
    P.o_sl_k0 = take(sizeof(uint64_t) * P.cap_s);
    P.o_sl_k1 = take(sizeof(uint64_t) * P.cap_s);
    P.o_sl_act = take(sizeof(uint32_t) * P.cap_s);
    P.o_sl_a = take(sizeof(uint32_t) * P.cap_s);
    P.o_sl_b = take(sizeof(uint32_t) * P.cap_s);
    P.o_sl_map = take(sizeof(uint32_t) * P.cap_s);
    P.o_sl_sub0 = take(sizeof(uint32_t) * P.cap_r0);
    P.o_sl_sub1 = take(sizeof(uint32_t) * P.cap_rt);
    P.o_sl_died0 = take(sizeof(uint32_t) * P.cap_r0);
    P.o_sl_died1 = take(sizeof(uint32_t) * P.cap_rt);
    P.bytes = o;
}

int plan_slabs(Plan& P, int S) {
    if (S < 1 || S > (1 << 16)) return CP_ERR_ARG;
    if (P.tab.n2d > 0 && P.tab.cross2d) return CP_ERR_ARG;
    if (P.h1) return CP_ERR_ARG;
    P.slabs = S;
    plan_split_buffers(P);
    return CP_OK;
}

// The Borůvka variant's arrays (calls whose two lists run side by side and
// without H1).
void plan_boruvka(Plan& P) {
    if (P.h1 || (P.tab.n2d > 0 && P.tab.cross2d)) return;
    plan_split_buffers(P);
    size_t o = P.bytes;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    P.boruvka = true;
    P.o_bv_comp0 = take(sizeof(uint32_t) * P.cap_r0);
    P.o_bv_comp1 = take(sizeof(uint32_t) * P.cap_rt);
    P.o_bv_best0 = take(sizeof(uint32_t) * P.cap_r0);
    P.o_bv_best1 = take(sizeof(uint32_t) * P.cap_rt);
    P.o_bv_hook0 = take(sizeof(uint32_t) * P.cap_r0);
    P.o_bv_hook1 = take(sizeof(uint32_t) * P.cap_rt);
    P.o_bv_act0 = take(sizeof(uint32_t) * P.cap_s);
    P.o_bv_act1 = take(sizeof(uint32_t) * P.cap_s);
    P.bytes = o;
}

template <class T>
T* at(void* ws, size_t off) {
    return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}

int status_to_code(uint32_t st) {
    if (st & kStNonfinite) return CP_ERR_NONFINITE;
    if (st & kStTimeout) return CP_ERR_TIMEOUT;
    if (st & kStCapacity) return CP_ERR_CAPACITY;
    if (st & (kStInternal | kStBounds)) return CP_ERR_INTERNAL;
    return CP_OK;
}

// T-filtration calls: the images' extents and dual images, and the input
// check's flag (run() flattens the frames after the pruning pass and maps the
// pairs of J back before the output sort).
struct TMode {
    TItems items;
    const uint32_t* bad;
};

int run(const Plan& P, cp_pair* d_out, int64_t capacity, int64_t* h_out_count, int64_t* d_out_count, void* ws,
        size_t ws_bytes, cudaStream_t s, bool prune_only = false, const TMode* tm = nullptr) {
    if (!ws || ws_bytes < P.bytes || (!d_out && capacity > 0) || capacity < 0) return CP_ERR_ARG;
    int rc = ensure_device_tables();
    if (rc != CP_OK) return rc;
    Counters* ctr = at<Counters>(ws, P.o_ctr);
    uint32_t* uf0 = at<uint32_t>(ws, P.o_uf0);
    uint32_t* uft = at<uint32_t>(ws, P.o_uft);
    uint64_t* s0 = at<uint64_t>(ws, P.o_s0);
    uint64_t* st = at<uint64_t>(ws, P.o_st);
    uint64_t* salt = at<uint64_t>(ws, P.o_salt);
    uint64_t* age0 = at<uint64_t>(ws, P.o_age0);
    uint64_t* res0 = at<uint64_t>(ws, P.o_res0);
    uint64_t* aget = at<uint64_t>(ws, P.o_aget);
    uint64_t* rest = at<uint64_t>(ws, P.o_rest);
    uint32_t* act0 = at<uint32_t>(ws, P.o_act0);
    uint32_t* act1 = at<uint32_t>(ws, P.o_act1);
    cp_pair* pairs = at<cp_pair>(ws, P.o_pairs);
    uint32_t* hist = at<uint32_t>(ws, P.o_hist);
    uint64_t* status = at<uint64_t>(ws, P.o_status);

#define CP_TRY(x)                                  \
    do {                                           \
        if ((x) != cudaSuccess) return CP_ERR_CUDA; \
    } while (0)
    StageRanges nv;
    nv.next("cp.prune");
    CP_TRY(cudaMemsetAsync(ctr, 0, sizeof(Counters), s));
    CP_TRY(launch_init(P.tab, ctr, uft, aget, rest, s));
    mark(0, s);
    if (prune_only) {
        PruneOuts po;
        po.uf0 = uf0;
        po.uft = uft;
        po.s0 = s0;
        po.st = st;
        po.age0 = age0;
        po.res0 = res0;
        po.aget = aget;
        po.rest = rest;
        po.cap_s = P.cap_s;
        po.cap_r0 = P.cap_r0;
        po.cap_rt = P.cap_rt;
        po.ctr = ctr;
        po.n_uf0 = uint32_t(P.ntot);
        po.n_uft = uint32_t(P.ttot);
        CP_TRY(launch_prune(P.tab, po, P.tma, s));
        mark(1, s);
        return CP_OK;
    }

    H1Bufs hb = {};
    if (P.h1) {
        hb.neg_e = at<uint32_t>(ws, P.o_h1_neg);
        hb.pos_q = at<uint32_t>(ws, P.o_h1_pos);
        hb.map_words = P.h1_words;
        hb.ctl = at<H1Ctl>(ws, P.o_h1_ctl);
        hb.cmask = at<uint32_t>(ws, P.o_h1_cmask);
        hb.coff = at<uint64_t>(ws, P.o_h1_coff);
        hb.clen = at<uint32_t>(ws, P.o_h1_clen);
        hb.ccap = at<uint32_t>(ws, P.o_h1_ccap);
        hb.list0 = at<uint32_t>(ws, P.o_h1_list0);
        hb.list[0] = at<uint32_t>(ws, P.o_h1_l0);
        hb.list[1] = at<uint32_t>(ws, P.o_h1_l1);
        hb.pivot = at<uint64_t>(ws, P.o_h1_piv);
        hb.pool = at<uint64_t>(ws, P.o_h1_pool);
        hb.pool_cap = P.h1_pool;
        hb.mcap = P.h1_mcap;
        hb.exp_neg_e = P.h1_neg;
        hb.exp_pos_q = P.h1_posq;
        hb.n_ids = uint32_t(3 * P.ntot);
        // the union-finds mark their committed survivors in these
        CP_TRY(cudaMemsetAsync(hb.neg_e, 0, sizeof(uint32_t) * P.h1_words, s));
        CP_TRY(cudaMemsetAsync(hb.pos_q, 0, sizeof(uint32_t) * P.h1_words, s));
    }

    PruneOuts po;
    po.uf0 = uf0;
    po.uft = uft;
    po.s0 = s0;
    po.st = st;
    po.age0 = age0;
    po.res0 = res0;
    po.aget = aget;
    po.rest = rest;
    po.cap_s = P.cap_s;
    po.cap_r0 = P.cap_r0;
    po.cap_rt = P.cap_rt;
    po.ctr = ctr;
    po.n_uf0 = uint32_t(P.ntot);
    po.n_uft = uint32_t(P.ttot);
    CP_TRY(launch_prune(P.tab, po, P.tma, s));
    if (tm) CP_TRY(launch_t_flatten(uf0, tm->items, s));
    mark(1, s);
    nv.next("cp.roots+sort");

    // First-round root walks over the unsorted survivors (tile order), then the
    // sort carrying each survivor's position, then the first active list.
    // Scratch while a list is being prepared: na1 / nb1 hold the endpoints'
    // root ids and act1 / ynode the sort payload (none of these is live yet).
    uint32_t* na0 = at<uint32_t>(ws, P.o_na0);
    uint32_t* na1 = at<uint32_t>(ws, P.o_na1);
    uint32_t* nb0 = at<uint32_t>(ws, P.o_nb0);
    uint32_t* nb1 = at<uint32_t>(ws, P.o_nb1);
    uint32_t* ynode = at<uint32_t>(ws, P.o_yn);
    RootArgs ra;
    ra.tab = P.tab;
    ra.cap = P.cap_s;
    ra.ra = na1;
    ra.rb = nb1;
    ra.pos = act1;
    ra.sorted_pos = act1;  // an even number of passes leaves the payload in place
    ra.scratch_cap = P.cap_s;
    ra.act = act0;
    ra.na = na0;
    ra.nb = nb0;
    ra.ctr = ctr;
    ra.n_nodes = uint32_t(P.ntot);
    SortBufs sb;
    sb.keys_alt = salt;
    sb.vals = act1;
    sb.vals_alt = ynode;
    sb.cap = P.cap_s;
    sb.hist = hist;
    sb.status = status;
    sb.ctr = ctr;
    auto prepare = [&](int dual, const uint32_t* d_n_before) -> cudaError_t {
        ra.keys = dual ? st : s0;
        ra.d_n = dual ? &ctr->n_st : &ctr->n_s0;
        ra.uf = dual ? uft : uf0;
        ra.n_nodes = uint32_t(dual ? P.ttot : P.ntot);
        ra.dual = dual;
        ra.d_n_before = d_n_before;
        cudaError_t e = launch_roots(ra, s);
        if (e != cudaSuccess) return e;
        sb.keys = dual ? st : s0;
        sb.d_count = ra.d_n;
        sb.tile_ctr = ctr->sort_tile + (dual ? 8 : 0);
        e = sort_keys(sb, 0, 8, dual ? 9 : 1, s);
        if (e != cudaSuccess) return e;
        return launch_place_roots(ra, s);
    };
    // The two lists are independent unless 2D items use cross-pruning (their
    // dual list then waits for the H0 union-find).
    const bool joint = P.tab.n2d == 0 || !P.tab.cross2d;
    if (joint) {
        // both lists walked, then sorted together (one launch per pass), then
        // placed side by side; the dual list's scratch sits in the pairs buffer
        uint64_t* salt2 = reinterpret_cast<uint64_t*>(pairs);
        uint32_t* raT = reinterpret_cast<uint32_t*>(salt2 + P.cap_s);
        uint32_t* rbT = raT + P.cap_s;
        uint32_t* posT = rbT + P.cap_s;
        RootArgs rt = ra;
        rt.keys = st;
        rt.d_n = &ctr->n_st;
        rt.uf = uft;
        rt.n_nodes = uint32_t(P.ttot);
        rt.dual = 1;
        rt.ra = raT;
        rt.rb = rbT;
        rt.pos = posT;
        rt.sorted_pos = posT;
        rt.d_n_before = &ctr->n_s0;
        ra.keys = s0;
        ra.d_n = &ctr->n_s0;
        ra.uf = uf0;
        ra.n_nodes = uint32_t(P.ntot);
        ra.dual = 0;
        ra.d_n_before = nullptr;
        CP_TRY(launch_roots2(ra, rt, s));
        SortBufs two[2] = {sb, sb};
        two[0].keys = s0;
        two[0].d_count = &ctr->n_s0;
        two[0].tile_ctr = ctr->sort_tile;
        two[1].keys = st;
        two[1].keys_alt = salt2;
        two[1].vals = posT;
        two[1].vals_alt = at<uint32_t>(ws, P.o_on);
        two[1].d_count = &ctr->n_st;
        two[1].hist = at<uint32_t>(ws, P.o_hist2);
        two[1].status = at<uint64_t>(ws, P.o_status2);
        CP_TRY(sort_keys_multi(two, 2, 0, 8, 1, s));
        CP_TRY(launch_place_roots(ra, s));
        CP_TRY(launch_place_roots(rt, s));
    } else {
        CP_TRY(prepare(0, nullptr));
    }
    mark(2, s);
    nv.next("cp.union-find");

    UfParams up[2];
    up[0].keys = s0;
    up[0].d_nkeys = &ctr->n_s0;
    up[0].cap_keys = P.cap_s;
    up[0].uf = uf0;
    up[0].age = age0;
    up[0].res = res0;
    up[0].act[0] = act0;
    up[0].act[1] = act1;
    up[0].na[0] = na0;
    up[0].na[1] = na1;
    up[0].nb[0] = nb0;
    up[0].nb[1] = nb1;
    up[0].ynode = ynode;
    up[0].onode = at<uint32_t>(ws, P.o_on);
    up[0].scratch_cap = P.cap_s;
    up[0].log = salt;  // the sort's spare buffer is free from here to the pair sort
    up[0].pairs = pairs;
    up[0].pair_cap = P.cap_p;
    up[0].dual_keys = joint ? nullptr : st;  // cross-pruning feeds the dual list of 2D items
    up[0].d_ndual = &ctr->n_st;
    up[0].dual_cap = P.cap_s;
    up[0].ctr = ctr;
    up[0].dual = 0;
    up[1] = up[0];
    up[1].keys = st;
    up[1].d_nkeys = &ctr->n_st;
    up[1].uf = uft;
    up[1].age = aget;
    up[1].res = rest;
    up[1].dual_keys = nullptr;
    up[1].d_ndual = nullptr;
    up[1].dual_cap = 0;
    up[1].dual = 1;
    up[0].h1flags = P.h1 ? hb.neg_e : nullptr;
    up[1].h1flags = P.h1 ? hb.pos_q : nullptr;
    up[0].n_nodes = uint32_t(P.ntot);
    up[0].n_rids = P.cap_r0;
    up[1].n_nodes = uint32_t(P.ttot);
    up[1].n_rids = P.cap_rt;

    if (!joint) {
        // the H0 union-find appends positive edges of 2D items to the dual list
        // (cross-pruning): the dual list is prepared after it
        g_ev_joint = false;
        CP_TRY(launch_uf(P.tab, &up[0], 1, s));
        mark(3, s);
        CP_TRY(prepare(1, nullptr));
        mark(4, s);
        CP_TRY(launch_uf(P.tab, &up[1], 1, s));
        mark(5, s);
    } else if (P.slabs > 0) {
        // slab split: each slab's union-find over the survivors inside it (one
        // launch for all slabs), then one union-find over what they committed
        // and the survivors between slabs
        mark(3, s);
        g_ev_joint = true;
        SlabCtr* sc = at<SlabCtr>(ws, P.o_sl_ctr);
        CP_TRY(cudaMemsetAsync(sc, 0, sizeof(SlabCtr), s));
        SlabArgs sa;
        sa.tab = P.tab;
        sa.S = P.slabs;
        sa.d_n[0] = &ctr->n_s0;
        sa.d_n[1] = &ctr->n_st;
        sa.cap = P.cap_s;
        sa.keys[0] = s0;
        sa.keys[1] = st;
        sa.age[0] = age0;
        sa.age[1] = aget;
        sa.n_rids[0] = P.cap_r0;
        sa.n_rids[1] = P.cap_rt;
        sa.res[0] = res0;
        sa.res[1] = rest;
        sa.na = na0;
        sa.nb = nb0;
        sa.sub[0] = at<uint32_t>(ws, P.o_sl_sub0);
        sa.sub[1] = at<uint32_t>(ws, P.o_sl_sub1);
        sa.died[0] = at<uint32_t>(ws, P.o_sl_died0);
        sa.died[1] = at<uint32_t>(ws, P.o_sl_died1);
        sa.pairs = pairs;
        sa.pair_cap = P.cap_p;
        sa.flag = at<uint8_t>(ws, P.o_sl_flag);
        sa.vcnt = at<uint32_t>(ws, P.o_sl_vcnt);
        sa.sc = sc;
        sa.ctr = ctr;
        sa.ko[0] = at<uint64_t>(ws, P.o_sl_k0);
        sa.ko[1] = at<uint64_t>(ws, P.o_sl_k1);
        sa.act = at<uint32_t>(ws, P.o_sl_act);
        sa.oa = at<uint32_t>(ws, P.o_sl_a);
        sa.ob = at<uint32_t>(ws, P.o_sl_b);
        sa.map = at<uint32_t>(ws, P.o_sl_map);
        sa.log = salt;
        CP_TRY(launch_slab_classify(sa, s));
        CP_TRY(launch_slab_compact(sa, 0, sc->n_in, s));
        // stage 1 works on its own active lists: the full lists' root ids in
        // na0 / nb0 stay for stage 2 (the marking pass rewrites the slots of
        // the commits it hands on)
        UfParams u[2] = {up[0], up[1]};
        for (int q = 0; q < 2; ++q) {
            u[q].keys = sa.ko[q];
            u[q].d_nkeys = &sc->n_in[q];
            u[q].act[0] = sa.act;
            u[q].na[0] = sa.oa;
            u[q].nb[0] = sa.ob;
            u[q].pairs = nullptr;
            u[q].h1flags = nullptr;
            u[q].dual_keys = nullptr;
            u[q].d_ndual = nullptr;
        }
        CP_TRY(launch_uf(P.tab, u, 2, s));
        mark(4, s);  // stage times: stage 1 in the union-find slot, stage 2 in the dual one
        CP_TRY(launch_slab_mark(sa, s));
        sa.map = nullptr;
        CP_TRY(launch_slab_compact(sa, 1, sc->n_merge, s));
        for (int q = 0; q < 2; ++q) {
            u[q].d_nkeys = &sc->n_merge[q];
            u[q].pairs = up[q].pairs;
        }
        CP_TRY(launch_uf(P.tab, u, 2, s));
        mark(5, s);
    } else if (P.boruvka) {
        // Borůvka's forest of both lists, then the union-find rounds over its
        // edges alone (compacted in order); stage times: the forest in the
        // union-find slot, compaction and pairing in the dual one
        mark(3, s);
        g_ev_joint = true;
        SlabCtr* sc = at<SlabCtr>(ws, P.o_sl_ctr);
        CP_TRY(cudaMemsetAsync(sc, 0, sizeof(SlabCtr), s));
        BoruvkaArgs ba;
        ba.d_n[0] = &ctr->n_s0;
        ba.d_n[1] = &ctr->n_st;
        ba.cap = P.cap_s;
        ba.n_rids[0] = P.cap_r0;
        ba.n_rids[1] = P.cap_rt;
        ba.na = na0;
        ba.nb = nb0;
        ba.comp[0] = at<uint32_t>(ws, P.o_bv_comp0);
        ba.comp[1] = at<uint32_t>(ws, P.o_bv_comp1);
        ba.best[0] = at<uint32_t>(ws, P.o_bv_best0);
        ba.best[1] = at<uint32_t>(ws, P.o_bv_best1);
        ba.hook[0] = at<uint32_t>(ws, P.o_bv_hook0);
        ba.hook[1] = at<uint32_t>(ws, P.o_bv_hook1);
        ba.act[0] = at<uint32_t>(ws, P.o_bv_act0);
        ba.act[1] = at<uint32_t>(ws, P.o_bv_act1);
        ba.flag = at<uint8_t>(ws, P.o_sl_flag);
        ba.d_rounds = &ctr->mst_rounds;
        ba.ctr = ctr;
        CP_TRY(launch_boruvka(ba, s));
        mark(4, s);
        SlabArgs sa = {};
        sa.tab = P.tab;
        sa.S = 1;
        sa.d_n[0] = &ctr->n_s0;
        sa.d_n[1] = &ctr->n_st;
        sa.cap = P.cap_s;
        sa.keys[0] = s0;
        sa.keys[1] = st;
        sa.n_rids[0] = P.cap_r0;
        sa.n_rids[1] = P.cap_rt;
        sa.na = na0;
        sa.nb = nb0;
        sa.flag = ba.flag;
        sa.vcnt = at<uint32_t>(ws, P.o_sl_vcnt);
        sa.sc = sc;
        sa.ctr = ctr;
        sa.ko[0] = at<uint64_t>(ws, P.o_sl_k0);
        sa.ko[1] = at<uint64_t>(ws, P.o_sl_k1);
        sa.act = at<uint32_t>(ws, P.o_sl_act);
        sa.oa = at<uint32_t>(ws, P.o_sl_a);
        sa.ob = at<uint32_t>(ws, P.o_sl_b);
        sa.map = nullptr;
        CP_TRY(launch_slab_compact(sa, 0, sc->n_in, s));
        UfParams u[2] = {up[0], up[1]};
        for (int q = 0; q < 2; ++q) {
            u[q].keys = sa.ko[q];
            u[q].d_nkeys = &sc->n_in[q];
            u[q].act[0] = sa.act;
            u[q].na[0] = sa.oa;
            u[q].nb[0] = sa.ob;
        }
        CP_TRY(launch_uf(P.tab, u, 2, s));
        mark(5, s);
    } else {
        // both union-finds share one launch and its rounds (the dual list after
        // the H0 list)
        mark(3, s);
        g_ev_joint = true;
        CP_TRY(launch_uf(P.tab, up, 2, s));
        mark(4, s);
        mark(5, s);
    }

    nv.next("cp.emit");
    CP_TRY(launch_essential(P.tab, ctr, pairs, P.cap_p, s));
    if (P.h1) {
        nv.next("cp.h1");
        CP_TRY(launch_h1(P.tab, hb, ctr, pairs, P.cap_p, s));
        nv.next("cp.emit");
    }
    uint32_t* pvals = at<uint32_t>(ws, P.o_pvals);
    uint32_t* pvalt = at<uint32_t>(ws, P.o_pvalt);
    // output order (item, dim, birth cell): only as many key bytes as this call's
    // item count and largest doubled grid need (4 for one 512^3 volume)
    int cell_bits = 1, item_bits = 0;
    for (int i = 0; i < P.tab.n; ++i) {
        const Item& it = P.tab.it[i];
        int64_t G = int64_t(2 * it.D - 1) * (2 * it.H - 1) * (2 * it.W - 1);
        if (tm) {  // the T-complex of the original image
            const TDims& d = tm->items.d[it.user];
            G = (d.ndim == 3 ? 2 * d.D + 1 : 1) * (2 * d.H + 1) * (2 * d.W + 1);
        }
        while ((int64_t(1) << cell_bits) < G) ++cell_bits;
    }
    if (tm) CP_TRY(launch_t_map(pairs, &ctr->n_pairs, P.cap_p, tm->items, tm->bad, ctr, s));
    // T calls: one more item index, for the dropped frame classes
    while ((1 << item_bits) < P.tab.n + (tm ? 1 : 0)) ++item_bits;
    const int dim_bits = P.h1 ? 2 : 1;
    int pair_passes = (item_bits + dim_bits + cell_bits + 7) / 8;
    pair_passes += pair_passes & 1;  // an even count leaves the result in place
    CP_TRY(launch_pair_keys(pairs, &ctr->n_pairs, P.cap_p, s0, pvals, cell_bits, dim_bits, s));
    sb.keys = s0;
    sb.keys_alt = salt;
    sb.vals = pvals;
    sb.vals_alt = pvalt;
    sb.d_count = &ctr->n_pairs;
    sb.cap = P.cap_p;
    sb.tile_ctr = ctr->sort_tile + 16;
    CP_TRY(sort_keys(sb, 0, pair_passes, 17, s));
    CP_TRY(launch_gather(pairs, pvals, tm ? &ctr->t_keep : &ctr->n_pairs, P.cap_p, d_out, capacity, d_out_count, ctr,
                         s));
    mark(6, s);
#undef CP_TRY
    if (h_out_count) {
        Counters h;
        if (cudaMemcpyAsync(&h, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CP_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return CP_ERR_CUDA;
        *h_out_count = h.out_count;
        return status_to_code(h.status);
    }
    return CP_OK;
}

int single(int ndim, const float* d_image, const int64_t* dims, cp_pair* d_out, int64_t capacity,
           int64_t* h_out_count, int64_t* d_out_count, void* ws, size_t ws_bytes, int64_t max_survivors,
           void* stream, bool h1 = false, int64_t h1_pool = 0) {
    if (!d_image || !dims) return CP_ERR_ARG;
    int32_t nd = ndim;
    int64_t d3[3] = {ndim == 3 ? dims[0] : 1, dims[ndim - 2], dims[ndim - 1]};
    Plan P;
    int rc = make_plan(1, &nd, d3, &d_image, max_survivors, P, h1, h1_pool);
    if (rc != CP_OK) return rc;
    return run(P, d_out, capacity, h_out_count, d_out_count, ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

// T-filtration: workspace = [the V workspace of the dual images][256 B
// scratch][J of item 0][J of item 1]... (each 256-byte aligned).
bool t_extents(int n_items, const int32_t* ndims, const int64_t* dims, TItems& t, std::vector<int64_t>& jdims) {
    if (n_items < 1 || n_items > kMaxItems || !ndims || !dims) return false;
    t.n = n_items;
    jdims.assign(size_t(3 * n_items), 1);
    for (int i = 0; i < n_items; ++i) {
        if (ndims[i] != 2 && ndims[i] != 3) return false;
        TDims& d = t.d[i];
        d.ndim = ndims[i];
        d.D = d.ndim == 3 ? dims[3 * i] : 1;
        d.H = dims[3 * i + 1];
        d.W = dims[3 * i + 2];
        if (d.D < 1 || d.H < 1 || d.W < 1) return false;
        jdims[3 * i] = d.ndim == 3 ? d.D + 2 : 1;
        jdims[3 * i + 1] = d.H + 2;
        jdims[3 * i + 2] = d.W + 2;
    }
    return true;
}

size_t t_workspace(int n_items, const int32_t* ndims, const int64_t* dims, int64_t max_survivors,
                   size_t* v_bytes) {
    TItems t;
    std::vector<int64_t> jd;
    if (!t_extents(n_items, ndims, dims, t, jd)) return 0;
    Plan P;
    if (make_plan(n_items, ndims, jd.data(), nullptr, max_survivors, P) != CP_OK) return 0;
    if (v_bytes) *v_bytes = P.bytes;
    size_t b = align_up(P.bytes) + 256;
    for (int i = 0; i < n_items; ++i) b += align_up(sizeof(float) * size_t(jd[3 * i] * jd[3 * i + 1] * jd[3 * i + 2]));
    return b;
}

int t_run(int n_items, const float* const* h_images, const int32_t* ndims, const int64_t* dims, cp_pair* d_out,
          int64_t capacity, int64_t* h_out_count, int64_t* d_out_count, void* ws, size_t ws_bytes,
          int64_t max_survivors, void* stream) {
    if (!h_images || !ws) return CP_ERR_ARG;
    TMode tm;
    std::vector<int64_t> jd;
    if (!t_extents(n_items, ndims, dims, tm.items, jd)) return CP_ERR_ARG;
    size_t v_bytes = 0;
    const size_t need = t_workspace(n_items, ndims, dims, max_survivors, &v_bytes);
    if (need == 0 || ws_bytes < need) return CP_ERR_ARG;
    int rc = ensure_device_tables();
    if (rc != CP_OK) return rc;
    char* base = static_cast<char*>(ws);
    uint32_t* bad = reinterpret_cast<uint32_t*>(base + align_up(v_bytes));
    size_t off = align_up(v_bytes) + 256;
    std::vector<const float*> jptr(static_cast<size_t>(n_items));
    for (int i = 0; i < n_items; ++i) {
        if (!h_images[i]) return CP_ERR_ARG;
        tm.items.img[i] = h_images[i];
        tm.items.J[i] = reinterpret_cast<float*>(base + off);
        jptr[size_t(i)] = tm.items.J[i];
        off += align_up(sizeof(float) * size_t(jd[3 * i] * jd[3 * i + 1] * jd[3 * i + 2]));
    }
    Plan P;
    rc = make_plan(n_items, ndims, jd.data(), jptr.data(), max_survivors, P);
    if (rc != CP_OK) return rc;
    for (int j = 0; j < P.tab.n; ++j) tm.items.voff[P.tab.it[j].user] = P.tab.it[j].voff;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (launch_t_build(tm.items, bad, s) != cudaSuccess) return CP_ERR_CUDA;
    tm.bad = bad;
    return run(P, d_out, capacity, h_out_count, d_out_count, ws, v_bytes, s, false, &tm);
}

int t_single(int ndim, const float* d_image, const int64_t* dims, cp_pair* d_out, int64_t capacity,
             int64_t* h_out_count, int64_t* d_out_count, void* ws, size_t ws_bytes, int64_t max_survivors,
             void* stream) {
    if (!d_image || !dims || (ndim != 2 && ndim != 3)) return CP_ERR_ARG;
    const int32_t nd = ndim;
    const int64_t d3[3] = {ndim == 3 ? dims[0] : 1, dims[ndim - 2], dims[ndim - 1]};
    return t_run(1, &d_image, &nd, d3, d_out, capacity, h_out_count, d_out_count, ws, ws_bytes, max_survivors,
                 stream);
}

}  // namespace

void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int device_sm_count() {
    static std::atomic<int> cached[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64) {
        const int c = cached[dev].load(std::memory_order_relaxed);
        if (c) return c;
    }
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
    if (dev >= 0 && dev < 64) cached[dev].store(n, std::memory_order_relaxed);
    return n;
}

int device_cached(int slot, int (*init)()) {
    static std::atomic<int> cache[64][kCacheSlots];
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || slot < 0 || slot >= kCacheSlots) return init();
    int v = cache[dev][slot].load(std::memory_order_acquire);
    if (v) return v;
    std::lock_guard<std::mutex> lk(mu);
    v = cache[dev][slot].load(std::memory_order_relaxed);
    if (!v) {
        v = init();
        cache[dev][slot].store(v, std::memory_order_release);
    }
    return v;
}

}  // namespace cp

using namespace cp;

extern "C" {

int cp_version(void) { return 100; }

const char* cp_error_string(int code) {
    switch (code) {
        case CP_OK: return "ok";
        case CP_ERR_ARG: return "invalid argument";
        case CP_ERR_NONFINITE: return "non-finite value in the input";
        case CP_ERR_CAPACITY: return "capacity exceeded";
        case CP_ERR_CUDA: return "CUDA runtime error";
        case CP_ERR_TIMEOUT: return "bounded device wait gave up";
        case CP_ERR_INTERNAL: return "internal consistency check failed";
        default: return "unknown error";
    }
}

int cp_lut_num_classes(int ndim) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!build_host_luts()) return -1;
    if (ndim == 2) return g_lut2d_classes;
    if (ndim == 3) return g_lut3d.nclasses;
    return -1;
}

int cp_lut_lookup(int ndim, uint32_t raw, uint32_t* relevant, uint64_t* entry) {
    if (ndim != 2 && ndim != 3) return CP_ERR_ARG;
    const Stencil& st = stencil(ndim);
    raw &= ~(1u << st.center);
    raw &= (1u << st.nbits) - 1u;
    uint32_t rel = collapse(st, raw);
    if (relevant) *relevant = rel;
    if (entry) *entry = classify(st, rel);
    return CP_OK;
}

int cp_lut_check_layout(uint64_t* n_mismatch) {
    if (!n_mismatch) return CP_ERR_ARG;
    *n_mismatch = check_mask3_layout();
    return CP_OK;
}

size_t cubical_persistence_workspace_size(int ndim, const int64_t* dims, int64_t max_survivors) {
    if ((ndim != 2 && ndim != 3) || !dims) return 0;
    int32_t nd = ndim;
    int64_t d3[3] = {ndim == 3 ? dims[0] : 1, dims[ndim - 2], dims[ndim - 1]};
    Plan P;
    if (make_plan(1, &nd, d3, nullptr, max_survivors, P) != CP_OK) return 0;
    return P.bytes;
}

int cubical_persistence_2d(const float* d_image, const int64_t dims[2], cp_pair* d_out_pairs, int64_t capacity,
                           int64_t* h_out_count, int64_t* d_out_count, void* d_workspace, size_t ws_bytes,
                           int64_t max_survivors, void* stream) {
    return single(2, d_image, dims, d_out_pairs, capacity, h_out_count, d_out_count, d_workspace, ws_bytes,
                  max_survivors, stream);
}

int cubical_persistence_3d(const float* d_image, const int64_t dims[3], cp_pair* d_out_pairs, int64_t capacity,
                           int64_t* h_out_count, int64_t* d_out_count, void* d_workspace, size_t ws_bytes,
                           int64_t max_survivors, void* stream) {
    return single(3, d_image, dims, d_out_pairs, capacity, h_out_count, d_out_count, d_workspace, ws_bytes,
                  max_survivors, stream);
}

size_t cubical_persistence_slabs_workspace_size(int ndim, const int64_t* dims, int n_slabs, int64_t max_survivors) {
    if ((ndim != 2 && ndim != 3) || !dims) return 0;
    int32_t nd = ndim;
    int64_t d3[3] = {ndim == 3 ? dims[0] : 1, dims[ndim - 2], dims[ndim - 1]};
    Plan P;
    if (make_plan(1, &nd, d3, nullptr, max_survivors, P) != CP_OK) return 0;
    if (plan_slabs(P, n_slabs) != CP_OK) return 0;
    return P.bytes;
}

int cubical_persistence_slabs(int ndim, const float* d_image, const int64_t* dims, int n_slabs, cp_pair* d_out_pairs,
                              int64_t capacity, int64_t* h_out_count, int64_t* d_out_count, void* d_workspace,
                              size_t ws_bytes, int64_t max_survivors, void* stream, cp_slab_stats* h_stats) {
    if ((ndim != 2 && ndim != 3) || !d_image || !dims) return CP_ERR_ARG;
    int32_t nd = ndim;
    int64_t d3[3] = {ndim == 3 ? dims[0] : 1, dims[ndim - 2], dims[ndim - 1]};
    Plan P;
    int rc = make_plan(1, &nd, d3, &d_image, max_survivors, P);
    if (rc != CP_OK) return rc;
    rc = plan_slabs(P, n_slabs);
    if (rc != CP_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = run(P, d_out_pairs, capacity, h_out_count, d_out_count, d_workspace, ws_bytes, s);
    if (!h_stats || rc == CP_ERR_ARG || rc == CP_ERR_CUDA) return rc;
    Counters h;
    SlabCtr hs;
    if (cudaMemcpyAsync(&h, at<Counters>(d_workspace, P.o_ctr), sizeof(Counters), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(&hs, at<SlabCtr>(d_workspace, P.o_sl_ctr), sizeof(SlabCtr), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CP_ERR_CUDA;
    std::memset(h_stats, 0, sizeof(*h_stats));
    h_stats->survivors[0] = h.n_s0;
    h_stats->survivors[1] = h.n_st;
    h_stats->rounds_merge[0] = h.rounds0;
    h_stats->rounds_merge[1] = h.roundst;
    for (int q = 0; q < 2; ++q) {
        h_stats->internal[q] = hs.n_in[q];
        h_stats->crossing[q] = hs.n_cross[q];
        h_stats->committed[q] = int64_t(hs.n_sent[q]) + hs.n_final[q];
        h_stats->final_pairs[q] = hs.n_final[q];
        h_stats->merged[q] = hs.n_merge[q];
        h_stats->rounds_slab[q] = hs.rounds_slab[q];
    }
    return rc != CP_OK ? rc : status_to_code(h.status);
}

size_t cubical_persistence_t_workspace_size(int ndim, const int64_t* dims, int64_t max_survivors) {
    if ((ndim != 2 && ndim != 3) || !dims) return 0;
    const int32_t nd = ndim;
    const int64_t d3[3] = {ndim == 3 ? dims[0] : 1, dims[ndim - 2], dims[ndim - 1]};
    return t_workspace(1, &nd, d3, max_survivors, nullptr);
}

size_t cubical_persistence_t_batched_workspace_size(int n_items, const int32_t* ndims, const int64_t* dims,
                                                    int64_t max_survivors) {
    return t_workspace(n_items, ndims, dims, max_survivors, nullptr);
}

int cubical_persistence_t_batched(int n_items, const float* const* h_images, const int32_t* ndims,
                                  const int64_t* dims, cp_pair* d_out_pairs, int64_t capacity, int64_t* h_out_count,
                                  int64_t* d_out_count, void* d_workspace, size_t ws_bytes, int64_t max_survivors,
                                  void* stream) {
    return t_run(n_items, h_images, ndims, dims, d_out_pairs, capacity, h_out_count, d_out_count, d_workspace,
                 ws_bytes, max_survivors, stream);
}

int cubical_persistence_t_2d(const float* d_image, const int64_t dims[2], cp_pair* d_out_pairs, int64_t capacity,
                             int64_t* h_out_count, int64_t* d_out_count, void* d_workspace, size_t ws_bytes,
                             int64_t max_survivors, void* stream) {
    return t_single(2, d_image, dims, d_out_pairs, capacity, h_out_count, d_out_count, d_workspace, ws_bytes,
                    max_survivors, stream);
}

int cubical_persistence_t_3d(const float* d_image, const int64_t dims[3], cp_pair* d_out_pairs, int64_t capacity,
                             int64_t* h_out_count, int64_t* d_out_count, void* d_workspace, size_t ws_bytes,
                             int64_t max_survivors, void* stream) {
    return t_single(3, d_image, dims, d_out_pairs, capacity, h_out_count, d_out_count, d_workspace, ws_bytes,
                    max_survivors, stream);
}

int cubical_persistence_debug_prune(int n_items, const float* const* h_images, const int32_t* ndims,
                                    const int64_t* dims, void* d_workspace, size_t ws_bytes, int64_t max_survivors,
                                    void* stream) {
    if (!h_images) return CP_ERR_ARG;
    Plan P;
    int rc = make_plan(n_items, ndims, dims, h_images, max_survivors, P);
    if (rc != CP_OK) return rc;
    return run(P, nullptr, 0, nullptr, nullptr, d_workspace, ws_bytes, static_cast<cudaStream_t>(stream), true);
}

int cubical_persistence_debug_layout(int n_items, const int32_t* ndims, const int64_t* dims, int64_t max_survivors,
                                     int64_t* h_offsets, int cap) {
    if (!h_offsets || cap < 12) return CP_ERR_ARG;
    Plan P;
    int rc = make_plan(n_items, ndims, dims, nullptr, max_survivors, P);
    if (rc != CP_OK) return rc;
    const int64_t v[13] = {int64_t(P.o_ctr), int64_t(P.o_uf0),  int64_t(P.o_uft),  int64_t(P.o_s0),
                           int64_t(P.o_st),  int64_t(P.o_age0), int64_t(P.o_aget), int64_t(P.ntot),
                           int64_t(P.ttot),  int64_t(P.cap_s),  int64_t(P.cap_r0), int64_t(P.cap_rt),
                           int64_t(P.o_ctr + offsetof(Counters, tma_tasks))};
    const int n = cap >= 13 ? 13 : 12;
    for (int i = 0; i < n; ++i) h_offsets[i] = v[i];
    return n;
}

size_t cubical_persistence_batched_workspace_size(int n_items, const int32_t* ndims, const int64_t* dims,
                                                  int64_t max_survivors) {
    Plan P;
    if (make_plan(n_items, ndims, dims, nullptr, max_survivors, P) != CP_OK) return 0;
    return P.bytes;
}

int cubical_persistence_batched(int n_items, const float* const* h_images, const int32_t* ndims, const int64_t* dims,
                                cp_pair* d_out_pairs, int64_t capacity, int64_t* h_out_count, int64_t* d_out_count,
                                void* d_workspace, size_t ws_bytes, int64_t max_survivors, void* stream) {
    if (!h_images) return CP_ERR_ARG;
    Plan P;
    int rc = make_plan(n_items, ndims, dims, h_images, max_survivors, P);
    if (rc != CP_OK) return rc;
    return run(P, d_out_pairs, capacity, h_out_count, d_out_count, d_workspace, ws_bytes,
               static_cast<cudaStream_t>(stream));
}

size_t cubical_persistence_full_batched_workspace_size(int n_items, const int32_t* ndims, const int64_t* dims,
                                                       int64_t max_survivors, int64_t pool_entries) {
    Plan P;
    if (make_plan(n_items, ndims, dims, nullptr, max_survivors, P, true, pool_entries) != CP_OK) return 0;
    return P.bytes;
}

int cubical_persistence_full_batched(int n_items, const float* const* h_images, const int32_t* ndims,
                                     const int64_t* dims, cp_pair* d_out_pairs, int64_t capacity,
                                     int64_t* h_out_count, int64_t* d_out_count, void* d_workspace, size_t ws_bytes,
                                     int64_t max_survivors, int64_t pool_entries, void* stream) {
    if (!h_images) return CP_ERR_ARG;
    Plan P;
    int rc = make_plan(n_items, ndims, dims, h_images, max_survivors, P, true, pool_entries);
    if (rc != CP_OK) return rc;
    return run(P, d_out_pairs, capacity, h_out_count, d_out_count, d_workspace, ws_bytes,
               static_cast<cudaStream_t>(stream));
}

size_t cubical_persistence_full_workspace_size(int ndim, const int64_t* dims, int64_t max_survivors,
                                               int64_t pool_entries) {
    if ((ndim != 2 && ndim != 3) || !dims) return 0;
    const int32_t nd = ndim;
    const int64_t d3[3] = {ndim == 3 ? dims[0] : 1, dims[ndim - 2], dims[ndim - 1]};
    return cubical_persistence_full_batched_workspace_size(1, &nd, d3, max_survivors, pool_entries);
}

int cubical_persistence_full_3d(const float* d_image, const int64_t dims[3], cp_pair* d_out_pairs, int64_t capacity,
                                int64_t* h_out_count, int64_t* d_out_count, void* d_workspace, size_t ws_bytes,
                                int64_t max_survivors, int64_t pool_entries, void* stream) {
    return single(3, d_image, dims, d_out_pairs, capacity, h_out_count, d_out_count, d_workspace, ws_bytes,
                  max_survivors, stream, true, pool_entries);
}

int cubical_persistence_full_info(const void* d_workspace, int n_items, const int32_t* ndims, const int64_t* dims,
                                  int64_t max_survivors, int64_t pool_entries, int64_t* h_info, int cap,
                                  void* stream) {
    if (!d_workspace || !h_info || cap < 4) return CP_ERR_ARG;
    Plan P;
    int rc = make_plan(n_items, ndims, dims, nullptr, max_survivors, P, true, pool_entries);
    if (rc != CP_OK) return rc;
    h_info[0] = h_info[1] = h_info[2] = 0;
    h_info[3] = int64_t(P.h1_pool);
    if (!P.h1) return CP_OK;
    H1Ctl c;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&c, static_cast<const char*>(d_workspace) + P.o_h1_ctl, sizeof(c), cudaMemcpyDeviceToHost,
                        s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CP_ERR_CUDA;
    h_info[0] = c.m;
    h_info[1] = c.rounds;
    h_info[2] = int64_t(c.grown);
    if (cap >= 10) {
        h_info[4] = c.neg_e;
        h_info[5] = c.pos_q;
        h_info[6] = c.pos_e;
        h_info[7] = int64_t(P.o_h1_neg);
        h_info[8] = int64_t(P.o_h1_pos);
        h_info[9] = c.nl;
    }
    if (cap >= 13) {
        h_info[10] = c.solo_round;
        h_info[11] = int64_t(c.t_grid_ns);
        h_info[12] = int64_t(c.t_solo_ns);
    }
    for (int k = 0; k < 16 && 13 + k < cap; ++k) h_info[13 + k] = c.nw_hist[k];
    for (int k = 0; k < 4 && 29 + k < cap; ++k) h_info[29 + k] = int64_t(c.t_phase_ns[k]);
    if (cap >= 36) {
        h_info[33] = int64_t(c.additions);
        h_info[34] = int64_t(c.merged);
        h_info[35] = c.solo_entries;
    }
    return CP_OK;
}

int cubical_persistence_stats(const void* d_workspace, cp_stats* h_stats, void* stream) {
    if (!d_workspace || !h_stats) return CP_ERR_ARG;
    Counters h;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&h, d_workspace, sizeof(Counters), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CP_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CP_ERR_CUDA;
    std::memset(h_stats, 0, sizeof(*h_stats));
    h_stats->h0_survivors = h.n_s0;
    h_stats->top_survivors = h.n_st;
    h_stats->h0_roots = h.n_r0;
    h_stats->top_roots = h.n_rt;
    h_stats->h0_rounds = h.rounds0;
    h_stats->top_rounds = h.roundst;
    h_stats->pairs = h.out_count;
    h_stats->status = h.status;
    h_stats->mst_rounds = h.mst_rounds;
    return status_to_code(h.status);
}

long long cp_launch_count(void) { return g_launches.load(); }

int cubical_persistence_debug_wait_timeout(void* d_workspace, size_t ws_bytes, int64_t limit_us, void* stream) {
    if (!d_workspace || ws_bytes < sizeof(Counters) + 256 || limit_us <= 0 || limit_us > 2000000) return CP_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Counters* ctr = static_cast<Counters*>(d_workspace);
    const uint32_t* flag = reinterpret_cast<const uint32_t*>(static_cast<char*>(d_workspace) + align_up(sizeof(Counters)));
    if (cudaMemsetAsync(d_workspace, 0, align_up(sizeof(Counters)) + 4, s) != cudaSuccess) return CP_ERR_CUDA;
    if (launch_wait_test(ctr, flag, uint64_t(limit_us) * 1000u, s) != cudaSuccess) return CP_ERR_CUDA;
    Counters h;
    if (cudaMemcpyAsync(&h, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CP_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CP_ERR_CUDA;
    return status_to_code(h.status);
}

int cp_set_tuning(int key, int value) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (key == CP_TUNE_H1_BUDGET_MS) {
        if (value < 0 || value > 3600000) return CP_ERR_ARG;
        set_h1_budget_ms(value);
        return CP_OK;
    }
    if (key == CP_TUNE_H1_SOLO) {
        if (value < 0 || value > 1024) return CP_ERR_ARG;
        set_h1_solo_cols(value);
        return CP_OK;
    }
    return set_tuning(key, value) == 0 ? CP_OK : CP_ERR_ARG;
}

int cp_get_tuning(int key) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (key == CP_TUNE_H1_BUDGET_MS) return get_h1_budget_ms();
    if (key == CP_TUNE_H1_SOLO) return get_h1_solo_cols();
    return get_tuning(key);
}

int cubical_persistence_uf_trace(const void* d_workspace, int dual, uint32_t* h_active, double* h_us, int cap,
                                 void* stream) {
    return cubical_persistence_uf_trace2(d_workspace, dual, h_active, h_us, nullptr, nullptr, cap, stream);
}

int cubical_persistence_uf_trace2(const void* d_workspace, int dual, uint32_t* h_active, double* h_us,
                                  double* h_us_phase_a, uint64_t* h_hops, int cap, void* stream) {
    if (!d_workspace || !h_active || !h_us || cap <= 0 || (dual != 0 && dual != 1)) return CP_ERR_ARG;
    Counters h;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&h, d_workspace, sizeof(Counters), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CP_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CP_ERR_CUDA;
    uint32_t rounds = dual ? h.roundst : h.rounds0;
    int n = int(std::min<uint32_t>(rounds + 1, uint32_t(kTraceRounds)));
    n = std::min(n, cap);
    for (int i = 0; i < n; ++i) {
        h_active[i] = h.trace_active[dual][i];
        h_us[i] = double(h.trace_t[dual][i] - h.trace_t[dual][0]) * 1e-3;
        if (h_us_phase_a)
            h_us_phase_a[i] = h.trace_ta[dual][i] ? double(h.trace_ta[dual][i] - h.trace_t[dual][0]) * 1e-3 : 0.0;
        if (h_hops) h_hops[i] = h.trace_hops[dual][i];
    }
    return n;
}

int cp_profile(int enable) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (enable && !g_ev_made) {
        for (int i = 0; i <= kStages; ++i)
            if (cudaEventCreate(&g_ev[i]) != cudaSuccess) return CP_ERR_CUDA;
        g_ev_made = true;
    }
    g_profile = enable != 0;
    return CP_OK;
}

int cp_stage_times(float* ms, int cap) {
    if (!ms || cap < kStages) return CP_ERR_ARG;
    if (!g_ev_made) return CP_ERR_ARG;
    if (cudaEventSynchronize(g_ev[kStages]) != cudaSuccess) return CP_ERR_CUDA;
    // event intervals of (prune, sort H0, union-find H0, sort dual, union-find dual, emit)
    static const int seq[kStages] = {0, 1, 2, 3, 4, 5};
    static const int joint[kStages] = {0, 1, 3, 2, 4, 5};  // events: sort H0 | sort dual | both | - | emit
    const int* order = g_ev_joint ? joint : seq;
    for (int i = 0; i < kStages; ++i)
        if (cudaEventElapsedTime(&ms[i], g_ev[order[i]], g_ev[order[i] + 1]) != cudaSuccess) return CP_ERR_CUDA;
    return kStages;
}

size_t cubical_persistence_loss_backward_workspace_size(int64_t n_pixels) {
    if (n_pixels <= 0) return 0;
    return align_up(sizeof(double) * size_t(n_pixels)) + align_up(sizeof(double) * size_t(loss_partials()));
}

int cubical_persistence_loss_backward(const cp_pair* d_pairs, int64_t n_pairs, const int64_t* d_n_pairs,
                                      float min_persistence, double* d_loss, const int64_t* d_item_offsets,
                                      float* d_grad_image, int64_t n_pixels, void* d_workspace, size_t ws_bytes,
                                      void* stream) {
    if (n_pairs < 0 || n_pixels <= 0 || !d_grad_image || !d_workspace || !d_loss) return CP_ERR_ARG;
    if (n_pairs > 0 && !d_pairs) return CP_ERR_ARG;
    if (ws_bytes < cubical_persistence_loss_backward_workspace_size(n_pixels)) return CP_ERR_ARG;
    double* acc = static_cast<double*>(d_workspace);
    double* parts = reinterpret_cast<double*>(static_cast<char*>(d_workspace) + align_up(sizeof(double) * size_t(n_pixels)));
    nvtxRangePushA("cp.loss_backward");
    cudaError_t e = launch_loss_backward(d_pairs, n_pairs, d_n_pairs, min_persistence, d_item_offsets, acc, parts,
                                         loss_partials(), d_loss, d_grad_image, n_pixels,
                                         static_cast<cudaStream_t>(stream));
    nvtxRangePop();
    return e == cudaSuccess ? CP_OK : CP_ERR_CUDA;
}

size_t cubical_persistence_backward_workspace_size(int64_t n_pixels) {
    if (n_pixels <= 0) return 0;
    return align_up(sizeof(double) * size_t(n_pixels));
}

int cubical_persistence_backward(const cp_pair* d_pairs, int64_t n_pairs, const float* d_grad_birth,
                                 const float* d_grad_death, const int64_t* d_item_offsets, float* d_grad_image,
                                 int64_t n_pixels, void* d_workspace, size_t ws_bytes, void* stream) {
    if (n_pairs < 0 || n_pixels <= 0 || !d_grad_image || !d_workspace) return CP_ERR_ARG;
    if (n_pairs > 0 && (!d_pairs || !d_grad_birth || !d_grad_death)) return CP_ERR_ARG;
    if (ws_bytes < cubical_persistence_backward_workspace_size(n_pixels)) return CP_ERR_ARG;
    nvtxRangePushA("cp.backward");
    cudaError_t e = launch_backward(d_pairs, n_pairs, d_grad_birth, d_grad_death, d_item_offsets,
                                    static_cast<double*>(d_workspace), d_grad_image, n_pixels,
                                    static_cast<cudaStream_t>(stream));
    nvtxRangePop();
    return e == cudaSuccess ? CP_OK : CP_ERR_CUDA;
}

}  // extern "C"
