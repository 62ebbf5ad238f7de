/*
 * Plain, slow, single-threaded CPU oracle for V-filtration cubical persistence
 * over F2 on 2D and 3D images: the H0 pairs and the top-dimension pairs
 * (H1 in 2D, H2 in 3D), and for volumes also the middle dimension (H1 in 3D).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this code.  The product path never
 * calls it and shares no code, header or table with it.
 *
 * What it computes is the persistence of the fully refined V-filtration,
 * written out from its definition with no pruning and no lookup table:
 *
 *   - V-filtration: a cell takes the largest value of its vertices
 *     (Sec. 2.2, the definition of f_V).
 *   - Fully refined order (Sec. 2.3): cells are compared through the vertex
 *     whose lower star holds them, then by the first-order tie-break, then by
 *     the second-order tie-break.  Readings used here (the paper leaves both
 *     tie-breaks unspecified):
 *       first order : equal pixel values are ordered by linear pixel index;
 *       second order: inside one lower star, lower dimension first, then
 *                     ascending index in the doubled grid.
 *     So the refined key of a cell s is R(s) = (f(m), m, dim s, idx s) with
 *     m the vertex of s that is largest under (f, linear index).
 *   - H0 (Sec. 4.1 step 3, Sec. 4.2 step 2): Kruskal over all edges in
 *     ascending R; a merging edge kills the younger of the two component
 *     roots (elder rule), the root of a component being its oldest vertex.
 *   - Top dimension (Sec. 3.1, Appendix A): union-find on the dual graph
 *     whose vertices are the top cells plus one extra vertex standing for
 *     the outside, and whose edges are the facets, processed in descending R.
 *     A facet with one cofacet joins it to the outside vertex.  The outside
 *     vertex is the oldest (first in the reversed order) and is never paired
 *     (Appendix A.4: the extra cofacet must never be paired).  A merging
 *     facet is paired with the younger of the two component representatives
 *     (Appendix A.4 pairing rule), the representative of a component being
 *     its top cell with the largest R.
 *   - H1 of a volume (oracle_persistence_full): the textbook column
 *     reduction over F2 (Sec. 2.1) of the boundary matrix of all squares
 *     (columns, ascending R) over all edges (rows, ascending R), nothing
 *     cleared or pruned.  A column that reduces to zero is a square that
 *     closes a 2-cycle (it is paired in H2); a nonzero reduced column pairs
 *     its lowest edge (the one with the largest R) with its square.
 *   - Pairs whose birth and death values are equal are omitted (Sec. 2.3,
 *     last paragraph).  One essential H0 class (global minimum, +inf) is
 *     reported.
 *
 * Cell indices are indices in the doubled grid: for an image of extents
 * (D, H, W) (D = 1 for 2D) the cell with doubled coordinates (Z, Y, X) has
 * index (Z*(2H-1) + Y)*(2W-1) + X and dimension = number of odd coordinates.
 *
 * Floating point: values are only compared and copied, never combined.
 * -0.0 is read as +0.0; NaN and +-inf are rejected.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    float birth, death;
    int64_t birth_cell, death_cell;
    int64_t birth_pixel, death_pixel;
    int32_t dim, pad;
} oracle_pair;

enum { ORACLE_OK = 0, ORACLE_EARG = -1, ORACLE_ENONFINITE = -2, ORACLE_ECAP = -3, ORACLE_ENOMEM = -4 };

typedef struct {
    const float *f;     /* canonicalised copy of the image (-0 -> +0) */
    int ndim;           /* 2 or 3 */
    int64_t D, H, W;    /* D = 1 for 2D */
    int64_t GD, GH, GW; /* doubled-grid extents */
} grid_t;

/* ---- vertex order K(v) = (f(v), v) (Sec. 2.3 first-order tie-break) ---- */
static int vertex_less(const grid_t *g, int64_t a, int64_t b) {
    float fa = g->f[a], fb = g->f[b];
    if (fa < fb) return 1;
    if (fa > fb) return 0;
    return a < b;
}

static void cell_coords(const grid_t *g, int64_t c, int64_t *Z, int64_t *Y, int64_t *X) {
    *X = c % g->GW;
    *Y = (c / g->GW) % g->GH;
    *Z = c / (g->GW * g->GH);
}

static int cell_dim(const grid_t *g, int64_t c) {
    int64_t Z, Y, X;
    cell_coords(g, c, &Z, &Y, &X);
    return (int)((Z & 1) + (Y & 1) + (X & 1));
}

/* m(s): the vertex of cell s that is largest in the vertex order (Sec. 2.2). */
static int64_t cell_max_vertex(const grid_t *g, int64_t c) {
    int64_t Z, Y, X;
    cell_coords(g, c, &Z, &Y, &X);
    int64_t best = -1;
    for (int dz = 0; dz <= (int)(Z & 1); ++dz)
        for (int dy = 0; dy <= (int)(Y & 1); ++dy)
            for (int dx = 0; dx <= (int)(X & 1); ++dx) {
                int64_t z = Z / 2 + dz, y = Y / 2 + dy, x = X / 2 + dx;
                int64_t v = (z * g->H + y) * g->W + x;
                if (best < 0 || vertex_less(g, best, v)) best = v;
            }
    return best;
}

/* Refined key R(s) = (f(m), m, dim, idx) as a struct compared field by field. */
typedef struct {
    float fm;
    int32_t dim;
    int64_t m;
    int64_t idx;
} rkey;

static rkey cell_key(const grid_t *g, int64_t c) {
    rkey k;
    k.m = cell_max_vertex(g, c);
    k.fm = g->f[k.m];
    k.dim = cell_dim(g, c);
    k.idx = c;
    return k;
}

static int rkey_cmp(const void *pa, const void *pb) {
    const rkey *a = (const rkey *)pa, *b = (const rkey *)pb;
    if (a->fm < b->fm) return -1;
    if (a->fm > b->fm) return 1;
    if (a->m != b->m) return a->m < b->m ? -1 : 1;
    if (a->dim != b->dim) return a->dim < b->dim ? -1 : 1;
    if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;
    return 0;
}

static int rkey_less(const rkey *a, const rkey *b) { return rkey_cmp(a, b) < 0; }

static int64_t vertex_cell_index(const grid_t *g, int64_t v) {
    int64_t x = v % g->W, y = (v / g->W) % g->H, z = v / (g->W * g->H);
    return ((2 * z) * g->GH + 2 * y) * g->GW + 2 * x;
}

/* ---- union-find with path compression; the caller decides link direction ---- */
static int64_t uf_find(int64_t *parent, int64_t x) {
    int64_t r = x;
    while (parent[r] != r) r = parent[r];
    while (parent[x] != r) {
        int64_t n = parent[x];
        parent[x] = r;
        x = n;
    }
    return r;
}

static int emit(oracle_pair *out, int64_t cap, int64_t *n, int keep_zero, float b, float d, int64_t bc,
                int64_t dc, int64_t bp, int64_t dp, int dim) {
    if (!keep_zero && b == d) return 0; /* zero persistence: omitted (Sec. 2.3) */
    if (*n < cap && out) {
        oracle_pair *p = &out[*n];
        p->birth = b;
        p->death = d;
        p->birth_cell = bc;
        p->death_cell = dc;
        p->birth_pixel = bp;
        p->death_pixel = dp;
        p->dim = dim;
        p->pad = 0;
    }
    ++*n;
    return 0;
}

/* H0: Kruskal over every edge in ascending R, elder rule. */
static int h0_pairs(const grid_t *g, oracle_pair *out, int64_t cap, int64_t *n, int keep_zero) {
    int64_t N = g->D * g->H * g->W;
    int64_t ncells = g->GD * g->GH * g->GW;
    int64_t nedges = 0;
    for (int64_t c = 0; c < ncells; ++c)
        if (cell_dim(g, c) == 1) ++nedges;
    rkey *edges = (rkey *)malloc(sizeof(rkey) * (size_t)(nedges ? nedges : 1));
    int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    if (!edges || !parent) {
        free(edges);
        free(parent);
        return ORACLE_ENOMEM;
    }
    int64_t k = 0;
    for (int64_t c = 0; c < ncells; ++c)
        if (cell_dim(g, c) == 1) edges[k++] = cell_key(g, c);
    qsort(edges, (size_t)nedges, sizeof(rkey), rkey_cmp);
    for (int64_t v = 0; v < N; ++v) parent[v] = v;
    for (int64_t i = 0; i < nedges; ++i) {
        int64_t Z, Y, X;
        cell_coords(g, edges[i].idx, &Z, &Y, &X);
        /* the two endpoints: round the one odd coordinate down and up */
        int64_t z0 = Z / 2, y0 = Y / 2, x0 = X / 2;
        int64_t z1 = z0 + (Z & 1), y1 = y0 + (Y & 1), x1 = x0 + (X & 1);
        int64_t a = (z0 * g->H + y0) * g->W + x0;
        int64_t b = (z1 * g->H + y1) * g->W + x1;
        int64_t ra = uf_find(parent, a), rb = uf_find(parent, b);
        if (ra == rb) continue; /* positive edge: creates a cycle */
        int64_t young = vertex_less(g, ra, rb) ? rb : ra;
        int64_t old = young == ra ? rb : ra;
        parent[young] = old;
        emit(out, cap, n, keep_zero, g->f[young], edges[i].fm, vertex_cell_index(g, young), edges[i].idx,
             young, edges[i].m, 0);
    }
    /* the one essential class: the global minimum never dies */
    int64_t gmin = 0;
    for (int64_t v = 1; v < N; ++v)
        if (vertex_less(g, v, gmin)) gmin = v;
    emit(out, cap, n, 1, g->f[gmin], INFINITY, vertex_cell_index(g, gmin), -1, gmin, -1, 0);
    free(edges);
    free(parent);
    return 0;
}

/* Dense id of a top cell (all coordinates odd on the image's axes). */
static int64_t top_id(const grid_t *g, int64_t Z, int64_t Y, int64_t X) {
    int64_t tz = g->ndim == 3 ? (Z - 1) / 2 : 0;
    int64_t ty = (Y - 1) / 2, tx = (X - 1) / 2;
    int64_t TH = g->H - 1, TW = g->W - 1;
    return (tz * TH + ty) * TW + tx;
}

/* Top dimension: union-find on the dual graph, facets in descending R. */
static int top_pairs(const grid_t *g, oracle_pair *out, int64_t cap, int64_t *n, int keep_zero) {
    int d = g->ndim;
    int64_t ncells = g->GD * g->GH * g->GW;
    int64_t T = (g->ndim == 3 ? g->D - 1 : 1) * (g->H - 1) * (g->W - 1);
    int64_t OUT = T;
    int64_t nfacets = 0;
    for (int64_t c = 0; c < ncells; ++c)
        if (cell_dim(g, c) == d - 1) ++nfacets;
    rkey *facets = (rkey *)malloc(sizeof(rkey) * (size_t)(nfacets ? nfacets : 1));
    int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * (size_t)(T + 1));
    rkey *rep = (rkey *)malloc(sizeof(rkey) * (size_t)(T + 1)); /* representative key per root */
    int64_t *tcell = (int64_t *)malloc(sizeof(int64_t) * (size_t)(T + 1));
    if (!facets || !parent || !rep || !tcell) {
        free(facets);
        free(parent);
        free(rep);
        free(tcell);
        return ORACLE_ENOMEM;
    }
    int64_t k = 0;
    for (int64_t c = 0; c < ncells; ++c) {
        int dim = cell_dim(g, c);
        if (dim == d - 1) facets[k++] = cell_key(g, c);
        if (dim == d) {
            int64_t Z, Y, X;
            cell_coords(g, c, &Z, &Y, &X);
            int64_t t = top_id(g, Z, Y, X);
            rep[t] = cell_key(g, c);
            tcell[t] = c;
        }
    }
    qsort(facets, (size_t)nfacets, sizeof(rkey), rkey_cmp);
    for (int64_t t = 0; t <= T; ++t) parent[t] = t;
    for (int64_t i = nfacets - 1; i >= 0; --i) { /* descending R: the reversed (cohomology) order */
        int64_t Z, Y, X;
        cell_coords(g, facets[i].idx, &Z, &Y, &X);
        /* the facet has exactly one even coordinate among the image's axes;
           its cofacets step that coordinate by -1 and +1 */
        int64_t co[2];
        int nco = 0;
        int64_t C[3] = {Z, Y, X}, G[3] = {g->GD, g->GH, g->GW};
        int first_axis = g->ndim == 3 ? 0 : 1;
        for (int ax = first_axis; ax < 3; ++ax) {
            if (C[ax] & 1) continue;
            for (int s = -1; s <= 1; s += 2) {
                int64_t q[3] = {C[0], C[1], C[2]};
                q[ax] += s;
                if (q[ax] < 0 || q[ax] >= G[ax]) {
                    co[nco++] = OUT;
                } else {
                    co[nco++] = top_id(g, q[0], q[1], q[2]);
                }
            }
        }
        int64_t ra = uf_find(parent, co[0]), rb = uf_find(parent, co[1]);
        if (ra == rb) continue; /* dual cycle: this facet is negative in homology */
        int64_t young, old;
        if (ra == OUT) {
            young = rb;
            old = ra;
        } else if (rb == OUT) {
            young = ra;
            old = rb;
        } else if (rkey_less(&rep[ra], &rep[rb])) {
            young = ra;
            old = rb;
        } else {
            young = rb;
            old = ra;
        }
        parent[young] = old; /* representative of the merged class stays `old` */
        emit(out, cap, n, keep_zero, facets[i].fm, rep[young].fm, facets[i].idx, tcell[young], facets[i].m,
             rep[young].m, d - 1);
    }
    free(facets);
    free(parent);
    free(rep);
    free(tcell);
    return 0;
}


/* ---- H1 of a volume: column reduction of the square-edge boundary matrix ---- */

/* Symmetric difference of two ascending arrays (F2 column addition). */
static int64_t *symdiff(const int64_t *a, int64_t na, const int64_t *b, int64_t nb, int64_t *nout) {
    int64_t *o = (int64_t *)malloc(sizeof(int64_t) * (size_t)(na + nb > 0 ? na + nb : 1));
    if (!o) return NULL;
    int64_t i = 0, j = 0, k = 0;
    while (i < na || j < nb) {
        if (j >= nb || (i < na && a[i] < b[j])) o[k++] = a[i++];
        else if (i >= na || b[j] < a[i]) o[k++] = b[j++];
        else { /* equal entries cancel */
            ++i;
            ++j;
        }
    }
    *nout = k;
    return o;
}

static int cmp_i64(const void *pa, const void *pb) {
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    return a < b ? -1 : (a > b ? 1 : 0);
}

static int h1_pairs(const grid_t *g, oracle_pair *out, int64_t cap, int64_t *n, int keep_zero) {
    int64_t ncells = g->GD * g->GH * g->GW;
    int64_t nedges = 0, nsq = 0;
    for (int64_t c = 0; c < ncells; ++c) {
        int d = cell_dim(g, c);
        if (d == 1) ++nedges;
        if (d == 2) ++nsq;
    }
    rkey *edges = (rkey *)malloc(sizeof(rkey) * (size_t)(nedges ? nedges : 1));
    rkey *sq = (rkey *)malloc(sizeof(rkey) * (size_t)(nsq ? nsq : 1));
    int64_t *erank = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncells); /* edge cell -> row (rank in R) */
    int64_t *owner = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nedges ? nedges : 1)); /* row -> column */
    int64_t **col = (int64_t **)calloc((size_t)(nsq ? nsq : 1), sizeof(int64_t *));
    int64_t *len = (int64_t *)calloc((size_t)(nsq ? nsq : 1), sizeof(int64_t));
    int rc = 0;
    if (!edges || !sq || !erank || !owner || !col || !len) {
        rc = ORACLE_ENOMEM;
        goto done;
    }
    int64_t ke = 0, ks = 0;
    for (int64_t c = 0; c < ncells; ++c) {
        int d = cell_dim(g, c);
        if (d == 1) edges[ke++] = cell_key(g, c);
        if (d == 2) sq[ks++] = cell_key(g, c);
    }
    qsort(edges, (size_t)nedges, sizeof(rkey), rkey_cmp);
    qsort(sq, (size_t)nsq, sizeof(rkey), rkey_cmp);
    for (int64_t i = 0; i < nedges; ++i) {
        erank[edges[i].idx] = i;
        owner[i] = -1;
    }
    for (int64_t j = 0; j < nsq; ++j) {
        /* the boundary of square j: step each of its two odd coordinates by -1 and +1 */
        int64_t Z, Y, X;
        cell_coords(g, sq[j].idx, &Z, &Y, &X);
        int64_t C[3] = {Z, Y, X};
        int64_t *c = (int64_t *)malloc(sizeof(int64_t) * 4);
        if (!c) {
            rc = ORACLE_ENOMEM;
            goto done;
        }
        int64_t nc = 0;
        for (int ax = 0; ax < 3; ++ax) {
            if (!(C[ax] & 1)) continue;
            for (int s = -1; s <= 1; s += 2) {
                int64_t q[3] = {C[0], C[1], C[2]};
                q[ax] += s;
                c[nc++] = erank[(q[0] * g->GH + q[1]) * g->GW + q[2]];
            }
        }
        qsort(c, (size_t)nc, sizeof(int64_t), cmp_i64);
        /* add earlier reduced columns while the lowest row has an owner */
        while (nc > 0 && owner[c[nc - 1]] >= 0) {
            int64_t k = owner[c[nc - 1]], nn = 0;
            int64_t *r = symdiff(c, nc, col[k], len[k], &nn);
            free(c);
            if (!r) {
                rc = ORACLE_ENOMEM;
                goto done;
            }
            c = r;
            nc = nn;
        }
        if (nc == 0) { /* closes a 2-cycle: paired in H2, not here */
            free(c);
            continue;
        }
        const rkey *e = &edges[c[nc - 1]];
        owner[c[nc - 1]] = j;
        col[j] = c;
        len[j] = nc;
        emit(out, cap, n, keep_zero, e->fm, sq[j].fm, e->idx, sq[j].idx, e->m, sq[j].m, 1);
    }
done:
    if (col)
        for (int64_t j = 0; j < nsq; ++j) free(col[j]);
    free(col);
    free(len);
    free(owner);
    free(erank);
    free(sq);
    free(edges);
    return rc;
}

static int pair_cmp(const void *pa, const void *pb) {
    const oracle_pair *a = (const oracle_pair *)pa, *b = (const oracle_pair *)pb;
    if (a->dim != b->dim) return a->dim < b->dim ? -1 : 1;
    if (a->birth_cell != b->birth_cell) return a->birth_cell < b->birth_cell ? -1 : 1;
    return 0;
}

/*
 * Persistence pairs of one image.
 *   img       : C-order float32 image, extents dims[0..ndim-1] ((H,W) or (D,H,W))
 *   keep_zero : 1 keeps zero-persistence pairs (for comparison with a full
 *               matrix reduction); 0 omits them as the method does.
 *   out, cap  : caller-owned output array; pairs are sorted by (dim, birth_cell).
 * Returns the number of pairs (which may exceed cap: then only cap were
 * written and the call should be repeated), or a negative error.
 */
static int64_t persistence_v(const float *img, int ndim, const int64_t *dims, int keep_zero, oracle_pair *out,
                             int64_t cap, int with_h1) {
    if (!img || !dims || (ndim != 2 && ndim != 3)) return ORACLE_EARG;
    grid_t g;
    g.ndim = ndim;
    g.D = ndim == 3 ? dims[0] : 1;
    g.H = dims[ndim - 2];
    g.W = dims[ndim - 1];
    if (g.H < 2 || g.W < 2 || (ndim == 3 && g.D < 2)) return ORACLE_EARG;
    g.GD = 2 * g.D - 1;
    g.GH = 2 * g.H - 1;
    g.GW = 2 * g.W - 1;
    int64_t N = g.D * g.H * g.W;
    float *f = (float *)malloc(sizeof(float) * (size_t)N);
    if (!f) return ORACLE_ENOMEM;
    for (int64_t i = 0; i < N; ++i) {
        float x = img[i];
        if (!isfinite(x)) {
            free(f);
            return ORACLE_ENONFINITE;
        }
        f[i] = x == 0.0f ? 0.0f : x; /* -0.0 reads as +0.0 */
    }
    g.f = f;
    int64_t n = 0;
    int rc = h0_pairs(&g, out, cap, &n, keep_zero);
    if (rc == 0 && with_h1 && ndim == 3) rc = h1_pairs(&g, out, cap, &n, keep_zero);
    if (rc == 0) rc = top_pairs(&g, out, cap, &n, keep_zero);
    free(f);
    if (rc) return rc;
    if (out && n <= cap) qsort(out, (size_t)n, sizeof(oracle_pair), pair_cmp);
    return n;
}

int64_t oracle_persistence(const float *img, int ndim, const int64_t *dims, int keep_zero, oracle_pair *out,
                           int64_t cap) {
    return persistence_v(img, ndim, dims, keep_zero, out, cap, 0);
}

/*
 * The whole diagram: as oracle_persistence, plus the H1 pairs of a volume
 * (dim 1, between the H0 and the H2 pairs in the output order).  For a 2D
 * image it equals oracle_persistence (H1 is the top dimension there).
 */
int64_t oracle_persistence_full(const float *img, int ndim, const int64_t *dims, int keep_zero, oracle_pair *out,
                                int64_t cap) {
    return persistence_v(img, ndim, dims, keep_zero, out, cap, 1);
}

/* Refined key of one cell, exposed so tests can check that R is a filtration order. */
int oracle_cell_key(const float *img, int ndim, const int64_t *dims, int64_t cell, float *fm, int64_t *m,
                    int32_t *dim) {
    grid_t g;
    g.ndim = ndim;
    g.D = ndim == 3 ? dims[0] : 1;
    g.H = dims[ndim - 2];
    g.W = dims[ndim - 1];
    g.GD = 2 * g.D - 1;
    g.GH = 2 * g.H - 1;
    g.GW = 2 * g.W - 1;
    g.f = img;
    if (cell < 0 || cell >= g.GD * g.GH * g.GW) return ORACLE_EARG;
    rkey k = cell_key(&g, cell);
    *fm = k.fm;
    *m = k.m;
    *dim = k.dim;
    return 0;
}

/* ==================================================================== T-filtration
 *
 * T-construction (Sec. 2.2): the pixel values sit on the top cells -- the
 * unit squares (2D) or cubes (3D) of the lattice [0,H]x[0,W] (x[0,D]) -- and
 * every lower-dimensional cell takes the smallest value among the top cells
 * that contain it (f_T).  The paper leaves the T-filtration to future work
 * (Sec. 6); the refined order used here is the reading that mirrors the V
 * one: a cell enters with the top cell of smallest (value, linear pixel
 * index) containing it, p(s); inside the set of cells entering with one top
 * cell, lower dimension first, then ascending doubled-grid index:
 *   R_T(s) = (f(p), p, dim s, idx s).
 * It is a filtration order: a face is contained in every top cell that holds
 * its coface, so its p is no later, and when equal its dimension is lower.
 * The doubled grid of the T-complex has extents 2n+1 along each image axis
 * (lattice points at even, pixels at odd coordinates); the cell with doubled
 * coordinates (Z, Y, X) has index (Z*(2H+1) + Y)*(2W+1) + X (Z = 0 in 2D).
 *   - H0: Kruskal over every edge in ascending R_T; a merging edge kills the
 *     younger root (larger R_T), a root being the oldest vertex of its class.
 *   - Top dimension: the dual union-find of Sec. 3.1 / Appendix A on this
 *     complex: top cells plus the outside vertex, facets in descending R_T,
 *     the younger representative (smaller R_T) paired with the facet.
 *   - Pairs with equal birth and death values are omitted; one essential H0
 *     class (the oldest vertex, +inf).
 * Pixels carried by the pairs are p(birth cell) and p(death cell).
 */
typedef struct {
    const float *f;
    int ndim;
    int64_t D, H, W;    /* pixel extents, D = 1 in 2D */
    int64_t GD, GH, GW; /* doubled extents: 2n+1 per image axis, GD = 1 in 2D */
} tgrid_t;

static void tcell_coords(const tgrid_t *g, int64_t c, int64_t *Z, int64_t *Y, int64_t *X) {
    *X = c % g->GW;
    *Y = (c / g->GW) % g->GH;
    *Z = c / (g->GW * g->GH);
}

static int tcell_dim(const tgrid_t *g, int64_t c) {
    int64_t Z, Y, X;
    tcell_coords(g, c, &Z, &Y, &X);
    return (int)((g->ndim == 3 ? (Z & 1) : 0) + (Y & 1) + (X & 1));
}

/* pixels along one axis that contain doubled coordinate C: one at an odd C,
   the (up to) two on either side at an even C */
static int axis_pixels(int64_t C, int64_t n, int64_t *k) {
    if (C & 1) {
        k[0] = (C - 1) / 2;
        return 1;
    }
    int m = 0;
    if (C / 2 - 1 >= 0) k[m++] = C / 2 - 1;
    if (C / 2 < n) k[m++] = C / 2;
    return m;
}

/* p(s): the top cell containing s that is smallest under (f, linear index). */
static int64_t tcell_min_pixel(const tgrid_t *g, int64_t c) {
    int64_t Z, Y, X, kz[2] = {0, 0}, ky[2], kx[2];
    tcell_coords(g, c, &Z, &Y, &X);
    int nz = g->ndim == 3 ? axis_pixels(Z, g->D, kz) : 1;
    int ny = axis_pixels(Y, g->H, ky), nx = axis_pixels(X, g->W, kx);
    int64_t best = -1;
    for (int a = 0; a < nz; ++a)
        for (int b = 0; b < ny; ++b)
            for (int e = 0; e < nx; ++e) {
                int64_t p = (kz[a] * g->H + ky[b]) * g->W + kx[e];
                if (best < 0 || g->f[p] < g->f[best] || (g->f[p] == g->f[best] && p < best)) best = p;
            }
    return best;
}

static rkey tcell_key(const tgrid_t *g, int64_t c) {
    rkey k;
    k.m = tcell_min_pixel(g, c);
    k.fm = g->f[k.m];
    k.dim = tcell_dim(g, c);
    k.idx = c;
    return k;
}

/* Dense id of a lattice point (all image-axis coordinates even). */
static int64_t tvertex_id(const tgrid_t *g, int64_t Z, int64_t Y, int64_t X) {
    return ((Z / 2) * (g->H + 1) + Y / 2) * (g->W + 1) + X / 2;
}

/* Dense id of a top cell (all image-axis coordinates odd). */
static int64_t tpixel_id(const tgrid_t *g, int64_t Z, int64_t Y, int64_t X) {
    int64_t z = g->ndim == 3 ? (Z - 1) / 2 : 0;
    return (z * g->H + (Y - 1) / 2) * g->W + (X - 1) / 2;
}

static int h0_pairs_t(const tgrid_t *g, oracle_pair *out, int64_t cap, int64_t *n, int keep_zero) {
    int64_t ncells = g->GD * g->GH * g->GW;
    int64_t NV = (g->ndim == 3 ? g->D + 1 : 1) * (g->H + 1) * (g->W + 1);
    int64_t nedges = 0;
    for (int64_t c = 0; c < ncells; ++c)
        if (tcell_dim(g, c) == 1) ++nedges;
    rkey *edges = (rkey *)malloc(sizeof(rkey) * (size_t)(nedges ? nedges : 1));
    rkey *vkey = (rkey *)malloc(sizeof(rkey) * (size_t)NV);
    int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * (size_t)NV);
    if (!edges || !vkey || !parent) {
        free(edges);
        free(vkey);
        free(parent);
        return ORACLE_ENOMEM;
    }
    int64_t k = 0;
    for (int64_t c = 0; c < ncells; ++c) {
        int dim = tcell_dim(g, c);
        if (dim == 1) edges[k++] = tcell_key(g, c);
        if (dim == 0) {
            int64_t Z, Y, X;
            tcell_coords(g, c, &Z, &Y, &X);
            vkey[tvertex_id(g, Z, Y, X)] = tcell_key(g, c);
        }
    }
    qsort(edges, (size_t)nedges, sizeof(rkey), rkey_cmp);
    for (int64_t v = 0; v < NV; ++v) parent[v] = v;
    for (int64_t i = 0; i < nedges; ++i) {
        int64_t Z, Y, X;
        tcell_coords(g, edges[i].idx, &Z, &Y, &X);
        /* the two endpoints: the one odd coordinate stepped down and up */
        int64_t a, b;
        if (X & 1) {
            a = tvertex_id(g, Z, Y, X - 1);
            b = tvertex_id(g, Z, Y, X + 1);
        } else if (Y & 1) {
            a = tvertex_id(g, Z, Y - 1, X);
            b = tvertex_id(g, Z, Y + 1, X);
        } else {
            a = tvertex_id(g, Z - 1, Y, X);
            b = tvertex_id(g, Z + 1, Y, X);
        }
        int64_t ra = uf_find(parent, a), rb = uf_find(parent, b);
        if (ra == rb) continue;
        int64_t young = rkey_less(&vkey[ra], &vkey[rb]) ? rb : ra;
        int64_t old = young == ra ? rb : ra;
        parent[young] = old;
        emit(out, cap, n, keep_zero, vkey[young].fm, edges[i].fm, vkey[young].idx, edges[i].idx, vkey[young].m,
             edges[i].m, 0);
    }
    int64_t oldest = 0;
    for (int64_t v = 1; v < NV; ++v)
        if (rkey_less(&vkey[v], &vkey[oldest])) oldest = v;
    emit(out, cap, n, 1, vkey[oldest].fm, INFINITY, vkey[oldest].idx, -1, vkey[oldest].m, -1, 0);
    free(edges);
    free(vkey);
    free(parent);
    return 0;
}

static int top_pairs_t(const tgrid_t *g, oracle_pair *out, int64_t cap, int64_t *n, int keep_zero) {
    int d = g->ndim;
    int64_t ncells = g->GD * g->GH * g->GW;
    int64_t T = g->D * g->H * g->W;
    int64_t OUT = T;
    int64_t nfacets = 0;
    for (int64_t c = 0; c < ncells; ++c)
        if (tcell_dim(g, c) == d - 1) ++nfacets;
    rkey *facets = (rkey *)malloc(sizeof(rkey) * (size_t)(nfacets ? nfacets : 1));
    int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * (size_t)(T + 1));
    rkey *rep = (rkey *)malloc(sizeof(rkey) * (size_t)(T + 1));
    int64_t *tcell = (int64_t *)malloc(sizeof(int64_t) * (size_t)(T + 1));
    if (!facets || !parent || !rep || !tcell) {
        free(facets);
        free(parent);
        free(rep);
        free(tcell);
        return ORACLE_ENOMEM;
    }
    int64_t k = 0;
    for (int64_t c = 0; c < ncells; ++c) {
        int dim = tcell_dim(g, c);
        if (dim == d - 1) facets[k++] = tcell_key(g, c);
        if (dim == d) {
            int64_t Z, Y, X;
            tcell_coords(g, c, &Z, &Y, &X);
            int64_t t = tpixel_id(g, Z, Y, X);
            rep[t] = tcell_key(g, c);
            tcell[t] = c;
        }
    }
    qsort(facets, (size_t)nfacets, sizeof(rkey), rkey_cmp);
    for (int64_t t = 0; t <= T; ++t) parent[t] = t;
    for (int64_t i = nfacets - 1; i >= 0; --i) {
        int64_t Z, Y, X;
        tcell_coords(g, facets[i].idx, &Z, &Y, &X);
        int64_t C[3] = {Z, Y, X}, G[3] = {g->GD, g->GH, g->GW};
        int64_t co[2];
        int nco = 0;
        for (int ax = 3 - d; ax < 3; ++ax) {
            if (C[ax] & 1) continue;
            for (int s = -1; s <= 1; s += 2) {
                int64_t q[3] = {C[0], C[1], C[2]};
                q[ax] += s;
                co[nco++] = (q[ax] < 0 || q[ax] >= G[ax]) ? OUT : tpixel_id(g, q[0], q[1], q[2]);
            }
        }
        int64_t ra = uf_find(parent, co[0]), rb = uf_find(parent, co[1]);
        if (ra == rb) continue;
        int64_t young, old;
        if (ra == OUT) {
            young = rb;
            old = ra;
        } else if (rb == OUT) {
            young = ra;
            old = rb;
        } else if (rkey_less(&rep[ra], &rep[rb])) {
            young = ra;
            old = rb;
        } else {
            young = rb;
            old = ra;
        }
        parent[young] = old;
        emit(out, cap, n, keep_zero, facets[i].fm, rep[young].fm, facets[i].idx, tcell[young], facets[i].m,
             rep[young].m, d - 1);
    }
    free(facets);
    free(parent);
    free(rep);
    free(tcell);
    return 0;
}

/*
 * Persistence pairs of one image under the T-filtration.  Same arguments,
 * output and errors as oracle_persistence; every extent may be 1 here (a
 * single top cell is a complex), cells are indices in the T doubled grid.
 */
int64_t oracle_persistence_t(const float *img, int ndim, const int64_t *dims, int keep_zero, oracle_pair *out,
                             int64_t cap) {
    if (!img || !dims || (ndim != 2 && ndim != 3)) return ORACLE_EARG;
    tgrid_t g;
    g.ndim = ndim;
    g.D = ndim == 3 ? dims[0] : 1;
    g.H = dims[ndim - 2];
    g.W = dims[ndim - 1];
    if (g.H < 1 || g.W < 1 || g.D < 1) return ORACLE_EARG;
    g.GD = ndim == 3 ? 2 * g.D + 1 : 1;
    g.GH = 2 * g.H + 1;
    g.GW = 2 * g.W + 1;
    int64_t N = g.D * g.H * g.W;
    float *f = (float *)malloc(sizeof(float) * (size_t)N);
    if (!f) return ORACLE_ENOMEM;
    for (int64_t i = 0; i < N; ++i) {
        float x = img[i];
        if (!isfinite(x)) {
            free(f);
            return ORACLE_ENONFINITE;
        }
        f[i] = x == 0.0f ? 0.0f : x;
    }
    g.f = f;
    int64_t n = 0;
    int rc = h0_pairs_t(&g, out, cap, &n, keep_zero);
    if (rc == 0) rc = top_pairs_t(&g, out, cap, &n, keep_zero);
    free(f);
    if (rc) return rc;
    if (out && n <= cap) qsort(out, (size_t)n, sizeof(oracle_pair), pair_cmp);
    return n;
}
