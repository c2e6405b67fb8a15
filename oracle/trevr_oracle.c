/*
 * TREVR oracle: a plain, slow CPU restatement of the reverse ray tracer of
 * Grond, Woods, Wadsley & Couchman (2019), "TREVR: A general N log^2 N
 * radiative transfer algorithm" (arXiv:1902.08083).
 *
 * THIS IS TEST INFRASTRUCTURE. Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it. The product path (the CUDA
 * library) shares no code with it and never calls it.
 *
 * Precision. Every value (cell moments, segment lengths, optical depths,
 * fluxes) is computed in FP64. The discrete decisions of the method -- the
 * Morton quantisation of a position, the opening-angle test (Eq. openangle),
 * the refinement test (Eq. refcrit), "does the ray touch this cell" and the
 * coincident-source skip -- are taken in IEEE fp32 with the operation
 * sequences written out below, because those decisions turn floating point
 * into integers and both implementations must take them in the same
 * precision. They work in coordinates relative to the domain's lower corner
 * (u = x - lo, cell planes g*h, rounded once each in fp32), so that their
 * rounding depends on the size of the domain and not on its distance from the
 * origin. The FP64 values use the positions and planes as given (lo + g*h).
 * The FP64 relative margin of each decision is recorded so a reader can see
 * how close each call was.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (contraction must
 * stay off so every fp32 expression rounds after each operation).
 *
 * Pins (tests/test_oracle_*.py): brute-force direct sum at theta=0 without
 * absorption (Sec. 3.1.2: theta=0 is an O(N^2) ray trace); brute-force
 * cell-by-cell optical depth at tau_ref<=0 (Sec. 2.2.3, full refinement);
 * the uniform-medium closed form L exp(-alpha r)/(4 pi r^2) (Eqs. ient,
 * simpint); an opaque occluder casts a shadow; hand-worked alpha_min /
 * alpha_max and cell-density examples; tiling of space by the leaves.
 * Beyond the flux:
 *   - the adjoint: finite differences of a replayed frozen forward pass;
 *   - the moments: direct sums, the trace identity and a single-source
 *     direction;
 *   - background sources: the shell formula (Eq. cosmof), and moved sources
 *     that lie on the sphere;
 *   - early termination: a closed form, the interaction-list definition and
 *     the exp(-tau_stop) bound;
 *   - bands: one band, proportional bands, full refinement and a
 *     transparent band;
 *   - the sub-bucket trace: a tree-free line integral of the SPH field, the
 *     kernel column and an opaque sink.
 * The glass stand-in is checked against the cost and error ratios that the
 * paper prints (Sec. 3.1.2, 3.1.3).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GRID_BITS 21
#define GRID_MAX ((int32_t)1 << GRID_BITS) /* 2^21 cells per axis */
#define ROOT 0                            /* preorder numbering: root first */
#define MAXDEPTH 80

enum {
    ORC_OK = 0,
    ORC_ERR_INVALID_ARGUMENT = 1,
    ORC_ERR_OUT_OF_DOMAIN = 2,
    ORC_ERR_NO_MEMORY = 6
};

/* ------------------------------------------------------------------------ */
/* Tree held by the oracle.  Node numbering is preorder (lower child first). */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n_gas, n_src, n_nodes, cap;
    int bucket;
    float lo32[3], side32, h32; /* domain as given (fp32) and cell size */
    double lo[3], side, h;      /* the same in FP64 */

    /* particles in Morton order */
    uint64_t *key;
    int64_t *perm;    /* perm[i] = caller index of the i-th sorted particle */
    int64_t *rank;    /* rank[caller index] = sorted position */
    int64_t *leaf_of; /* leaf node of the i-th sorted particle */
    float *px, *py, *pz, *alpha, *w;
    /* the same positions relative to the domain's lower corner, u = x - lo in fp32:
       the frame of every fp32 decision (the cell planes are g * h in it) */
    float *ux, *uy, *uz;

    /* nodes */
    int64_t *first, *count, *parent, *lower; /* lower child (upper = next subtree) */
    int64_t *upper;
    int32_t *split_bit, *depth; /* split_bit = -1 for a leaf */
    int32_t (*glo)[3], (*ghi)[3];
    double *W, *abar, (*amin_d)[3], (*amax_d)[3], *amin, *amax;
    double *L, (*cen)[3], *lrad;
    float *abar32, *dalpha32, *L32, (*cen32)[3], *l2_32;
    float (*blo32)[3], (*bhi32)[3];
    int64_t *src_first, *src_count; /* contiguous range in the sorted sources */

    /* sources, sorted by (first particle of their leaf, caller index) */
    int64_t *src_order, *src_leaf;
    float *sx, *sy, *sz, *slum;
    float *usx, *usy, *usz; /* source positions relative to lo (fp32), as ux */

    /* several bands (orc_build_bands; nb = 0 otherwise): per cell and band the mean
       absorption and the luminosity, per sorted source and band the luminosity */
    int nb;
    double *babar, *bL;
    float *bslum;

    /* smoothing lengths (orc_set_smoothing; NULL otherwise): per sorted particle,
       and per leaf the spread max - min of its particles' alpha (fp32) */
    float *hsml, *dbk;
} orc_tree;

#define ORC_MAXB 8

/* ------------------------------------------------------------------------ */
/* Morton key: q_d = floor((x_d - lo_d) * (2^21/side)), clamped to 2^21-1,    */
/* computed in fp32 (one subtraction and one multiplication, each rounded).   */
/* Key bit 62 is x's top bit, then y, then z, down to bit 0 (z's bit 0).      */
/* The tree is the binary tree of Morton prefixes: bisecting the longest axis */
/* of a cube in x, y, z order (Sec. 2.3) is the Morton subdivision.           */
/* ------------------------------------------------------------------------ */
static int in_domain32(float x, float lo, float hi) { return x >= lo && x < hi; }

static uint32_t quantize32(float x, float lo, float scale)
{
    float t = (x - lo) * scale;
    uint32_t q = (uint32_t)t; /* t >= 0 by the domain check */
    if (q > (uint32_t)(GRID_MAX - 1)) q = (uint32_t)(GRID_MAX - 1);
    return q;
}

static uint64_t interleave3(uint32_t qx, uint32_t qy, uint32_t qz)
{
    uint64_t k = 0;
    for (int b = GRID_BITS - 1; b >= 0; --b) {
        k = (k << 1) | ((qx >> b) & 1u);
        k = (k << 1) | ((qy >> b) & 1u);
        k = (k << 1) | ((qz >> b) & 1u);
    }
    return k;
}

static uint32_t coord_of_key(uint64_t key, int axis)
{
    uint32_t g = 0;
    for (int b = GRID_BITS - 1; b >= 0; --b) {
        int pos = 3 * b + (2 - axis);
        g = (g << 1) | (uint32_t)((key >> pos) & 1u);
    }
    return g;
}

static float domain_scale32(float side) { return 2097152.0f / side; }

int orc_morton_keys(const float *x, const float *y, const float *z, int64_t n,
                    const float lo[3], float side, uint64_t *keys)
{
    const float scale = domain_scale32(side);
    float hi[3];
    for (int d = 0; d < 3; ++d) hi[d] = lo[d] + side;
    int bad = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!in_domain32(x[i], lo[0], hi[0]) || !in_domain32(y[i], lo[1], hi[1]) ||
            !in_domain32(z[i], lo[2], hi[2])) {
            bad = 1;
            keys[i] = 0;
            continue;
        }
        keys[i] = interleave3(quantize32(x[i], lo[0], scale), quantize32(y[i], lo[1], scale),
                              quantize32(z[i], lo[2], scale));
    }
    return bad ? ORC_ERR_OUT_OF_DOMAIN : ORC_OK;
}

/* Stable sort of (key, index): ties keep the caller's order. */
typedef struct {
    uint64_t key;
    int64_t idx;
} kv_t;

static int kv_cmp(const void *a, const void *b)
{
    const kv_t *p = (const kv_t *)a, *q = (const kv_t *)b;
    if (p->key < q->key) return -1;
    if (p->key > q->key) return 1;
    return (p->idx > q->idx) - (p->idx < q->idx);
}

/* ------------------------------------------------------------------------ */
/* Top-down tree.  A node over the sorted range [i, j) is a leaf when it      */
/* holds at most N_B particles (the bucket, Sec. 2.2) or when all its keys    */
/* are equal.  Otherwise it splits at the highest key bit b in which key[i]   */
/* and key[j-1] differ: the lower child takes the particles whose bit b is 0. */
/* The cut is a plane on axis (62-b) mod 3 at the middle of the Morton cell   */
/* of the common prefix; the children are the parent box cut by that plane,  */
/* so the leaves fill space (Sec. 2.2.2, 2.3).                                */
/* ------------------------------------------------------------------------ */
static int64_t build_rec(orc_tree *T, int64_t i, int64_t j, const int32_t glo[3],
                         const int32_t ghi[3], int64_t parent, int32_t depth)
{
    int64_t id = T->n_nodes++;
    T->first[id] = i;
    T->count[id] = j - i;
    T->parent[id] = parent;
    T->depth[id] = depth;
    for (int d = 0; d < 3; ++d) {
        T->glo[id][d] = glo[d];
        T->ghi[id][d] = ghi[d];
    }
    T->lower[id] = -1;
    T->upper[id] = -1;
    T->split_bit[id] = -1;
    for (int64_t k = i; k < j; ++k) T->leaf_of[k] = id; /* overwritten by descendants */
    if (j - i <= T->bucket || T->key[i] == T->key[j - 1]) return id;

    uint64_t diff = T->key[i] ^ T->key[j - 1];
    int b = 63;
    while (!((diff >> b) & 1u)) --b;
    int64_t k = i;
    while (!((T->key[k] >> b) & 1u)) ++k; /* first particle of the upper side */
    int axis = (62 - b) % 3;
    int level = (62 - b) / 3;
    int shift = GRID_BITS - 1 - level;
    uint32_t g = coord_of_key(T->key[i], axis);
    int32_t plane = (int32_t)(((g >> shift) | 1u) << shift);
    T->split_bit[id] = b;

    int32_t lo1[3], hi1[3], lo2[3], hi2[3];
    for (int d = 0; d < 3; ++d) {
        lo1[d] = lo2[d] = glo[d];
        hi1[d] = hi2[d] = ghi[d];
    }
    hi1[axis] = plane;
    lo2[axis] = plane;
    T->lower[id] = build_rec(T, i, k, lo1, hi1, id, depth + 1);
    T->upper[id] = build_rec(T, k, j, lo2, hi2, id, depth + 1);
    return id;
}

static int split_axis_of(int32_t b) { return (62 - b) % 3; }

/* fp32 coordinate of grid plane g relative to the domain's lower corner: g*h,
   h = side * 2^-21. Every fp32 decision works in this frame (positions u = x - lo),
   so a plane's rounding depends on the domain's size only, not on its offset from
   the origin; far from the origin, lo + g*h in fp32 would merge distinct planes. */
static float rel32(float h, int32_t g) { return (float)g * h; }

/* ------------------------------------------------------------------------ */
/* Cell moments (Sec. 2.2.3, 2.3).                                           */
/* ------------------------------------------------------------------------ */
static void node_moments(orc_tree *T)
{
    const int64_t nn = T->n_nodes;
    /* absorption: volume-weighted mean of alpha = kappa*rho, weight w = m/rho */
    for (int64_t X = 0; X < nn; ++X) {
        double sw = 0.0, swa = 0.0;
        for (int64_t i = T->first[X]; i < T->first[X] + T->count[X]; ++i) {
            sw += (double)T->w[i];
            swa += (double)T->w[i] * (double)T->alpha[i];
        }
        T->W[X] = sw;
        T->abar[X] = swa / sw;
    }
    /* directional alpha_min/alpha_max, children before parents (reverse preorder) */
    for (int64_t X = nn - 1; X >= 0; --X) {
        if (T->split_bit[X] < 0) {
            for (int d = 0; d < 3; ++d) T->amin_d[X][d] = T->amax_d[X][d] = T->abar[X];
        } else {
            int64_t c1 = T->lower[X], c2 = T->upper[X];
            int a = split_axis_of(T->split_bit[X]);
            for (int d = 0; d < 3; ++d) {
                if (d == a) {
                    /* the ray crosses both children: optical depths add, then divide by width */
                    double w1 = (double)(T->ghi[c1][d] - T->glo[c1][d]);
                    double w2 = (double)(T->ghi[c2][d] - T->glo[c2][d]);
                    double Wd = (double)(T->ghi[X][d] - T->glo[X][d]);
                    T->amin_d[X][d] = (T->amin_d[c1][d] * w1 + T->amin_d[c2][d] * w2) / Wd;
                    T->amax_d[X][d] = (T->amax_d[c1][d] * w1 + T->amax_d[c2][d] * w2) / Wd;
                } else {
                    /* the ray crosses one child or the other */
                    T->amin_d[X][d] = fmin(T->amin_d[c1][d], T->amin_d[c2][d]);
                    T->amax_d[X][d] = fmax(T->amax_d[c1][d], T->amax_d[c2][d]);
                }
            }
        }
        T->amin[X] = fmin(fmin(T->amin_d[X][0], T->amin_d[X][1]), T->amin_d[X][2]);
        T->amax[X] = fmax(fmax(T->amax_d[X][0], T->amax_d[X][1]), T->amax_d[X][2]);
    }
    /* sources: total luminosity and centre of luminosity (Sec. 2.2.1) */
    for (int64_t X = 0; X < nn; ++X) {
        double sl = 0.0, sy[3] = {0.0, 0.0, 0.0}, su[3] = {0.0, 0.0, 0.0};
        for (int64_t s = T->src_first[X]; s < T->src_first[X] + T->src_count[X]; ++s) {
            double Lj = (double)T->slum[s];
            sl += Lj;
            sy[0] += Lj * (double)T->sx[s];
            sy[1] += Lj * (double)T->sy[s];
            sy[2] += Lj * (double)T->sz[s];
            su[0] += Lj * (double)T->usx[s];
            su[1] += Lj * (double)T->usy[s];
            su[2] += Lj * (double)T->usz[s];
        }
        T->L[X] = sl;
        for (int d = 0; d < 3; ++d) {
            T->cen[X][d] = sl > 0.0 ? sy[d] / sl : 0.0;
            /* the decisions' centre: from the sources' fp32 relative positions */
            T->cen32[X][d] = sl > 0.0 ? (float)(su[d] / sl) : 0.0f;
        }
    }
    /* fp32 copies used by the decisions, and l = furthest vertex from the centroid */
    for (int64_t X = 0; X < nn; ++X) {
        T->abar32[X] = (float)T->abar[X];
        T->dalpha32[X] = (float)(T->amax[X] - T->amin[X]);
        T->L32[X] = (float)T->L[X];
        for (int d = 0; d < 3; ++d) {
            T->blo32[X][d] = rel32(T->h32, T->glo[X][d]);
            T->bhi32[X][d] = rel32(T->h32, T->ghi[X][d]);
        }
        float l2 = 0.0f;
        double l2d = 0.0;
        for (int d = 0; d < 3; ++d) {
            float a = fmaxf(T->cen32[X][d] - T->blo32[X][d], T->bhi32[X][d] - T->cen32[X][d]);
            l2 = l2 + a * a;
            double lod = T->lo[d] + (double)T->glo[X][d] * T->h;
            double hid = T->lo[d] + (double)T->ghi[X][d] * T->h;
            double ad = fmax(T->cen[X][d] - lod, hid - T->cen[X][d]);
            l2d += ad * ad;
        }
        T->l2_32[X] = l2;
        T->lrad[X] = sqrt(l2d);
    }
}

/* Descend from the root to the leaf whose box holds grid point g. */
static int64_t leaf_of_point(const orc_tree *T, const uint32_t g[3])
{
    int64_t X = ROOT;
    while (T->split_bit[X] >= 0) {
        int a = split_axis_of(T->split_bit[X]);
        int64_t up = T->upper[X];
        X = ((int32_t)g[a] >= T->glo[up][a]) ? up : T->lower[X];
    }
    return X;
}

static int64_t lower_bound_i64(const int64_t *a, int64_t n, int64_t v)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t m = lo + (hi - lo) / 2;
        if (a[m] < v) lo = m + 1;
        else hi = m;
    }
    return lo;
}

void orc_tree_free(orc_tree *T);

#define ALLOC(ptr, n) \
    do { \
        (ptr) = calloc((size_t)((n) > 0 ? (n) : 1), sizeof(*(ptr))); \
        if (!(ptr)) goto nomem; \
    } while (0)

/*
 * Build the oracle's tree.  gas_x/y/z, alpha, weight (NULL = all 1) have
 * n_gas entries in the caller's order; src_* have n_src entries.
 */
int orc_build(const float *gas_x, const float *gas_y, const float *gas_z, const float *alpha,
              const float *weight, int64_t n_gas, const float *src_x, const float *src_y,
              const float *src_z, const float *src_lum, int64_t n_src, const float lo[3],
              float side, int bucket, orc_tree **out)
{
    *out = NULL;
    if (n_gas <= 0 || n_src < 0 || bucket < 1 || !(side > 0.0f) || !isfinite(side))
        return ORC_ERR_INVALID_ARGUMENT;
    for (int64_t i = 0; i < n_gas; ++i) {
        if (!isfinite(alpha[i]) || alpha[i] < 0.0f) return ORC_ERR_INVALID_ARGUMENT;
        if (weight && (!isfinite(weight[i]) || !(weight[i] > 0.0f))) return ORC_ERR_INVALID_ARGUMENT;
    }
    for (int64_t s = 0; s < n_src; ++s)
        if (!isfinite(src_lum[s]) || src_lum[s] < 0.0f) return ORC_ERR_INVALID_ARGUMENT;

    orc_tree *T = calloc(1, sizeof(orc_tree));
    if (!T) return ORC_ERR_NO_MEMORY;
    T->n_gas = n_gas;
    T->n_src = n_src;
    T->bucket = bucket;
    T->side32 = side;
    T->h32 = side * (1.0f / 2097152.0f);
    T->side = (double)side;
    T->h = (double)side / 2097152.0;
    for (int d = 0; d < 3; ++d) {
        T->lo32[d] = lo[d];
        T->lo[d] = (double)lo[d];
    }
    int64_t cap = 2 * n_gas;
    T->cap = cap;
    ALLOC(T->key, n_gas);
    ALLOC(T->perm, n_gas);
    ALLOC(T->rank, n_gas);
    ALLOC(T->leaf_of, n_gas);
    ALLOC(T->px, n_gas);
    ALLOC(T->py, n_gas);
    ALLOC(T->pz, n_gas);
    ALLOC(T->ux, n_gas);
    ALLOC(T->uy, n_gas);
    ALLOC(T->uz, n_gas);
    ALLOC(T->alpha, n_gas);
    ALLOC(T->w, n_gas);
    ALLOC(T->first, cap);
    ALLOC(T->count, cap);
    ALLOC(T->parent, cap);
    ALLOC(T->lower, cap);
    ALLOC(T->upper, cap);
    ALLOC(T->split_bit, cap);
    ALLOC(T->depth, cap);
    ALLOC(T->glo, cap);
    ALLOC(T->ghi, cap);
    ALLOC(T->W, cap);
    ALLOC(T->abar, cap);
    ALLOC(T->amin_d, cap);
    ALLOC(T->amax_d, cap);
    ALLOC(T->amin, cap);
    ALLOC(T->amax, cap);
    ALLOC(T->L, cap);
    ALLOC(T->cen, cap);
    ALLOC(T->lrad, cap);
    ALLOC(T->abar32, cap);
    ALLOC(T->dalpha32, cap);
    ALLOC(T->L32, cap);
    ALLOC(T->cen32, cap);
    ALLOC(T->l2_32, cap);
    ALLOC(T->blo32, cap);
    ALLOC(T->bhi32, cap);
    ALLOC(T->src_first, cap);
    ALLOC(T->src_count, cap);
    ALLOC(T->src_order, n_src);
    ALLOC(T->src_leaf, n_src);
    ALLOC(T->sx, n_src);
    ALLOC(T->sy, n_src);
    ALLOC(T->sz, n_src);
    ALLOC(T->usx, n_src);
    ALLOC(T->usy, n_src);
    ALLOC(T->usz, n_src);
    ALLOC(T->slum, n_src);

    {
        uint64_t *k0 = malloc((size_t)n_gas * sizeof(uint64_t));
        kv_t *kv = malloc((size_t)n_gas * sizeof(kv_t));
        if (!k0 || !kv) {
            free(k0);
            free(kv);
            goto nomem;
        }
        int rc = orc_morton_keys(gas_x, gas_y, gas_z, n_gas, lo, side, k0);
        if (rc != ORC_OK) {
            free(k0);
            free(kv);
            orc_tree_free(T);
            return rc;
        }
        for (int64_t i = 0; i < n_gas; ++i) {
            kv[i].key = k0[i];
            kv[i].idx = i;
        }
        qsort(kv, (size_t)n_gas, sizeof(kv_t), kv_cmp);
        for (int64_t i = 0; i < n_gas; ++i) {
            int64_t o = kv[i].idx;
            T->key[i] = kv[i].key;
            T->perm[i] = o;
            T->rank[o] = i;
            T->px[i] = gas_x[o];
            T->py[i] = gas_y[o];
            T->pz[i] = gas_z[o];
            T->ux[i] = gas_x[o] - T->lo32[0];
            T->uy[i] = gas_y[o] - T->lo32[1];
            T->uz[i] = gas_z[o] - T->lo32[2];
            T->alpha[i] = alpha[o];
            T->w[i] = weight ? weight[o] : 1.0f;
        }
        free(k0);
        free(kv);
    }

    {
        int32_t glo[3] = {0, 0, 0}, ghi[3] = {GRID_MAX, GRID_MAX, GRID_MAX};
        T->n_nodes = 0;
        build_rec(T, 0, n_gas, glo, ghi, -1, 0);
    }

    /* sources: quantise like particles, descend to their leaf, sort by
       (first particle of the leaf, caller index) */
    if (n_src > 0) {
        const float scale = domain_scale32(side);
        float hi[3];
        for (int d = 0; d < 3; ++d) hi[d] = lo[d] + side;
        kv_t *kv = malloc((size_t)n_src * sizeof(kv_t));
        int64_t *leaf0 = malloc((size_t)n_src * sizeof(int64_t));
        if (!kv || !leaf0) {
            free(kv);
            free(leaf0);
            goto nomem;
        }
        for (int64_t s = 0; s < n_src; ++s) {
            if (!in_domain32(src_x[s], lo[0], hi[0]) || !in_domain32(src_y[s], lo[1], hi[1]) ||
                !in_domain32(src_z[s], lo[2], hi[2])) {
                free(kv);
                free(leaf0);
                orc_tree_free(T);
                return ORC_ERR_OUT_OF_DOMAIN;
            }
            uint32_t g[3] = {quantize32(src_x[s], lo[0], scale), quantize32(src_y[s], lo[1], scale),
                             quantize32(src_z[s], lo[2], scale)};
            leaf0[s] = leaf_of_point(T, g);
            kv[s].key = (uint64_t)T->first[leaf0[s]];
            kv[s].idx = s;
        }
        qsort(kv, (size_t)n_src, sizeof(kv_t), kv_cmp);
        for (int64_t s = 0; s < n_src; ++s) {
            int64_t o = kv[s].idx;
            T->src_order[s] = o;
            T->src_leaf[s] = leaf0[o];
            T->sx[s] = src_x[o];
            T->sy[s] = src_y[o];
            T->sz[s] = src_z[o];
            T->usx[s] = src_x[o] - T->lo32[0];
            T->usy[s] = src_y[o] - T->lo32[1];
            T->usz[s] = src_z[o] - T->lo32[2];
            T->slum[s] = src_lum[o];
        }
        free(kv);
        free(leaf0);
    }
    {
        /* source range of each node: sources whose leaf starts inside the node's particle range */
        int64_t *lf = malloc((size_t)(n_src > 0 ? n_src : 1) * sizeof(int64_t));
        if (!lf) goto nomem;
        for (int64_t s = 0; s < n_src; ++s) lf[s] = T->first[T->src_leaf[s]];
        for (int64_t X = 0; X < T->n_nodes; ++X) {
            int64_t a = lower_bound_i64(lf, n_src, T->first[X]);
            int64_t b = lower_bound_i64(lf, n_src, T->first[X] + T->count[X]);
            T->src_first[X] = a;
            T->src_count[X] = b - a;
        }
        free(lf);
    }
    node_moments(T);
    *out = T;
    return ORC_OK;
nomem:
    orc_tree_free(T);
    return ORC_ERR_NO_MEMORY;
}

/*
 * Several bands (Sec. 4: many bands for a constant factor in cost). Band b has its
 * own absorption alpha_b (band-major, n_bands x n_gas) and its own source
 * luminosities L_b (n_bands x n_src). Reading: the walk and the rays are shared
 * by the bands. The tree, the centres of luminosity and the opening-angle test
 * use the summed luminosity L = sum_b L_b (FP64 in band order, rounded to fp32
 * per source). Each band keeps its own optical depth along the shared segments.
 * A cell is refined when any band asks for it: the refinement test uses
 * max_b (alpha_max,b - alpha_min,b). With one band this is the plain method.
 */
int orc_build_bands(const float *gas_x, const float *gas_y, const float *gas_z,
                    const float *alpha_bands, const float *weight, int64_t n_gas,
                    const float *src_x, const float *src_y, const float *src_z,
                    const float *lum_bands, int64_t n_src, int n_bands, const float lo[3],
                    float side, int bucket, orc_tree **out)
{
    *out = NULL;
    if (n_bands < 1 || n_bands > ORC_MAXB || n_gas <= 0 || n_src < 0)
        return ORC_ERR_INVALID_ARGUMENT;
    for (int64_t k = 0; k < (int64_t)n_bands * n_gas; ++k)
        if (!isfinite(alpha_bands[k]) || alpha_bands[k] < 0.0f) return ORC_ERR_INVALID_ARGUMENT;
    for (int64_t k = 0; k < (int64_t)n_bands * n_src; ++k)
        if (!isfinite(lum_bands[k]) || lum_bands[k] < 0.0f) return ORC_ERR_INVALID_ARGUMENT;
    float *lsum = malloc((size_t)(n_src > 0 ? n_src : 1) * sizeof(float));
    if (!lsum) return ORC_ERR_NO_MEMORY;
    for (int64_t j = 0; j < n_src; ++j) {
        double t = 0.0;
        for (int b = 0; b < n_bands; ++b) t += (double)lum_bands[(int64_t)b * n_src + j];
        lsum[j] = (float)t;
    }
    orc_tree *T = NULL;
    int rc = orc_build(gas_x, gas_y, gas_z, alpha_bands, weight, n_gas, src_x, src_y, src_z,
                       lsum, n_src, lo, side, bucket, &T);
    free(lsum);
    if (rc != ORC_OK) return rc;
    const int64_t nn = T->n_nodes, B = n_bands;
    double *dmax = calloc((size_t)nn, sizeof(double));
    T->nb = n_bands;
    T->babar = calloc((size_t)(nn * B), sizeof(double));
    T->bL = calloc((size_t)(nn * B), sizeof(double));
    T->bslum = calloc((size_t)(n_src > 0 ? n_src * B : 1), sizeof(float));
    if (!dmax || !T->babar || !T->bL || !T->bslum) {
        free(dmax);
        orc_tree_free(T);
        return ORC_ERR_NO_MEMORY;
    }
    for (int64_t s = 0; s < n_src; ++s)
        for (int64_t b = 0; b < B; ++b)
            T->bslum[s * B + b] = lum_bands[b * n_src + T->src_order[s]];
    for (int64_t b = 0; b < B; ++b) {
        /* this band's absorption: mean and directional spread of every cell */
        for (int64_t i = 0; i < n_gas; ++i) T->alpha[i] = alpha_bands[b * n_gas + T->perm[i]];
        node_moments(T);
        for (int64_t X = 0; X < nn; ++X) {
            T->babar[X * B + b] = T->abar[X];
            const double d = T->amax[X] - T->amin[X];
            if (b == 0 || d > dmax[X]) dmax[X] = d;
            double sl = 0.0;
            for (int64_t s = T->src_first[X]; s < T->src_first[X] + T->src_count[X]; ++s)
                sl += (double)T->bslum[s * B + b];
            T->bL[X * B + b] = sl;
        }
    }
    /* band 0 in the single-band fields; the refinement test takes the largest spread */
    for (int64_t i = 0; i < n_gas; ++i) T->alpha[i] = alpha_bands[T->perm[i]];
    node_moments(T);
    for (int64_t X = 0; X < nn; ++X) {
        T->amin[X] = 0.0;
        T->amax[X] = dmax[X];
        T->dalpha32[X] = (float)dmax[X];
    }
    free(dmax);
    *out = T;
    return ORC_OK;
}

void orc_tree_free(orc_tree *T)
{
    if (!T) return;
    void *ptrs[] = {T->key, T->perm, T->rank, T->leaf_of, T->px, T->py, T->pz, T->ux, T->uy,
                    T->uz, T->usx, T->usy, T->usz, T->alpha, T->w,
                    T->first, T->count, T->parent, T->lower, T->upper, T->split_bit, T->depth,
                    T->glo, T->ghi, T->W, T->abar, T->amin_d, T->amax_d, T->amin, T->amax, T->L,
                    T->cen, T->lrad, T->abar32, T->dalpha32, T->L32, T->cen32, T->l2_32, T->blo32,
                    T->bhi32, T->src_first, T->src_count, T->src_order, T->src_leaf, T->sx, T->sy,
                    T->sz, T->slum, T->babar, T->bL, T->bslum, T->hsml, T->dbk};
    for (size_t k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); ++k) free(ptrs[k]);
    free(T);
}

int64_t orc_n_nodes(const orc_tree *T) { return T->n_nodes; }

/* Copy the tree out (caller allocates n_nodes / n_gas / n_src sized arrays; any may be NULL). */
void orc_export_nodes(const orc_tree *T, int64_t *first, int64_t *count, int64_t *parent,
                      int64_t *lower, int64_t *upper, int32_t *split_bit, int32_t *depth,
                      int32_t *glo, int32_t *ghi, double *W, double *abar, double *amin,
                      double *amax, double *L, double *cen, double *lrad, int64_t *src_first,
                      int64_t *src_count)
{
    for (int64_t X = 0; X < T->n_nodes; ++X) {
        if (first) first[X] = T->first[X];
        if (count) count[X] = T->count[X];
        if (parent) parent[X] = T->parent[X];
        if (lower) lower[X] = T->lower[X];
        if (upper) upper[X] = T->upper[X];
        if (split_bit) split_bit[X] = T->split_bit[X];
        if (depth) depth[X] = T->depth[X];
        for (int d = 0; d < 3; ++d) {
            if (glo) glo[3 * X + d] = T->glo[X][d];
            if (ghi) ghi[3 * X + d] = T->ghi[X][d];
            if (cen) cen[3 * X + d] = T->cen[X][d];
        }
        if (W) W[X] = T->W[X];
        if (abar) abar[X] = T->abar[X];
        if (amin) amin[X] = T->amin[X];
        if (amax) amax[X] = T->amax[X];
        if (L) L[X] = T->L[X];
        if (lrad) lrad[X] = T->lrad[X];
        if (src_first) src_first[X] = T->src_first[X];
        if (src_count) src_count[X] = T->src_count[X];
    }
}

/* fp32 node values the decisions use. */
void orc_export_nodes32(const orc_tree *T, float *abar32, float *dalpha32, float *L32,
                        float *cen32, float *l2_32, float *blo32, float *bhi32)
{
    for (int64_t X = 0; X < T->n_nodes; ++X) {
        if (abar32) abar32[X] = T->abar32[X];
        if (dalpha32) dalpha32[X] = T->dalpha32[X];
        if (L32) L32[X] = T->L32[X];
        if (l2_32) l2_32[X] = T->l2_32[X];
        for (int d = 0; d < 3; ++d) {
            if (cen32) cen32[3 * X + d] = T->cen32[X][d];
            if (blo32) blo32[3 * X + d] = T->blo32[X][d];
            if (bhi32) bhi32[3 * X + d] = T->bhi32[X][d];
        }
    }
}

/* Directional alpha_min / alpha_max (x, y, z) of every node. */
void orc_export_directional(const orc_tree *T, double *amin_d, double *amax_d)
{
    for (int64_t X = 0; X < T->n_nodes; ++X)
        for (int d = 0; d < 3; ++d) {
            amin_d[3 * X + d] = T->amin_d[X][d];
            amax_d[3 * X + d] = T->amax_d[X][d];
        }
}

void orc_export_particles(const orc_tree *T, uint64_t *key, int64_t *perm, int64_t *leaf_of)
{
    for (int64_t i = 0; i < T->n_gas; ++i) {
        if (key) key[i] = T->key[i];
        if (perm) perm[i] = T->perm[i];
        if (leaf_of) leaf_of[i] = T->leaf_of[i];
    }
}

void orc_export_sources(const orc_tree *T, int64_t *src_order, int64_t *src_leaf)
{
    for (int64_t s = 0; s < T->n_src; ++s) {
        if (src_order) src_order[s] = T->src_order[s];
        if (src_leaf) src_leaf[s] = T->src_leaf[s];
    }
}

/* ------------------------------------------------------------------------ */
/* Reverse ray (Sec. 2.2.2-2.2.3).                                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    /* fp32 ray for the decisions */
    float p[3], d[3], inv[3], len;
    /* FP64 ray for the values */
    double P[3], D[3], LEN;
    /* the receiving particle (sorted index) and the sub-bucket switch */
    int64_t sink;
    int sub;
} ray_t;

typedef struct {
    double sum, comp; /* Neumaier summation */
} nsum_t;

static void nsum_add(nsum_t *s, double x)
{
    double t = s->sum + x;
    if (fabs(s->sum) >= fabs(x)) s->comp += (s->sum - t) + x;
    else s->comp += (x - t) + s->sum;
    s->sum = t;
}
static double nsum_get(const nsum_t *s) { return s->sum + s->comp; }

typedef struct {
    int64_t interactions, segments, visited, refinements, terminated, subbucket;
    double margin;
    /* optional record of the frozen decisions */
    int record;
} counters_t;

static void note_margin(counters_t *c, double m)
{
    if (m < c->margin) c->margin = m;
}

/* fp32 length of the ray inside the node box (slab method); 0 if it misses.
   Along an axis the ray does not move on (d_k = 0) the box is half-open,
   [lo, hi): a ray lying in a face between two cells belongs to the upper one
   only, so the cells still tile the ray exactly. */
static float clip32(const ray_t *R, const float blo[3], const float bhi[3])
{
    float t0 = 0.0f, t1 = 1.0f;
    for (int k = 0; k < 3; ++k) {
        if (R->d[k] != 0.0f) {
            float ta = (blo[k] - R->p[k]) * R->inv[k];
            float tb = (bhi[k] - R->p[k]) * R->inv[k];
            t0 = fmaxf(t0, fminf(ta, tb));
            t1 = fminf(t1, fmaxf(ta, tb));
        } else if (R->p[k] < blo[k] || R->p[k] >= bhi[k]) {
            return 0.0f;
        }
    }
    return t1 > t0 ? (t1 - t0) * R->len : 0.0f;
}

/* FP64 length of the ray inside the node box. */
static double clip64(const orc_tree *T, const ray_t *R, int64_t X)
{
    double t0 = 0.0, t1 = 1.0;
    for (int k = 0; k < 3; ++k) {
        double lo = T->lo[k] + (double)T->glo[X][k] * T->h;
        double hi = T->lo[k] + (double)T->ghi[X][k] * T->h;
        if (R->D[k] != 0.0) {
            double ta = (lo - R->P[k]) / R->D[k];
            double tb = (hi - R->P[k]) / R->D[k];
            t0 = fmax(t0, fmin(ta, tb));
            t1 = fmin(t1, fmax(ta, tb));
        } else if (R->P[k] < lo || R->P[k] >= hi) {
            return 0.0;
        }
    }
    return t1 > t0 ? (t1 - t0) * R->LEN : 0.0;
}

/* FP64 parameter range [t0, t1] of the ray inside the node box (as clip64). */
static void clip64_range(const orc_tree *T, const ray_t *R, int64_t X, double *t0o, double *t1o)
{
    double t0 = 0.0, t1 = 1.0;
    for (int k = 0; k < 3; ++k) {
        double lo = T->lo[k] + (double)T->glo[X][k] * T->h;
        double hi = T->lo[k] + (double)T->ghi[X][k] * T->h;
        if (R->D[k] != 0.0) {
            double ta = (lo - R->P[k]) / R->D[k];
            double tb = (hi - R->P[k]) / R->D[k];
            t0 = fmax(t0, fmin(ta, tb));
            t1 = fmin(t1, fmax(ta, tb));
        } else if (R->P[k] < lo || R->P[k] >= hi) {
            t1 = t0;
        }
    }
    *t0o = t0;
    *t1o = t1 > t0 ? t1 : t0;
}

/*
 * Sub-bucket particle trace (Sec. 2.2.3, 3.1.3). The absorption below the bucket
 * scale is the SPH field alpha(x) = sum_j alpha_j w_j W(|x - x_j|, h_j): alpha_j w_j
 * = kappa_j m_j is particle j's absorbing mass, and W is the cubic spline
 * W(r, h) = (1/(pi h^3)) (1 - 3/2 q^2 + 3/4 q^3) for q = r/h < 1,
 * (1/(pi h^3)) (2 - q)^3 / 4 for 1 <= q < 2, and 0 beyond. Along a ray at impact
 * parameter b from x_j, r = sqrt(b^2 + s^2). The integral over s uses closed-form
 * antiderivatives of r^n (the integral of r^n du from 0 to s):
 *   n = 0: s
 *   n = 1: (s r + b^2 ln((s + r)/b)) / 2
 *   n = 2: b^2 s + s^3 / 3
 *   n = 3: s r^3 / 4 + 3 b^2 s r / 8 + 3 b^4 ln((s + r)/b) / 8
 */
static double rpow_int(int n, double b, double s)
{
    const double r = sqrt(b * b + s * s);
    const double lg = b > 0.0 ? log((s + r) / b) : 0.0;
    switch (n) {
    case 0: return s;
    case 1: return 0.5 * (s * r + b * b * lg);
    case 2: return b * b * s + s * s * s / 3.0;
    default: return s * r * r * r / 4.0 + 3.0 * b * b * s * r / 8.0 + 3.0 * b * b * b * b * lg / 8.0;
    }
}

/* integral of W(sqrt(b^2 + u^2), h) du over [0, s], s >= 0 */
static double kernel_half_line(double b, double s, double h)
{
    const double u1 = b < h ? sqrt(h * h - b * b) : 0.0;         /* r = h */
    const double u2 = b < 2.0 * h ? sqrt(4.0 * h * h - b * b) : 0.0; /* r = 2h */
    const double a1 = fmin(s, u1), a2 = fmin(s, u2);
    double in = 0.0, out = 0.0;
    if (a1 > 0.0)
        in = rpow_int(0, b, a1) - 1.5 / (h * h) * rpow_int(2, b, a1) +
             0.75 / (h * h * h) * rpow_int(3, b, a1);
    if (a2 > a1)
        out = 2.0 * (rpow_int(0, b, a2) - rpow_int(0, b, a1)) -
              3.0 / h * (rpow_int(1, b, a2) - rpow_int(1, b, a1)) +
              1.5 / (h * h) * (rpow_int(2, b, a2) - rpow_int(2, b, a1)) -
              0.25 / (h * h * h) * (rpow_int(3, b, a2) - rpow_int(3, b, a1));
    return (in + out) / (M_PI * h * h * h);
}

/* integral of W along the line from s0 to s1 (s measured from the closest approach) */
static double kernel_line(double b, double s0, double s1, double h)
{
    const double g1 = s1 >= 0.0 ? kernel_half_line(b, s1, h) : -kernel_half_line(b, -s1, h);
    const double g0 = s0 >= 0.0 ? kernel_half_line(b, s0, h) : -kernel_half_line(b, -s0, h);
    return g1 - g0;
}

/* optical depth of the chord t in [t0, t1] of the ray through the SPH field, the
   receiving particle R->sink left out (it does not shadow itself) */
static double sph_chord(const orc_tree *T, const ray_t *R, double t0, double t1)
{
    if (!(t1 > t0)) return 0.0;
    const double D2 = R->D[0] * R->D[0] + R->D[1] * R->D[1] + R->D[2] * R->D[2];
    double lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
        const double e0 = R->P[k] + t0 * R->D[k], e1 = R->P[k] + t1 * R->D[k];
        lo[k] = fmin(e0, e1);
        hi[k] = fmax(e0, e1);
    }
    nsum_t tau = {0.0, 0.0};
    for (int64_t j = 0; j < T->n_gas; ++j) {
        if (j == R->sink) continue;
        const double a = (double)T->alpha[j] * (double)T->w[j];
        if (!(a > 0.0)) continue;
        const double H = (double)T->hsml[j];
        const double x[3] = {T->px[j], T->py[j], T->pz[j]};
        double g2 = 0.0; /* squared distance from x_j to the chord's bounding box */
        for (int k = 0; k < 3; ++k) {
            const double e = fmax(fmax(lo[k] - x[k], x[k] - hi[k]), 0.0);
            g2 += e * e;
        }
        if (g2 >= 4.0 * H * H) continue;
        double ud = 0.0;
        for (int k = 0; k < 3; ++k) ud += (x[k] - R->P[k]) * R->D[k];
        const double tc = ud / D2;
        double b2 = 0.0;
        for (int k = 0; k < 3; ++k) {
            const double e = x[k] - (R->P[k] + tc * R->D[k]);
            b2 += e * e;
        }
        if (b2 >= 4.0 * H * H) continue;
        const double L = sqrt(D2);
        nsum_add(&tau, a * kernel_line(sqrt(b2), (t0 - tc) * L, (t1 - tc) * L, H));
    }
    return nsum_get(&tau);
}

typedef struct {
    nsum_t tau;
    double len_sum; /* sum of the FP64 lengths of the used segments (tiling check) */
    int64_t nseg;
    nsum_t taub[ORC_MAXB]; /* optical depth of each band (trees with bands) */
} raysum_t;

/* Optical depth through node X: use its mean absorption unless the
   refinement criterion (Eq. refcrit, fp32) asks for its children. */
static void seg(const orc_tree *T, const ray_t *R, int64_t X, float tau_ref, counters_t *c,
                raysum_t *rs)
{
    float l32 = clip32(R, T->blo32[X], T->bhi32[X]);
    if (!(l32 > 0.0f)) return;
    if (R->sub && T->split_bit[X] < 0 && (tau_ref <= 0.0f || T->dbk[X] * l32 > tau_ref)) {
        /* a bucket that still asks for refinement: trace its particles */
        double t0, t1;
        clip64_range(T, R, X, &t0, &t1);
        nsum_add(&rs->tau, sph_chord(T, R, t0, t1));
        rs->len_sum += (t1 - t0) * R->LEN;
        rs->nseg++;
        c->segments++;
        c->subbucket++;
        return;
    }
    if (T->split_bit[X] >= 0) {
        int refine = (tau_ref <= 0.0f) || (T->dalpha32[X] * l32 > tau_ref);
        if (tau_ref > 0.0f) {
            double crit = (T->amax[X] - T->amin[X]) * clip64(T, R, X);
            note_margin(c, fabs(crit - (double)tau_ref) / (double)tau_ref);
        }
        if (refine) {
            c->refinements++;
            seg(T, R, T->lower[X], tau_ref, c, rs);
            seg(T, R, T->upper[X], tau_ref, c, rs);
            return;
        }
    }
    double l64 = clip64(T, R, X);
    nsum_add(&rs->tau, T->abar[X] * l64);
    for (int b = 0; b < T->nb; ++b) nsum_add(&rs->taub[b], T->babar[X * T->nb + b] * l64);
    rs->len_sum += l64;
    rs->nseg++;
    c->segments++;
}

static int64_t sibling_of(const orc_tree *T, int64_t U)
{
    int64_t P = T->parent[U];
    return T->lower[P] == U ? T->upper[P] : T->lower[P];
}

/*
 * Optical depth from the sink (in leaf S) to the point q (in node C).  The
 * segments are S, C, and the siblings of the nodes on the two paths up to
 * (not including) the children of their lowest common ancestor A: these
 * boxes tile box A, which holds the whole ray (Sec. 3.1.3: the walk goes up
 * from the sink's bucket and from the source cell).
 */
static void ray_tau(const orc_tree *T, const ray_t *R, int64_t S, int64_t C, float tau_ref,
                    counters_t *c, raysum_t *rs)
{
    seg(T, R, S, tau_ref, c, rs);
    if (S == C) return;
    seg(T, R, C, tau_ref, c, rs);
    int64_t u = S, v = C;
    while (T->depth[u] > T->depth[v]) {
        seg(T, R, sibling_of(T, u), tau_ref, c, rs);
        u = T->parent[u];
    }
    while (T->depth[v] > T->depth[u]) {
        seg(T, R, sibling_of(T, v), tau_ref, c, rs);
        v = T->parent[v];
    }
    while (T->parent[u] != T->parent[v]) {
        seg(T, R, sibling_of(T, u), tau_ref, c, rs);
        seg(T, R, sibling_of(T, v), tau_ref, c, rs);
        u = T->parent[u];
        v = T->parent[v];
    }
}

/*
 * Top-down ray walk (Sec. 3.1.3, last paragraph of "Refinement Criterion"; Sec. 4,
 * Discussion). The paper's own walk above goes up from the sink's bucket and from
 * the source cell, and so always splits the ray into the cells along both paths;
 * the paper notes that a walk going down the tree instead would rest more, or
 * solely, on the refinement criterion, and could scale better than N log^2 N in
 * optically thin media. Here the ray starts as one segment in A, the lowest common
 * ancestor of S and C (the smallest cell that holds the whole ray; every cell
 * above it holds the ray whole too), and seg() refines it by Eq. refcrit alone:
 * a cell whose (alpha_max - alpha_min) l exceeds tau_ref is replaced by its two
 * children, down to the buckets. tau_ref <= 0 refines to the buckets everywhere,
 * as the bottom-up walk does. S == C gives the single segment S, as there.
 */
static void ray_tau_topdown(const orc_tree *T, const ray_t *R, int64_t S, int64_t C, float tau_ref,
                            counters_t *c, raysum_t *rs)
{
    int64_t u = S, v = C;
    while (T->depth[u] > T->depth[v]) u = T->parent[u];
    while (T->depth[v] > T->depth[u]) v = T->parent[v];
    while (u != v) {
        u = T->parent[u];
        v = T->parent[v];
    }
    seg(T, R, u, tau_ref, c, rs);
}

typedef struct {
    int64_t node;  /* C */
    double q[3];   /* pseudo-source position */
    double L;      /* luminosity */
    double tau;    /* optical depth along the ray */
    double len_sum;
    double flux;   /* contribution */
    int64_t nseg;
    int64_t src;   /* sorted source index, or -1 for a merged node */
} inter_t;

typedef struct {
    inter_t *buf;
    int64_t n, cap;
} inter_log_t;

/* Moments of the intensity beyond Eq. simpint (Sec. 2.1): the flux vector
   sum f n (Eq. simpflux, n the unit vector from the source to the sink) and the
   second moment sum f n n^T (radiation pressure tensor; xx, yy, zz, xy, xz, yz). */
typedef struct {
    nsum_t v[9];
} moments_t;

/* Options of one walk beyond theta and tau_ref (all off when zero). */
typedef struct {
    float bg_radius;  /* > 0: background sources on this sphere (Sec. 2.2.4) */
    float tau_stop;   /* > 0: early ray termination (Sec. 4) */
    int sub_bucket;   /* particle trace below the buckets (Sec. 2.2.3, 3.1.3) */
    nsum_t *bandF;    /* per-band flux accumulators (trees with bands) */
    int topdown;      /* 1: the top-down ray walk (ray_tau_topdown), 0: bottom-up */
} walkopt_t;

static const walkopt_t NO_OPTS = {0.0f, 0.0f, 0, NULL, 0};

/* One pseudo-source (L at q, inside node C) seen from sorted particle i.
   tau_stop > 0: early ray termination (Sec. 4, proposed there). The optical depth
   sum of a ray is abandoned once it passes tau_stop, and the ray then adds nothing.
   Every term of the sum is non-negative, so a partial sum passes tau_stop exactly
   when the complete sum does: here the complete sum decides.
   bandF (trees with bands): each band's flux L_b exp(-tau_b) / (4 pi s^2) is added to
   bandF[b], L_b the band luminosity of the source (src >= 0) or of the merged cell C. */
static double contribute_m(const orc_tree *T, int64_t i, int64_t S, int64_t C, const float q32[3],
                           const double q64[3], double L, float tau_ref, float smin2,
                           counters_t *c, inter_log_t *log, int64_t src, moments_t *mom,
                           const walkopt_t *o)
{
    const float tau_stop = o->tau_stop;
    nsum_t *bandF = o->bandF;
    ray_t R;
    memset(&R, 0, sizeof(R));
    R.sink = i;
    R.sub = o->sub_bucket;
    R.p[0] = T->ux[i];
    R.p[1] = T->uy[i];
    R.p[2] = T->uz[i];
    R.P[0] = (double)T->px[i];
    R.P[1] = (double)T->py[i];
    R.P[2] = (double)T->pz[i];
    for (int k = 0; k < 3; ++k) {
        R.d[k] = q32[k] - R.p[k];
        R.inv[k] = R.d[k] != 0.0f ? 1.0f / R.d[k] : 0.0f;
        R.D[k] = q64[k] - R.P[k];
    }
    float s2 = R.d[0] * R.d[0] + R.d[1] * R.d[1] + R.d[2] * R.d[2];
    if (s2 < smin2) return 0.0; /* a source on top of the sink adds nothing */
    R.len = sqrtf(s2);
    double S2 = R.D[0] * R.D[0] + R.D[1] * R.D[1] + R.D[2] * R.D[2];
    R.LEN = sqrt(S2);
    raysum_t rs;
    memset(&rs, 0, sizeof(rs));
    if (o->topdown)
        ray_tau_topdown(T, &R, S, C, tau_ref, c, &rs);
    else
        ray_tau(T, &R, S, C, tau_ref, c, &rs);
    double tau = nsum_get(&rs.tau);
    const int cut = tau_stop > 0.0f && tau > (double)tau_stop;
    /* Eq. simpint: I = L exp(-tau) / (4 pi s^2) */
    double f = cut ? 0.0 : L * exp(-tau) / (4.0 * M_PI * S2);
    c->interactions++;
    c->terminated += cut;
    if (bandF) {
        for (int b = 0; b < T->nb; ++b) {
            const double Lb = src >= 0 ? (double)T->bslum[src * T->nb + b] : T->bL[C * T->nb + b];
            nsum_add(&bandF[b], Lb * exp(-nsum_get(&rs.taub[b])) / (4.0 * M_PI * S2));
        }
    }
    if (mom) {
        const double n[3] = {-R.D[0] / R.LEN, -R.D[1] / R.LEN, -R.D[2] / R.LEN};
        for (int k = 0; k < 3; ++k) nsum_add(&mom->v[k], f * n[k]);
        nsum_add(&mom->v[3], f * n[0] * n[0]);
        nsum_add(&mom->v[4], f * n[1] * n[1]);
        nsum_add(&mom->v[5], f * n[2] * n[2]);
        nsum_add(&mom->v[6], f * n[0] * n[1]);
        nsum_add(&mom->v[7], f * n[0] * n[2]);
        nsum_add(&mom->v[8], f * n[1] * n[2]);
    }
    if (log && log->n < log->cap) {
        inter_t *e = &log->buf[log->n];
        e->node = C;
        for (int k = 0; k < 3; ++k) e->q[k] = q64[k];
        e->L = L;
        e->tau = tau;
        e->len_sum = rs.len_sum;
        e->flux = f;
        e->nseg = rs.nseg;
        e->src = src;
    }
    if (log) log->n++;
    return f;
}

/*
 * Source walk for the sink at sorted position i (Sec. 2.2.1): a node whose
 * cell satisfies the opening-angle criterion theta > l/r (Eq. openangle)
 * acts as one source of luminosity L_X at its centre of luminosity;
 * otherwise it is opened; a leaf that is opened contributes its sources one
 * by one.  fp32 decision: l^2 < theta^2 r^2.
 */
static double sink_flux_m(const orc_tree *T, int64_t i, float theta, float tau_ref,
                          counters_t *c, inter_log_t *log, moments_t *mom, const walkopt_t *o);

static double sink_flux(const orc_tree *T, int64_t i, float theta, float tau_ref,
                        counters_t *c, inter_log_t *log)
{
    return sink_flux_m(T, i, theta, tau_ref, c, log, NULL, &NO_OPTS);
}

/* Leaf holding a point that may sit a rounding step outside the domain: its grid
   coordinates are clamped to the grid. */
static int64_t leaf_of_point_clamped(const orc_tree *T, const float q[3])
{
    const float scale = domain_scale32(T->side32);
    uint32_t g[3];
    for (int d = 0; d < 3; ++d) {
        float t = q[d] * scale; /* q relative to lo */
        if (!(t >= 0.0f)) t = 0.0f;
        uint32_t v = (uint32_t)t;
        g[d] = v > (uint32_t)(GRID_MAX - 1) ? (uint32_t)(GRID_MAX - 1) : v;
    }
    return leaf_of_point(T, g);
}

/*
 * Background sources (Sec. 2.2.4): all sources lie on a sphere of radius R
 * around the centre of the domain, and a merged cell's centre of luminosity,
 * which lies inside the sphere, is moved radially onto it before the ray is
 * traced; the ray then ends in the leaf that holds the moved point. fp32
 * position (it drives the decisions), relative to lo like every fp32 decision:
 * d = c - o; s = sqrt((dx^2 + dy^2) + dz^2); k = R / s; q = o + d * k, with the
 * centre o = side * 0.5. A centroid at the centre itself is not moved.
 */
static void bg_project(const orc_tree *T, const float c32[3], const double c64[3], float R,
                       float q32[3], double q64[3])
{
    float o[3], d[3];
    double O[3], D[3];
    for (int k = 0; k < 3; ++k) {
        o[k] = T->side32 * 0.5f; /* the centre, relative to lo */
        d[k] = c32[k] - o[k];
        O[k] = T->lo[k] + 0.5 * T->side;
        D[k] = c64[k] - O[k];
    }
    float s = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double S = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
    for (int k = 0; k < 3; ++k) {
        q32[k] = s > 0.0f ? o[k] + d[k] * (R / s) : c32[k];
        q64[k] = S > 0.0 ? O[k] + D[k] * ((double)R / S) : c64[k];
    }
}

static double sink_flux_m(const orc_tree *T, int64_t i, float theta, float tau_ref,
                          counters_t *c, inter_log_t *log, moments_t *mom, const walkopt_t *o)
{
    const float bg_radius = o->bg_radius;
    const float theta2 = theta * theta;
    const float smin = 1e-12f * T->side32;
    const float smin2 = smin * smin;
    const float p[3] = {T->ux[i], T->uy[i], T->uz[i]};
    const int64_t S = T->leaf_of[i];
    nsum_t F = {0.0, 0.0};
    int64_t stack[MAXDEPTH + 2];
    int sp = 0;
    stack[sp++] = ROOT;
    while (sp > 0) {
        int64_t X = stack[--sp];
        if (!(T->L[X] > 0.0)) continue;
        c->visited++;
        float r2 = 0.0f;
        double r2d = 0.0;
        for (int d = 0; d < 3; ++d) {
            float e = fmaxf(fmaxf(T->blo32[X][d] - p[d], p[d] - T->bhi32[X][d]), 0.0f);
            r2 = r2 + e * e;
            double lod = T->lo[d] + (double)T->glo[X][d] * T->h;
            double hid = T->lo[d] + (double)T->ghi[X][d] * T->h;
            double ed = fmax(fmax(lod - (double)p[d], (double)p[d] - hid), 0.0);
            r2d += ed * ed;
        }
        int accept = T->l2_32[X] < theta2 * r2;
        {
            double tr = (double)theta * sqrt(r2d), l = T->lrad[X];
            double den = fmax(tr, l);
            if (den > 0.0) note_margin(c, fabs(l - tr) / den);
        }
        if (accept && bg_radius > 0.0f) {
            float q32[3];
            double q64[3];
            bg_project(T, T->cen32[X], T->cen[X], bg_radius, q32, q64);
            const int64_t Cq = leaf_of_point_clamped(T, q32);
            nsum_add(&F, contribute_m(T, i, S, Cq, q32, q64, T->L[X], tau_ref, smin2, c, log, -1,
                                      mom, o));
        } else if (accept) {
            nsum_add(&F, contribute_m(T, i, S, X, T->cen32[X], T->cen[X], T->L[X], tau_ref, smin2,
                                      c, log, -1, mom, o));
        } else if (T->split_bit[X] < 0) {
            for (int64_t s = T->src_first[X]; s < T->src_first[X] + T->src_count[X]; ++s) {
                if (!(T->slum[s] > 0.0f)) continue;
                const float q32[3] = {T->usx[s], T->usy[s], T->usz[s]};
                const double q64[3] = {(double)T->sx[s], (double)T->sy[s], (double)T->sz[s]};
                nsum_add(&F, contribute_m(T, i, S, X, q32, q64, (double)T->slum[s], tau_ref, smin2,
                                          c, log, s, mom, o));
            }
        } else {
            stack[sp++] = T->upper[X];
            stack[sp++] = T->lower[X];
        }
    }
    return nsum_get(&F);
}

/*
 * Flux (Eq. simpint summed over pseudo-sources) for the sinks given by their
 * caller indices.  counters (nullable) gets 4 int64 per sink: interactions,
 * segments, visited source nodes, refinements.  margin (nullable) gets the
 * smallest FP64 relative margin of any decision taken for that sink.
 */
int orc_flux(const orc_tree *T, const int64_t *sinks, int64_t n_sink, float theta, float tau_ref,
             double *flux, int64_t *counters, double *margin, int nthreads)
{
    if (T->nb > 1) return ORC_ERR_INVALID_ARGUMENT; /* a tree with bands: orc_flux_bands */
    if (!(theta >= 0.0f) || !isfinite(theta) || isnan(tau_ref)) return ORC_ERR_INVALID_ARGUMENT;
    for (int64_t k = 0; k < n_sink; ++k)
        if (sinks[k] < 0 || sinks[k] >= T->n_gas) return ORC_ERR_INVALID_ARGUMENT;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t k = 0; k < n_sink; ++k) {
        counters_t c;
        memset(&c, 0, sizeof(c));
        c.margin = INFINITY;
        int64_t i = T->rank[sinks[k]];
        flux[k] = sink_flux(T, i, theta, tau_ref, &c, NULL);
        if (counters) {
            counters[4 * k + 0] = c.interactions;
            counters[4 * k + 1] = c.segments;
            counters[4 * k + 2] = c.visited;
            counters[4 * k + 3] = c.refinements;
        }
        if (margin) margin[k] = c.margin;
    }
    return ORC_OK;
}

/*
 * Flux and its first two direction moments at the sinks: flux[k] (Eq. simpint),
 * fvec[3k..3k+2] = sum f n (Eq. simpflux) and press[6k..6k+5] = sum f n n^T
 * (xx, yy, zz, xy, xz, yz), n the unit vector from the pseudo-source to the sink.
 */
int orc_flux_moments(const orc_tree *T, const int64_t *sinks, int64_t n_sink, float theta,
                     float tau_ref, double *flux, double *fvec, double *press, int nthreads)
{
    if (T->nb > 1) return ORC_ERR_INVALID_ARGUMENT; /* a tree with bands: orc_flux_bands */
    if (!(theta >= 0.0f) || !isfinite(theta) || isnan(tau_ref)) return ORC_ERR_INVALID_ARGUMENT;
    for (int64_t k = 0; k < n_sink; ++k)
        if (sinks[k] < 0 || sinks[k] >= T->n_gas) return ORC_ERR_INVALID_ARGUMENT;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t k = 0; k < n_sink; ++k) {
        counters_t c;
        memset(&c, 0, sizeof(c));
        c.margin = INFINITY;
        moments_t m;
        memset(&m, 0, sizeof(m));
        flux[k] = sink_flux_m(T, T->rank[sinks[k]], theta, tau_ref, &c, NULL, &m, &NO_OPTS);
        for (int q = 0; q < 3; ++q)
            if (fvec) fvec[3 * k + q] = nsum_get(&m.v[q]);
        for (int q = 0; q < 6; ++q)
            if (press) press[6 * k + q] = nsum_get(&m.v[3 + q]);
    }
    return ORC_OK;
}

/* Flux with every source treated as a background source on the sphere of radius
   bg_radius around the domain centre (merged centroids moved onto the sphere). */
int orc_flux_background(const orc_tree *T, const int64_t *sinks, int64_t n_sink, float theta,
                        float tau_ref, float bg_radius, double *flux, int64_t *counters,
                        int nthreads)
{
    if (T->nb > 1) return ORC_ERR_INVALID_ARGUMENT; /* a tree with bands: orc_flux_bands */
    if (!(theta >= 0.0f) || !isfinite(theta) || isnan(tau_ref) || !(bg_radius > 0.0f))
        return ORC_ERR_INVALID_ARGUMENT;
    for (int64_t k = 0; k < n_sink; ++k)
        if (sinks[k] < 0 || sinks[k] >= T->n_gas) return ORC_ERR_INVALID_ARGUMENT;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t k = 0; k < n_sink; ++k) {
        counters_t c;
        memset(&c, 0, sizeof(c));
        c.margin = INFINITY;
        const walkopt_t o = {bg_radius, 0.0f, 0, NULL};
        flux[k] = sink_flux_m(T, T->rank[sinks[k]], theta, tau_ref, &c, NULL, NULL, &o);
        if (counters) {
            counters[4 * k + 0] = c.interactions;
            counters[4 * k + 1] = c.segments;
            counters[4 * k + 2] = c.visited;
            counters[4 * k + 3] = c.refinements;
        }
    }
    return ORC_OK;
}

/* Flux with early ray termination at optical depth tau_stop > 0 (Sec. 4), and
   with background sources on the sphere of radius bg_radius when it is > 0.
   counters (nullable) gets 5 int64 per sink: interactions, segments, visited
   source nodes, refinements and terminated rays (segments and refinements
   count the complete rays). */
int orc_flux_terminated(const orc_tree *T, const int64_t *sinks, int64_t n_sink, float theta,
                        float tau_ref, float tau_stop, float bg_radius, double *flux,
                        int64_t *counters, int nthreads)
{
    if (T->nb > 1) return ORC_ERR_INVALID_ARGUMENT; /* a tree with bands: orc_flux_bands */
    if (!(theta >= 0.0f) || !isfinite(theta) || isnan(tau_ref) || !(tau_stop > 0.0f) ||
        !(bg_radius >= 0.0f))
        return ORC_ERR_INVALID_ARGUMENT;
    for (int64_t k = 0; k < n_sink; ++k)
        if (sinks[k] < 0 || sinks[k] >= T->n_gas) return ORC_ERR_INVALID_ARGUMENT;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t k = 0; k < n_sink; ++k) {
        counters_t c;
        memset(&c, 0, sizeof(c));
        c.margin = INFINITY;
        const walkopt_t o = {bg_radius, tau_stop, 0, NULL};
        flux[k] = sink_flux_m(T, T->rank[sinks[k]], theta, tau_ref, &c, NULL, NULL, &o);
        if (counters) {
            counters[5 * k + 0] = c.interactions;
            counters[5 * k + 1] = c.segments;
            counters[5 * k + 2] = c.visited;
            counters[5 * k + 3] = c.refinements;
            counters[5 * k + 4] = c.terminated;
        }
    }
    return ORC_OK;
}

/* Flux with the top-down ray walk (ray_tau_topdown). counters (nullable) gets 4
   int64 per sink as in orc_flux: interactions, segments, visited source nodes and
   refinements. */
int orc_flux_topdown(const orc_tree *T, const int64_t *sinks, int64_t n_sink, float theta,
                     float tau_ref, double *flux, int64_t *counters, int nthreads)
{
    if (T->nb > 1) return ORC_ERR_INVALID_ARGUMENT; /* a tree with bands: orc_flux_bands */
    if (!(theta >= 0.0f) || !isfinite(theta) || isnan(tau_ref)) return ORC_ERR_INVALID_ARGUMENT;
    for (int64_t k = 0; k < n_sink; ++k)
        if (sinks[k] < 0 || sinks[k] >= T->n_gas) return ORC_ERR_INVALID_ARGUMENT;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t k = 0; k < n_sink; ++k) {
        counters_t c;
        memset(&c, 0, sizeof(c));
        c.margin = INFINITY;
        const walkopt_t o = {0.0f, 0.0f, 0, NULL, 1};
        flux[k] = sink_flux_m(T, T->rank[sinks[k]], theta, tau_ref, &c, NULL, NULL, &o);
        if (counters) {
            counters[4 * k + 0] = c.interactions;
            counters[4 * k + 1] = c.segments;
            counters[4 * k + 2] = c.visited;
            counters[4 * k + 3] = c.refinements;
        }
    }
    return ORC_OK;
}

/* Flux of every band of a tree built by orc_build_bands: flux[b * n_sink + k].
   counters (nullable): 4 int64 per sink as in orc_flux. */
int orc_flux_bands(const orc_tree *T, const int64_t *sinks, int64_t n_sink, float theta,
                   float tau_ref, double *flux, int64_t *counters, int nthreads)
{
    if (T->nb < 1 || !(theta >= 0.0f) || !isfinite(theta) || isnan(tau_ref))
        return ORC_ERR_INVALID_ARGUMENT;
    for (int64_t k = 0; k < n_sink; ++k)
        if (sinks[k] < 0 || sinks[k] >= T->n_gas) return ORC_ERR_INVALID_ARGUMENT;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t k = 0; k < n_sink; ++k) {
        counters_t c;
        memset(&c, 0, sizeof(c));
        c.margin = INFINITY;
        nsum_t F[ORC_MAXB];
        memset(F, 0, sizeof(F));
        const walkopt_t o = {0.0f, 0.0f, 0, F};
        sink_flux_m(T, T->rank[sinks[k]], theta, tau_ref, &c, NULL, NULL, &o);
        for (int b = 0; b < T->nb; ++b) flux[(int64_t)b * n_sink + k] = nsum_get(&F[b]);
        if (counters) {
            counters[4 * k + 0] = c.interactions;
            counters[4 * k + 1] = c.segments;
            counters[4 * k + 2] = c.visited;
            counters[4 * k + 3] = c.refinements;
        }
    }
    return ORC_OK;
}

/* Smoothing lengths h (n_gas, caller order, > 0) for the sub-bucket trace; also
   the spread max - min of alpha over each bucket's particles, the sub-bucket
   refinement test's alpha_max - alpha_min (fp32). */
int orc_set_smoothing(orc_tree *T, const float *h)
{
    if (T->nb > 1) return ORC_ERR_INVALID_ARGUMENT;
    for (int64_t i = 0; i < T->n_gas; ++i)
        if (!(h[i] > 0.0f) || !isfinite(h[i])) return ORC_ERR_INVALID_ARGUMENT;
    if (!T->hsml) T->hsml = calloc((size_t)T->n_gas, sizeof(float));
    if (!T->dbk) T->dbk = calloc((size_t)T->n_nodes, sizeof(float));
    if (!T->hsml || !T->dbk) return ORC_ERR_NO_MEMORY;
    for (int64_t i = 0; i < T->n_gas; ++i) T->hsml[i] = h[T->perm[i]];
    for (int64_t X = 0; X < T->n_nodes; ++X) {
        T->dbk[X] = 0.0f;
        if (T->split_bit[X] >= 0) continue;
        float mn = INFINITY, mx = -INFINITY;
        for (int64_t i = T->first[X]; i < T->first[X] + T->count[X]; ++i) {
            mn = fminf(mn, T->alpha[i]);
            mx = fmaxf(mx, T->alpha[i]);
        }
        T->dbk[X] = mx - mn;
    }
    return ORC_OK;
}

/* Flux with the sub-bucket particle trace (needs orc_set_smoothing). counters
   (nullable): 5 int64 per sink, those of orc_flux and the sub-bucket segments. */
int orc_flux_sub(const orc_tree *T, const int64_t *sinks, int64_t n_sink, float theta,
                 float tau_ref, double *flux, int64_t *counters, int nthreads)
{
    if (T->nb > 1 || !T->hsml || !(theta >= 0.0f) || !isfinite(theta) || isnan(tau_ref))
        return ORC_ERR_INVALID_ARGUMENT;
    for (int64_t k = 0; k < n_sink; ++k)
        if (sinks[k] < 0 || sinks[k] >= T->n_gas) return ORC_ERR_INVALID_ARGUMENT;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int64_t k = 0; k < n_sink; ++k) {
        counters_t c;
        memset(&c, 0, sizeof(c));
        c.margin = INFINITY;
        const walkopt_t o = {0.0f, 0.0f, 1, NULL};
        flux[k] = sink_flux_m(T, T->rank[sinks[k]], theta, tau_ref, &c, NULL, NULL, &o);
        if (counters) {
            counters[5 * k + 0] = c.interactions;
            counters[5 * k + 1] = c.segments;
            counters[5 * k + 2] = c.visited;
            counters[5 * k + 3] = c.refinements;
            counters[5 * k + 4] = c.subbucket;
        }
    }
    return ORC_OK;
}

/* Interaction list of one sink (caller index): returns the number of
   interactions; fills at most cap entries. */
int64_t orc_sink_interactions(const orc_tree *T, int64_t sink, float theta, float tau_ref,
                              float bg_radius, int64_t cap, int64_t *node, double *q, double *L,
                              double *tau, double *len_sum, double *flux, int64_t *nseg,
                              int64_t *src)
{
    inter_log_t log;
    log.n = 0;
    log.cap = cap;
    log.buf = cap > 0 ? calloc((size_t)cap, sizeof(inter_t)) : NULL;
    if (cap > 0 && !log.buf) return -1;
    counters_t c;
    memset(&c, 0, sizeof(c));
    c.margin = INFINITY;
    const walkopt_t o = {bg_radius, 0.0f, 0, NULL};
    sink_flux_m(T, T->rank[sink], theta, tau_ref, &c, &log, NULL, &o);
    for (int64_t k = 0; k < log.n && k < cap; ++k) {
        const inter_t *e = &log.buf[k];
        if (node) node[k] = e->node;
        if (q)
            for (int d = 0; d < 3; ++d) q[3 * k + d] = e->q[d];
        if (L) L[k] = e->L;
        if (tau) tau[k] = e->tau;
        if (len_sum) len_sum[k] = e->len_sum;
        if (flux) flux[k] = e->flux;
        if (nseg) nseg[k] = e->nseg;
        if (src) src[k] = e->src;
    }
    free(log.buf);
    return log.n;
}

/* Optical depth of the ray from sorted particle (caller index) sink to the
   point q inside node C, with the segment set of the bottom-up walk (topdown = 0)
   or of the top-down walk (topdown = 1). */
double orc_ray_tau_walk(const orc_tree *T, int64_t sink, int64_t C, const float q[3],
                        float tau_ref, int topdown, double *len_sum, int64_t *nseg)
{
    int64_t i = T->rank[sink];
    ray_t R;
    memset(&R, 0, sizeof(R));
    R.p[0] = T->ux[i];
    R.p[1] = T->uy[i];
    R.p[2] = T->uz[i];
    R.P[0] = (double)T->px[i];
    R.P[1] = (double)T->py[i];
    R.P[2] = (double)T->pz[i];
    for (int k = 0; k < 3; ++k) {
        const float qu = q[k] - T->lo32[k]; /* q is given in world coordinates */
        R.d[k] = qu - R.p[k];
        R.inv[k] = R.d[k] != 0.0f ? 1.0f / R.d[k] : 0.0f;
        R.D[k] = (double)q[k] - R.P[k];
    }
    R.len = sqrtf(R.d[0] * R.d[0] + R.d[1] * R.d[1] + R.d[2] * R.d[2]);
    R.LEN = sqrt(R.D[0] * R.D[0] + R.D[1] * R.D[1] + R.D[2] * R.D[2]);
    counters_t c;
    memset(&c, 0, sizeof(c));
    c.margin = INFINITY;
    raysum_t rs;
    memset(&rs, 0, sizeof(rs));
    if (topdown)
        ray_tau_topdown(T, &R, T->leaf_of[i], C, tau_ref, &c, &rs);
    else
        ray_tau(T, &R, T->leaf_of[i], C, tau_ref, &c, &rs);
    if (len_sum) *len_sum = rs.len_sum;
    if (nseg) *nseg = rs.nseg;
    return nsum_get(&rs.tau);
}

double orc_ray_tau(const orc_tree *T, int64_t sink, int64_t C, const float q[3], float tau_ref,
                   double *len_sum, int64_t *nseg)
{
    return orc_ray_tau_walk(T, sink, C, q, tau_ref, 0, len_sum, nseg);
}

/* Leaf holding the grid point of (x,y,z) (same quantisation as the keys). */
int64_t orc_leaf_of_point(const orc_tree *T, float x, float y, float z)
{
    const float scale = domain_scale32(T->side32);
    uint32_t g[3] = {quantize32(x, T->lo32[0], scale), quantize32(y, T->lo32[1], scale),
                     quantize32(z, T->lo32[2], scale)};
    return leaf_of_point(T, g);
}

/* ======================================================================== */
/* Adjoint with frozen decisions (differentiation of Eq. simpint).          */
/*                                                                          */
/* For a loss with dLoss/dF_p = g_p, every interaction (p, C) contributes   */
/* f = L_C exp(-tau) / (4 pi s^2), s = |q - p|, tau = sum_X abar_X l_X(q).  */
/* The accept / refine / touch decisions are held fixed; the centre of      */
/* luminosity q = c_C = sum_j L_j y_j / L_C moves with the luminosities.    */
/*   df/dL_C = f / L_C ;  dc_C/dL_j = (y_j - c_C) / L_C   (j in C)          */
/*   grad_q f = f (-2 (q - p)/s^2 - sum_X abar_X grad_q l_X)                */
/*   df/dabar_X = -f l_X ;  dabar_X/dalpha_i = w_i / W_X    (i in X)        */
/* l_X = (t_exit - t_enter) |q - p|, with t of a slab plane b on axis k     */
/* equal to (b - p_k)/(q_k - p_k), so dt/dq_k = -t/(q_k - p_k); a t clamped */
/* to 0 or 1 (the ray starts or ends inside X) does not move.               */
/* ======================================================================== */

typedef struct {
    double *a;     /* per node: sum g f / L_C over merged interactions with C */
    double *b;     /* per node, 3: sum g grad_q f / L_C */
    double *e;     /* per sorted source: sum g f / L_j over single-source interactions */
    double *G;     /* per node: sum -g f l_X over segments using X */
} adj_acc_t;

/* FP64 length and its gradient w.r.t. the ray's end point q. */
static double clip64_grad(const orc_tree *T, const ray_t *R, int64_t X, double grad[3])
{
    double t0 = 0.0, t1 = 1.0;
    int k0 = -1, k1 = -1;
    for (int k = 0; k < 3; ++k) {
        double lo = T->lo[k] + (double)T->glo[X][k] * T->h;
        double hi = T->lo[k] + (double)T->ghi[X][k] * T->h;
        if (R->D[k] != 0.0) {
            double ta = (lo - R->P[k]) / R->D[k];
            double tb = (hi - R->P[k]) / R->D[k];
            double tn = fmin(ta, tb), tx = fmax(ta, tb);
            if (tn > t0) { t0 = tn; k0 = k; }
            if (tx < t1) { t1 = tx; k1 = k; }
        } else if (R->P[k] < lo || R->P[k] >= hi) {
            grad[0] = grad[1] = grad[2] = 0.0;
            return 0.0;
        }
    }
    if (!(t1 > t0)) {
        grad[0] = grad[1] = grad[2] = 0.0;
        return 0.0;
    }
    double dt[3] = {0.0, 0.0, 0.0};
    if (k1 >= 0) dt[k1] += -t1 / R->D[k1];
    if (k0 >= 0) dt[k0] -= -t0 / R->D[k0];
    for (int k = 0; k < 3; ++k) grad[k] = dt[k] * R->LEN + (t1 - t0) * R->D[k] / R->LEN;
    return (t1 - t0) * R->LEN;
}

typedef struct {
    int64_t *box;
    double *len;
    int64_t n, cap;
} seglist_t;

static void seglist_push(seglist_t *s, int64_t X, double l)
{
    if (s->n == s->cap) {
        int64_t nc = s->cap ? 2 * s->cap : 64;
        s->box = realloc(s->box, (size_t)nc * sizeof(int64_t));
        s->len = realloc(s->len, (size_t)nc * sizeof(double));
        s->cap = nc;
    }
    s->box[s->n] = X;
    s->len[s->n] = l;
    s->n++;
}

/* the unrefined segments of a ray, with the same decisions as seg() */
static void seg_list(const orc_tree *T, const ray_t *R, int64_t X, float tau_ref, seglist_t *out)
{
    float l32 = clip32(R, T->blo32[X], T->bhi32[X]);
    if (!(l32 > 0.0f)) return;
    if (T->split_bit[X] >= 0 && ((tau_ref <= 0.0f) || (T->dalpha32[X] * l32 > tau_ref))) {
        seg_list(T, R, T->lower[X], tau_ref, out);
        seg_list(T, R, T->upper[X], tau_ref, out);
        return;
    }
    seglist_push(out, X, 0.0);
}

static void ray_segments(const orc_tree *T, const ray_t *R, int64_t S, int64_t C, float tau_ref,
                         seglist_t *out)
{
    seg_list(T, R, S, tau_ref, out);
    if (S == C) return;
    seg_list(T, R, C, tau_ref, out);
    int64_t u = S, v = C;
    while (T->depth[u] > T->depth[v]) {
        seg_list(T, R, sibling_of(T, u), tau_ref, out);
        u = T->parent[u];
    }
    while (T->depth[v] > T->depth[u]) {
        seg_list(T, R, sibling_of(T, v), tau_ref, out);
        v = T->parent[v];
    }
    while (T->parent[u] != T->parent[v]) {
        seg_list(T, R, sibling_of(T, u), tau_ref, out);
        seg_list(T, R, sibling_of(T, v), tau_ref, out);
        u = T->parent[u];
        v = T->parent[v];
    }
}

static void make_ray(const orc_tree *T, int64_t i, const float q32[3], const double q64[3], ray_t *R)
{
    memset(R, 0, sizeof(*R));
    R->sink = i;
    R->p[0] = T->ux[i];
    R->p[1] = T->uy[i];
    R->p[2] = T->uz[i];
    R->P[0] = (double)T->px[i];
    R->P[1] = (double)T->py[i];
    R->P[2] = (double)T->pz[i];
    for (int k = 0; k < 3; ++k) {
        R->d[k] = q32[k] - R->p[k];
        R->inv[k] = R->d[k] != 0.0f ? 1.0f / R->d[k] : 0.0f;
        R->D[k] = q64[k] - R->P[k];
    }
    R->len = sqrtf(R->d[0] * R->d[0] + R->d[1] * R->d[1] + R->d[2] * R->d[2]);
    R->LEN = sqrt(R->D[0] * R->D[0] + R->D[1] * R->D[1] + R->D[2] * R->D[2]);
}

#define ATOMIC_ADD(ptr, v) \
    do { \
        double _v = (v); \
        _Pragma("omp atomic") *(ptr) += _v; \
    } while (0)

/* one interaction of the adjoint: accumulate into acc */
static void adj_interaction(const orc_tree *T, int64_t i, int64_t S, int64_t C, const float q32[3],
                            const double q64[3], double L, float tau_ref, float smin2, double g,
                            int64_t src, adj_acc_t *acc)
{
    ray_t R;
    make_ray(T, i, q32, q64, &R);
    float s2 = R.d[0] * R.d[0] + R.d[1] * R.d[1] + R.d[2] * R.d[2];
    if (s2 < smin2) return;
    seglist_t sl = {NULL, NULL, 0, 0};
    ray_segments(T, &R, S, C, tau_ref, &sl);
    nsum_t tau = {0.0, 0.0};
    double gtau[3] = {0.0, 0.0, 0.0};
    for (int64_t k = 0; k < sl.n; ++k) {
        double gl[3];
        double l = clip64_grad(T, &R, sl.box[k], gl);
        sl.len[k] = l;
        nsum_add(&tau, T->abar[sl.box[k]] * l);
        for (int d = 0; d < 3; ++d) gtau[d] += T->abar[sl.box[k]] * gl[d];
    }
    double S2 = R.D[0] * R.D[0] + R.D[1] * R.D[1] + R.D[2] * R.D[2];
    double f = L * exp(-nsum_get(&tau)) / (4.0 * M_PI * S2);
    for (int64_t k = 0; k < sl.n; ++k) ATOMIC_ADD(&acc->G[sl.box[k]], -g * f * sl.len[k]);
    if (src >= 0) {
        ATOMIC_ADD(&acc->e[src], g * f / L);
    } else {
        ATOMIC_ADD(&acc->a[C], g * f / L);
        for (int d = 0; d < 3; ++d) {
            double gq = f * (-2.0 * R.D[d] / S2 - gtau[d]);
            ATOMIC_ADD(&acc->b[3 * C + d], g * gq / L);
        }
    }
    free(sl.box);
    free(sl.len);
}

static void adj_sink(const orc_tree *T, int64_t i, float theta, float tau_ref, double g,
                     adj_acc_t *acc)
{
    const float theta2 = theta * theta;
    const float smin = 1e-12f * T->side32;
    const float smin2 = smin * smin;
    const float p[3] = {T->ux[i], T->uy[i], T->uz[i]};
    const int64_t S = T->leaf_of[i];
    int64_t stack[MAXDEPTH + 2];
    int sp = 0;
    stack[sp++] = ROOT;
    while (sp > 0) {
        int64_t X = stack[--sp];
        if (!(T->L[X] > 0.0)) continue;
        float r2 = 0.0f;
        for (int d = 0; d < 3; ++d) {
            float e = fmaxf(fmaxf(T->blo32[X][d] - p[d], p[d] - T->bhi32[X][d]), 0.0f);
            r2 = r2 + e * e;
        }
        if (T->l2_32[X] < theta2 * r2) {
            adj_interaction(T, i, S, X, T->cen32[X], T->cen[X], T->L[X], tau_ref, smin2, g, -1,
                            acc);
        } else if (T->split_bit[X] < 0) {
            for (int64_t s = T->src_first[X]; s < T->src_first[X] + T->src_count[X]; ++s) {
                if (!(T->slum[s] > 0.0f)) continue;
                const float q32[3] = {T->usx[s], T->usy[s], T->usz[s]};
                const double q64[3] = {(double)T->sx[s], (double)T->sy[s], (double)T->sz[s]};
                adj_interaction(T, i, S, X, q32, q64, (double)T->slum[s], tau_ref, smin2, g, s,
                                acc);
            }
        } else {
            stack[sp++] = T->upper[X];
            stack[sp++] = T->lower[X];
        }
    }
}

/*
 * Gradients of a loss with dLoss/dF = grad_flux (one entry per sink in
 * `sinks`, caller indices) with respect to the source luminosities
 * (grad_lum, n_src, caller order) and the particle absorption coefficients
 * (grad_alpha, n_gas, caller order). Decisions frozen (see above).
 */
int orc_adjoint(const orc_tree *T, const int64_t *sinks, int64_t n_sink, const double *grad_flux,
                float theta, float tau_ref, double *grad_lum, double *grad_alpha, int nthreads)
{
    if (T->nb > 1) return ORC_ERR_INVALID_ARGUMENT; /* a tree with bands: orc_flux_bands */
    for (int64_t k = 0; k < n_sink; ++k)
        if (sinks[k] < 0 || sinks[k] >= T->n_gas) return ORC_ERR_INVALID_ARGUMENT;
    const int64_t nn = T->n_nodes;
    adj_acc_t acc;
    acc.a = calloc((size_t)nn, sizeof(double));
    acc.b = calloc((size_t)(3 * nn), sizeof(double));
    acc.e = calloc((size_t)(T->n_src > 0 ? T->n_src : 1), sizeof(double));
    acc.G = calloc((size_t)nn, sizeof(double));
    if (!acc.a || !acc.b || !acc.e || !acc.G) {
        free(acc.a);
        free(acc.b);
        free(acc.e);
        free(acc.G);
        return ORC_ERR_NO_MEMORY;
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t k = 0; k < n_sink; ++k)
        if (grad_flux[k] != 0.0) adj_sink(T, T->rank[sinks[k]], theta, tau_ref, grad_flux[k], &acc);

    /* luminosities: single-source terms plus, for every ancestor C of the
       source's leaf (the leaf included), a_C + b_C . (y_j - c_C) */
    for (int64_t s = 0; s < T->n_src; ++s) {
        double gsum = acc.e[s];
        const double y[3] = {(double)T->sx[s], (double)T->sy[s], (double)T->sz[s]};
        for (int64_t C = T->src_leaf[s]; C >= 0; C = T->parent[C]) {
            gsum += acc.a[C];
            for (int d = 0; d < 3; ++d) gsum += acc.b[3 * C + d] * (y[d] - T->cen[C][d]);
        }
        grad_lum[T->src_order[s]] = gsum;
    }
    /* absorption: w_i sum over the cells X holding i of G_X / W_X */
    for (int64_t i = 0; i < T->n_gas; ++i) {
        double gsum = 0.0;
        for (int64_t X = T->leaf_of[i]; X >= 0; X = T->parent[X]) gsum += acc.G[X] / T->W[X];
        grad_alpha[T->perm[i]] = (double)T->w[i] * gsum;
    }
    free(acc.a);
    free(acc.b);
    free(acc.e);
    free(acc.G);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Replay: the loss sum_p w_p log F_p re-evaluated with the decisions of the */
/* unperturbed forward pass (interactions and segment cells recorded), for   */
/* one perturbed input. Used for central finite differences of the adjoint.  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n_sink;
    int64_t *sink_i;     /* sorted particle index of each sink */
    int64_t *ia_start;   /* n_sink+1: range of interactions */
    int64_t *ia_node;    /* C */
    int64_t *ia_src;     /* sorted source index or -1 */
    int64_t *ia_seg0;    /* n_ia+1: range of segment cells */
    int64_t *seg_box;
    int64_t n_ia, n_seg;
} orc_replay;

void orc_replay_free(orc_replay *r)
{
    if (!r) return;
    free(r->sink_i);
    free(r->ia_start);
    free(r->ia_node);
    free(r->ia_src);
    free(r->ia_seg0);
    free(r->seg_box);
    free(r);
}

typedef struct {
    int64_t *node, *src, *nseg;
    int64_t n, cap;
    seglist_t segs;
} rec_buf_t;

static void rec_interaction(const orc_tree *T, int64_t i, int64_t S, int64_t C, const float q32[3],
                            const double q64[3], float tau_ref, float smin2, int64_t src,
                            rec_buf_t *rb)
{
    ray_t R;
    make_ray(T, i, q32, q64, &R);
    float s2 = R.d[0] * R.d[0] + R.d[1] * R.d[1] + R.d[2] * R.d[2];
    if (s2 < smin2) return;
    int64_t before = rb->segs.n;
    ray_segments(T, &R, S, C, tau_ref, &rb->segs);
    if (rb->n == rb->cap) {
        int64_t nc = rb->cap ? 2 * rb->cap : 64;
        rb->node = realloc(rb->node, (size_t)nc * sizeof(int64_t));
        rb->src = realloc(rb->src, (size_t)nc * sizeof(int64_t));
        rb->nseg = realloc(rb->nseg, (size_t)nc * sizeof(int64_t));
        rb->cap = nc;
    }
    rb->node[rb->n] = C;
    rb->src[rb->n] = src;
    rb->nseg[rb->n] = rb->segs.n - before;
    rb->n++;
}

int orc_replay_record(const orc_tree *T, const int64_t *sinks, int64_t n_sink, float theta,
                      float tau_ref, orc_replay **out)
{
    if (T->nb > 1) return ORC_ERR_INVALID_ARGUMENT; /* a tree with bands: orc_flux_bands */
    *out = NULL;
    orc_replay *r = calloc(1, sizeof(orc_replay));
    rec_buf_t rb;
    memset(&rb, 0, sizeof(rb));
    r->n_sink = n_sink;
    r->sink_i = malloc((size_t)(n_sink + 1) * sizeof(int64_t));
    r->ia_start = malloc((size_t)(n_sink + 1) * sizeof(int64_t));
    const float theta2 = theta * theta;
    const float smin = 1e-12f * T->side32;
    const float smin2 = smin * smin;
    for (int64_t k = 0; k < n_sink; ++k) {
        int64_t i = T->rank[sinks[k]];
        r->sink_i[k] = i;
        r->ia_start[k] = rb.n;
        const float p[3] = {T->ux[i], T->uy[i], T->uz[i]};
        const int64_t S = T->leaf_of[i];
        int64_t stack[MAXDEPTH + 2];
        int sp = 0;
        stack[sp++] = ROOT;
        while (sp > 0) {
            int64_t X = stack[--sp];
            if (!(T->L[X] > 0.0)) continue;
            float r2 = 0.0f;
            for (int d = 0; d < 3; ++d) {
                float e = fmaxf(fmaxf(T->blo32[X][d] - p[d], p[d] - T->bhi32[X][d]), 0.0f);
                r2 = r2 + e * e;
            }
            if (T->l2_32[X] < theta2 * r2) {
                rec_interaction(T, i, S, X, T->cen32[X], T->cen[X], tau_ref, smin2, -1, &rb);
            } else if (T->split_bit[X] < 0) {
                for (int64_t s = T->src_first[X]; s < T->src_first[X] + T->src_count[X]; ++s) {
                    if (!(T->slum[s] > 0.0f)) continue;
                    const float q32[3] = {T->usx[s], T->usy[s], T->usz[s]};
                    const double q64[3] = {(double)T->sx[s], (double)T->sy[s], (double)T->sz[s]};
                    rec_interaction(T, i, S, X, q32, q64, tau_ref, smin2, s, &rb);
                }
            } else {
                stack[sp++] = T->upper[X];
                stack[sp++] = T->lower[X];
            }
        }
    }
    r->ia_start[n_sink] = rb.n;
    r->n_ia = rb.n;
    r->n_seg = rb.segs.n;
    r->ia_node = rb.node;
    r->ia_src = rb.src;
    r->seg_box = rb.segs.box;
    free(rb.segs.len);
    r->ia_seg0 = malloc((size_t)(rb.n + 1) * sizeof(int64_t));
    int64_t acc = 0;
    for (int64_t q = 0; q < rb.n; ++q) {
        r->ia_seg0[q] = acc;
        acc += rb.nseg[q];
    }
    r->ia_seg0[rb.n] = acc;
    free(rb.nseg);
    *out = r;
    return ORC_OK;
}

/* FP64 length of the segment p->q inside node X (no decisions). */
static double seg_len64(const orc_tree *T, const double P[3], const double Q[3], int64_t X)
{
    double D[3] = {Q[0] - P[0], Q[1] - P[1], Q[2] - P[2]};
    double t0 = 0.0, t1 = 1.0;
    for (int k = 0; k < 3; ++k) {
        double lo = T->lo[k] + (double)T->glo[X][k] * T->h;
        double hi = T->lo[k] + (double)T->ghi[X][k] * T->h;
        if (D[k] != 0.0) {
            double ta = (lo - P[k]) / D[k], tb = (hi - P[k]) / D[k];
            t0 = fmax(t0, fmin(ta, tb));
            t1 = fmin(t1, fmax(ta, tb));
        } else if (P[k] < lo || P[k] >= hi) {
            return 0.0;
        }
    }
    return t1 > t0 ? (t1 - t0) * sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]) : 0.0;
}

/* Bounding planes of the segment p->q inside node X (FP64, as seg_len64): plane
   2k+0 is the box's lower face on axis k, 2k+1 its upper face; *e0 is the plane
   that sets the entry t0 and *e1 the one that sets the exit t1, -1 where the ray
   starts or ends inside X (t clamped to 0 or 1). Returns 0 when the ray misses X. */
static int seg_planes64(const orc_tree *T, const double P[3], const double Q[3], int64_t X,
                        int *e0, int *e1)
{
    double D[3] = {Q[0] - P[0], Q[1] - P[1], Q[2] - P[2]};
    double t0 = 0.0, t1 = 1.0;
    *e0 = -1;
    *e1 = -1;
    for (int k = 0; k < 3; ++k) {
        double lo = T->lo[k] + (double)T->glo[X][k] * T->h;
        double hi = T->lo[k] + (double)T->ghi[X][k] * T->h;
        if (D[k] != 0.0) {
            double ta = (lo - P[k]) / D[k], tb = (hi - P[k]) / D[k];
            int pa = 2 * k, pb = 2 * k + 1;
            double tn = ta, tx = tb;
            int pn = pa, px = pb;
            if (tb < ta) {
                tn = tb; tx = ta; pn = pb; px = pa;
            }
            if (tn > t0) { t0 = tn; *e0 = pn; }
            if (tx < t1) { t1 = tx; *e1 = px; }
        } else if (P[k] < lo || P[k] >= hi) {
            return 0;
        }
    }
    return t1 > t0;
}

/* FP64 length of the segment p->q inside X with its bounding planes given (as
   seg_planes64 found them for another end point): (t1 - t0) |q - p| with t of
   plane b on axis k equal to (b - p_k)/(q_k - p_k). An analytic function of q. */
static double seg_len64_planes(const orc_tree *T, const double P[3], const double Q[3],
                               int64_t X, int e0, int e1)
{
    double D[3] = {Q[0] - P[0], Q[1] - P[1], Q[2] - P[2]};
    double t0 = 0.0, t1 = 1.0;
    if (e0 >= 0) {
        int k = e0 / 2;
        double b = T->lo[k] + (double)(e0 % 2 ? T->ghi[X][k] : T->glo[X][k]) * T->h;
        t0 = (b - P[k]) / D[k];
    }
    if (e1 >= 0) {
        int k = e1 / 2;
        double b = T->lo[k] + (double)(e1 % 2 ? T->ghi[X][k] : T->glo[X][k]) * T->h;
        t1 = (b - P[k]) / D[k];
    }
    return (t1 - t0) * sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
}

/* The perturbed moments of one replay evaluation: luminosity and centre of every
   cell, the luminosity of the perturbed source, and the change of every cell's
   mean absorption (kind 0: source `index` has L += h; kind 1: particle `index`
   has alpha += h; kind -1: none). */
typedef struct {
    double *dabar, *Lp, (*cp)[3];
    int64_t psrc;
    double srcL;
} replay_pert_t;

static void replay_perturb(const orc_tree *T, int kind, int64_t index, double h, replay_pert_t *o)
{
    const int64_t nn = T->n_nodes;
    o->dabar = calloc((size_t)nn, sizeof(double));
    o->Lp = malloc((size_t)nn * sizeof(double));
    o->cp = malloc((size_t)nn * sizeof(*o->cp));
    for (int64_t X = 0; X < nn; ++X) {
        o->Lp[X] = T->L[X];
        for (int d = 0; d < 3; ++d) o->cp[X][d] = T->cen[X][d];
    }
    o->psrc = -1;
    o->srcL = 0.0;
    if (kind == 0) {
        for (int64_t s = 0; s < T->n_src; ++s)
            if (T->src_order[s] == index) o->psrc = s;
        const int64_t ps = o->psrc;
        const double y[3] = {(double)T->sx[ps], (double)T->sy[ps], (double)T->sz[ps]};
        for (int64_t C = T->src_leaf[ps]; C >= 0; C = T->parent[C]) {
            double Ln = T->L[C] + h;
            for (int d = 0; d < 3; ++d) o->cp[C][d] = (T->L[C] * T->cen[C][d] + h * y[d]) / Ln;
            o->Lp[C] = Ln;
        }
        o->srcL = (double)T->slum[ps] + h;
    } else if (kind == 1) {
        int64_t i = T->rank[index];
        for (int64_t X = T->leaf_of[i]; X >= 0; X = T->parent[X])
            o->dabar[X] = (double)T->w[i] * h / T->W[X];
    }
}

static void replay_pert_free(replay_pert_t *o)
{
    free(o->dabar);
    free(o->Lp);
    free(o->cp);
}

/*
 * Loss sum_k w[k] log F_k over the recorded sinks, with one input perturbed:
 * kind 0: luminosity of source `index` (caller order) += h;
 * kind 1: alpha of particle `index` (caller order) += h;
 * kind -1: no perturbation.  Moments are updated exactly for the perturbation.
 * frozen_planes = 0: each segment's length is the FP64 clip of the moved ray (the
 * loss whose decisions are frozen; it has kinks where a bounding plane switches).
 * frozen_planes = 1: each segment keeps the bounding planes of the unperturbed
 * ray, so the loss is analytic in h; its derivative at h = 0 is the same, and it
 * is the function the adjoint differentiates.
 */
double orc_replay_loss_planes(const orc_tree *T, const orc_replay *r, const double *w, int kind,
                              int64_t index, double h, int frozen_planes)
{
    replay_pert_t pt;
    replay_perturb(T, kind, index, h, &pt);
    double loss = 0.0;
#ifdef _OPENMP
#pragma omp parallel for reduction(+ : loss) schedule(dynamic, 16)
#endif
    for (int64_t k = 0; k < r->n_sink; ++k) {
        int64_t i = r->sink_i[k];
        const double P[3] = {(double)T->px[i], (double)T->py[i], (double)T->pz[i]};
        nsum_t F = {0.0, 0.0};
        for (int64_t q = r->ia_start[k]; q < r->ia_start[k + 1]; ++q) {
            int64_t C = r->ia_node[q], s = r->ia_src[q];
            double Q[3], Q0[3], L;
            if (s >= 0) {
                Q[0] = (double)T->sx[s];
                Q[1] = (double)T->sy[s];
                Q[2] = (double)T->sz[s];
                L = (s == pt.psrc) ? pt.srcL : (double)T->slum[s];
            } else {
                for (int d = 0; d < 3; ++d) Q[d] = pt.cp[C][d];
                L = pt.Lp[C];
            }
            for (int d = 0; d < 3; ++d) Q0[d] = s >= 0 ? Q[d] : T->cen[C][d];
            nsum_t tau = {0.0, 0.0};
            for (int64_t g = r->ia_seg0[q]; g < r->ia_seg0[q + 1]; ++g) {
                int64_t X = r->seg_box[g];
                double l;
                if (frozen_planes) {
                    int e0, e1;
                    l = seg_planes64(T, P, Q0, X, &e0, &e1) ?
                        seg_len64_planes(T, P, Q, X, e0, e1) : 0.0;
                } else {
                    l = seg_len64(T, P, Q, X);
                }
                nsum_add(&tau, (T->abar[X] + pt.dabar[X]) * l);
            }
            double s2 = 0.0;
            for (int d = 0; d < 3; ++d) s2 += (Q[d] - P[d]) * (Q[d] - P[d]);
            nsum_add(&F, L * exp(-nsum_get(&tau)) / (4.0 * M_PI * s2));
        }
        loss += w[k] * log(nsum_get(&F));
    }
    replay_pert_free(&pt);
    return loss;
}

double orc_replay_loss(const orc_tree *T, const orc_replay *r, const double *w, int kind,
                       int64_t index, double h)
{
    return orc_replay_loss_planes(T, r, w, kind, index, h, 0);
}

/*
 * Number of recorded segments whose bounding planes (seg_planes64) differ between
 * the perturbations -h and +h of input `index` (kind as orc_replay_loss): each is a
 * kink of the frozen-decision loss inside the central-difference step. Only a
 * luminosity moves a ray (through the centres of luminosity), so kind 1 gives 0.
 */
int64_t orc_replay_kinks(const orc_tree *T, const orc_replay *r, int kind, int64_t index,
                         double h)
{
    if (kind != 0) return 0;
    replay_pert_t pm, pp;
    replay_perturb(T, kind, index, -h, &pm);
    replay_perturb(T, kind, index, h, &pp);
    int64_t kinks = 0;
#ifdef _OPENMP
#pragma omp parallel for reduction(+ : kinks) schedule(dynamic, 16)
#endif
    for (int64_t k = 0; k < r->n_sink; ++k) {
        int64_t i = r->sink_i[k];
        const double P[3] = {(double)T->px[i], (double)T->py[i], (double)T->pz[i]};
        for (int64_t q = r->ia_start[k]; q < r->ia_start[k + 1]; ++q) {
            int64_t C = r->ia_node[q];
            if (r->ia_src[q] >= 0) continue; /* a single source does not move */
            const double *Qm = pm.cp[C], *Qp = pp.cp[C];
            if (Qm[0] == Qp[0] && Qm[1] == Qp[1] && Qm[2] == Qp[2]) continue;
            for (int64_t g = r->ia_seg0[q]; g < r->ia_seg0[q + 1]; ++g) {
                int a0, a1, b0, b1;
                int hm = seg_planes64(T, P, Qm, r->seg_box[g], &a0, &a1);
                int hp = seg_planes64(T, P, Qp, r->seg_box[g], &b0, &b1);
                if (hm != hp || (hm && (a0 != b0 || a1 != b1))) ++kinks;
            }
        }
    }
    replay_pert_free(&pm);
    replay_pert_free(&pp);
    return kinks;
}
