/*
 * zd_oracle.c -- plain, slow CPU oracle for the zd-tree k-NN path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or helper with the CUDA
 * library; the two meet only on the arrays produced by the seeded generators.
 *
 * What it computes, and where the paper defines it (Blelloch & Dobson,
 * "Parallel Nearest Neighbors in Low Dimensions with Batch Updates"):
 *
 *   morton_key        Sec. 1.1 "Morton ordering" + Sec. 2 "Construction"
 *                     (random shift, kept for the tree's lifetime).
 *   sort              Sec. 2 "Construction": points sorted by Morton order.
 *                     Ties (equal keys) keep ascending id.
 *   build             Algorithm 1 (buildTree / splitUsingBit) with the
 *                     empty-cut pruning of Sec. 2.1 ("pruned zd-tree").
 *   boxes             Sec. 2 "Data structure": every node stores the corners
 *                     of the bounding box of its points.
 *   search_down       Algorithm 2 (searchDown, withinBox, distance, insert).
 *   search_up         Algorithm 3 (searchUp); leaf-based mode of Sec. 2.
 *   bit / root mode   Sec. 2 "Upward search algorithm", last paragraph.
 *   brute force       the plain definition of exact k-NN (no tree).
 *   gradient          d/dx of a sum of Euclidean k-NN distances (no paper
 *                     counterpart; plain calculus in fp64).
 *
 * Readings where the paper is silent or loose (each listed in the design
 * notes):  leaf iff size <= L (Alg. 1 "size < sizeCutoff" with
 * sizeCutoff = L+1); the candidate inserted in Alg. 2/3 is q, not p;
 * neighbours are ranked by the total order (squared distance, id); a node is
 * visited iff its box distance^2 <= the current k-th distance^2; the climb of
 * Alg. 3 stops once no point outside the current node's box can be within the
 * k-th distance; fewer than k candidates pad with id -1.
 *
 * Arithmetic: integer coordinates use exact int64 squared distances.  Float
 * coordinates rank by an fp64 squared distance evaluated left to right,
 * ((dx*dx + dy*dy) + dz*dz) with dx = (double)q.x - (double)p.x; this file
 * must be compiled with -ffp-contract=off so no FMA changes the rounding.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ZDO_OK 0
#define ZDO_ERR_INVALID 1
#define ZDO_ERR_RANGE 2
#define ZDO_ERR_OOM 3

/* ------------------------------------------------------------------------ */
/* Morton key (Sec. 1.1): read the bits of the shifted integer coordinates   */
/* from the top level down; within one level the first coordinate comes     */
/* first.  Level b of coordinate j lands on key bit d*b + (d-1-j).          */
/* ------------------------------------------------------------------------ */
static uint64_t morton_key(const int64_t *c, int dim, int coord_bits)
{
    uint64_t key = 0;
    for (int b = coord_bits - 1; b >= 0; --b)
        for (int j = 0; j < dim; ++j)
            key = (key << 1) | (uint64_t)((c[j] >> b) & 1);
    return key;
}

static int params_ok(int dim, int coord_bits)
{
    if (dim != 2 && dim != 3) return 0;
    if (coord_bits < 1 || coord_bits * dim > 64) return 0;
    return 1;
}

/* Integer points: shift, range-check against [0, 2^coord_bits), encode. */
int zdo_morton_keys_i32(const int32_t *pts, int64_t n, int dim, int coord_bits,
                        const uint32_t *shift, uint64_t *keys)
{
    if (!params_ok(dim, coord_bits) || n < 0) return ZDO_ERR_INVALID;
    const int64_t lim = (int64_t)1 << coord_bits;
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3] = {0, 0, 0};
        for (int j = 0; j < dim; ++j) {
            c[j] = (int64_t)pts[i * dim + j] + (int64_t)(shift ? shift[j] : 0u);
            if (c[j] < 0 || c[j] >= lim) return ZDO_ERR_RANGE;
        }
        keys[i] = morton_key(c, dim, coord_bits);
    }
    return ZDO_OK;
}

/* Float points (Sec. 3.1 "Numerical details": coordinates are rounded to
 * integers for the tree and the Morton order).  Reading: per dimension
 * q = floor((x - lo_j) * scale), clamped to [0, 2^coord_bits - 1], in fp64.
 * It only shapes the tree; the neighbour ranking uses the float values. */
int zdo_quantize_f32(const float *pts, int64_t n, int dim, const double *lo,
                     double scale, int coord_bits, int32_t *q)
{
    if (!params_ok(dim, coord_bits) || coord_bits > 31) return ZDO_ERR_INVALID;
    const double top = (double)(((int64_t)1 << coord_bits) - 1);
    for (int64_t i = 0; i < n; ++i)
        for (int j = 0; j < dim; ++j) {
            double v = floor(((double)pts[i * dim + j] - lo[j]) * scale);
            if (!(v >= 0.0)) v = 0.0; /* also maps NaN to 0 */
            if (v > top) v = top;
            q[i * dim + j] = (int32_t)v;
        }
    return ZDO_OK;
}

/* ------------------------------------------------------------------------ */
/* Sort by Morton order (Sec. 2 "Construction"); equal keys by ascending id. */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t key;
    int64_t id;
    int64_t pos;
} sort_rec;

static int cmp_rec(const void *a, const void *b)
{
    const sort_rec *x = (const sort_rec *)a, *y = (const sort_rec *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

/* perm[i] = input position of the i-th point in (key, id) order. */
int zdo_sort_perm(const uint64_t *keys, const int32_t *ids, int64_t n, int64_t *perm)
{
    sort_rec *r = (sort_rec *)malloc(sizeof(sort_rec) * (size_t)(n > 0 ? n : 1));
    if (!r) return ZDO_ERR_OOM;
    for (int64_t i = 0; i < n; ++i) {
        r[i].key = keys[i];
        r[i].id = ids ? ids[i] : i;
        r[i].pos = i;
    }
    qsort(r, (size_t)n, sizeof(sort_rec), cmp_rec);
    for (int64_t i = 0; i < n; ++i) perm[i] = r[i].pos;
    free(r);
    return ZDO_OK;
}

/* ------------------------------------------------------------------------ */
/* The tree (Sec. 2 "Data structure").                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t lo, hi;             /* points [lo, hi) of the sorted order */
    int bit;                    /* split bit of an internal node, -1 for a leaf */
    int64_t left, right, parent; /* -1 where absent */
    int64_t ibox_lo[3], ibox_hi[3]; /* integer mode: tight box of the points */
    double fbox_lo[3], fbox_hi[3];  /* float mode: tight box of the points */
} onode;

typedef struct {
    int64_t n;
    int dim, coord_bits, leaf_size, is_float;
    uint32_t shift[3];
    double qlo[3], qscale;      /* float mode quantization */
    uint64_t *keys;             /* sorted keys */
    int32_t *ids;               /* sorted ids */
    int64_t *icoord;            /* sorted integer coordinates [n, dim] */
    double *fcoord;             /* sorted float coordinates (as double) [n, dim] */
    onode *nodes;
    int64_t nnodes, cap;
    int64_t root;
    int oom;
} otree;

static int64_t new_node(otree *t)
{
    if (t->nnodes == t->cap) {
        int64_t nc = t->cap ? 2 * t->cap : 64;
        onode *nn = (onode *)realloc(t->nodes, sizeof(onode) * (size_t)nc);
        if (!nn) {
            t->oom = 1;
            return -1;
        }
        t->nodes = nn;
        t->cap = nc;
    }
    int64_t id = t->nnodes++;
    onode *v = &t->nodes[id];
    memset(v, 0, sizeof(*v));
    v->left = v->right = v->parent = -1;
    v->bit = -1;
    return id;
}

/* splitUsingBit (Alg. 1): the points of a node share every key bit above b,
 * so along the sorted range bit b is 0...0 1...1; binary search for the first
 * 1.  Returns hi if there is none. */
static int64_t split_using_bit(const uint64_t *keys, int64_t lo, int64_t hi, int b)
{
    int64_t a = lo, z = hi;
    while (a < z) {
        int64_t mid = a + (z - a) / 2;
        if ((keys[mid] >> b) & 1) z = mid;
        else a = mid + 1;
    }
    return a;
}

/* buildTree(P, b) of Alg. 1.  `b` counts the key bits not yet used; the bit
 * examined is b-1.  A leaf is made when the node holds at most L points or
 * no bits remain (then all its keys are equal).  A cut that leaves one side
 * empty makes no node: the same points are split on the next bit instead
 * (Sec. 2.1, the pruned zd-tree). */
static int64_t build_rec(otree *t, int64_t lo, int64_t hi, int b, int64_t parent)
{
    for (;;) {
        if (hi - lo <= t->leaf_size || b == 0) {
            int64_t id = new_node(t);
            if (id < 0) return -1;
            t->nodes[id].lo = lo;
            t->nodes[id].hi = hi;
            t->nodes[id].parent = parent;
            return id;
        }
        int64_t s = split_using_bit(t->keys, lo, hi, b - 1);
        if (s == lo || s == hi) {
            b -= 1; /* empty cut: pruned */
            continue;
        }
        int64_t id = new_node(t);
        if (id < 0) return -1;
        t->nodes[id].lo = lo;
        t->nodes[id].hi = hi;
        t->nodes[id].bit = b - 1;
        t->nodes[id].parent = parent;
        int64_t l = build_rec(t, lo, s, b - 1, id);
        int64_t r = build_rec(t, s, hi, b - 1, id);
        if (l < 0 || r < 0) return -1;
        t->nodes[id].left = l;
        t->nodes[id].right = r;
        return id;
    }
}

/* Bounding box of every node: a leaf's from its points, an internal node's
 * as the union of its children's boxes (post-order). */
static void boxes_rec(otree *t, int64_t v)
{
    onode *x = &t->nodes[v];
    const int d = t->dim;
    for (int j = 0; j < 3; ++j) {
        x->ibox_lo[j] = INT64_MAX;
        x->ibox_hi[j] = INT64_MIN;
        x->fbox_lo[j] = INFINITY;
        x->fbox_hi[j] = -INFINITY;
    }
    if (x->bit < 0) {
        for (int64_t i = x->lo; i < x->hi; ++i)
            for (int j = 0; j < d; ++j) {
                if (t->is_float) {
                    double c = t->fcoord[i * d + j];
                    if (c < x->fbox_lo[j]) x->fbox_lo[j] = c;
                    if (c > x->fbox_hi[j]) x->fbox_hi[j] = c;
                } else {
                    int64_t c = t->icoord[i * d + j];
                    if (c < x->ibox_lo[j]) x->ibox_lo[j] = c;
                    if (c > x->ibox_hi[j]) x->ibox_hi[j] = c;
                }
            }
        return;
    }
    boxes_rec(t, x->left);
    boxes_rec(t, x->right);
    x = &t->nodes[v]; /* no realloc happens here, but keep it obvious */
    const onode *l = &t->nodes[x->left], *r = &t->nodes[x->right];
    for (int j = 0; j < d; ++j) {
        x->ibox_lo[j] = l->ibox_lo[j] < r->ibox_lo[j] ? l->ibox_lo[j] : r->ibox_lo[j];
        x->ibox_hi[j] = l->ibox_hi[j] > r->ibox_hi[j] ? l->ibox_hi[j] : r->ibox_hi[j];
        x->fbox_lo[j] = l->fbox_lo[j] < r->fbox_lo[j] ? l->fbox_lo[j] : r->fbox_lo[j];
        x->fbox_hi[j] = l->fbox_hi[j] > r->fbox_hi[j] ? l->fbox_hi[j] : r->fbox_hi[j];
    }
}

void zdo_free(void *h)
{
    otree *t = (otree *)h;
    if (!t) return;
    free(t->keys);
    free(t->ids);
    free(t->icoord);
    free(t->fcoord);
    free(t->nodes);
    free(t);
}

/* Build the tree over n points.  Exactly one of pts_i32 / pts_f32 is given.
 * ids may be NULL (then ids are 0..n-1).  For float points, qlo[dim] and
 * qscale define the quantization that feeds the Morton keys. */
void *zdo_build(const int32_t *pts_i32, const float *pts_f32, const int32_t *ids, int64_t n,
                int dim, int coord_bits, const uint32_t *shift, const double *qlo,
                double qscale, int leaf_size, int *status)
{
    *status = ZDO_OK;
    if (!params_ok(dim, coord_bits) || leaf_size < 1 || n < 0 || (!pts_i32 && !pts_f32)) {
        *status = ZDO_ERR_INVALID;
        return NULL;
    }
    otree *t = (otree *)calloc(1, sizeof(otree));
    if (!t) {
        *status = ZDO_ERR_OOM;
        return NULL;
    }
    t->n = n;
    t->dim = dim;
    t->coord_bits = coord_bits;
    t->leaf_size = leaf_size;
    t->is_float = pts_f32 != NULL;
    for (int j = 0; j < 3; ++j) {
        t->shift[j] = shift ? shift[j] : 0u;
        t->qlo[j] = (qlo && j < dim) ? qlo[j] : 0.0;
    }
    t->qscale = qscale;
    size_t nn = (size_t)(n > 0 ? n : 1);
    uint64_t *k0 = (uint64_t *)malloc(sizeof(uint64_t) * nn);
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * nn);
    int32_t *qi = NULL;
    t->keys = (uint64_t *)malloc(sizeof(uint64_t) * nn);
    t->ids = (int32_t *)malloc(sizeof(int32_t) * nn);
    if (t->is_float) t->fcoord = (double *)malloc(sizeof(double) * nn * (size_t)dim);
    else t->icoord = (int64_t *)malloc(sizeof(int64_t) * nn * (size_t)dim);
    if (!k0 || !perm || !t->keys || !t->ids || (!t->fcoord && !t->icoord)) {
        *status = ZDO_ERR_OOM;
        goto fail;
    }
    if (t->is_float) {
        qi = (int32_t *)malloc(sizeof(int32_t) * nn * (size_t)dim);
        if (!qi) {
            *status = ZDO_ERR_OOM;
            goto fail;
        }
        *status = zdo_quantize_f32(pts_f32, n, dim, t->qlo, qscale, coord_bits, qi);
        if (*status) goto fail;
        *status = zdo_morton_keys_i32(qi, n, dim, coord_bits, t->shift, k0);
    } else {
        *status = zdo_morton_keys_i32(pts_i32, n, dim, coord_bits, t->shift, k0);
    }
    if (*status) goto fail;
    *status = zdo_sort_perm(k0, ids, n, perm);
    if (*status) goto fail;
    for (int64_t i = 0; i < n; ++i) {
        int64_t p = perm[i];
        t->keys[i] = k0[p];
        t->ids[i] = ids ? ids[p] : (int32_t)p;
        for (int j = 0; j < dim; ++j) {
            if (t->is_float) t->fcoord[i * dim + j] = (double)pts_f32[p * dim + j];
            else t->icoord[i * dim + j] = (int64_t)pts_i32[p * dim + j];
        }
    }
    t->root = build_rec(t, 0, n, dim * coord_bits, -1);
    if (t->root < 0 || t->oom) {
        *status = ZDO_ERR_OOM;
        goto fail;
    }
    boxes_rec(t, t->root);
    free(k0);
    free(perm);
    free(qi);
    return t;
fail:
    free(k0);
    free(perm);
    free(qi);
    zdo_free(t);
    return NULL;
}

int64_t zdo_num_nodes(void *h) { return ((otree *)h)->nnodes; }
int64_t zdo_root(void *h) { return ((otree *)h)->root; }

/* Export: sorted keys, sorted ids, and per node (lo, hi, bit, left, right,
 * parent) plus its box (integer or float, dim values each).  Any output may
 * be NULL. */
void zdo_export(void *h, uint64_t *keys, int32_t *ids, int64_t *lo, int64_t *hi, int32_t *bit,
                int64_t *left, int64_t *right, int64_t *parent, int64_t *ibox_lo,
                int64_t *ibox_hi, double *fbox_lo, double *fbox_hi)
{
    otree *t = (otree *)h;
    const int d = t->dim;
    for (int64_t i = 0; i < t->n; ++i) {
        if (keys) keys[i] = t->keys[i];
        if (ids) ids[i] = t->ids[i];
    }
    for (int64_t v = 0; v < t->nnodes; ++v) {
        const onode *x = &t->nodes[v];
        if (lo) lo[v] = x->lo;
        if (hi) hi[v] = x->hi;
        if (bit) bit[v] = x->bit;
        if (left) left[v] = x->left;
        if (right) right[v] = x->right;
        if (parent) parent[v] = x->parent;
        for (int j = 0; j < d; ++j) {
            if (ibox_lo) ibox_lo[v * d + j] = x->ibox_lo[j];
            if (ibox_hi) ibox_hi[v * d + j] = x->ibox_hi[j];
            if (fbox_lo) fbox_lo[v * d + j] = x->fbox_lo[j];
            if (fbox_hi) fbox_hi[v * d + j] = x->fbox_hi[j];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* The k-best set N of Alg. 2/3, kept sorted by (distance^2, id).           */
/* ------------------------------------------------------------------------ */
typedef struct {
    int k, cnt;
    int64_t *id;
    int64_t *i2; /* integer squared distances */
    double *f2;  /* float-mode squared distances */
} kbest;

/* The query context. */
typedef struct {
    int64_t ic[3];
    double fc[3];
    int64_t self_id; /* all-points mode: the query's own id; -1 otherwise */
} query;

/* Lexicographic "strictly better than the current k-th" test (the order
 * (d^2, id) replaces the strict '<' of Alg. 2 line "distance(q,p) <
 * distance(p,N,k)" so that ties have one answer). */
static int kb_accepts_i(const kbest *N, int64_t d2, int64_t id)
{
    if (N->cnt < N->k) return 1;
    int64_t wd = N->i2[N->k - 1], wi = N->id[N->k - 1];
    return d2 < wd || (d2 == wd && id < wi);
}
static int kb_accepts_f(const kbest *N, double d2, int64_t id)
{
    if (N->cnt < N->k) return 1;
    double wd = N->f2[N->k - 1];
    int64_t wi = N->id[N->k - 1];
    return d2 < wd || (d2 == wd && id < wi);
}

/* insert(N, q, k): keep the k best. */
static void kb_insert_i(kbest *N, int64_t d2, int64_t id)
{
    int pos = N->cnt < N->k ? N->cnt : N->k - 1;
    while (pos > 0 && (N->i2[pos - 1] > d2 || (N->i2[pos - 1] == d2 && N->id[pos - 1] > id))) {
        N->i2[pos] = N->i2[pos - 1];
        N->id[pos] = N->id[pos - 1];
        --pos;
    }
    N->i2[pos] = d2;
    N->id[pos] = id;
    if (N->cnt < N->k) N->cnt++;
}
static void kb_insert_f(kbest *N, double d2, int64_t id)
{
    int pos = N->cnt < N->k ? N->cnt : N->k - 1;
    while (pos > 0 && (N->f2[pos - 1] > d2 || (N->f2[pos - 1] == d2 && N->id[pos - 1] > id))) {
        N->f2[pos] = N->f2[pos - 1];
        N->id[pos] = N->id[pos - 1];
        --pos;
    }
    N->f2[pos] = d2;
    N->id[pos] = id;
    if (N->cnt < N->k) N->cnt++;
}

static int64_t dist2_i(const int64_t *a, const int64_t *b, int dim)
{
    int64_t s = 0;
    for (int j = 0; j < dim; ++j) s += (a[j] - b[j]) * (a[j] - b[j]);
    return s;
}
/* ((dx*dx + dy*dy) + dz*dz), left to right, no contraction. */
static double dist2_f(const double *a, const double *b, int dim)
{
    double s = 0.0;
    for (int j = 0; j < dim; ++j) {
        double dx = a[j] - b[j];
        double sq = dx * dx;
        s = (j == 0) ? sq : s + sq;
    }
    return s;
}

/* Consider point i of the sorted order as a candidate for N. */
static void consider(const otree *t, int64_t i, const query *q, kbest *N)
{
    int64_t id = t->ids[i];
    if (q->self_id >= 0 && id == q->self_id) return; /* "if q != p" */
    if (t->is_float) {
        double d2 = dist2_f(q->fc, &t->fcoord[i * t->dim], t->dim);
        if (kb_accepts_f(N, d2, id)) kb_insert_f(N, d2, id);
    } else {
        int64_t d2 = dist2_i(q->ic, &t->icoord[i * t->dim], t->dim);
        if (kb_accepts_i(N, d2, id)) kb_insert_i(N, d2, id);
    }
}

/* withinBox(T, p, r) of Alg. 2: true while N is not full, else iff the
 * squared distance from p to T's box is <= the k-th squared distance. */
static int within_box(const otree *t, const onode *v, const query *q, const kbest *N)
{
    if (N->cnt < N->k) return 1;
    if (v->hi <= v->lo) return 0; /* empty node: nothing to find */
    if (t->is_float) {
        double s = 0.0;
        for (int j = 0; j < t->dim; ++j) {
            double c = 0.0;
            if (q->fc[j] < v->fbox_lo[j]) c = v->fbox_lo[j] - q->fc[j];
            else if (q->fc[j] > v->fbox_hi[j]) c = q->fc[j] - v->fbox_hi[j];
            double sq = c * c;
            s = (j == 0) ? sq : s + sq;
        }
        return s <= N->f2[N->k - 1];
    }
    int64_t s = 0;
    for (int j = 0; j < t->dim; ++j) {
        int64_t c = 0;
        if (q->ic[j] < v->ibox_lo[j]) c = v->ibox_lo[j] - q->ic[j];
        else if (q->ic[j] > v->ibox_hi[j]) c = q->ic[j] - v->ibox_hi[j];
        s += c * c;
    }
    return s <= N->i2[N->k - 1];
}

/* withinBox(C, p, -r) of Alg. 3: true iff N is full and no point outside C's
 * box can be within the k-th distance, i.e. in every dimension the gap from
 * p to the outside of the box, squared, exceeds the k-th squared distance.
 * Integer points outside [lo, hi] lie at lo-1 or hi+1 or beyond. */
static int inside_box(const otree *t, const onode *v, const query *q, const kbest *N)
{
    if (N->cnt < N->k) return 0;
    if (v->hi <= v->lo) return 0;
    for (int j = 0; j < t->dim; ++j) {
        if (t->is_float) {
            double a = q->fc[j] - v->fbox_lo[j], b = v->fbox_hi[j] - q->fc[j];
            double m = a < b ? a : b;
            if (!(m >= 0.0)) return 0;
            if (!(m * m > N->f2[N->k - 1])) return 0;
        } else {
            int64_t a = q->ic[j] - v->ibox_lo[j] + 1, b = v->ibox_hi[j] + 1 - q->ic[j];
            int64_t m = a < b ? a : b;
            if (m <= 0) return 0;
            if (!(m * m > N->i2[N->k - 1])) return 0;
        }
    }
    return 1;
}

/* Distance ordering of Alg. 2's children: squared distance from p to a box
 * centre, computed on doubled coordinates so it stays integral. */
static double centre_dist(const otree *t, const onode *v, const query *q)
{
    double s = 0.0;
    for (int j = 0; j < t->dim; ++j) {
        double c = t->is_float ? 2.0 * q->fc[j] - v->fbox_lo[j] - v->fbox_hi[j]
                               : (double)(2 * q->ic[j] - v->ibox_lo[j] - v->ibox_hi[j]);
        s += c * c;
    }
    return s;
}

/* searchDown (Alg. 2). */
static void search_down(const otree *t, int64_t vi, const query *q, kbest *N)
{
    const onode *v = &t->nodes[vi];
    if (!within_box(t, v, q, N)) return;
    if (v->bit < 0) {
        for (int64_t i = v->lo; i < v->hi; ++i) consider(t, i, q, N);
        return;
    }
    const onode *L = &t->nodes[v->left], *R = &t->nodes[v->right];
    double dl = centre_dist(t, L, q), dr = centre_dist(t, R, q);
    if (dl < dr) {
        search_down(t, v->left, q, N);
        search_down(t, v->right, q, N);
    } else {
        search_down(t, v->right, q, N);
        search_down(t, v->left, q, N);
    }
}

/* searchUp (Alg. 3) from leaf c. */
static void search_up(const otree *t, int64_t c, const query *q, kbest *N)
{
    const onode *C = &t->nodes[c];
    for (int64_t i = C->lo; i < C->hi; ++i) consider(t, i, q, N);
    int64_t p = C->parent;
    while (!inside_box(t, &t->nodes[c], q, N) && p >= 0) {
        const onode *P = &t->nodes[p];
        search_down(t, P->left == c ? P->right : P->left, q, N);
        c = p;
        p = t->nodes[c].parent;
    }
}

/* Bit-based leaf location (Sec. 2): from the root, go right iff the query's
 * Morton key has the node's split bit set. */
static int64_t locate_leaf(const otree *t, uint64_t key)
{
    int64_t v = t->root;
    while (t->nodes[v].bit >= 0) v = ((key >> t->nodes[v].bit) & 1) ? t->nodes[v].right : t->nodes[v].left;
    return v;
}

/* k-NN over the tree.
 *   mode 0: all points (leaf-based; queries are the tree's own points, self
 *           excluded by id; output row r belongs to sorted position r0 + r,
 *           whose id zdo_export reports; [r0, r1) selects a range of sorted
 *           positions, r1 < 0 meaning all);
 *   mode 1: external queries, bit-based leaf location then Alg. 3;
 *   mode 2: external queries, root-based Alg. 2.
 * External queries come as q_i32 or q_f32 [m, dim].  Outputs [m, k]: ids
 * (-1 padding) and squared distances (int64, or fp64 in float mode; padding
 * INT64_MAX / +inf).  Returns ZDO_ERR_RANGE if a query key is out of range. */
int zdo_knn(void *h, const int32_t *q_i32, const float *q_f32, int64_t m, int k, int mode,
            int64_t r0, int64_t r1, int32_t *out_idx, int64_t *out_d2, double *out_d2f,
            int nthreads)
{
    otree *t = (otree *)h;
    const int d = t->dim;
    if (k < 1 || (mode < 0 || mode > 2)) return ZDO_ERR_INVALID;
    if (mode == 0) {
        if (r1 < 0 || r1 > t->n) r1 = t->n;
        if (r0 < 0 || r0 > r1) return ZDO_ERR_INVALID;
        m = r1 - r0;
    }
    uint64_t *qkeys = NULL;
    if (mode == 1) {
        /* query Morton keys for the bit-based descent */
        qkeys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1));
        if (!qkeys) return ZDO_ERR_OOM;
        int st;
        if (t->is_float) {
            int32_t *qq = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1) * (size_t)d);
            if (!qq) {
                free(qkeys);
                return ZDO_ERR_OOM;
            }
            zdo_quantize_f32(q_f32, m, d, t->qlo, t->qscale, t->coord_bits, qq);
            st = zdo_morton_keys_i32(qq, m, d, t->coord_bits, t->shift, qkeys);
            free(qq);
        } else {
            st = zdo_morton_keys_i32(q_i32, m, d, t->coord_bits, t->shift, qkeys);
        }
        if (st) {
            free(qkeys);
            return st;
        }
    }
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        kbest N;
        N.k = k;
        N.id = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
        N.i2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
        N.f2 = (double *)malloc(sizeof(double) * (size_t)k);
        if (!N.id || !N.i2 || !N.f2) err = 1;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 256)
#endif
        for (int64_t r = 0; r < m; ++r) {
            if (err) continue;
            query q;
            memset(&q, 0, sizeof(q));
            q.self_id = -1;
            int64_t start = -1;
            int64_t row = r;
            if (mode == 0) {
                /* sorted position sp = r0 + r; self excluded by its id */
                const int64_t sp = r0 + r;
                for (int j = 0; j < d; ++j) {
                    if (t->is_float) q.fc[j] = t->fcoord[sp * d + j];
                    else q.ic[j] = t->icoord[sp * d + j];
                }
                q.self_id = t->ids[sp];
                /* the leaf that holds sorted position sp */
                int64_t v = t->root;
                while (t->nodes[v].bit >= 0) {
                    const onode *x = &t->nodes[v];
                    v = (sp < t->nodes[x->left].hi) ? x->left : x->right;
                }
                start = v;
            } else {
                for (int j = 0; j < d; ++j) {
                    if (t->is_float) q.fc[j] = (double)q_f32[r * d + j];
                    else q.ic[j] = (int64_t)q_i32[r * d + j];
                }
                if (mode == 1) start = locate_leaf(t, qkeys[r]);
            }
            N.cnt = 0;
            if (t->n > 0) {
                if (mode == 2) search_down(t, t->root, &q, &N);
                else search_up(t, start, &q, &N);
            }
            for (int j = 0; j < k; ++j) {
                int have = j < N.cnt;
                out_idx[row * k + j] = have ? (int32_t)N.id[j] : -1;
                if (out_d2) out_d2[row * k + j] = have ? N.i2[j] : INT64_MAX;
                if (out_d2f) out_d2f[row * k + j] = have ? N.f2[j] : INFINITY;
            }
        }
        free(N.id);
        free(N.i2);
        free(N.f2);
    }
    free(qkeys);
    return err ? ZDO_ERR_OOM : ZDO_OK;
}

/* ------------------------------------------------------------------------ */
/* Plain definition of exact k-NN (no tree): for each query, rank every     */
/* reference point by (squared distance, id), skipping the reference whose  */
/* id equals the query's id when q_ids is given; take the first k.          */
/* ------------------------------------------------------------------------ */
int zdo_knn_brute(const int32_t *ref_i32, const float *ref_f32, const int32_t *ref_ids,
                  int64_t n, const int32_t *q_i32, const float *q_f32, const int32_t *q_ids,
                  int64_t m, int dim, int k, int32_t *out_idx, int64_t *out_d2,
                  double *out_d2f, int nthreads)
{
    if (k < 1 || (dim != 2 && dim != 3)) return ZDO_ERR_INVALID;
    const int is_float = ref_f32 != NULL;
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        kbest N;
        N.k = k;
        N.id = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
        N.i2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
        N.f2 = (double *)malloc(sizeof(double) * (size_t)k);
        if (!N.id || !N.i2 || !N.f2) err = 1;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t r = 0; r < m; ++r) {
            if (err) continue;
            N.cnt = 0;
            int64_t qi[3] = {0, 0, 0};
            double qf[3] = {0, 0, 0};
            for (int j = 0; j < dim; ++j) {
                if (is_float) qf[j] = (double)q_f32[r * dim + j];
                else qi[j] = (int64_t)q_i32[r * dim + j];
            }
            for (int64_t i = 0; i < n; ++i) {
                int64_t id = ref_ids ? ref_ids[i] : i;
                if (q_ids && id == q_ids[r]) continue;
                if (is_float) {
                    double p[3] = {0, 0, 0};
                    for (int j = 0; j < dim; ++j) p[j] = (double)ref_f32[i * dim + j];
                    double d2 = dist2_f(qf, p, dim);
                    if (kb_accepts_f(&N, d2, id)) kb_insert_f(&N, d2, id);
                } else {
                    int64_t p[3] = {0, 0, 0};
                    for (int j = 0; j < dim; ++j) p[j] = (int64_t)ref_i32[i * dim + j];
                    int64_t d2 = dist2_i(qi, p, dim);
                    if (kb_accepts_i(&N, d2, id)) kb_insert_i(&N, d2, id);
                }
            }
            for (int j = 0; j < k; ++j) {
                int have = j < N.cnt;
                out_idx[r * k + j] = have ? (int32_t)N.id[j] : -1;
                if (out_d2) out_d2[r * k + j] = have ? N.i2[j] : INT64_MAX;
                if (out_d2f) out_d2f[r * k + j] = have ? N.f2[j] : INFINITY;
            }
        }
        free(N.id);
        free(N.i2);
        free(N.f2);
    }
    return err ? ZDO_ERR_OOM : ZDO_OK;
}

/* ------------------------------------------------------------------------ */
/* Loss and gradient of  sum_{i,j} || a_i - b_{idx(i,j)} ||  in fp64.        */
/* gout is a scalar (gout_per == 0) or one weight per (i, j) (gout_per == 1).*/
/* A zero distance contributes a zero gradient; idx < 0 contributes nothing. */
/* ------------------------------------------------------------------------ */
double zdo_knn_dist_grad(const float *a, const float *b, const int32_t *idx, int64_t m,
                         int64_t nb, int dim, int k, const double *gout, int gout_per,
                         double *ga, double *gb)
{
    double loss = 0.0;
    for (int64_t i = 0; i < m * dim; ++i) ga[i] = 0.0;
    for (int64_t i = 0; i < nb * dim; ++i) gb[i] = 0.0;
    for (int64_t i = 0; i < m; ++i)
        for (int j = 0; j < k; ++j) {
            int32_t t = idx[i * k + j];
            if (t < 0 || t >= nb) continue;
            double diff[3] = {0, 0, 0}, s = 0.0;
            for (int c = 0; c < dim; ++c) {
                diff[c] = (double)a[i * dim + c] - (double)b[(int64_t)t * dim + c];
                s += diff[c] * diff[c];
            }
            double dist = sqrt(s);
            loss += dist;
            if (dist == 0.0) continue;
            double g = gout_per ? gout[i * k + j] : gout[0];
            for (int c = 0; c < dim; ++c) {
                double u = g * diff[c] / dist;
                ga[i * dim + c] += u;
                gb[(int64_t)t * dim + c] -= u;
            }
        }
    return loss;
}
