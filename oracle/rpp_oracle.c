/*
 * rpp_oracle.c -- reference CPU oracle for Vietoris-Rips persistence barcodes
 * over Z/2 (Zhang, Xiao, Wang: "GPU-Accelerated Computation of Vietoris-Rips
 * Persistence Barcodes", arXiv 2003.07989).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this library. The GPU library never links, loads or
 * calls it, and the two share no source, header, table or helper.
 *
 * Plain, slow code written from the paper's definitions:
 *   - Rips filtration: the simplices with diam <= t, where diam is the largest
 *     pairwise distance of the simplex's vertices (Sec. 2, definition of Rips_t).
 *   - Simplex-wise refinement: increasing diameter, then increasing dimension,
 *     then decreasing combinatorial index (Sec. "The Simplex-wise Refinement").
 *     The combinatorial index order is the lexicographic order of the
 *     decreasingly sorted vertex tuple (Sec. "The Combinatorial Number System",
 *     remark after the bijection). The oracle compares the tuples themselves:
 *     a simplex is stored as its vertices packed most-significant-first, so
 *     integer order of the packed key is that lexicographic order. No binomial
 *     coefficient is ever formed here.
 *   - Alg. 1 (standard reduction, low = largest nonzero row) on
 *       HOM         the explicit boundary matrix of all simplices;
 *       COHOM       the coboundary matrix (anti-transposed boundary matrix,
 *                   Sec. "The Coboundary Matrix"), one dimension at a time,
 *                   without clearing;
 *       COHOM_CLEAR H0 by Kruskal's union-find in filtration order (Sec.
 *                   "Zero-Dimensional Persistence Computation") and H_q, q >= 1,
 *                   by the coboundary reduction with the clearing lemma (Sec.
 *                   "Clearing Lemma"): the columns of dim-q simplices that were
 *                   deaths in dim q-1 are skipped.
 *     No apparent pairs, emergent pairs or enclosing radius are used by any mode.
 *   - Apparent pairs by their definition (Definition "apparent pair"): sigma is
 *     the youngest facet of tau and tau is the oldest cofacet of sigma.
 *   - Distances from points: s = 0; s = s + (x_k - y_k) * (x_k - y_k) for
 *     k = 0..dim-1 in float32 round-to-nearest with no fused multiply-add, then
 *     a correctly rounded float32 square root. The paper takes the distance
 *     matrix as its input; this is the reading this project fixes for points.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (see build.py).
 * OpenMP only parallelises independent per-column scans whose results are
 * combined in a fixed order, so results never depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAXV 8 /* vertices per simplex in the output records */

enum { MODE_HOM = 0, MODE_COHOM = 1, MODE_COHOM_CLEAR = 2 };

/* ------------------------------------------------------------------------ */
/* distances                                                                 */

/* Distance matrix from points (row-major n x dim) into D (row-major n x n). */
int oracle_distance_matrix(const float *X, int64_t n, int32_t dim, float *D) {
    if (n < 0 || dim < 1) return 1;
    for (int64_t i = 0; i < n; ++i) {
        D[i * n + i] = 0.0f;
        for (int64_t j = i + 1; j < n; ++j) {
            float s = 0.0f;
            for (int32_t k = 0; k < dim; ++k) {
                float d = X[i * dim + k] - X[j * dim + k];
                float sq = d * d;
                s = s + sq;
            }
            float r = sqrtf(s);
            D[i * n + j] = r;
            D[j * n + i] = r;
        }
    }
    return 0;
}

/* Enclosing radius min_x max_y d(x, y) (Sec. "Filtering Out Simplices by
 * Diameter Equal to the Enclosing Radius"). */
float oracle_enclosing_radius(const float *D, int64_t n) {
    float best = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        float m = 0.0f;
        for (int64_t j = 0; j < n; ++j)
            if (D[i * n + j] > m) m = D[i * n + j];
        if (m < best) best = m;
    }
    return n > 0 ? best : 0.0f;
}

static int cmp_float(const void *a, const void *b) {
    float x = *(const float *)a, y = *(const float *)b;
    return (x > y) - (x < y);
}

/* Nearest-rank q-quantile of the C(n,2) distances above the diagonal:
 * the ceil(q*m)-th smallest (1-based), clamped to [1, m]. */
float oracle_distance_quantile(const float *D, int64_t n, double q) {
    int64_t m = n * (n - 1) / 2;
    if (m <= 0) return 0.0f;
    float *v = (float *)malloc((size_t)m * sizeof(float));
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) v[c++] = D[i * n + j];
    qsort(v, (size_t)m, sizeof(float), cmp_float);
    int64_t r = (int64_t)ceil(q * (double)m);
    if (r < 1) r = 1;
    if (r > m) r = m;
    float out = v[r - 1];
    free(v);
    return out;
}

/* ------------------------------------------------------------------------ */
/* simplices as packed vertex tuples                                          */

typedef struct {
    int64_t n;
    int bits;             /* bits per vertex in a packed key */
    const float *D;
} space;

/* Pack vertices given in decreasing order (v[0] > v[1] > ... > v[k-1]). */
static uint64_t pack(const space *S, const int32_t *v, int k) {
    uint64_t key = 0;
    for (int i = 0; i < k; ++i) key = (key << S->bits) | (uint64_t)v[i];
    return key;
}

static void unpack(const space *S, uint64_t key, int k, int32_t *v) {
    uint64_t mask = (S->bits >= 64) ? ~0ull : ((1ull << S->bits) - 1ull);
    for (int i = k - 1; i >= 0; --i) {
        v[i] = (int32_t)(key & mask);
        key >>= S->bits;
    }
}

static float diam_of(const space *S, const int32_t *v, int k) {
    float m = 0.0f;
    for (int a = 0; a < k; ++a)
        for (int b = a + 1; b < k; ++b) {
            float d = S->D[(int64_t)v[a] * S->n + v[b]];
            if (d > m) m = d;
        }
    return m;
}

/* Insert vertex w (not in v) into the decreasing tuple v of length k. */
static void insert_vertex(const int32_t *v, int k, int32_t w, int32_t *out) {
    int o = 0, placed = 0;
    for (int i = 0; i < k; ++i) {
        if (!placed && w > v[i]) { out[o++] = w; placed = 1; }
        out[o++] = v[i];
    }
    if (!placed) out[o++] = w;
}

/* Remove position r from the decreasing tuple v of length k. */
static void remove_vertex(const int32_t *v, int k, int r, int32_t *out) {
    int o = 0;
    for (int i = 0; i < k; ++i)
        if (i != r) out[o++] = v[i];
}

static int in_tuple(const int32_t *v, int k, int32_t w) {
    for (int i = 0; i < k; ++i)
        if (v[i] == w) return 1;
    return 0;
}

typedef struct {
    float diam;
    uint64_t key;
} ent; /* one simplex of a fixed dimension */

/* Filtration order within one dimension: older first = smaller diameter, then
 * larger combinatorial index (= larger packed key). Returns <0 if a is older. */
static int older(const ent *a, const ent *b) {
    if (a->diam < b->diam) return -1;
    if (a->diam > b->diam) return 1;
    if (a->key > b->key) return -1;
    if (a->key < b->key) return 1;
    return 0;
}

/* Coboundary (reverse filtration) order: younger first. */
static int cmp_younger_first(const void *pa, const void *pb) {
    return -older((const ent *)pa, (const ent *)pb);
}

/* Enumerate all k-subsets of {0..n-1} with diam <= t, in any order. */
static ent *all_simplices(const space *S, int k, float t, int64_t *count) {
    int64_t cap = 1024, c = 0;
    ent *out = (ent *)malloc((size_t)cap * sizeof(ent));
    int32_t idx[ORACLE_MAXV + 2], v[ORACLE_MAXV + 2];
    if (k > S->n) { *count = 0; return out; }
    for (int i = 0; i < k; ++i) idx[i] = i; /* increasing combination */
    for (;;) {
        for (int i = 0; i < k; ++i) v[i] = idx[k - 1 - i];
        float d = diam_of(S, v, k);
        if (d <= t) {
            if (c == cap) { cap *= 2; out = (ent *)realloc(out, (size_t)cap * sizeof(ent)); }
            out[c].diam = d;
            out[c].key = pack(S, v, k);
            ++c;
        }
        int i = k - 1;
        while (i >= 0 && idx[i] == S->n - k + i) --i;
        if (i < 0) break;
        ++idx[i];
        for (int j = i + 1; j < k; ++j) idx[j] = idx[j - 1] + 1;
    }
    *count = c;
    return out;
}

/* ------------------------------------------------------------------------ */
/* hash map from packed key to int64 (open addressing)                        */

typedef struct {
    uint64_t *keys;
    int64_t *vals;
    int64_t cap, size;
} kmap;

#define EMPTY_KEY (~0ull)

static uint64_t hmix(uint64_t z) {
    z = (z ^ (z >> 33)) * 0xff51afd7ed558ccdull;
    z = (z ^ (z >> 33)) * 0xc4ceb9fe1a85ec53ull;
    return z ^ (z >> 33);
}

static void kmap_init(kmap *m, int64_t cap) {
    int64_t c = 16;
    while (c < 2 * cap) c <<= 1;
    m->cap = c;
    m->size = 0;
    m->keys = (uint64_t *)malloc((size_t)c * sizeof(uint64_t));
    m->vals = (int64_t *)malloc((size_t)c * sizeof(int64_t));
    for (int64_t i = 0; i < c; ++i) m->keys[i] = EMPTY_KEY;
}

static void kmap_free(kmap *m) {
    free(m->keys);
    free(m->vals);
}

static void kmap_put(kmap *m, uint64_t key, int64_t val);

static void kmap_grow(kmap *m) {
    kmap bigger;
    kmap_init(&bigger, m->cap);
    for (int64_t i = 0; i < m->cap; ++i)
        if (m->keys[i] != EMPTY_KEY) kmap_put(&bigger, m->keys[i], m->vals[i]);
    kmap_free(m);
    *m = bigger;
}

static void kmap_put(kmap *m, uint64_t key, int64_t val) {
    if (2 * (m->size + 1) > m->cap) kmap_grow(m);
    uint64_t h = hmix(key) & (uint64_t)(m->cap - 1);
    while (m->keys[h] != EMPTY_KEY && m->keys[h] != key) h = (h + 1) & (uint64_t)(m->cap - 1);
    if (m->keys[h] == EMPTY_KEY) { m->keys[h] = key; ++m->size; }
    m->vals[h] = val;
}

static int kmap_get(const kmap *m, uint64_t key, int64_t *val) {
    uint64_t h = hmix(key) & (uint64_t)(m->cap - 1);
    while (m->keys[h] != EMPTY_KEY) {
        if (m->keys[h] == key) { if (val) *val = m->vals[h]; return 1; }
        h = (h + 1) & (uint64_t)(m->cap - 1);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* result records                                                             */

typedef struct {
    int32_t dim;       /* homology dimension of the pair */
    float birth, death; /* death = +INFINITY for an essential class */
    int32_t bv[ORACLE_MAXV]; /* birth simplex vertices, decreasing, -1 padded */
    int32_t dv[ORACLE_MAXV]; /* death simplex vertices, -1 padded (all -1 if essential) */
} oracle_pair;

typedef struct {
    oracle_pair *pairs;
    int64_t count, cap;
    int64_t additions; /* column additions performed (work counter) */
} oracle_result;

static void add_pair(const space *S, oracle_result *R, int dim, const ent *b, const ent *d) {
    if (R->count == R->cap) {
        R->cap = R->cap ? 2 * R->cap : 1024;
        R->pairs = (oracle_pair *)realloc(R->pairs, (size_t)R->cap * sizeof(oracle_pair));
    }
    oracle_pair *P = &R->pairs[R->count++];
    P->dim = dim;
    for (int i = 0; i < ORACLE_MAXV; ++i) P->bv[i] = P->dv[i] = -1;
    P->birth = b->diam;
    unpack(S, b->key, dim + 1, P->bv);
    if (d) {
        P->death = d->diam;
        unpack(S, d->key, dim + 2, P->dv);
    } else {
        P->death = INFINITY;
    }
}

/* ------------------------------------------------------------------------ */
/* HOM: Alg. 1 on the explicit boundary matrix of the whole filtration        */

typedef struct {
    ent e;
    int dim;
} sx;

static int cmp_filtration(const void *pa, const void *pb) {
    const sx *a = (const sx *)pa, *b = (const sx *)pb;
    if (a->e.diam != b->e.diam) return a->e.diam < b->e.diam ? -1 : 1;
    if (a->dim != b->dim) return a->dim < b->dim ? -1 : 1;
    if (a->e.key != b->e.key) return a->e.key > b->e.key ? -1 : 1;
    return 0;
}

typedef struct {
    int64_t *v;
    int64_t len, cap;
} ivec;

static void ivec_push(ivec *c, int64_t x) {
    if (c->len == c->cap) {
        c->cap = c->cap ? 2 * c->cap : 8;
        c->v = (int64_t *)realloc(c->v, (size_t)c->cap * sizeof(int64_t));
    }
    c->v[c->len++] = x;
}

static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* c <- c + o over Z/2; both sorted ascending. */
static void ivec_symdiff(ivec *c, const ivec *o) {
    int64_t *out = (int64_t *)malloc((size_t)(c->len + o->len + 1) * sizeof(int64_t));
    int64_t i = 0, j = 0, k = 0;
    while (i < c->len && j < o->len) {
        if (c->v[i] < o->v[j]) out[k++] = c->v[i++];
        else if (c->v[i] > o->v[j]) out[k++] = o->v[j++];
        else { ++i; ++j; }
    }
    while (i < c->len) out[k++] = c->v[i++];
    while (j < o->len) out[k++] = o->v[j++];
    free(c->v);
    c->v = out;
    c->len = k;
    c->cap = c->len + o->len + 1;
}

static void run_hom(const space *S, int max_dim, float t, oracle_result *R) {
    int top = max_dim + 1;
    int64_t total = 0, counts[ORACLE_MAXV];
    ent *per[ORACLE_MAXV];
    for (int q = 0; q <= top; ++q) {
        per[q] = all_simplices(S, q + 1, t, &counts[q]);
        total += counts[q];
    }
    sx *all = (sx *)malloc((size_t)(total > 0 ? total : 1) * sizeof(sx));
    int64_t c = 0;
    for (int q = 0; q <= top; ++q)
        for (int64_t i = 0; i < counts[q]; ++i) { all[c].e = per[q][i]; all[c].dim = q; ++c; }
    qsort(all, (size_t)total, sizeof(sx), cmp_filtration);
    /* per-dim position lookup by key */
    kmap pos[ORACLE_MAXV];
    for (int q = 0; q <= top; ++q) kmap_init(&pos[q], counts[q] + 1);
    for (int64_t i = 0; i < total; ++i) kmap_put(&pos[all[i].dim], all[i].e.key, i);
    ivec *col = (ivec *)calloc((size_t)(total > 0 ? total : 1), sizeof(ivec));
    int64_t *owner = (int64_t *)malloc((size_t)(total > 0 ? total : 1) * sizeof(int64_t));
    char *is_low = (char *)calloc((size_t)(total > 0 ? total : 1), 1);
    for (int64_t i = 0; i < total; ++i) owner[i] = -1;
    int32_t v[ORACLE_MAXV + 2], f[ORACLE_MAXV + 2];
    for (int64_t j = 0; j < total; ++j) {
        int q = all[j].dim;
        if (q == 0) continue;
        unpack(S, all[j].e.key, q + 1, v);
        for (int r = 0; r <= q; ++r) {
            remove_vertex(v, q + 1, r, f);
            int64_t p;
            kmap_get(&pos[q - 1], pack(S, f, q), &p);
            ivec_push(&col[j], p);
        }
        qsort(col[j].v, (size_t)col[j].len, sizeof(int64_t), cmp_i64);
        while (col[j].len > 0) {
            int64_t low = col[j].v[col[j].len - 1];
            if (owner[low] < 0) break;
            ivec_symdiff(&col[j], &col[owner[low]]);
            ++R->additions;
        }
        if (col[j].len > 0) {
            int64_t low = col[j].v[col[j].len - 1];
            owner[low] = j;
            is_low[low] = 1;
            is_low[j] = 2; /* j is a death */
            add_pair(S, R, q - 1, &all[low].e, &all[j].e);
        }
    }
    for (int64_t j = 0; j < total; ++j)
        if (is_low[j] == 0 && col[j].len == 0 && all[j].dim <= max_dim)
            add_pair(S, R, all[j].dim, &all[j].e, NULL);
    for (int64_t j = 0; j < total; ++j) free(col[j].v);
    free(col); free(owner); free(is_low); free(all);
    for (int q = 0; q <= top; ++q) { free(per[q]); kmap_free(&pos[q]); }
}

/* ------------------------------------------------------------------------ */
/* COHOM / COHOM_CLEAR: Alg. 1 on the coboundary matrix, one dimension at a time */

typedef struct {
    ent *v;
    int64_t len;
} ecol; /* a coboundary column: entries sorted younger-first, low = last */

/* Coboundary of a dim-q simplex: its cofacets with diam <= t, younger first. */
static ecol coboundary(const space *S, const ent *s, int q, float t) {
    int32_t v[ORACLE_MAXV + 2], w[ORACLE_MAXV + 2];
    unpack(S, s->key, q + 1, v);
    ecol c;
    c.v = (ent *)malloc((size_t)(S->n + 1) * sizeof(ent));
    c.len = 0;
    for (int32_t x = 0; x < S->n; ++x) {
        if (in_tuple(v, q + 1, x)) continue;
        float d = s->diam;
        for (int i = 0; i <= q; ++i) {
            float e = S->D[(int64_t)v[i] * S->n + x];
            if (e > d) d = e;
        }
        if (d > t) continue;
        insert_vertex(v, q + 1, x, w);
        c.v[c.len].diam = d;
        c.v[c.len].key = pack(S, w, q + 2);
        ++c.len;
    }
    qsort(c.v, (size_t)c.len, sizeof(ent), cmp_younger_first);
    return c;
}

/* The low (oldest cofacet) of the unreduced coboundary, without storing it. */
static int coboundary_low(const space *S, const ent *s, int q, float t, ent *low) {
    int32_t v[ORACLE_MAXV + 2], w[ORACLE_MAXV + 2];
    unpack(S, s->key, q + 1, v);
    int found = 0;
    for (int32_t x = 0; x < S->n; ++x) {
        if (in_tuple(v, q + 1, x)) continue;
        float d = s->diam;
        for (int i = 0; i <= q; ++i) {
            float e = S->D[(int64_t)v[i] * S->n + x];
            if (e > d) d = e;
        }
        if (d > t) continue;
        if (found && d > low->diam) continue; /* cannot be older than the current low */
        insert_vertex(v, q + 1, x, w);
        ent e;
        e.diam = d;
        e.key = pack(S, w, q + 2);
        if (!found || older(&e, low) < 0) { *low = e; found = 1; }
    }
    return found;
}

/* The working column of a reduction: a binary heap holding the entries of a
 * Z/2 sum with repetitions, oldest entry on top. An entry present an even
 * number of times is zero; cancellation happens when the low is read. */
typedef struct {
    ent *v;
    int64_t len, cap;
} eheap;

static void heap_push(eheap *h, ent e) {
    if (h->len == h->cap) {
        h->cap = h->cap ? 2 * h->cap : 1024;
        h->v = (ent *)realloc(h->v, (size_t)h->cap * sizeof(ent));
    }
    int64_t i = h->len++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (older(&e, &h->v[p]) >= 0) break;
        h->v[i] = h->v[p];
        i = p;
    }
    h->v[i] = e;
}

static ent heap_pop(eheap *h) {
    ent top = h->v[0];
    ent last = h->v[--h->len];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= h->len) break;
        if (c + 1 < h->len && older(&h->v[c + 1], &h->v[c]) < 0) ++c;
        if (older(&h->v[c], &last) >= 0) break;
        h->v[i] = h->v[c];
        i = c;
    }
    if (h->len > 0) h->v[i] = last;
    return top;
}

/* The low (oldest nonzero entry) of the sum; 0 if the sum is zero. The low
 * stays in the heap. */
static int heap_low(eheap *h, ent *low) {
    while (h->len > 0) {
        ent e = heap_pop(h);
        if (h->len > 0 && h->v[0].key == e.key) { heap_pop(h); continue; }
        heap_push(h, e);
        *low = e;
        return 1;
    }
    return 0;
}

static void heap_add(eheap *h, const ecol *c) {
    for (int64_t i = 0; i < c->len; ++i) heap_push(h, c->v[i]);
}

/* Drain the heap into a column holding each surviving entry once. */
static ecol heap_drain(eheap *h) {
    ecol c;
    c.v = (ent *)malloc((size_t)(h->len > 0 ? h->len : 1) * sizeof(ent));
    c.len = 0;
    ent e;
    while (heap_low(h, &e)) {
        heap_pop(h);
        c.v[c.len++] = e;
    }
    /* drained oldest-first; store younger-first like a coboundary */
    for (int64_t i = 0, j = c.len - 1; i < j; ++i, --j) {
        ent x = c.v[i];
        c.v[i] = c.v[j];
        c.v[j] = x;
    }
    return c;
}

/* Kruskal on the edges with diam <= t in filtration order; merging edges are
 * the H0 deaths. The dying vertex is the younger of the two components' oldest
 * vertices (older vertex = larger index, since all vertices have diameter 0). */
static void run_kruskal(const space *S, float t, oracle_result *R, kmap *deaths) {
    int64_t m;
    ent *E = all_simplices(S, 2, t, &m);
    qsort(E, (size_t)m, sizeof(ent), cmp_younger_first); /* reverse filtration */
    int64_t n = S->n;
    int64_t *parent = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *oldest = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) { parent[i] = i; oldest[i] = i; }
    int32_t v[2];
    for (int64_t k = m - 1; k >= 0; --k) { /* filtration order */
        unpack(S, E[k].key, 2, v);
        int64_t a = v[0], b = v[1];
        while (parent[a] != a) a = parent[a] = parent[parent[a]];
        while (parent[b] != b) b = parent[b] = parent[parent[b]];
        if (a == b) continue;
        int64_t oa = oldest[a], ob = oldest[b];
        int64_t young = oa < ob ? oa : ob, old = oa < ob ? ob : oa;
        ent vx;
        vx.diam = 0.0f;
        int32_t yv = (int32_t)young;
        vx.key = pack(S, &yv, 1);
        add_pair(S, R, 0, &vx, &E[k]);
        if (deaths) kmap_put(deaths, E[k].key, 1);
        parent[a] = b;
        oldest[b] = old;
    }
    for (int64_t i = 0; i < n; ++i)
        if (parent[i] == i) {
            ent vx;
            vx.diam = 0.0f;
            int32_t yv = (int32_t)oldest[i];
            vx.key = pack(S, &yv, 1);
            add_pair(S, R, 0, &vx, NULL);
        }
    free(parent); free(oldest); free(E);
}

static void run_cohom(const space *S, int max_dim, float t, int clearing, oracle_result *R) {
    kmap prev_deaths; /* dim-q simplices that are deaths of dim q-1 pairs */
    kmap_init(&prev_deaths, 16);
    int q0 = 0;
    if (clearing) {
        run_kruskal(S, t, R, &prev_deaths);
        q0 = 1;
    }
    for (int q = q0; q <= max_dim; ++q) {
        int64_t m;
        ent *cols = all_simplices(S, q + 1, t, &m);
        qsort(cols, (size_t)m, sizeof(ent), cmp_younger_first);
        char *skip = (char *)calloc((size_t)(m > 0 ? m : 1), 1);
        for (int64_t j = 0; j < m; ++j)
            if (kmap_get(&prev_deaths, cols[j].key, NULL)) skip[j] = clearing ? 1 : 2;
        /* independent per-column scans: the low of each unreduced column */
        ent *low0 = (ent *)malloc((size_t)(m > 0 ? m : 1) * sizeof(ent));
        char *has0 = (char *)calloc((size_t)(m > 0 ? m : 1), 1);
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t j = 0; j < m; ++j)
            if (skip[j] != 1) has0[j] = (char)coboundary_low(S, &cols[j], q, t, &low0[j]);
        kmap owner, deaths;
        kmap_init(&owner, 1024);
        kmap_init(&deaths, 1024);
        ecol *stored = (ecol *)calloc((size_t)(m > 0 ? m : 1), sizeof(ecol));
        for (int64_t j = 0; j < m; ++j) {
            if (skip[j] == 1) continue; /* cleared: this column reduces to zero */
            int64_t k;
            if (!has0[j] || !kmap_get(&owner, low0[j].key, &k)) {
                if (has0[j]) { /* no addition needed: the low is free */
                    kmap_put(&owner, low0[j].key, j);
                    kmap_put(&deaths, low0[j].key, 1);
                    add_pair(S, R, q, &cols[j], &low0[j]);
                } else if (skip[j] == 0) {
                    add_pair(S, R, q, &cols[j], NULL); /* empty column, not a death */
                }
                continue;
            }
            eheap h = {0};
            ecol c = coboundary(S, &cols[j], q, t);
            heap_add(&h, &c);
            free(c.v);
            ent low;
            int nonzero;
            while ((nonzero = heap_low(&h, &low)) && kmap_get(&owner, low.key, &k)) {
                if (stored[k].v) {
                    heap_add(&h, &stored[k]);
                } else {
                    ecol o = coboundary(S, &cols[k], q, t);
                    heap_add(&h, &o);
                    free(o.v);
                }
                ++R->additions;
            }
            if (nonzero) {
                kmap_put(&owner, low.key, j);
                kmap_put(&deaths, low.key, 1);
                add_pair(S, R, q, &cols[j], &low);
                stored[j] = heap_drain(&h); /* keep the reduced column: it was modified */
            } else if (skip[j] == 0) {
                add_pair(S, R, q, &cols[j], NULL);
            }
            free(h.v);
        }
        for (int64_t j = 0; j < m; ++j) free(stored[j].v);
        free(stored); free(low0); free(has0); free(skip); free(cols);
        kmap_free(&owner);
        kmap_free(&prev_deaths);
        prev_deaths = deaths;
    }
    kmap_free(&prev_deaths);
}

static int setup_space(space *S, const float *D, int64_t n, int kmax) {
    S->n = n;
    S->D = D;
    int b = 1;
    while ((1ll << b) <= n) ++b;
    if (kmax < 1) kmax = 1;
    if (b * kmax > 64) return 1;
    S->bits = 64 / kmax;
    if (S->bits > 32) S->bits = 32;
    if (S->bits < b) return 1;
    return 0;
}

/* Barcodes of dims 0..max_dim of Rips_t (all pairs, zero-length ones included).
 * Returns a result handle (free with oracle_result_free) or NULL on bad input. */
oracle_result *oracle_barcodes(const float *D, int64_t n, int32_t max_dim, float t, int32_t mode) {
    if (n < 1 || max_dim < 0 || max_dim + 2 > ORACLE_MAXV || !(t >= 0.0f)) return NULL;
    space S;
    if (setup_space(&S, D, n, max_dim + 2)) return NULL;
    oracle_result *R = (oracle_result *)calloc(1, sizeof(oracle_result));
    if (mode == MODE_HOM) run_hom(&S, max_dim, t, R);
    else if (mode == MODE_COHOM) run_cohom(&S, max_dim, t, 0, R);
    else if (mode == MODE_COHOM_CLEAR) run_cohom(&S, max_dim, t, 1, R);
    else { free(R); return NULL; }
    return R;
}

/* H0 alone by Kruskal (used as an independent pin of the reductions). */
oracle_result *oracle_kruskal(const float *D, int64_t n, float t) {
    space S;
    if (n < 1 || setup_space(&S, D, n, 2)) return NULL;
    oracle_result *R = (oracle_result *)calloc(1, sizeof(oracle_result));
    run_kruskal(&S, t, R, NULL);
    return R;
}

int64_t oracle_result_count(const oracle_result *R) { return R ? R->count : -1; }
const oracle_pair *oracle_result_pairs(const oracle_result *R) { return R ? R->pairs : NULL; }
int64_t oracle_result_additions(const oracle_result *R) { return R ? R->additions : -1; }
void oracle_result_free(oracle_result *R) {
    if (!R) return;
    free(R->pairs);
    free(R);
}

/* ------------------------------------------------------------------------ */
/* columns and apparent pairs                                                 */

/* All dim-p simplices with diam <= t in coboundary order (decreasing diameter,
 * then increasing combinatorial index). verts: count x (p+1), decreasing. */
int64_t oracle_columns(const float *D, int64_t n, int32_t p, float t,
                       float *diam, int32_t *verts, int64_t cap) {
    space S;
    if (n < 1 || p < 0 || p + 1 > ORACLE_MAXV || setup_space(&S, D, n, p + 1)) return -1;
    int64_t m;
    ent *c = all_simplices(&S, p + 1, t, &m);
    qsort(c, (size_t)m, sizeof(ent), cmp_younger_first);
    if (diam && verts && m <= cap)
        for (int64_t i = 0; i < m; ++i) {
            diam[i] = c[i].diam;
            unpack(&S, c[i].key, p + 1, verts + i * (p + 1));
        }
    free(c);
    return m;
}

/* Test one dim-p simplex sigma (vertices decreasing) against the definition of
 * an apparent pair. Returns 1 and fills tau (p+2 vertices, decreasing) if
 * apparent, 0 if not, -1 on bad input. */
int oracle_apparent_one(const float *D, int64_t n, int32_t p, float t,
                        const int32_t *sigma, int32_t *tau) {
    space S;
    if (p < 0 || p + 2 > ORACLE_MAXV || setup_space(&S, D, n, p + 2)) return -1;
    ent s;
    s.diam = diam_of(&S, sigma, p + 1);
    s.key = pack(&S, sigma, p + 1);
    if (s.diam > t) return 0;
    ent oldest;
    if (!coboundary_low(&S, &s, p, t, &oldest)) return 0; /* no cofacet */
    int32_t w[ORACLE_MAXV + 2], f[ORACLE_MAXV + 2];
    unpack(&S, oldest.key, p + 2, w);
    /* youngest facet of tau: larger diameter, then smaller index */
    ent young;
    int have = 0;
    for (int r = 0; r < p + 2; ++r) {
        remove_vertex(w, p + 2, r, f);
        ent e;
        e.diam = diam_of(&S, f, p + 1);
        e.key = pack(&S, f, p + 1);
        if (!have || older(&e, &young) > 0) { young = e; have = 1; }
    }
    if (young.key != s.key) return 0;
    if (tau) memcpy(tau, w, (size_t)(p + 2) * sizeof(int32_t));
    return 1;
}

/* Every apparent pair (sigma, tau) with sigma of dim p and diam <= t, sigma in
 * coboundary order. Returns the count; fills up to cap records. */
int64_t oracle_apparent_pairs(const float *D, int64_t n, int32_t p, float t,
                              int32_t *sigma_out, int32_t *tau_out, int64_t cap) {
    space S;
    if (n < 1 || p < 0 || p + 2 > ORACLE_MAXV || setup_space(&S, D, n, p + 2)) return -1;
    int64_t m;
    ent *c = all_simplices(&S, p + 1, t, &m);
    qsort(c, (size_t)m, sizeof(ent), cmp_younger_first);
    char *ok = (char *)calloc((size_t)(m > 0 ? m : 1), 1);
    int32_t *taus = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * (size_t)(p + 2) * sizeof(int32_t));
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < m; ++i) {
        int32_t v[ORACLE_MAXV + 2];
        unpack(&S, c[i].key, p + 1, v);
        ok[i] = (char)(oracle_apparent_one(D, n, p, t, v, taus + i * (p + 2)) == 1);
    }
    int64_t k = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (!ok[i]) continue;
        if (k < cap && sigma_out && tau_out) {
            unpack(&S, c[i].key, p + 1, sigma_out + k * (p + 1));
            memcpy(tau_out + k * (p + 2), taus + i * (p + 2), (size_t)(p + 2) * sizeof(int32_t));
        }
        ++k;
    }
    free(ok); free(taus); free(c);
    return k;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
