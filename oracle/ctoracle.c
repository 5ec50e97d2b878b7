/*
 * ctoracle.c -- CPU oracle for the exact ε-graph (test infrastructure only).
 *
 * This file is test infrastructure.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may call it.  It shares no code with the
 * CUDA library and is deliberately plain: FP64, sequential loops, no blocking.
 * Compile with -ffp-contract=off (no FMA contraction) so every floating-point
 * operation below is one IEEE round-to-nearest operation in program order.
 *
 * Contents (paper sections in brackets):
 *   - the L2 predicate (definition of the ε-graph, Sec. III) pinned as
 *     s = sum_k (x_k - y_k)^2 in FP64, ascending k, edge iff s <= fl(eps*eps);
 *   - Levenshtein distance (edit distance, named in Sec. I and Sec. III) by the
 *     Wagner-Fischer dynamic programme, and a banded cutoff variant (Ukkonen);
 *   - Hamming distance of bit strings (the binary datasets of Sec. V-A,
 *     Table I): the number of positions whose bits differ, bit by bit;
 *   - brute-force all-pairs ε-graph (the ground truth, Sec. III "ε-graph");
 *   - the plain cover tree: batch construction by vertex splitting
 *     (Algorithm 1, SplitVertex) applied level by level (Algorithm 2,
 *     BuildLevel), and the stack-based ε query (Algorithm 3);
 *   - an invariant checker for any tree in the flat export format
 *     (cover-tree invariants of Sec. III: nesting, covering, separation; the
 *     vertex-triple radius of Sec. IV-A as an upper bound on descendants).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_L2 0
#define ORC_LEV 1
#define ORC_HAM 2

typedef struct {
    int32_t metric;        /* ORC_L2, ORC_LEV or ORC_HAM */
    int64_t n;
    int32_t dim;           /* L2: coordinates per point; Hamming: bits per row */
    const float *X;        /* L2: n*dim row-major */
    const uint8_t *S;      /* Lev: concatenated strings; Hamming: n rows of ceil(dim/8) bytes,
                              bit j of a row = bit (j mod 8) of its byte j/8 */
    const int64_t *off;    /* Lev: n+1 offsets */
} orc_space;

/* ------------------------------------------------------------------ metrics */

/* Squared L2 distance, the pinned predicate's sum: inputs converted exactly
 * fp32 -> fp64, t = x - y, s = s + t*t for k = 0..dim-1 in order. */
double orc_sq_l2(const float *x, const float *y, int32_t dim)
{
    double s = 0.0;
    for (int32_t k = 0; k < dim; ++k) {
        double t = (double)x[k] - (double)y[k];
        double t2 = t * t;
        s = s + t2;
    }
    return s;
}

/* Wagner-Fischer edit distance, unit costs for insertion, deletion and
 * substitution; this is the definition of Levenshtein distance. */
int32_t orc_lev_full(const uint8_t *a, int32_t la, const uint8_t *b, int32_t lb)
{
    int32_t *prev = (int32_t *)malloc(sizeof(int32_t) * (size_t)(lb + 1));
    int32_t *cur = (int32_t *)malloc(sizeof(int32_t) * (size_t)(lb + 1));
    for (int32_t j = 0; j <= lb; ++j) prev[j] = j;
    for (int32_t i = 1; i <= la; ++i) {
        cur[0] = i;
        for (int32_t j = 1; j <= lb; ++j) {
            int32_t sub = prev[j - 1] + (a[i - 1] != b[j - 1]);
            int32_t del = prev[j] + 1;
            int32_t ins = cur[j - 1] + 1;
            int32_t v = sub < del ? sub : del;
            cur[j] = v < ins ? v : ins;
        }
        int32_t *t = prev; prev = cur; cur = t;
    }
    int32_t r = prev[lb];
    free(prev); free(cur);
    return r;
}

/* Banded edit distance with cutoff k (Ukkonen 1985): only cells with
 * |i - j| <= k are computed; the result equals the edit distance when it is
 * <= k and is k + 1 otherwise. */
int32_t orc_lev_banded(const uint8_t *a, int32_t la, const uint8_t *b, int32_t lb,
                       int32_t k)
{
    if (k < 0) return 0 == la && 0 == lb ? 0 : k + 1;
    int32_t dl = la > lb ? la - lb : lb - la;
    const int32_t INF = k + 1;
    if (dl > k) return INF;
    int32_t *prev = (int32_t *)malloc(sizeof(int32_t) * (size_t)(lb + 2));
    int32_t *cur = (int32_t *)malloc(sizeof(int32_t) * (size_t)(lb + 2));
    for (int32_t j = 0; j <= lb + 1; ++j) prev[j] = (j <= k && j <= lb) ? j : INF;
    for (int32_t j = 0; j <= lb + 1; ++j) cur[j] = INF;
    for (int32_t i = 1; i <= la; ++i) {
        int32_t jlo = i - k > 1 ? i - k : 1;
        int32_t jhi = i + k < lb ? i + k : lb;
        int32_t rowmin;
        if (jlo - 1 == 0) cur[0] = i <= k ? i : INF;
        else cur[jlo - 1] = INF;
        rowmin = cur[jlo - 1];
        for (int32_t j = jlo; j <= jhi; ++j) {
            int32_t sub = prev[j - 1] + (a[i - 1] != b[j - 1]);
            int32_t del = prev[j] + 1;
            int32_t ins = cur[j - 1] + 1;
            int32_t v = sub < del ? sub : del;
            v = v < ins ? v : ins;
            if (v > INF) v = INF;
            cur[j] = v;
            if (v < rowmin) rowmin = v;
        }
        if (jhi + 1 <= lb) cur[jhi + 1] = INF;
        if (rowmin > k) { free(prev); free(cur); return INF; }
        int32_t *t = prev; prev = cur; cur = t;
    }
    int32_t r = prev[lb] < INF ? prev[lb] : INF;
    free(prev); free(cur);
    return r;
}

/* Hamming distance of two rows of `dim` bits: the number of positions j <
 * dim whose bits differ, counted one bit at a time (the definition). */
int32_t orc_hamming(const uint8_t *a, const uint8_t *b, int32_t dim)
{
    int32_t d = 0;
    for (int32_t j = 0; j < dim; ++j) {
        int32_t x = (a[j >> 3] >> (j & 7)) & 1;
        int32_t y = (b[j >> 3] >> (j & 7)) & 1;
        d += x != y;
    }
    return d;
}

static inline const uint8_t *bits_at(const orc_space *sp, int64_t i)
{
    return sp->S + (size_t)i * (size_t)((sp->dim + 7) / 8);
}

static inline const uint8_t *str_at(const orc_space *sp, int64_t i, int32_t *len)
{
    *len = (int32_t)(sp->off[i + 1] - sp->off[i]);
    return sp->S + sp->off[i];
}

/* Metric value as a double: sqrt of the pinned sum for L2, the exact integer
 * for Levenshtein and Hamming. */
static double metric_dist(const orc_space *sp, int64_t i, int64_t j)
{
    if (sp->metric == ORC_L2)
        return sqrt(orc_sq_l2(sp->X + (size_t)i * sp->dim, sp->X + (size_t)j * sp->dim, sp->dim));
    if (sp->metric == ORC_HAM)
        return (double)orc_hamming(bits_at(sp, i), bits_at(sp, j), sp->dim);
    int32_t la, lb;
    const uint8_t *a = str_at(sp, i, &la), *b = str_at(sp, j, &lb);
    return (double)orc_lev_full(a, la, b, lb);
}

/* Edge predicate d(i,j) <= eps, with its distance.  L2 compares the pinned sum
 * against fl(eps*eps); Levenshtein uses the banded cutoff at floor(eps);
 * Hamming compares the integer distance with floor(eps). */
static int edge_pred(const orc_space *sp, int64_t i, int64_t j, double eps, double eps2,
                     double *dist)
{
    if (sp->metric == ORC_L2) {
        double s = orc_sq_l2(sp->X + (size_t)i * sp->dim, sp->X + (size_t)j * sp->dim, sp->dim);
        *dist = sqrt(s);
        return s <= eps2;
    }
    if (sp->metric == ORC_HAM) {
        int32_t v = orc_hamming(bits_at(sp, i), bits_at(sp, j), sp->dim);
        *dist = (double)v;
        return (double)v <= floor(eps);
    }
    int32_t la, lb;
    const uint8_t *a = str_at(sp, i, &la), *b = str_at(sp, j, &lb);
    int32_t k = (int32_t)floor(eps);
    int32_t v = orc_lev_banded(a, la, b, lb, k);
    *dist = (double)v;
    return v <= k;
}

/* ------------------------------------------------------------ CSR assembly */

typedef struct { int64_t *col; double *dist; int64_t len, cap; } vec_t;

static void vec_push(vec_t *v, int64_t c, double d)
{
    if (v->len == v->cap) {
        v->cap = v->cap ? 2 * v->cap : 64;
        v->col = (int64_t *)realloc(v->col, sizeof(int64_t) * (size_t)v->cap);
        v->dist = (double *)realloc(v->dist, sizeof(double) * (size_t)v->cap);
    }
    v->col[v->len] = c;
    v->dist[v->len] = d;
    v->len++;
}

typedef struct {
    int64_t n_rows, nnz;
    int64_t *row_ptr;  /* n_rows + 1 */
    int64_t *col;
    double *dist;
    int64_t dist_evals; /* metric evaluations performed */
} orc_csr;

static int cmp_pair(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* Sort one row by column (pairs of (col, dist-bits)). */
static void sort_row(int64_t *col, double *dist, int64_t len)
{
    if (len < 2) return;
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)len);
    for (int64_t i = 0; i < len; ++i) {
        tmp[2 * i] = col[i];
        memcpy(&tmp[2 * i + 1], &dist[i], sizeof(double));
    }
    qsort(tmp, (size_t)len, 2 * sizeof(int64_t), cmp_pair);
    for (int64_t i = 0; i < len; ++i) {
        col[i] = tmp[2 * i];
        memcpy(&dist[i], &tmp[2 * i + 1], sizeof(double));
    }
    free(tmp);
}

/* Gather per-row vectors into a CSR with ascending columns in each row. */
static orc_csr *assemble(int64_t n, vec_t *rows)
{
    orc_csr *o = (orc_csr *)calloc(1, sizeof(orc_csr));
    o->n_rows = n;
    o->row_ptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    o->row_ptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) o->row_ptr[i + 1] = o->row_ptr[i] + rows[i].len;
    o->nnz = o->row_ptr[n];
    o->col = (int64_t *)malloc(sizeof(int64_t) * (size_t)(o->nnz ? o->nnz : 1));
    o->dist = (double *)malloc(sizeof(double) * (size_t)(o->nnz ? o->nnz : 1));
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        int64_t b = o->row_ptr[i];
        if (rows[i].len) {
            memcpy(o->col + b, rows[i].col, sizeof(int64_t) * (size_t)rows[i].len);
            memcpy(o->dist + b, rows[i].dist, sizeof(double) * (size_t)rows[i].len);
            sort_row(o->col + b, o->dist + b, rows[i].len);
        }
        free(rows[i].col);
        free(rows[i].dist);
    }
    free(rows);
    return o;
}

void orc_csr_free(orc_csr *o)
{
    if (!o) return;
    free(o->row_ptr); free(o->col); free(o->dist); free(o);
}

/* ------------------------------------------------------------- brute force */

/* Ground truth: every ordered pair (i, j), j != i unless include_self, with
 * d(p_i, p_j) <= eps (the ε-graph definition, closed ball). */
orc_csr *orc_brute_force(const orc_space *sp, double eps, int32_t include_self)
{
    int64_t n = sp->n;
    double eps2 = eps * eps;
    vec_t *rows = (vec_t *)calloc((size_t)(n ? n : 1), sizeof(vec_t));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            if (j == i && !include_self) continue;
            double d;
            if (edge_pred(sp, i, j, eps, eps2, &d)) vec_push(&rows[i], j, d);
        }
    }
    orc_csr *o = assemble(n, rows);
    o->dist_evals = n * n;
    return o;
}

/* Brute force restricted to the query rows `rows[0..k)` (ascending columns);
 * row r of the result is the neighbour list of point rows[r]. */
orc_csr *orc_brute_rows(const orc_space *sp, double eps, int32_t include_self, const int64_t *rows,
                        int64_t k)
{
    int64_t n = sp->n;
    double eps2 = eps * eps;
    vec_t *out = (vec_t *)calloc((size_t)(k ? k : 1), sizeof(vec_t));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < k; ++r) {
        int64_t i = rows[r];
        for (int64_t j = 0; j < n; ++j) {
            if (j == i && !include_self) continue;
            double d;
            if (edge_pred(sp, i, j, eps, eps2, &d)) vec_push(&out[r], j, d);
        }
    }
    orc_csr *o = assemble(k, out);
    o->dist_evals = k * n;
    return o;
}

/* --------------------------------------------------------- landmarks */

/* Voronoi cells of the centres (point indices centres[0..m)): cell[i] is the
 * index k of the nearest centre (the lowest k among equals) and dmin[i] its
 * distance -- step (1) of the landmark construction (Sec. IV-D). */
void orc_voronoi(const orc_space *sp, const int64_t *centres, int32_t m, int32_t *cell, double *dmin)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < sp->n; ++i) {
        int32_t best = 0;
        double bd = metric_dist(sp, i, centres[0]);
        for (int32_t k = 1; k < m; ++k) {
            double d = metric_dist(sp, i, centres[k]);
            if (d < bd) { bd = d; best = k; }
        }
        cell[i] = best;
        dmin[i] = bd;
    }
}

/* The ε-graph by landmarks (Sec. IV-D, Algorithms 5 and 6 on one processor):
 * Voronoi cells V_k of the centres; the ε-ghosts of V_k are the points p
 * outside it with d(p, c_k) <= d(p, C) + factor * eps (Lemma 1: factor 2
 * catches every p with a neighbour in V_k); each point's row is the brute
 * force over its own cell and that cell's ghosts.  factor < 2 is for tests
 * that show Lemma 1's bound is needed. */
orc_csr *orc_landmark_graph(const orc_space *sp, const int64_t *centres, int32_t m, double eps,
                            int32_t include_self, double factor)
{
    int64_t n = sp->n;
    double eps2 = eps * eps;
    int32_t *cell = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    double *dmin = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    if (n) orc_voronoi(sp, centres, m, cell, dmin);
    /* members of every cell: its own points and its ghosts */
    vec_t *mem = (vec_t *)calloc((size_t)m, sizeof(vec_t));
    for (int64_t p = 0; p < n; ++p) {
        for (int32_t k = 0; k < m; ++k) {
            if (k == cell[p]) { vec_push(&mem[k], p, 0.0); continue; }
            double d = metric_dist(sp, p, centres[k]);
            if (d <= dmin[p] + factor * eps) vec_push(&mem[k], p, 1.0);
        }
    }
    /* rows of each cell's own points, by brute force over the cell's members */
    vec_t *rows = (vec_t *)calloc((size_t)(n ? n : 1), sizeof(vec_t));
    int64_t evals = 0;
    for (int32_t k = 0; k < m; ++k) {
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : evals)
        for (int64_t a = 0; a < mem[k].len; ++a) {
            int64_t p = mem[k].col[a];
            if (mem[k].dist[a] != 0.0) continue;   /* a ghost: its row is made in its own cell */
            for (int64_t b = 0; b < mem[k].len; ++b) {
                int64_t q = mem[k].col[b];
                if (q == p && !include_self) continue;
                double d;
                evals++;
                if (edge_pred(sp, p, q, eps, eps2, &d)) vec_push(&rows[p], q, d);
            }
        }
        free(mem[k].col);
        free(mem[k].dist);
    }
    free(mem); free(cell); free(dmin);
    orc_csr *o = assemble(n, rows);
    o->dist_evals = evals;
    return o;
}

/* ------------------------------------------------------------- cover tree */

/* Flat tree export, shared format between this oracle and the GPU library's
 * export routine (the format is plain arrays; no code is shared):
 *   node 0 is the root; children of a node are contiguous node ids;
 *   a leaf block has child_count == 0 and lists its points in
 *   leaf_pts[pts_begin .. pts_begin + pts_count). */
typedef struct {
    int64_t n_nodes, n_points;
    int64_t *center;       /* point id of the vertex */
    double *radius;        /* vertex-triple radius (upper bound on descendants) */
    int32_t *level;        /* split level l (threshold 2^(l-1)); INT32_MIN for radius 0 */
    int64_t *child_begin, *child_count;
    int64_t *pts_begin, *pts_count;
    int64_t *leaf_pts;     /* n_points */
    int64_t dist_evals;
} orc_tree;

typedef struct {
    int64_t node;          /* tree node this hub will fill */
    int64_t *H;            /* point ids in scan order */
    double *D;             /* D[i] = d(H[i], centre) */
    int64_t m;             /* |H| */
    int32_t level;
} hub_t;

static int64_t tree_new_nodes(orc_tree *t, int64_t k, int64_t *cap)
{
    int64_t first = t->n_nodes;
    if (t->n_nodes + k > *cap) {
        int64_t nc = *cap ? *cap : 64;
        while (nc < t->n_nodes + k) nc *= 2;
        t->center = (int64_t *)realloc(t->center, sizeof(int64_t) * (size_t)nc);
        t->radius = (double *)realloc(t->radius, sizeof(double) * (size_t)nc);
        t->level = (int32_t *)realloc(t->level, sizeof(int32_t) * (size_t)nc);
        t->child_begin = (int64_t *)realloc(t->child_begin, sizeof(int64_t) * (size_t)nc);
        t->child_count = (int64_t *)realloc(t->child_count, sizeof(int64_t) * (size_t)nc);
        t->pts_begin = (int64_t *)realloc(t->pts_begin, sizeof(int64_t) * (size_t)nc);
        t->pts_count = (int64_t *)realloc(t->pts_count, sizeof(int64_t) * (size_t)nc);
        *cap = nc;
    }
    for (int64_t i = first; i < first + k; ++i) {
        t->child_begin[i] = 0; t->child_count[i] = 0;
        t->pts_begin[i] = 0; t->pts_count[i] = 0;
    }
    t->n_nodes += k;
    return first;
}

/* ceil(log2 r) for r > 0, exact for powers of two. */
static int32_t ceil_log2(double r)
{
    int e;
    double m = frexp(r, &e);   /* r = m * 2^e, m in [0.5, 1) */
    return m == 0.5 ? e - 1 : e;
}

/* Builds the cover tree by vertex splitting.
 * Root: point `root` (the paper selects one point as the root).  A vertex
 * triple (H, p, r) with |H| > zeta and r > 0 is a hub at level ceil(log2 r)
 * (levels with a single nested child are not materialised); its split adds
 * farthest points as new centres until every point of H lies within
 * 2^(l-1) of its nearest centre (Algorithm 1), then partitions H by label.
 * A child with |H_i| <= zeta, or with radius 0 (duplicates), is a leaf block
 * (Algorithm 2). */
orc_tree *orc_build_tree(const orc_space *sp, int32_t zeta, int64_t root)
{
    orc_tree *t = (orc_tree *)calloc(1, sizeof(orc_tree));
    int64_t n = sp->n, cap = 0;
    t->n_points = n;
    t->leaf_pts = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    int64_t n_leaf_pts = 0;
    if (n == 0) return t;
    if (zeta < 1) zeta = 1;
    int64_t evals = 0;

    /* root triple: D[p] = d(p, root) */
    hub_t h0;
    h0.node = tree_new_nodes(t, 1, &cap);
    h0.m = n;
    h0.H = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    h0.D = (double *)malloc(sizeof(double) * (size_t)n);
    h0.H[0] = root;
    for (int64_t i = 0, j = 1; i < n; ++i) if (i != root) h0.H[j++] = i;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) h0.D[i] = metric_dist(sp, h0.H[i], root);
    evals += n;
    double r0 = 0.0;
    for (int64_t i = 0; i < n; ++i) if (h0.D[i] > r0) r0 = h0.D[i];
    t->center[h0.node] = root;
    t->radius[h0.node] = r0;

    /* work list of pending triples (hub or leaf decided on pop) */
    int64_t qcap = 64, qlen = 0;
    hub_t *queue = (hub_t *)malloc(sizeof(hub_t) * (size_t)qcap);
    h0.level = r0 > 0 ? ceil_log2(r0) : INT32_MIN;
    queue[qlen++] = h0;
    int64_t qhead = 0;

    while (qhead < qlen) {
        hub_t h = queue[qhead++];
        int64_t u = h.node;
        double r = t->radius[u];
        if (h.m <= zeta || r == 0.0) {
            /* leaf block: its points are the leaf vertices B(p, 0) */
            t->level[u] = r > 0 ? ceil_log2(r) : INT32_MIN;
            t->pts_begin[u] = n_leaf_pts;
            t->pts_count[u] = h.m;
            for (int64_t i = 0; i < h.m; ++i) t->leaf_pts[n_leaf_pts++] = h.H[i];
            free(h.H); free(h.D);
            continue;
        }
        int32_t l = h.level;
        t->level[u] = l;
        double thr = ldexp(1.0, l - 1);

        /* SplitVertex: L[i] = index of nearest centre so far */
        int64_t *L = (int64_t *)calloc((size_t)h.m, sizeof(int64_t));
        int64_t ccap = 16, nc = 1;
        int64_t *cent = (int64_t *)malloc(sizeof(int64_t) * (size_t)ccap);
        cent[0] = 0;  /* position of pi_1 in H: the hub's own centre */
        for (;;) {
            /* farthest point: first maximum in scan order (strict >) */
            double rs = 0.0;
            int64_t far = -1;
            for (int64_t i = 0; i < h.m; ++i)
                if (h.D[i] > rs) { rs = h.D[i]; far = i; }
            if (far < 0 || h.D[far] <= thr) break;
            if (nc == ccap) { ccap *= 2; cent = (int64_t *)realloc(cent, sizeof(int64_t) * (size_t)ccap); }
            cent[nc] = far;
            int64_t lab = nc++;
            int64_t pc = h.H[far];
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < h.m; ++i) {
                double d = metric_dist(sp, h.H[i], pc);
                if (d < h.D[i]) { h.D[i] = d; L[i] = lab; }
            }
            evals += h.m;
        }
        /* partition H by label into the children, preserving scan order;
         * child c's centre is placed first in its list */
        int64_t first = tree_new_nodes(t, nc, &cap);
        t->child_begin[u] = first;
        t->child_count[u] = nc;
        int64_t *cnt = (int64_t *)calloc((size_t)nc, sizeof(int64_t));
        for (int64_t i = 0; i < h.m; ++i) cnt[L[i]]++;
        for (int64_t c = 0; c < nc; ++c) {
            hub_t ch;
            ch.node = first + c;
            ch.m = cnt[c];
            ch.H = (int64_t *)malloc(sizeof(int64_t) * (size_t)ch.m);
            ch.D = (double *)malloc(sizeof(double) * (size_t)ch.m);
            int64_t ci = cent[c], w = 1;
            ch.H[0] = h.H[ci];
            ch.D[0] = h.D[ci];
            double rc = 0.0;
            for (int64_t i = 0; i < h.m; ++i) {
                if (L[i] != c || i == ci) continue;
                ch.H[w] = h.H[i];
                ch.D[w] = h.D[i];
                if (h.D[i] > rc) rc = h.D[i];
                w++;
            }
            t->center[ch.node] = ch.H[0];
            t->radius[ch.node] = rc;
            ch.level = rc > 0 ? ceil_log2(rc) : INT32_MIN;
            if (qlen == qcap) { qcap *= 2; queue = (hub_t *)realloc(queue, sizeof(hub_t) * (size_t)qcap); }
            queue[qlen++] = ch;
        }
        free(cnt); free(L); free(cent); free(h.H); free(h.D);
    }
    free(queue);
    t->dist_evals = evals;
    return t;
}

void orc_tree_free(orc_tree *t)
{
    if (!t) return;
    free(t->center); free(t->radius); free(t->level);
    free(t->child_begin); free(t->child_count);
    free(t->pts_begin); free(t->pts_count); free(t->leaf_pts);
    free(t);
}

/* Relative slack on the subtree test: FP64 rounding of the computed distances
 * may break the triangle inequality by a few ulps; the test keeps a subtree
 * whenever d(q, v) <= (radius(v) + eps) (1 + PRUNE_SLACK). */
#define PRUNE_SLACK 1e-12

/* ε query of every point against the tree (Algorithm 3), stack walk from the
 * root.  A child vertex v is pushed iff d(q, v) <= radius(v) + eps; the points
 * of a leaf block are leaf vertices B(p, 0), reported iff d(q, p) <= eps (the
 * pinned predicate). */
orc_csr *orc_tree_query_rows(const orc_space *sp, const orc_tree *t, double eps,
                             int32_t include_self, const int64_t *rows, int64_t n_rows)
{
    int64_t n = n_rows;
    double eps2 = eps * eps;
    vec_t *rows_out = (vec_t *)calloc((size_t)(n ? n : 1), sizeof(vec_t));
    int64_t evals = 0;
    if (n > 0) {
#pragma omp parallel reduction(+ : evals)
        {
            int64_t scap = 256;
            int64_t *stack = (int64_t *)malloc(sizeof(int64_t) * (size_t)scap);
#pragma omp for schedule(dynamic, 64)
            for (int64_t qr = 0; qr < n; ++qr) {
                int64_t q = rows ? rows[qr] : qr;
                vec_t *row = &rows_out[qr];
                int64_t sp_top = 0;
                stack[sp_top++] = 0;
                while (sp_top > 0) {
                    int64_t u = stack[--sp_top];
                    if (t->child_count[u] == 0) {
                        /* leaf block: its children are the point vertices */
                        for (int64_t k = 0; k < t->pts_count[u]; ++k) {
                            int64_t p = t->leaf_pts[t->pts_begin[u] + k];
                            if (p == q && !include_self) continue;
                            double d;
                            evals++;
                            if (edge_pred(sp, q, p, eps, eps2, &d)) vec_push(row, p, d);
                        }
                        continue;
                    }
                    for (int64_t c = 0; c < t->child_count[u]; ++c) {
                        int64_t v = t->child_begin[u] + c;
                        double dv;
                        evals++;
                        if (sp->metric == ORC_L2) {
                            dv = metric_dist(sp, q, t->center[v]);
                            if (!(dv <= (t->radius[v] + eps) * (1.0 + PRUNE_SLACK))) continue;
                        } else if (sp->metric == ORC_HAM) {
                            dv = metric_dist(sp, q, t->center[v]);
                            if (!(dv <= floor(t->radius[v] + eps))) continue;
                        } else {
                            int32_t la, lb;
                            const uint8_t *a = str_at(sp, q, &la);
                            const uint8_t *b = str_at(sp, t->center[v], &lb);
                            int32_t k = (int32_t)floor(t->radius[v] + eps);
                            if (orc_lev_banded(a, la, b, lb, k) > k) continue;
                        }
                        if (sp_top == scap) {
                            scap *= 2;
                            stack = (int64_t *)realloc(stack, sizeof(int64_t) * (size_t)scap);
                        }
                        stack[sp_top++] = v;
                    }
                }
            }
            free(stack);
        }
    }
    orc_csr *o = assemble(n, rows_out);
    o->dist_evals = evals;
    return o;
}

orc_csr *orc_tree_query(const orc_space *sp, const orc_tree *t, double eps, int32_t include_self)
{
    return orc_tree_query_rows(sp, t, eps, include_self, NULL, sp->n);
}

/* ---------------------------------------------------------- invariant check */

/* Checks a flat tree against the cover-tree invariants.  `tol` is the relative
 * tolerance for the net properties (covering within 2^l, separation above
 * 2^(l-1)): 0 for an FP64-built tree, about 1e-5 for an fp32-built one.  The
 * radius check is strict in FP64: every point below a vertex lies within its
 * stored radius, since the query's correctness depends on it.
 * Returns 0 when every check passes, otherwise a code and a message. */
int32_t orc_check_tree(const orc_space *sp, const orc_tree *t, double tol, char *msg,
                       int32_t msg_len)
{
    int64_t n = sp->n, N = t->n_nodes;
#define FAIL(code, ...) do { snprintf(msg, (size_t)msg_len, __VA_ARGS__); return code; } while (0)
    msg[0] = 0;
    if (n == 0) { if (N != 0) FAIL(1, "empty point set but %lld nodes", (long long)N); return 0; }
    if (N < 1) FAIL(1, "no root");
    /* structure: every node but the root has exactly one parent, children
     * ranges are in bounds, internal nodes list no points */
    int32_t *parents = (int32_t *)calloc((size_t)N, sizeof(int32_t));
    for (int64_t u = 0; u < N; ++u) {
        if (t->child_count[u] < 0 || t->child_begin[u] < 0 ||
            t->child_begin[u] + t->child_count[u] > N) { free(parents); FAIL(2, "node %lld: child range out of bounds", (long long)u); }
        if (t->child_count[u] > 0 && t->pts_count[u] != 0) { free(parents); FAIL(2, "node %lld: internal node with points", (long long)u); }
        if (t->child_count[u] == 0 && t->pts_count[u] <= 0) { free(parents); FAIL(2, "node %lld: empty leaf block", (long long)u); }
        for (int64_t c = 0; c < t->child_count[u]; ++c) {
            int64_t v = t->child_begin[u] + c;
            if (v == 0) { free(parents); FAIL(2, "root listed as a child"); }
            parents[v]++;
        }
    }
    for (int64_t u = 1; u < N; ++u)
        if (parents[u] != 1) { int32_t p = parents[u]; free(parents); FAIL(2, "node %lld has %d parents", (long long)u, p); }
    free(parents);
    /* every point in exactly one leaf block */
    int32_t *seen = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    int64_t total = 0;
    for (int64_t u = 0; u < N; ++u) {
        if (t->child_count[u]) continue;
        if (t->pts_begin[u] < 0 || t->pts_begin[u] + t->pts_count[u] > t->n_points) { free(seen); FAIL(3, "node %lld: point range out of bounds", (long long)u); }
        for (int64_t k = 0; k < t->pts_count[u]; ++k) {
            int64_t p = t->leaf_pts[t->pts_begin[u] + k];
            if (p < 0 || p >= n) { free(seen); FAIL(3, "node %lld: bad point id", (long long)u); }
            seen[p]++;
            total++;
        }
        /* the leaf block's centre is its first point */
        if (t->leaf_pts[t->pts_begin[u]] != t->center[u]) { free(seen); FAIL(4, "leaf block %lld: centre is not its first point", (long long)u); }
    }
    for (int64_t p = 0; p < n; ++p)
        if (seen[p] != 1) { int32_t s = seen[p]; free(seen); FAIL(3, "point %lld appears in %d leaf blocks", (long long)p, s); }
    free(seen);
    (void)total;

    int32_t code = 0;
    /* per internal node: nesting, covering, separation, child level order */
    for (int64_t u = 0; u < N && !code; ++u) {
        int64_t nc = t->child_count[u];
        if (!nc) continue;
        int64_t cb = t->child_begin[u];
        if (t->center[cb] != t->center[u]) { code = 5; snprintf(msg, (size_t)msg_len, "node %lld: first child does not share its point (nesting)", (long long)u); break; }
        if (t->level[u] == INT32_MIN) { code = 6; snprintf(msg, (size_t)msg_len, "node %lld: internal node with radius 0", (long long)u); break; }
        double cover = ldexp(1.0, t->level[u]);
        double sep = ldexp(1.0, t->level[u] - 1);
        if (t->radius[u] > cover * (1.0 + tol)) { code = 6; snprintf(msg, (size_t)msg_len, "node %lld: radius %.17g above 2^%d", (long long)u, t->radius[u], t->level[u]); break; }
        for (int64_t a = 0; a < nc && !code; ++a) {
            int64_t va = cb + a;
            if (t->child_count[va] && t->level[va] >= t->level[u]) { code = 6; snprintf(msg, (size_t)msg_len, "node %lld: child level not below parent", (long long)va); break; }
            double d = metric_dist(sp, t->center[u], t->center[va]);
            if (d > cover * (1.0 + tol)) { code = 7; snprintf(msg, (size_t)msg_len, "node %lld: child %lld at %.17g outside 2^%d (covering)", (long long)u, (long long)va, d, t->level[u]); break; }
            for (int64_t b = a + 1; b < nc; ++b) {
                double e = metric_dist(sp, t->center[va], t->center[cb + b]);
                if (!(e > sep * (1.0 - tol))) { code = 8; snprintf(msg, (size_t)msg_len, "node %lld: children %lld,%lld at %.17g not above 2^%d (separation)", (long long)u, (long long)va, (long long)(cb + b), e, t->level[u] - 1); break; }
            }
        }
    }
    if (code) return code;

    /* strict radius: walk each leaf point up to the root; needs parent links */
    int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    parent[0] = -1;
    for (int64_t u = 0; u < N; ++u)
        for (int64_t c = 0; c < t->child_count[u]; ++c) parent[t->child_begin[u] + c] = u;
    int64_t bad_u = -1, bad_p = -1;
    double bad_d = 0.0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t u = 0; u < N; ++u) {
        if (t->child_count[u]) continue;
        for (int64_t k = 0; k < t->pts_count[u]; ++k) {
            int64_t p = t->leaf_pts[t->pts_begin[u] + k];
            for (int64_t a = u; a >= 0; a = parent[a]) {
                double d = metric_dist(sp, t->center[a], p);
                if (!(d <= t->radius[a])) {
#pragma omp critical
                    { if (bad_u < 0) { bad_u = a; bad_p = p; bad_d = d; } }
                }
            }
        }
    }
    free(parent);
    if (bad_u >= 0)
        FAIL(9, "node %lld: point %lld at %.17g beyond stored radius %.17g", (long long)bad_u, (long long)bad_p, bad_d, t->radius[bad_u]);
    return 0;
#undef FAIL
}

int32_t orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
