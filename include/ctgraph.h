/*
 * ctgraph.h -- exact fixed-radius near-neighbour graphs (ε-graphs) with a
 * cover tree on one GB300 GPU (sm_103a).
 *
 * Problem (paper Sec. III, "ε-graph"): given n points P with a metric d and a
 * threshold eps, output every ordered pair (i, j), i != j, with
 * d(p_i, p_j) <= eps (closed ball).  The output is a CSR matrix whose row i
 * lists the original indices j in ascending order; it is symmetric, and nnz
 * counts both directions of every undirected edge, as Table I does.
 *
 * Method: a cover tree built level by level by vertex splitting
 * (Algorithms 1 and 2, Sec. IV-A), queried in batches (Algorithm 3 and the
 * batching remark of Sec. IV-B): each leaf block of the tree is one query
 * group; its candidate leaf blocks are found by a triangle-inequality walk of
 * the tree, then every (query, candidate point) pair is decided exactly.
 *
 * Conventions for every entry point:
 *  - Device pointers are CUDA device addresses on the current device; host
 *    pointers are ordinary process memory.  `stream` is a cudaStream_t (NULL
 *    is the legacy default stream).
 *  - Inputs are borrowed: the caller keeps them valid until the work enqueued
 *    on `stream` has completed.
 *  - Outputs are owned by the library and are released only by csr_free /
 *    ct_tree_free.  Device buffers are allocated stream-ordered on `stream`.
 *  - Every call returns a status and never aborts, traps or exits.  On error
 *    the out-parameters are zeroed and ct_last_error() describes the failure;
 *    a CUDA error maps to CT_ECUDA with the CUDA error string.
 *  - Calls synchronise `stream` where the size of an output must be known on
 *    the host (the edge count before the CSR is allocated).
 */
#ifndef CTGRAPH_H
#define CTGRAPH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CT_OK = 0,
    CT_EINVAL = 1,        /* invalid argument (null pointer, negative size, eps < 0, ...) */
    CT_ENOMEM = 2,        /* a device or host allocation failed */
    CT_ECUDA = 3,         /* a CUDA call or kernel failed; see ct_last_error() */
    CT_ETIMEOUT = 4,      /* a bounded device-side wait gave up */
    CT_EOVERFLOW = 5,     /* a size does not fit the index types (e.g. n >= 2^31) */
    CT_EUNSUPPORTED = 6   /* valid but unsupported input (e.g. a string above the length limit) */
} ct_status;

typedef enum {
    CT_L2_F32 = 0,        /* Euclidean distance over fp32 coordinates */
    CT_LEVENSHTEIN_U8 = 1, /* edit distance, unit costs, over byte strings */
    CT_HAMMING_B1 = 2     /* Hamming distance over bit strings (the number of differing bits) */
} ct_metric;

/* A cudaStream_t, passed as an opaque pointer so this header needs no CUDA headers. */
typedef void *ct_stream;

/* The point set P (paper Sec. III: a finite metric space).
 *  CT_L2_F32:         data    = device, n*dim fp32, row-major, rows contiguous;
 *                     offsets = NULL; 1 <= dim <= 4096.
 *  CT_LEVENSHTEIN_U8: data    = device, concatenated byte strings;
 *                     offsets = device, n+1 int64, string i is
 *                     data[offsets[i] .. offsets[i+1]); dim ignored;
 *                     every string at most CT_MAX_STRING_LEN bytes.
 *  CT_HAMMING_B1:     data    = device, n rows of ceil(dim/8) bytes, rows
 *                     contiguous; bit j of a row is bit (j mod 8) of its
 *                     byte j/8 (bits past dim are ignored); offsets = NULL;
 *                     1 <= dim <= 4096 bits.  Distances are integers; an
 *                     edge iff d <= floor(eps) (the binary datasets of the
 *                     paper's Sec. V-A, Table I).
 *  n may be 0.  n must be below 2^31 - 1. */
typedef struct {
    int32_t metric;
    int32_t dim;
    int64_t n;
    const void *data;
    const int64_t *offsets;
} ct_points;

#define CT_MAX_STRING_LEN 1024

/* Build options.  leaf_size is ζ of Algorithm 2: a vertex with at most ζ
 * points becomes a leaf block (<= 0 selects 32).  root is the index of the
 * root point (the paper selects one point as the root; default 0). */
typedef struct {
    int32_t leaf_size;
    int32_t root;
} ct_build_opts;

/* Query options.
 *  precision:     0 = plain FP32 direct-difference leaf tiles;
 *                 1 = tensor-core filter (tcgen05, fp16 rows centred on
 *                     the column means and scaled by a power of two,
 *                     prepared once per query) with FP32 recheck (L2 only;
 *                     rows above 128 floats use the FP32 tiles);
 *                 2 = per cloud, the count kernel and work-item length that
 *                     ct_autotune measured fastest for its row length (before
 *                     tuning: tensor-core tiles from 32 floats per row up).
 *                 All give the same edge set and distances.
 *  use_predictor: 0 = two-pass count -> scan -> emit;
 *                 1 = one-pass emit into row capacities predicted by
 *                     `predictor` (a fitted ct_predictor on the tree's
 *                     device); entries past a row's capacity go to an
 *                     overflow arena, rows that overflow the arena too are
 *                     emitted again exactly.  Same output.
 *  include_self:  1 adds the pair (i, i) to every row (d(p, p) = 0 <= eps).
 *  upper_triangle: 1 evaluates each pair of points of two different query
 *                 groups once, from the group that comes first in tree
 *                 order, and writes the edge into both rows (the symmetry
 *                 d(p, q) = d(q, p) the paper's ring uses to halve its
 *                 rounds, Sec. IV-C); pairs inside a group are evaluated
 *                 from both ends as before.  Same output, about half the
 *                 leaf pairs.
 *  predictor:     a ct_predictor* when use_predictor = 1, else NULL. */
typedef struct {
    int32_t precision;
    int32_t use_predictor;
    int32_t include_self;
    int32_t upper_triangle;
    const void *predictor;
} ct_query_opts;

/* CSR output.  row_ptr: device int64[n_rows + 1]; col: device int32[nnz]
 * (original point indices, ascending within a row); dist: device fp32[nnz]
 * (the distance; within 1e-6 relative of the FP64 value for L2, exact
 * integers for edit distance).  Pointers may be NULL when nnz == 0 (col,
 * dist) or n_rows == 0 is still given a one-entry row_ptr. */
typedef struct {
    int64_t n_rows;
    int64_t nnz;
    int64_t *row_ptr;
    int32_t *col;
    float *dist;
    void *priv;           /* library-owned; do not touch */
} ct_csr;

/* Counters of one query, read back with ct_csr_stats. */
typedef struct {
    int64_t traversal_evals;  /* distance evaluations in the tree walk (count pass) */
    int64_t leaf_pairs;       /* (query, candidate point) pairs decided (count pass) */
    int64_t guard_fp64;       /* pairs decided by the pinned FP64 sum */
    int64_t recheck_fp32;     /* pairs re-evaluated in FP32 after the tensor-core filter */
    int64_t candidates;       /* (group, candidate leaf block) entries */
    int64_t overflow_rows;    /* learned form: rows whose degree exceeded the predicted capacity */
    int64_t kernel_launches;  /* kernels this library launched for the query */
    int64_t emit_pairs;       /* pairs evaluated again by the emit pass */
    int64_t reemit_rows;      /* learned form: rows emitted again (overflow arena was full) */
    int64_t leaf_rows;        /* point rows loaded into the count pass's leaf tiles (L2) */
    int64_t guard_band;       /* pairs in the guard band |d - eps| <= 1e-3 eps (FP32 value); of
                                 these, only those the fp32 error bound cannot place on one side
                                 of eps go to FP64 */
    int64_t lev_columns;      /* edit distance, count pass: text characters the bit-parallel
                                 recurrence processed, times the pattern's 64-bit words */
} ct_query_stats;

typedef struct ct_tree ct_tree;           /* opaque, device-resident */

/* Cover-tree construction (Algorithms 1 and 2): level-wise vertex splitting on
 * the GPU.  The points are copied into tree order, so the tree does not alias
 * `points`.  Synchronises `stream` a few times per level (loop control).
 * Errors: CT_EINVAL (null pointers, n < 0, bad metric or dim),
 * CT_EUNSUPPORTED (string too long), CT_ENOMEM, CT_ECUDA. */
ct_status ct_build(const ct_points *points, const ct_build_opts *opts, ct_stream stream,
                   ct_tree **out);

/* The ε-graph of the tree's point set (Sec. III definition; query by
 * Algorithm 3 with batching, Sec. IV-B).  eps >= 0; for edit distance only
 * floor(eps) matters.  On success *out holds a CSR in library-owned device
 * memory (release with csr_free).  Synchronises `stream` once to learn nnz.
 * Errors: CT_EINVAL (null pointers, eps < 0 or NaN, precision 1 with a
 * non-L2 tree, use_predictor without predictor), CT_ENOMEM, CT_ECUDA. */
ct_status eps_graph_query(const ct_tree *tree, double eps, const ct_query_opts *opts,
                          ct_stream stream, ct_csr *out);

/* Many point clouds in one call: outs[c] is the ε-graph of trees[c] with
 * radius eps[c] (host array); the same output as n_clouds calls of
 * eps_graph_query.  L2 clouds go in batches of up to 64 that share every
 * launch: one walk over all their groups (in one global order), one leaf
 * launch over all their work items, one scan, one row sort.  Edit-distance
 * clouds run one at a time.  The CSRs of one batch view shared allocations,
 * released when the last of them is freed (each csr_free as usual); the
 * counters ct_csr_stats returns for them are those of the whole batch.
 * Errors: as eps_graph_query, for any cloud. */
ct_status eps_graph_query_batched(int32_t n_clouds, const ct_tree *const *trees,
                                  const double *eps, const ct_query_opts *opts,
                                  ct_stream stream, ct_csr *outs);

/* ------------------------------------------------------------------------
 * Plans: one batch of L2 clouds (the batched form above) queried again and
 * again over the same trees, with every buffer allocated once.  The paper's
 * batching of queries (Sec. IV-B) is carried across clouds: a run is one
 * sequence of launches with no host read-back and no allocation -- the walk
 * over every cloud's query groups, each group's candidates gathered into one
 * range, then the leaf stage as ONE persistent launch over all clouds'
 * (cloud, group) work items: each CTA first produces the work items of a
 * chunk of groups into a device work queue (groups in the walk order; item
 * lengths per row-length class from ct_autotune with precision 2), then
 * takes queue slots, waiting for a slot's producer with a bounded number of
 * polls -- then the scan, the emit pass (the same persistent launch over the
 * complete queue) and the row sorts (rows above 4096 entries by one radix
 * sort over a capacity sized like the others).  With use_graph the run is
 * captured once into a CUDA graph and every launch replays it.  A plan's leaf
 * tiles are the FP32 ones (precision 1 is taken as 0); use_predictor orders
 * the walk by predicted work; the output equals eps_graph_query_batched's.
 * The plan borrows the trees: they must outlive it and stay unchanged. */
typedef struct ct_plan ct_plan;

/* Runs the batch once with the exact query to size every buffer (candidate
 * list, work queue, edges: each times 1 + margin, plus a constant), then
 * allocates them (and captures the graph when use_graph != 0).  1 <= n_clouds
 * <= 64, L2 trees on the current device.  Synchronises `stream`.
 * Errors: CT_EINVAL (NULL arguments, a bad count, margin outside [0, 100],
 * a tree of another metric, options as eps_graph_query), CT_ENOMEM,
 * CT_ECUDA. */
ct_status ct_plan_create(int32_t n_clouds, const ct_tree *const *trees, const double *eps,
                         const ct_query_opts *opts, float margin, int32_t use_graph, ct_stream stream,
                         ct_plan **out);
/* Enqueues one run on `stream` (a graph launch with use_graph); returns at
 * once.  Runs on one plan must not overlap (they share its buffers). */
ct_status ct_plan_launch(ct_plan *plan, ct_stream stream);
/* Synchronises `stream` and reports the last run: CT_OK with outs[c] (host
 * array of n_clouds) the CSR of cloud c -- views into the plan's buffers,
 * valid until the next launch or ct_plan_free (csr_free releases only the
 * view) -- or CT_EOVERFLOW (the run outgrew a capacity: create a new plan),
 * CT_ETIMEOUT (a work-queue wait gave up), CT_ECUDA; on error outs are
 * zeroed. */
ct_status ct_plan_result(ct_plan *plan, ct_stream stream, ct_csr *outs);
/* Test control of the work queue's bounded waits, read by later runs
 * (replays included): withhold_producers != 0 makes the producers take their
 * groups and publish nothing, so that every consumer's wait runs out after
 * max_polls polls (about 1 us each; default 2^20) and the run reports
 * CT_ETIMEOUT.  Synchronises the device.  Errors: CT_EINVAL. */
ct_status ct_plan_set_wait(ct_plan *plan, int32_t withhold_producers, int32_t max_polls);
/* Releases a plan (synchronises its creation stream).  NULL-safe. */
void ct_plan_free(ct_plan *plan);

/* The ε-graph of one tree at several radii (the paper queries each dataset at
 * three radii, Table I; the tree does not depend on eps, so one build serves
 * them all).  outs[k] is exactly the CSR eps_graph_query(tree, eps[k], opts)
 * returns (the same entries and distances, bit for bit), each released with
 * csr_free.  The largest radius is queried in full; each smaller one is
 * derived from the CSR of the next larger one: an entry is decided again
 * from its stored distance when that distance lies outside the guard band
 * |d - r| <= 1e-3 r of both radii (the stored value is within 1e-6 of the
 * exact one), and from the points, by the query's own decision, inside it.
 * eps (host array of n_eps) may be in any order.  The counters of outs[k]
 * are the full query's for the largest radius; for the others leaf_pairs
 * counts the entries evaluated again from the points.  Synchronises
 * `stream` once per radius.  Errors: as eps_graph_query for any radius. */
ct_status eps_graph_query_sweep(const ct_tree *tree, int32_t n_eps, const double *eps,
                                const ct_query_opts *opts, ct_stream stream, ct_csr *outs);

/* Sizes of the landmark form's partition (eps_graph_query_landmark). */
typedef struct {
    int64_t cells;         /* m */
    int64_t members;       /* points over all cells: each point in its own cell plus its ghost cells */
    int64_t ghosts;        /* members - n */
    int64_t largest_cell;  /* members of the largest cell */
} ct_landmark_info;

/* The ε-graph through landmarks (Sec. IV-D, the paper's Voronoi-cell and
 * ghost-query algorithms on one GPU): the points' Voronoi cells of the m
 * centres (host int64 point indices, e.g. drawn at random as the paper
 * does); the ε-ghosts of every cell by Lemma 1 -- the points p outside it
 * with d(p, c_k) <= d(p, C) + 2 eps -- so that every neighbour of a cell's
 * point lies in the cell or among its ghosts; a cover tree per cell over its
 * points and ghosts (`bopts`), all cells queried as one batch with `qopts`
 * (the forms of eps_graph_query); each point's row from its own cell.  The
 * output equals eps_graph_query's on the whole set (the same entries and
 * distances), in library-owned memory (csr_free).  `points` as for ct_build
 * (L2 or Hamming; device memory).  info (may be NULL) receives the sizes.
 * n = 0 gives the empty graph.  Synchronises `stream`.  Errors: CT_EINVAL
 * (NULL arguments, m outside [1, n], a centre out of range, options as
 * eps_graph_query),
 * CT_EUNSUPPORTED (edit distance), CT_ENOMEM, CT_ECUDA. */
ct_status eps_graph_query_landmark(const ct_points *points, const int64_t *centres, int32_t m, double eps,
                                  const ct_build_opts *bopts, const ct_query_opts *qopts, ct_stream stream,
                                  ct_csr *out, ct_landmark_info *info);

/* Writes a tree to a file at `path` (a header with the sizes, every device
 * array of the tree, and a 64-bit FNV-1a checksum), so that a later process
 * can query it without building it again.  Synchronises the tree's stream.
 * Errors: CT_EINVAL (NULL argument, the file cannot be written), CT_ECUDA. */
ct_status ct_tree_save(const ct_tree *tree, const char *path);

/* Reads a tree written by ct_tree_save onto the current device (allocated
 * stream-ordered on `stream`, released with ct_tree_free).  Queries of the
 * loaded tree return what queries of the saved one return.  The header is
 * checked, the checksum compared and every index of the tree range-checked
 * on the device before the call returns.  Synchronises `stream`.
 * Errors: CT_EINVAL (NULL argument, unreadable, truncated or inconsistent
 * file, checksum mismatch), CT_ENOMEM, CT_ECUDA. */
ct_status ct_tree_load(const char *path, ct_stream stream, ct_tree **out);

/* Autotuner of precision 2.  For each class of row length present among the
 * L2 trees (dp = dim rounded up to 4: <= 4, 16, 32, 64, 128), times the
 * batched query of that class's clouds (eps_graph_query_batched with
 * `opts`, twice per candidate, outputs discarded) with each candidate --
 * count kernel (tensor-core or FP32 tiles) x work-item length (512 or 256
 * candidate blocks) -- and keeps the fastest in a process-wide table.
 * choices (host int32[n_clouds], may be NULL) receives each cloud's kernel
 * (1 tensor core, 0 FP32).  Synchronises `stream`.  ct_autotune_reset clears the
 * table.  Errors: as eps_graph_query_batched. */
ct_status ct_autotune(int32_t n_clouds, const ct_tree *const *trees, const double *eps,
                      const ct_query_opts *opts, ct_stream stream, int32_t *choices);
void ct_autotune_reset(void);

/* Size of the fixed device array used by eps_graph_degrees_noalloc. */
#define CT_NOALLOC_SCRATCH_BYTES (16u << 20)

/* Degree of every point of the ε-graph, without allocating device memory.
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot let a library allocate on the device (an application whose own
 * allocator owns the device and hands out fixed budgets, or a latency-bound
 * loop that cannot take an allocation's implicit synchronisation or its
 * possible failure).
 *  degrees: device int32[n], written by the call: degrees[i] is the number of
 *           j (j != i unless include_self) with d(p_i, p_j) <= eps, i.e.
 *           row_ptr[i+1] - row_ptr[i] of eps_graph_query with the same eps.
 * All temporaries live in one fixed array of CT_NOALLOC_SCRATCH_BYTES bytes
 * inside the library (every GPU that loads the library holds it until the
 * process exits).  The first call on a device looks up that array's device
 * address.  Calls never allocate or free device memory; they synchronise
 * `stream` twice and copy counters to host memory.  The candidate list holds
 * about 2.5 M (group, leaf block) entries, fewer for deep trees; the walk
 * runs with at most 64 blocks of 4 warps.
 * Every call reuses the same array and clears what must start at zero; calls
 * whose work overlaps on the GPU (other streams, other host threads) race on
 * it and must be serialised by the caller.
 * L2 trees only.  Errors: CT_EINVAL (null pointers, eps < 0 or NaN),
 * CT_EUNSUPPORTED (an edit-distance tree, or a problem whose temporaries do
 * not fit the fixed array: the message gives the need), CT_ECUDA. */
ct_status eps_graph_degrees_noalloc(const ct_tree *tree, double eps, int32_t include_self,
                                    int32_t *degrees, ct_stream stream);

/* Releases a CSR (stream-ordered on the stream it was produced on; that
 * stream must still exist).  Idempotent and NULL-safe: zeroes *csr. */
void csr_free(ct_csr *csr);

/* Host copy of the counters recorded with `csr`. */
ct_status ct_csr_stats(const ct_csr *csr, ct_query_stats *out);

/* Releases a tree (synchronises the device).  NULL-safe. */
void ct_tree_free(ct_tree *tree);

/* Sizes of a tree: number of vertices (internal + leaf blocks) and points. */
ct_status ct_tree_shape(const ct_tree *tree, int64_t *n_nodes, int64_t *n_points);

/* Copies the tree to host arrays in the flat format (vertex 0 is the root;
 * children of a vertex are consecutive ids; a leaf block lists its points
 * in leaf_pts[pts_begin .. pts_begin + pts_count)).  Every array is host
 * memory sized by ct_tree_shape: center, radius, level, child_begin,
 * child_count, pts_begin, pts_count have n_nodes entries; leaf_pts has
 * n_points.  Point ids are original indices.  Synchronises the device. */
ct_status ct_tree_export(const ct_tree *tree, int64_t *center, double *radius, int32_t *level,
                         int64_t *child_begin, int64_t *child_count, int64_t *pts_begin,
                         int64_t *pts_count, int64_t *leaf_pts);

/* ------------------------------------------------------------------------
 * Degree/work predictor of the learned form.  The paper has no learned
 * component: this is an extension that sizes the one-pass emit and orders the
 * traversal.  A small multilayer perceptron, CT_MLP_IN -> 64 -> 64 -> 2 with
 * ReLU after both hidden layers, maps 16 features of a query, read from the
 * tree before the query runs (e = max(eps, 1e-20)):
 *    0 log1p(d(q, leaf-block centre)/e)   1 log1p(d(q, group centre)/e)
 *                                           (L2; 0 for edit distance)
 *    2 log1p(group radius/e)              3 log2(points of the group)
 *    4..11 leaf block and its first three ancestors (the root repeats):
 *          log1p(points below), log1p(radius/e)
 *    12..15 log1p(points below the lowest ancestor of the leaf block,
 *          itself included, with radius >= e, 2e, 4e, 16e; the root if none)
 * (the group: the query's run of sibling leaf blocks, at most 32 points, or
 * a cut of 32 consecutive points of a larger block; its centre is its first
 * point) to
 *    output 0: log(1 + degree of the query),
 *    output 1: log(1 + vertices tested by the tree walk of its group).
 * Output 0 sizes the rows of the one-pass emit; output 1, averaged over a
 * group, orders the walks longest first.  Inputs and targets are
 * standardised with the mean and deviation of the training set.  Parameters
 * are one fp32 vector, W1 (64 x 16, row-major), b1, W2 (64 x 64), b2,
 * W3 (2 x 64), b3: CT_MLP_NPARAMS values.  Inference uses fp16 copies of the
 * weights with fp32 sums.
 * A predictor lives on the device that was current when it was created. */
#define CT_MLP_IN 16
#define CT_MLP_NPARAMS 5378
#define CT_MLP_NORM 36  /* feature mean[16], feature std[16], target mean[2], target std[2] */

typedef struct ct_predictor ct_predictor;

/* Fit options (zero fields select the defaults). */
typedef struct {
    int32_t steps;         /* Adam steps (default 1500) */
    int32_t batch;         /* samples per step, drawn uniformly (default 4096) */
    float lr;              /* initial learning rate, cosine-decayed to lr/10 (default 2e-3) */
    int32_t include_self;  /* the degrees to learn count the point itself */
    uint64_t seed;         /* batch sampling */
} ct_fit_opts;

/* New predictor with He-initialised weights drawn from `seed`.
 * Errors: CT_EINVAL (out NULL), CT_ENOMEM, CT_ECUDA. */
ct_status ct_predictor_create(uint64_t seed, ct_predictor **out);
/* Releases a predictor (synchronises its device).  NULL-safe. */
void ct_predictor_free(ct_predictor *p);

/* Labels every point of `tree` with its exact degree at `eps` and its group's
 * walk length (one traversal and one FP32 count pass of eps_graph_query),
 * then trains on the GPU (mean squared error, Adam).  *final_loss (may be NULL) receives the
 * mean standardised loss of the last 10% of the steps.  Synchronises `stream`.
 * Errors: CT_EINVAL (null pointers, eps < 0 or NaN, empty tree, predictor on
 * another device), CT_ENOMEM, CT_ECUDA. */
ct_status ct_predictor_fit(ct_predictor *p, const ct_tree *tree, double eps, const ct_fit_opts *opts,
                           ct_stream stream, double *final_loss);

/* Row capacity of the one-pass emit: ceil(predicted degree * (1 + margin)) +
 * pad (at most n); overflow arena: arena_frac * (sum of capacities) +
 * arena_min entries.  Defaults 0.5, 16, 0.25, 65536.  margin >= -1, pad >= 0,
 * arena_frac >= 0, arena_min >= 0, else CT_EINVAL. */
ct_status ct_predictor_set_capacity(ct_predictor *p, float margin, int32_t pad, float arena_frac,
                                    int64_t arena_min);

/* Order of the tree walks: 1 (default) = groups by decreasing predicted walk
 * length, 0 = by decreasing group radius (the order without a predictor).
 * Errors: CT_EINVAL. */
ct_status ct_predictor_set_order(ct_predictor *p, int32_t by_predicted_work);

/* Host copies of the parameters (CT_MLP_NPARAMS floats) and the
 * standardisation (CT_MLP_NORM floats); either pointer may be NULL.  set
 * marks the predictor fitted.  Errors: CT_EINVAL, CT_ECUDA. */
ct_status ct_predictor_get_params(const ct_predictor *p, float *params, float *norm);
ct_status ct_predictor_set_params(ct_predictor *p, const float *params, const float *norm);

/* Raw (unstandardised) features of every point of `tree` at `eps`: device
 * fp32 [n x CT_MLP_IN], 16-byte aligned, row i for the point at tree
 * position i (the order of ct_tree_export's leaf_pts).
 * Errors: CT_EINVAL, CT_ENOMEM, CT_ECUDA. */
ct_status ct_predictor_features(const ct_tree *tree, double eps, float *x, ct_stream stream);

/* Predicted degree and group walk length of every point (device fp32 [n]
 * each, by original index; either may be NULL).  Requires a fitted
 * predictor.  Errors: CT_EINVAL, CT_ENOMEM, CT_ECUDA. */
ct_status ct_predictor_predict(const ct_predictor *p, const ct_tree *tree, double eps, float *degree,
                               float *walk, ct_stream stream);

/* The perceptron itself, for checking (device buffers):
 * ct_mlp_loss_grad: loss = (1/n) sum over samples and both outputs of
 *   (y - t)^2 for x [n x 16], t [n x 2]; grad [CT_MLP_NPARAMS] is overwritten
 *   with d loss / d params (fp32 kernels); *loss (host, may be NULL) gets the
 *   loss.  Synchronises `stream`.
 * ct_mlp_forward_f16: y [n x 2] = forward pass with the parameters rounded
 *   to fp16 and fp32 sums (the inference kernel).
 * Errors: CT_EINVAL (null pointers, n < 0), CT_ENOMEM, CT_ECUDA. */
ct_status ct_mlp_loss_grad(const float *params, const float *x, const float *t, int64_t n, float *grad,
                           double *loss, ct_stream stream);
ct_status ct_mlp_forward_f16(const float *params, const float *x, int64_t n, float *y, ct_stream stream);

/* Stage timing.  When enabled, every later ct_build / eps_graph_query call
 * records a CUDA event pair around each of its stages on the caller's stream
 * and adds the elapsed device time to a process-wide table (stage name ->
 * total milliseconds, calls).  ct_profile_count() snapshots the table's names;
 * ct_profile_entry(i, ...) reads entry i of that snapshot (the name stays
 * valid until the next ct_profile_count).  Timing costs a few microseconds of
 * host time per stage. */
void ct_profile_enable(int32_t on);
void ct_profile_reset(void);
int32_t ct_profile_count(void);
ct_status ct_profile_entry(int32_t i, const char **name, double *total_ms, int64_t *calls);

/* Number of kernels this library has launched in this process so far. */
int64_t ct_kernel_launches(void);

/* Diagnostic for tests (the paper has none): while `rows` is set, every
 * count pass of later queries (L2, FP32 and tensor-core tiles) appends the
 * CSR rows of both ends of each pair it decides by the pinned FP64 sum --
 * the pairs nearest eps -- to rows (device int32[cap]), counting them in
 * *count (device uint64, zeroed by the caller; entries past cap are counted,
 * not written).  Process-wide; rows = NULL turns it off.  Synchronises the
 * device.  Errors: CT_EINVAL (rows without count, cap < 0), CT_ECUDA. */
ct_status ct_debug_guard_rows(int32_t *rows, uint64_t *count, int64_t cap);

/* Tensor-core self-test (a diagnostic; the paper has none): D = A * B^T for
 * A (128 x 128) and B (32 x 128) 16-bit row-major device matrices (fp16 = 0:
 * bf16, 1: fp16; both the same type) and D (128 x 32) fp32 row-major device
 * output, through one tcgen05 kind::f16 MMA chain with the accumulator in
 * tensor memory -- the primitive of the precision-1 leaf filter (fp16).
 * Synchronises `stream`.  CT_EINVAL for a NULL pointer or fp16 outside
 * {0, 1}; CT_ETIMEOUT if the bounded wait for the MMA's completion gives up. */
ct_status ct_selftest_tc_gemm(const void *A, const void *B, int32_t fp16, float *D, ct_stream stream);

/* The same self-test with the MMA withheld (a test of the failure path: no
 * MMA and no commit are issued, so the bounded wait for the completion runs
 * out, about a second): returns CT_ETIMEOUT and leaves the context usable. */
ct_status ct_selftest_tc_timeout(ct_stream stream);

/* Host-side fault injection for tests: the k-th next device allocation made
 * by the library (k >= 1, counted process-wide) fails as an out-of-memory
 * error would (the call returns CT_ENOMEM); k = 0 turns it off.
 * Errors: CT_EINVAL (k < 0). */
ct_status ct_debug_fail_alloc(int64_t k);

/* Bytes of the current device's default memory pool in use (the pool the
 * library allocates from), after synchronising the device: a test's check
 * that a failed call leaked nothing.  Errors: CT_EINVAL, CT_ECUDA. */
ct_status ct_debug_pool_used(uint64_t *bytes);

/* Test hook: the memory budget, in bytes, of the learned form's one-pass
 * buffers (the capacity region and the overflow arena), process-wide, in
 * place of the default -- a third of the free device memory; 0 restores the
 * default.  Predicted capacities that need more are scaled down to the budget
 * (entries past a row's capacity go to the arena, rows past the arena are
 * emitted again exactly); a budget below the arena's minimum takes the
 * two-pass emit.  Errors: CT_EINVAL (bytes < 0). */
ct_status ct_debug_capacity_budget(int64_t bytes);

/* Thread-local message for the last non-OK status of this thread. */
const char *ct_last_error(void);

/* Library version string. */
const char *ct_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CTGRAPH_H */
