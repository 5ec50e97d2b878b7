// query.cuh -- shared declarations of the query stages.
#pragma once

#include <memory>

#include "common.cuh"

struct ct_predictor;

namespace ct {

// Decision parameters of the L2 predicate d(q, p) <= eps.
//  mode 0: fp32 decides outside the guard band |d - eps| <= 1e-3 eps; inside
//          it fp32 still decides where its error bound certifies the side of
//          eps^2, else FP64 (the pinned sequential sum);
//  mode 1: eps == 0: no edge if the fp32 sum is positive (x != y), else FP64;
//  mode 2: every pair in FP64 (eps^2 outside [2^-100, 2^100]);
//  mode 3: every pair is an edge (eps^2 above any representable sum).
struct QParams {
    double eps64 = 0, eps2_64 = 0;
    float eps_up = 0;      // eps rounded up to fp32 (traversal bound)
    float lo2 = 0, hi2 = 0;  // guard band in squared distance, rounded outwards
    float c_lo = 0, c_hi = 0;  // inside it: fp32 sums outside [c_lo, c_hi] decide alone
    int mode = 0;
    int include_self = 0;
    int lev_k = 0;         // edit distance, Hamming: floor(eps)
    int half = 0;          // upper-triangle form: each pair of two query groups evaluated once, mirrored
};

QParams make_qparams(const ct_tree *t, double eps, int include_self);

// Device allocations shared by the CSRs of one batch; released (stream
// ordered) when the last of them is released.
struct SharedBlocks {
    explicit SharedBlocks(cudaStream_t st) : s(st) {}
    ~SharedBlocks() {
        for (void *q : p)
            if (q) cudaFreeAsync(q, s);
    }
    SharedBlocks(const SharedBlocks &) = delete;
    SharedBlocks &operator=(const SharedBlocks &) = delete;
    cudaStream_t s;
    void *p[3] = {nullptr, nullptr, nullptr};
};

// Per-query output and counters of one query.  With `shared` set the three
// arrays are views into a batch's shared allocations.
struct QueryOut {
    int64_t nnz = 0;
    int64_t *row_ptr = nullptr;
    int32_t *col = nullptr;
    float *dist = nullptr;
    ct_query_stats stats{};
    std::shared_ptr<SharedBlocks> shared;
};

// The plain FP32 path (precision 0) and the edit-distance path.
void query_plain(const ct_tree *t, const QParams &qp, cudaStream_t s, QueryOut &out);
void query_tc(const ct_tree *t, const QParams &qp, cudaStream_t s, QueryOut &out);

// Learned form.  A probe collects the labels for fitting the predictor: the
// query stops after the count pass.
struct Probe {
    int32_t *deg = nullptr;     // n, by original id: degree
    int32_t *gvisit = nullptr;  // G: vertices tested by each group's walk
};
// What the predictor decided before the traversal.
struct LearnedPlan {
    DBuf<int64_t> cap_off;      // n + 1 row capacity offsets by original id
    int64_t cap_total = 0;
    int64_t arena = 0;          // overflow arena entries
    DBuf<int32_t> group_order;  // groups by decreasing predicted walk length
    bool one_pass = false;
};
// The query of C clouds (1 <= C <= 64) in shared launches: outs[c] is the
// CSR of trees[c].  Several clouds must all be L2; a probe needs C = 1.
void query_multi(int C, const ct_tree *const *trees, const QParams *qps, cudaStream_t s, QueryOut *outs,
                 int precision, const ct_predictor *P, Probe *probe);
constexpr int kBatchClouds = 64;
// Count-pass kernel (1: tensor-core tiles, 0: FP32 tiles) and work-item
// length of a cloud; autotuned per class of row length (dp <= 4, 16, 32, 64,
// 128, wider).
struct LeafChoice {
    int use_tc;
    int item_len;
};
constexpr int kDpClasses = 6;
int dp_class(int dp);
LeafChoice leaf_choice(const ct_tree *t, int precision);
void tune_set(int cls, LeafChoice c);
void tune_reset();
void learned_plan(const ct_predictor *P, int C, const ct_tree *const *trees, const QParams *qps,
                  const int64_t *rbase, const int32_t *gbase, cudaStream_t s, LearnedPlan &lp);

// Plans: a batch of L2 clouds with every buffer allocated up front, so that a
// run (one graph-capturable sequence of launches, the leaf stage one
// persistent launch over a device work queue) needs no host read-back.
struct PlanImpl;
PlanImpl *plan_create(int C, const ct_tree *const *trees, const QParams *qps, int precision,
                      const ct_predictor *pred, float margin, bool use_graph, cudaStream_t s);
void plan_launch(PlanImpl *p, cudaStream_t s);
void plan_set_wait(PlanImpl *p, int withhold, int max_polls);
int plan_clouds(const PlanImpl *p);
int64_t plan_rows(const PlanImpl *p, int c);
ct_status plan_result(PlanImpl *p, cudaStream_t s, QueryOut *outs);
void plan_free(PlanImpl *p);

// Sorts every CSR row (n rows, columns below ncols) by column, moving dist
// along.
void sort_rows(const int64_t *row_ptr, int64_t n, int64_t ncols, int32_t *col, float *dist, int64_t nnz,
               cudaStream_t s);

// Stats slots accumulated on the device.
enum { ST_TRAV = 0, ST_PAIRS, ST_GUARD, ST_RECHECK, ST_CAND, ST_OVERFLOW, ST_ERR, ST_EMIT, ST_ROWS, ST_BAND, ST_COLS, ST_N };

}  // namespace ct
