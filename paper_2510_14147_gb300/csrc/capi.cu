// capi.cu -- the C-ABI of include/ctgraph.h: argument checks, status codes,
// ownership of trees and CSR outputs.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "mlp.cuh"
#include "query.cuh"

namespace ct {
ct_tree *build_tree(const ct_points *pts, int zeta, int root, cudaStream_t s);
void free_tree(ct_tree *t);
void query_tc(const ct_tree *t, const QParams &qp, cudaStream_t s, QueryOut &out);
void query_predicted(const ct_tree *t, const QParams &qp, const void *predictor, int precision,
                     cudaStream_t s, QueryOut &out);
void query_batched(int n_clouds, const ct_tree *const *trees, const QParams *qps, const ct_query_opts *opts,
                   cudaStream_t s, QueryOut *outs);
void autotune(int n_clouds, const ct_tree *const *trees, const QParams *qps, const ct_query_opts *opts,
              cudaStream_t s, int32_t *choices);
void degrees_noalloc(const ct_tree *t, const QParams &qp, int32_t *degrees, cudaStream_t s);
void tc_selftest(const void *A, const void *B, int fp16, float *D, cudaStream_t s, int withhold);
void save_tree(const ct_tree *t, const char *path);
ct_tree *load_tree(const char *path, cudaStream_t s);
void sweep_filter(const ct_tree *t, const QParams &qs, const QParams &qd, const QueryOut &src, cudaStream_t s,
                  QueryOut &out);
void set_guard_rows(int32_t *rows, unsigned long long *count, int64_t cap);
void landmark_query(const ct_points *pts, const int64_t *centres, int m, double eps, int zeta,
                    const ct_query_opts *opts, cudaStream_t s, QueryOut &out, ct_landmark_info *info);
}  // namespace ct

namespace {

struct CsrPriv {
    cudaStream_t stream;
    ct_query_stats stats;
    std::shared_ptr<ct::SharedBlocks> shared;  // batch allocations this CSR views (or null)
};

template <class F>
ct_status guarded(F &&f) {
    try {
        f();
        return CT_OK;
    } catch (const ct::Error &e) {
        return e.st;
    } catch (const std::bad_alloc &) {
        ct::set_error("host allocation failed");
        return CT_ENOMEM;
    } catch (...) {
        ct::set_error("unexpected internal error");
        return CT_ECUDA;
    }
}

void check_device(const ct_tree *t) {
    int dev = -1;
    CT_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev != t->device) CT_FAIL(CT_EINVAL, "tree lives on device %d, current device is %d", t->device, dev);
}

ct_query_opts default_query_opts() {
    ct_query_opts o;
    std::memset(&o, 0, sizeof(o));
    return o;
}

void validate_query(const ct_tree *tree, double eps, const ct_query_opts &o) {
    if (!tree) CT_FAIL(CT_EINVAL, "tree is NULL");
    if (!(eps >= 0.0)) CT_FAIL(CT_EINVAL, "eps must be >= 0 (got %g)", eps);
    if (o.precision < 0 || o.precision > 2) CT_FAIL(CT_EINVAL, "precision must be 0, 1 or 2");
    if (o.precision == 1 && tree->metric != CT_L2_F32)
        CT_FAIL(CT_EINVAL, "the tensor-core filter applies to L2 trees only");
    if (o.use_predictor && !o.predictor) CT_FAIL(CT_EINVAL, "use_predictor set without a predictor");
    if (o.include_self != 0 && o.include_self != 1) CT_FAIL(CT_EINVAL, "include_self must be 0 or 1");
    if (o.upper_triangle != 0 && o.upper_triangle != 1) CT_FAIL(CT_EINVAL, "upper_triangle must be 0 or 1");
}

void fill_csr(ct_csr *out, int64_t n, ct::QueryOut &q, cudaStream_t s) {
    CsrPriv *p = new CsrPriv();
    p->stream = s;
    p->stats = q.stats;
    p->shared = q.shared;
    out->n_rows = n;
    out->nnz = q.nnz;
    out->row_ptr = q.row_ptr;
    out->col = q.col;
    out->dist = q.dist;
    out->priv = p;
}

void release_query_out(ct::QueryOut &q, cudaStream_t s) {
    if (!q.shared) {
        ct::dfree(q.row_ptr, s);
        ct::dfree(q.col, s);
        ct::dfree(q.dist, s);
    }
    q.shared.reset();
    q.row_ptr = nullptr;
    q.col = nullptr;
    q.dist = nullptr;
}

}  // namespace

extern "C" {

ct_status ct_build(const ct_points *points, const ct_build_opts *opts, ct_stream stream, ct_tree **out) {
    if (out) *out = nullptr;
    return guarded([&] {
        if (!points || !out) CT_FAIL(CT_EINVAL, "points and out must not be NULL");
        const ct_points &p = *points;
        if (p.n < 0) CT_FAIL(CT_EINVAL, "n must be >= 0");
        if (p.n >= 0x7f7f7f00LL) CT_FAIL(CT_EOVERFLOW, "n = %lld is above the supported limit", (long long)p.n);
        if (p.metric == CT_L2_F32) {
            if (p.dim < 1 || p.dim > 4096) CT_FAIL(CT_EINVAL, "dim must be in [1, 4096] (got %d)", p.dim);
            if (p.n > 0 && !p.data) CT_FAIL(CT_EINVAL, "data is NULL");
            if ((double)p.n * (double)((p.dim + 3) / 4 * 4) > 4.0e9 * 4)
                CT_FAIL(CT_EOVERFLOW, "n * dim too large");
        } else if (p.metric == CT_LEVENSHTEIN_U8) {
            if (p.n > 0 && (!p.data || !p.offsets)) CT_FAIL(CT_EINVAL, "data and offsets must not be NULL");
        } else if (p.metric == CT_HAMMING_B1) {
            if (p.dim < 1 || p.dim > 4096) CT_FAIL(CT_EINVAL, "dim must be in [1, 4096] bits (got %d)", p.dim);
            if (p.n > 0 && !p.data) CT_FAIL(CT_EINVAL, "data is NULL");
        } else {
            CT_FAIL(CT_EINVAL, "unknown metric %d", p.metric);
        }
        int zeta = opts && opts->leaf_size > 0 ? opts->leaf_size : 32;
        int root = opts ? opts->root : 0;
        if (p.n > 0 && (root < 0 || root >= p.n)) CT_FAIL(CT_EINVAL, "root %d out of range", root);
        ct::g_launches = 0;
        *out = ct::build_tree(&p, zeta, root, (cudaStream_t)stream);
    });
}

ct_status eps_graph_query(const ct_tree *tree, double eps, const ct_query_opts *opts, ct_stream stream,
                          ct_csr *out) {
    if (out) std::memset(out, 0, sizeof(*out));
    cudaStream_t s = (cudaStream_t)stream;
    ct::QueryOut q;
    ct_status st = guarded([&] {
        if (!out) CT_FAIL(CT_EINVAL, "out is NULL");
        ct_query_opts o = opts ? *opts : default_query_opts();
        validate_query(tree, eps, o);
        check_device(tree);
        ct::g_launches = 0;
        ct::QParams qp = ct::make_qparams(tree, eps, o.include_self);
        qp.half = o.upper_triangle;
        if (o.use_predictor)
            ct::query_predicted(tree, qp, o.predictor, o.precision, s, q);
        else
            ct::query_multi(1, &tree, &qp, s, &q, o.precision, nullptr, nullptr);
        q.stats.kernel_launches = ct::g_launches;
        fill_csr(out, tree->n, q, s);
    });
    if (st != CT_OK) {
        release_query_out(q, s);
        if (out) std::memset(out, 0, sizeof(*out));
    }
    return st;
}

ct_status eps_graph_query_sweep(const ct_tree *tree, int32_t n_eps, const double *eps, const ct_query_opts *opts,
                                ct_stream stream, ct_csr *outs) {
    if (outs && n_eps > 0) std::memset(outs, 0, sizeof(ct_csr) * (size_t)n_eps);
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<ct::QueryOut> q((size_t)(n_eps > 0 ? n_eps : 0));
    ct_status st = guarded([&] {
        if (n_eps < 0) CT_FAIL(CT_EINVAL, "n_eps must be >= 0");
        if (n_eps == 0) return;
        if (!eps || !outs) CT_FAIL(CT_EINVAL, "eps and outs must not be NULL");
        ct_query_opts o = opts ? *opts : default_query_opts();
        for (int k = 0; k < n_eps; ++k) validate_query(tree, eps[k], o);
        check_device(tree);
        // radii in decreasing order; equal radii keep their input order
        std::vector<int> ord((size_t)n_eps);
        for (int k = 0; k < n_eps; ++k) ord[k] = k;
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return eps[a] > eps[b]; });
        std::vector<ct::QParams> qps((size_t)n_eps);
        for (int k = 0; k < n_eps; ++k) {
            qps[k] = ct::make_qparams(tree, eps[k], o.include_self);
            qps[k].half = o.upper_triangle;
        }
        ct::g_launches = 0;
        const int top = ord[0];
        if (o.use_predictor)
            ct::query_predicted(tree, qps[top], o.predictor, o.precision, s, q[top]);
        else
            ct::query_multi(1, &tree, &qps[top], s, &q[top], o.precision, nullptr, nullptr);
        q[top].stats.kernel_launches = ct::g_launches;
        for (size_t i = 1; i < ord.size(); ++i) {
            const int a = ord[i - 1], b = ord[i];
            ct::g_launches = 0;
            ct::sweep_filter(tree, qps[a], qps[b], q[a], s, q[b]);
            q[b].stats.kernel_launches = ct::g_launches;
        }
        for (int k = 0; k < n_eps; ++k) {
            fill_csr(&outs[k], tree->n, q[k], s);
            q[k] = ct::QueryOut();
        }
    });
    if (st != CT_OK) {
        for (auto &x : q) release_query_out(x, s);
        if (outs && n_eps > 0) std::memset(outs, 0, sizeof(ct_csr) * (size_t)n_eps);
    }
    return st;
}

struct ct_plan {
    ct::PlanImpl *impl;
};

ct_status ct_plan_create(int32_t n_clouds, const ct_tree *const *trees, const double *eps, const ct_query_opts *opts,
                         float margin, int32_t use_graph, ct_stream stream, ct_plan **out) {
    if (out) *out = nullptr;
    return guarded([&] {
        if (!out || !trees || !eps) CT_FAIL(CT_EINVAL, "trees, eps and out must not be NULL");
        if (n_clouds < 1 || n_clouds > ct::kBatchClouds)
            CT_FAIL(CT_EINVAL, "a plan takes 1 to %d clouds (got %d)", ct::kBatchClouds, n_clouds);
        if (!(margin >= 0.0f) || margin > 100.0f) CT_FAIL(CT_EINVAL, "margin must be in [0, 100]");
        ct_query_opts o = opts ? *opts : default_query_opts();
        std::vector<ct::QParams> qps((size_t)n_clouds);
        for (int c = 0; c < n_clouds; ++c) {
            validate_query(trees[c], eps[c], o);
            check_device(trees[c]);
            if (trees[c]->metric != CT_L2_F32) CT_FAIL(CT_EINVAL, "plans take L2 trees only");
            qps[c] = ct::make_qparams(trees[c], eps[c], o.include_self);
            qps[c].half = o.upper_triangle;
        }
        const ct_predictor *P = o.use_predictor ? static_cast<const ct_predictor *>(o.predictor) : nullptr;
        ct::g_launches = 0;
        std::unique_ptr<ct_plan> h(new ct_plan{nullptr});
        h->impl = ct::plan_create(n_clouds, trees, qps.data(), o.precision, P, margin, use_graph != 0,
                                  (cudaStream_t)stream);
        *out = h.release();
    });
}

ct_status ct_plan_launch(ct_plan *plan, ct_stream stream) {
    return guarded([&] {
        if (!plan || !plan->impl) CT_FAIL(CT_EINVAL, "plan is NULL");
        ct::g_launches = 0;
        ct::plan_launch(plan->impl, (cudaStream_t)stream);
    });
}

ct_status ct_plan_result(ct_plan *plan, ct_stream stream, ct_csr *outs) {
    cudaStream_t s = (cudaStream_t)stream;
    const int C = plan && plan->impl ? ct::plan_clouds(plan->impl) : 0;
    if (outs && C > 0) std::memset(outs, 0, sizeof(ct_csr) * (size_t)C);
    ct_status rs = CT_OK;
    ct_status st = guarded([&] {
        if (!plan || !plan->impl || !outs) CT_FAIL(CT_EINVAL, "plan and outs must not be NULL");
        std::vector<ct::QueryOut> q((size_t)C);
        rs = ct::plan_result(plan->impl, s, q.data());
        if (rs != CT_OK) return;
        const ct::PlanImpl *pi = plan->impl;
        (void)pi;
        for (int c = 0; c < C; ++c) fill_csr(&outs[c], ct::plan_rows(plan->impl, c), q[c], s);
    });
    if (st == CT_OK) st = rs;
    if (st != CT_OK && outs && C > 0) {
        for (int c = 0; c < C; ++c) csr_free(&outs[c]);
    }
    return st;
}

ct_status ct_plan_set_wait(ct_plan *plan, int32_t withhold_producers, int32_t max_polls) {
    return guarded([&] {
        if (!plan || !plan->impl) CT_FAIL(CT_EINVAL, "plan is NULL");
        if (max_polls < 1) CT_FAIL(CT_EINVAL, "max_polls must be >= 1");
        ct::plan_set_wait(plan->impl, withhold_producers, max_polls);
    });
}

void ct_plan_free(ct_plan *plan) {
    if (!plan) return;
    ct::plan_free(plan->impl);
    delete plan;
}

ct_status eps_graph_query_landmark(const ct_points *points, const int64_t *centres, int32_t m, double eps,
                                  const ct_build_opts *bopts, const ct_query_opts *qopts, ct_stream stream,
                                  ct_csr *out, ct_landmark_info *info) {
    if (out) std::memset(out, 0, sizeof(*out));
    if (info) std::memset(info, 0, sizeof(*info));
    cudaStream_t s = (cudaStream_t)stream;
    ct::QueryOut q;
    ct_status st = guarded([&] {
        if (!points || !out || (m > 0 && !centres)) CT_FAIL(CT_EINVAL, "points, centres and out must not be NULL");
        const ct_points &p = *points;
        if (p.n < 0 || p.n >= 0x7f7f7f00LL) CT_FAIL(CT_EINVAL, "bad n");
        if (p.metric != CT_L2_F32 && p.metric != CT_HAMMING_B1)
            CT_FAIL(CT_EUNSUPPORTED, "the landmark form takes L2 points or Hamming rows");
        if (p.dim < 1 || p.dim > 4096) CT_FAIL(CT_EINVAL, "dim must be in [1, 4096]");
        if (p.n > 0 && !p.data) CT_FAIL(CT_EINVAL, "data is NULL");
        if (!(eps >= 0.0)) CT_FAIL(CT_EINVAL, "eps must be >= 0 (got %g)", eps);
        ct_query_opts o = qopts ? *qopts : default_query_opts();
        if (o.precision < 0 || o.precision > 2) CT_FAIL(CT_EINVAL, "precision must be 0, 1 or 2");
        if (o.precision == 1 && p.metric != CT_L2_F32) CT_FAIL(CT_EINVAL, "the tensor-core filter applies to L2 only");
        if (o.use_predictor && !o.predictor) CT_FAIL(CT_EINVAL, "use_predictor set without a predictor");
        if (o.include_self != 0 && o.include_self != 1) CT_FAIL(CT_EINVAL, "include_self must be 0 or 1");
        if (o.upper_triangle != 0 && o.upper_triangle != 1) CT_FAIL(CT_EINVAL, "upper_triangle must be 0 or 1");
        const int zeta = bopts && bopts->leaf_size > 0 ? bopts->leaf_size : 32;
        ct::g_launches = 0;
        ct::landmark_query(&p, centres, m, eps, zeta, &o, s, q, info);
        q.stats.kernel_launches = ct::g_launches;
        fill_csr(out, p.n, q, s);
    });
    if (st != CT_OK) {
        release_query_out(q, s);
        if (out) std::memset(out, 0, sizeof(*out));
    }
    return st;
}

ct_status ct_tree_save(const ct_tree *tree, const char *path) {
    return guarded([&] {
        if (!tree || !path) CT_FAIL(CT_EINVAL, "tree and path must not be NULL");
        check_device(tree);
        ct::save_tree(tree, path);
    });
}

ct_status ct_tree_load(const char *path, ct_stream stream, ct_tree **out) {
    if (out) *out = nullptr;
    return guarded([&] {
        if (!path || !out) CT_FAIL(CT_EINVAL, "path and out must not be NULL");
        ct::g_launches = 0;
        *out = ct::load_tree(path, (cudaStream_t)stream);
    });
}

ct_status eps_graph_query_batched(int32_t n_clouds, const ct_tree *const *trees, const double *eps,
                                  const ct_query_opts *opts, ct_stream stream, ct_csr *outs) {
    if (outs && n_clouds > 0) std::memset(outs, 0, sizeof(ct_csr) * (size_t)n_clouds);
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<ct::QueryOut> q((size_t)(n_clouds > 0 ? n_clouds : 0));
    ct_status st = guarded([&] {
        if (n_clouds < 0) CT_FAIL(CT_EINVAL, "n_clouds must be >= 0");
        if (n_clouds == 0) return;
        if (!trees || !eps || !outs) CT_FAIL(CT_EINVAL, "trees, eps and outs must not be NULL");
        ct_query_opts o = opts ? *opts : default_query_opts();
        std::vector<ct::QParams> qps((size_t)n_clouds);
        for (int c = 0; c < n_clouds; ++c) {
            validate_query(trees[c], eps[c], o);
            check_device(trees[c]);
            qps[c] = ct::make_qparams(trees[c], eps[c], o.include_self);
            qps[c].half = o.upper_triangle;
        }
        ct::g_launches = 0;
        ct::query_batched(n_clouds, trees, qps.data(), &o, s, q.data());
        for (int c = 0; c < n_clouds; ++c) {
            q[c].stats.kernel_launches = ct::g_launches;
            fill_csr(&outs[c], trees[c]->n, q[c], s);
            q[c] = ct::QueryOut();
        }
    });
    if (st != CT_OK) {
        for (auto &x : q) release_query_out(x, s);
        if (outs && n_clouds > 0) {
            for (int c = 0; c < n_clouds; ++c) csr_free(&outs[c]);
        }
    }
    return st;
}

ct_status ct_autotune(int32_t n_clouds, const ct_tree *const *trees, const double *eps, const ct_query_opts *opts,
                      ct_stream stream, int32_t *choices) {
    return guarded([&] {
        if (n_clouds < 0) CT_FAIL(CT_EINVAL, "n_clouds must be >= 0");
        if (n_clouds == 0) return;
        if (!trees || !eps) CT_FAIL(CT_EINVAL, "trees and eps must not be NULL");
        ct_query_opts o = opts ? *opts : default_query_opts();
        std::vector<ct::QParams> qps((size_t)n_clouds);
        for (int c = 0; c < n_clouds; ++c) {
            validate_query(trees[c], eps[c], o);
            check_device(trees[c]);
            qps[c] = ct::make_qparams(trees[c], eps[c], o.include_self);
            qps[c].half = o.upper_triangle;
        }
        ct::autotune(n_clouds, trees, qps.data(), &o, (cudaStream_t)stream, choices);
    });
}

void ct_autotune_reset(void) { ct::tune_reset(); }

ct_status eps_graph_degrees_noalloc(const ct_tree *tree, double eps, int32_t include_self, int32_t *degrees,
                                    ct_stream stream) {
    return guarded([&] {
        if (!tree) CT_FAIL(CT_EINVAL, "tree is NULL");
        if (tree->n > 0 && !degrees) CT_FAIL(CT_EINVAL, "degrees is NULL");
        if (!(eps >= 0.0)) CT_FAIL(CT_EINVAL, "eps must be >= 0 (got %g)", eps);
        if (include_self != 0 && include_self != 1) CT_FAIL(CT_EINVAL, "include_self must be 0 or 1");
        check_device(tree);
        ct::QParams qp = ct::make_qparams(tree, eps, include_self);
        ct::degrees_noalloc(tree, qp, degrees, (cudaStream_t)stream);
    });
}

ct_status ct_debug_guard_rows(int32_t *rows, uint64_t *count, int64_t cap) {
    return guarded([&] {
        if (rows && (!count || cap < 0)) CT_FAIL(CT_EINVAL, "count must be given and cap >= 0");
        ct::set_guard_rows(rows, reinterpret_cast<unsigned long long *>(count), cap);
    });
}

ct_status ct_selftest_tc_gemm(const void *A, const void *B, int32_t fp16, float *D, ct_stream stream) {
    return guarded([&] {
        if (!A || !B || !D) CT_FAIL(CT_EINVAL, "NULL argument");
        if (fp16 != 0 && fp16 != 1) CT_FAIL(CT_EINVAL, "fp16 must be 0 or 1");
        ct::tc_selftest(A, B, fp16, D, (cudaStream_t)stream, 0);
    });
}

ct_status ct_selftest_tc_timeout(ct_stream stream) {
    cudaStream_t s = (cudaStream_t)stream;
    return guarded([&] {
        ct::DBuf<uint16_t> a(128 * 128, s), b(32 * 128, s);
        ct::DBuf<float> d(128 * 32, s);
        CT_CHECK_CUDA(cudaMemsetAsync(a.p, 0, 128 * 128 * sizeof(uint16_t), s));
        CT_CHECK_CUDA(cudaMemsetAsync(b.p, 0, 32 * 128 * sizeof(uint16_t), s));
        ct::tc_selftest(a.p, b.p, 1, d.p, s, 1);
    });
}

ct_status ct_debug_fail_alloc(int64_t k) {
    return guarded([&] {
        if (k < 0) CT_FAIL(CT_EINVAL, "k must be >= 0");
        ct::set_fail_alloc(k);
    });
}

ct_status ct_debug_capacity_budget(int64_t bytes) {
    return guarded([&] {
        if (bytes < 0) CT_FAIL(CT_EINVAL, "bytes must be >= 0");
        ct::set_capacity_budget(bytes);
    });
}

ct_status ct_debug_pool_used(uint64_t *bytes) {
    return guarded([&] {
        if (!bytes) CT_FAIL(CT_EINVAL, "bytes is NULL");
        int dev = 0;
        CT_CHECK_CUDA(cudaGetDevice(&dev));
        CT_CHECK_CUDA(cudaDeviceSynchronize());
        cudaMemPool_t pool;
        CT_CHECK_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
        uint64_t used = 0;
        CT_CHECK_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
        *bytes = used;
    });
}

void csr_free(ct_csr *csr) {
    if (!csr) return;
    CsrPriv *p = (CsrPriv *)csr->priv;
    cudaStream_t s = p ? p->stream : (cudaStream_t)0;
    if (!(p && p->shared)) {  // a batch's views are released with its last CSR
        if (csr->row_ptr) cudaFreeAsync(csr->row_ptr, s);
        if (csr->col) cudaFreeAsync(csr->col, s);
        if (csr->dist) cudaFreeAsync(csr->dist, s);
    }
    delete p;
    std::memset(csr, 0, sizeof(*csr));
}

ct_status ct_csr_stats(const ct_csr *csr, ct_query_stats *out) {
    return guarded([&] {
        if (!csr || !out) CT_FAIL(CT_EINVAL, "csr and out must not be NULL");
        if (!csr->priv) CT_FAIL(CT_EINVAL, "csr holds no query");
        *out = ((CsrPriv *)csr->priv)->stats;
    });
}

void ct_tree_free(ct_tree *tree) { ct::free_tree(tree); }

ct_status ct_tree_shape(const ct_tree *tree, int64_t *n_nodes, int64_t *n_points) {
    return guarded([&] {
        if (!tree || !n_nodes || !n_points) CT_FAIL(CT_EINVAL, "NULL argument");
        *n_nodes = tree->n_nodes;
        *n_points = tree->n;
    });
}

ct_status ct_tree_export(const ct_tree *tree, int64_t *center, double *radius, int32_t *level,
                         int64_t *child_begin, int64_t *child_count, int64_t *pts_begin, int64_t *pts_count,
                         int64_t *leaf_pts) {
    return guarded([&] {
        if (!tree) CT_FAIL(CT_EINVAL, "tree is NULL");
        const int N = tree->n_nodes;
        const int64_t n = tree->n;
        if (N > 0 && (!center || !radius || !level || !child_begin || !child_count || !pts_begin || !pts_count))
            CT_FAIL(CT_EINVAL, "NULL output array");
        if (n > 0 && !leaf_pts) CT_FAIL(CT_EINVAL, "NULL leaf_pts");
        check_device(tree);
        CT_CHECK_CUDA(cudaDeviceSynchronize());
        std::vector<int32_t> nb(N), nc(N), cb(N), cc(N), lv(N), perm(n);
        std::vector<float> rd(N);
        auto get = [&](void *h, const void *d, size_t bytes) {
            if (bytes) CT_CHECK_CUDA(cudaMemcpy(h, d, bytes, cudaMemcpyDeviceToHost));
        };
        get(nb.data(), tree->node_begin, N * sizeof(int32_t));
        get(nc.data(), tree->node_count, N * sizeof(int32_t));
        get(cb.data(), tree->child_begin, N * sizeof(int32_t));
        get(cc.data(), tree->child_count, N * sizeof(int32_t));
        get(lv.data(), tree->level, N * sizeof(int32_t));
        get(rd.data(), tree->radius, N * sizeof(float));
        get(perm.data(), tree->perm, n * sizeof(int32_t));
        for (int v = 0; v < N; ++v) {
            center[v] = perm[nb[v]];
            radius[v] = (double)rd[v];
            level[v] = lv[v];
            child_begin[v] = cb[v];
            child_count[v] = cc[v];
            pts_begin[v] = cc[v] == 0 ? nb[v] : 0;
            pts_count[v] = cc[v] == 0 ? nc[v] : 0;
        }
        for (int64_t i = 0; i < n; ++i) leaf_pts[i] = perm[i];
    });
}

ct_status ct_predictor_create(uint64_t seed, ct_predictor **out) {
    if (out) *out = nullptr;
    ct_predictor *p = nullptr;
    ct_status st = guarded([&] {
        if (!out) CT_FAIL(CT_EINVAL, "out is NULL");
        p = new ct_predictor();
        CT_CHECK_CUDA(cudaGetDevice(&p->device));
        ct::predictor_init(p, seed);
        *out = p;
    });
    if (st != CT_OK && p) {
        ct::predictor_release(p);
        delete p;
    }
    return st;
}

void ct_predictor_free(ct_predictor *p) {
    if (!p) return;
    ct::predictor_release(p);
    delete p;
}

namespace {
void check_predictor_device(const ct_predictor *p) {
    int dev = -1;
    CT_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev != p->device) CT_FAIL(CT_EINVAL, "predictor lives on device %d, current device is %d", p->device, dev);
}
}  // namespace

ct_status ct_predictor_fit(ct_predictor *p, const ct_tree *tree, double eps, const ct_fit_opts *opts,
                           ct_stream stream, double *final_loss) {
    return guarded([&] {
        if (!p || !tree) CT_FAIL(CT_EINVAL, "predictor and tree must not be NULL");
        if (!(eps >= 0.0)) CT_FAIL(CT_EINVAL, "eps must be >= 0 (got %g)", eps);
        if (tree->n == 0) CT_FAIL(CT_EINVAL, "cannot fit on an empty tree");
        check_device(tree);
        check_predictor_device(p);
        ct_fit_opts o;
        std::memset(&o, 0, sizeof(o));
        if (opts) o = *opts;
        if (o.include_self != 0 && o.include_self != 1) CT_FAIL(CT_EINVAL, "include_self must be 0 or 1");
        if (o.steps < 0 || o.batch < 0 || !(o.lr >= 0.f)) CT_FAIL(CT_EINVAL, "steps, batch and lr must be >= 0");
        ct::g_launches = 0;
        const double l = ct::predictor_fit(p, tree, eps, o, (cudaStream_t)stream);
        if (final_loss) *final_loss = l;
    });
}

ct_status ct_predictor_set_capacity(ct_predictor *p, float margin, int32_t pad, float arena_frac,
                                    int64_t arena_min) {
    return guarded([&] {
        if (!p) CT_FAIL(CT_EINVAL, "predictor is NULL");
        if (!(margin >= -1.0f) || pad < 0 || !(arena_frac >= 0.0f) || arena_min < 0 || !std::isfinite(margin) ||
            !std::isfinite(arena_frac))
            CT_FAIL(CT_EINVAL, "need margin >= -1, pad >= 0, arena_frac >= 0, arena_min >= 0");
        p->margin = margin;
        p->pad = pad;
        p->arena_frac = arena_frac;
        p->arena_min = arena_min;
    });
}

ct_status ct_predictor_set_order(ct_predictor *p, int32_t by_predicted_work) {
    return guarded([&] {
        if (!p) CT_FAIL(CT_EINVAL, "predictor is NULL");
        if (by_predicted_work != 0 && by_predicted_work != 1) CT_FAIL(CT_EINVAL, "by_predicted_work must be 0 or 1");
        p->order_by_work = by_predicted_work;
    });
}

ct_status ct_predictor_get_params(const ct_predictor *p, float *params, float *norm) {
    return guarded([&] {
        if (!p) CT_FAIL(CT_EINVAL, "predictor is NULL");
        check_predictor_device(p);
        if (params) {
            CT_CHECK_CUDA(cudaDeviceSynchronize());
            CT_CHECK_CUDA(cudaMemcpy(params, p->w, sizeof(float) * ct::MLP_NPARAMS, cudaMemcpyDeviceToHost));
        }
        if (norm) {
            std::memcpy(norm, p->fmean, sizeof(float) * ct::MLP_IN);
            std::memcpy(norm + ct::MLP_IN, p->fstd, sizeof(float) * ct::MLP_IN);
            std::memcpy(norm + 2 * ct::MLP_IN, p->tmean, sizeof(float) * ct::MLP_OUT);
            std::memcpy(norm + 2 * ct::MLP_IN + ct::MLP_OUT, p->tstd, sizeof(float) * ct::MLP_OUT);
        }
    });
}

ct_status ct_predictor_set_params(ct_predictor *p, const float *params, const float *norm) {
    return guarded([&] {
        if (!p) CT_FAIL(CT_EINVAL, "predictor is NULL");
        check_predictor_device(p);
        if (params) {
            CT_CHECK_CUDA(cudaDeviceSynchronize());
            CT_CHECK_CUDA(cudaMemcpy(p->w, params, sizeof(float) * ct::MLP_NPARAMS, cudaMemcpyHostToDevice));
            ct::mlp_to_half(p->w, p->wh, 0);
            CT_CHECK_CUDA(cudaDeviceSynchronize());
        }
        if (norm) {
            std::memcpy(p->fmean, norm, sizeof(float) * ct::MLP_IN);
            std::memcpy(p->fstd, norm + ct::MLP_IN, sizeof(float) * ct::MLP_IN);
            std::memcpy(p->tmean, norm + 2 * ct::MLP_IN, sizeof(float) * ct::MLP_OUT);
            std::memcpy(p->tstd, norm + 2 * ct::MLP_IN + ct::MLP_OUT, sizeof(float) * ct::MLP_OUT);
        }
        p->fitted = true;
    });
}

ct_status ct_predictor_features(const ct_tree *tree, double eps, float *x, ct_stream stream) {
    return guarded([&] {
        if (!tree) CT_FAIL(CT_EINVAL, "tree is NULL");
        if (!(eps >= 0.0)) CT_FAIL(CT_EINVAL, "eps must be >= 0 (got %g)", eps);
        if (tree->n > 0 && (!x || ((uintptr_t)x & 15))) CT_FAIL(CT_EINVAL, "x must be a 16-byte aligned device pointer");
        check_device(tree);
        ct::predictor_features(tree, eps, nullptr, x, (cudaStream_t)stream);
    });
}

ct_status ct_predictor_predict(const ct_predictor *p, const ct_tree *tree, double eps, float *degree, float *walk,
                               ct_stream stream) {
    return guarded([&] {
        if (!p || !tree) CT_FAIL(CT_EINVAL, "predictor and tree must not be NULL");
        if (!(eps >= 0.0)) CT_FAIL(CT_EINVAL, "eps must be >= 0 (got %g)", eps);
        if (!p->fitted) CT_FAIL(CT_EINVAL, "the predictor has not been fitted");
        check_device(tree);
        check_predictor_device(p);
        ct::predictor_predict(p, tree, eps, degree, walk, (cudaStream_t)stream);
    });
}

ct_status ct_mlp_loss_grad(const float *params, const float *x, const float *t, int64_t n, float *grad,
                           double *loss, ct_stream stream) {
    return guarded([&] {
        if (!params || !grad || n < 0 || (n > 0 && (!x || !t))) CT_FAIL(CT_EINVAL, "bad argument");
        cudaStream_t s = (cudaStream_t)stream;
        CT_CHECK_CUDA(cudaMemsetAsync(grad, 0, sizeof(float) * ct::MLP_NPARAMS, s));
        ct::DBuf<double> acc(1, s);
        CT_CHECK_CUDA(cudaMemsetAsync(acc.p, 0, sizeof(double), s));
        ct::mlp_accumulate_grad(params, x, t, n, (double)(n > 0 ? n : 1), grad, acc.p, s);
        double h = 0.0;
        ct::to_host(&h, acc.p, 1, s);
        if (loss) *loss = h / (double)(n > 0 ? n : 1);
    });
}

ct_status ct_mlp_forward_f16(const float *params, const float *x, int64_t n, float *y, ct_stream stream) {
    return guarded([&] {
        if (!params || n < 0 || (n > 0 && (!x || !y))) CT_FAIL(CT_EINVAL, "bad argument");
        cudaStream_t s = (cudaStream_t)stream;
        ct::DBuf<__half> wh(ct::MLP_NPARAMS, s);
        ct::mlp_to_half(params, wh.p, s);
        ct::mlp_predict(wh.p, x, n, y, s);
        CT_CHECK_CUDA(cudaStreamSynchronize(s));
    });
}

const char *ct_last_error(void) { return ct::get_error(); }

const char *ct_version(void) { return "ctgraph 0.1 (sm_103a)"; }

}  // extern "C"
