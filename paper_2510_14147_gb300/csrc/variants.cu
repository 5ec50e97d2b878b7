// variants.cu -- query forms that leave the output unchanged: the tensor-core
// filter, the learned one-pass emit and the many-cloud batch.
#include <vector>

#include "mlp.cuh"
#include "query.cuh"

namespace ct {

void query_predicted(const ct_tree *t, const QParams &qp, const void *predictor, int precision,
                     cudaStream_t s, QueryOut &out);

// Many clouds: edit-distance clouds one at a time; L2 clouds in batches of up
// to kBatchClouds that share every launch (items of all clouds in one grid).
void query_batched(int n_clouds, const ct_tree *const *trees, const QParams *qps, const ct_query_opts *opts,
                   cudaStream_t s, QueryOut *outs) {
    const ct_predictor *P = opts->use_predictor ? static_cast<const ct_predictor *>(opts->predictor) : nullptr;
    if (P && !P->fitted) CT_FAIL(CT_EINVAL, "the predictor has not been fitted");
    std::vector<int> l2;
    for (int c = 0; c < n_clouds; ++c)
        if (P && P->device != trees[c]->device) CT_FAIL(CT_EINVAL, "predictor and tree live on different devices");
    for (int c = 0; c < n_clouds; ++c) {
        if (trees[c]->metric == CT_L2_F32) {
            l2.push_back(c);
        } else if (P) {
            query_predicted(trees[c], qps[c], P, opts->precision, s, outs[c]);
        } else {
            query_plain(trees[c], qps[c], s, outs[c]);
        }
    }
    for (size_t b = 0; b < l2.size(); b += kBatchClouds) {
        const int C = (int)std::min<size_t>(kBatchClouds, l2.size() - b);
        std::vector<const ct_tree *> ts(C);
        std::vector<QParams> qs(C);
        std::vector<QueryOut> os(C);
        for (int i = 0; i < C; ++i) {
            ts[i] = trees[l2[b + i]];
            qs[i] = qps[l2[b + i]];
        }
        query_multi(C, ts.data(), qs.data(), s, os.data(), opts->precision, P, nullptr);
        for (int i = 0; i < C; ++i) outs[l2[b + i]] = std::move(os[i]);
    }
}

namespace {
void release(QueryOut &q, cudaStream_t s) {
    if (!q.shared) {
        dfree(q.row_ptr, s);
        dfree(q.col, s);
        dfree(q.dist, s);
    }
    q = QueryOut();
}
}  // namespace

// Autotuner: for every row-length class present among the L2 clouds, times
// the whole batched query of that class's clouds with each candidate (count
// kernel x work-item length) and keeps the fastest for precision 2.
void autotune(int n_clouds, const ct_tree *const *trees, const QParams *qps, const ct_query_opts *opts,
              cudaStream_t s, int32_t *choices) {
    static const LeafChoice cands[] = {{0, 512}, {0, 256}, {1, 512}, {1, 256}};
    ct_query_opts o = *opts;
    o.precision = 2;
    cudaEvent_t e0, e1;
    CT_CHECK_CUDA(cudaEventCreate(&e0));
    CT_CHECK_CUDA(cudaEventCreate(&e1));
    struct Ev {
        cudaEvent_t a, b;
        ~Ev() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } ev{e0, e1};
    for (int cls = 0; cls < kDpClasses; ++cls) {
        std::vector<const ct_tree *> ts;
        std::vector<QParams> qs;
        for (int c = 0; c < n_clouds; ++c)
            if (trees[c]->metric == CT_L2_F32 && trees[c]->dp <= 128 && dp_class(trees[c]->dp) == cls) {
                ts.push_back(trees[c]);
                qs.push_back(qps[c]);
            }
        if (ts.empty()) continue;
        float best = 1e30f;
        LeafChoice pick = cands[0];
        for (const LeafChoice &cd : cands) {
            tune_set(cls, cd);
            std::vector<QueryOut> outs(ts.size());
            for (int rep = 0; rep < 2; ++rep) {  // the first run warms up
                CT_CHECK_CUDA(cudaEventRecord(ev.a, s));
                query_batched((int)ts.size(), ts.data(), qs.data(), &o, s, outs.data());
                CT_CHECK_CUDA(cudaEventRecord(ev.b, s));
                for (auto &q : outs) release(q, s);
            }
            CT_CHECK_CUDA(cudaEventSynchronize(ev.b));
            float ms = 0.f;
            CT_CHECK_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
            if (ms < best) {
                best = ms;
                pick = cd;
            }
        }
        tune_set(cls, pick);
    }
    if (choices)
        for (int c = 0; c < n_clouds; ++c) choices[c] = leaf_choice(trees[c], 2).use_tc;
}

}  // namespace ct
