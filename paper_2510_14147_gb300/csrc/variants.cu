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

}  // namespace ct
