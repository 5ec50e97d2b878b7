// variants.cu -- query forms that leave the output unchanged: the tensor-core
// filter, the learned one-pass emit and the many-cloud batch.
#include "query.cuh"

namespace ct {

void query_predicted(const ct_tree *t, const QParams &qp, const void *predictor, int precision,
                     cudaStream_t s, QueryOut &out);

void query_batched(int n_clouds, const ct_tree *const *trees, const QParams *qps, const ct_query_opts *opts,
                   cudaStream_t s, QueryOut *outs) {
    for (int c = 0; c < n_clouds; ++c) {
        if (opts->use_predictor) query_predicted(trees[c], qps[c], opts->predictor, opts->precision, s, outs[c]);
        else if (opts->precision == 1) query_tc(trees[c], qps[c], s, outs[c]);
        else query_plain(trees[c], qps[c], s, outs[c]);
    }
}

}  // namespace ct
