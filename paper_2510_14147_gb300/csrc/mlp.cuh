// mlp.cuh -- the degree/work predictor (no counterpart in the paper): a
// 16 -> 64 -> 64 -> 2 multilayer perceptron with ReLU, trained on the GPU.
#pragma once

#include <cuda_fp16.h>

#include "common.cuh"

namespace ct {

constexpr int MLP_IN = 16, MLP_HID = 64, MLP_OUT = 2;
constexpr int MLP_NPARAMS = MLP_HID * MLP_IN + MLP_HID + MLP_HID * MLP_HID + MLP_HID + MLP_OUT * MLP_HID + MLP_OUT;
// offsets of the parameter blocks in the flat vector (W1, b1, W2, b2, W3, b3)
constexpr int P_W1 = 0, P_B1 = P_W1 + MLP_HID * MLP_IN, P_W2 = P_B1 + MLP_HID, P_B2 = P_W2 + MLP_HID * MLP_HID,
              P_W3 = P_B2 + MLP_HID, P_B3 = P_W3 + MLP_OUT * MLP_HID;

// Mean-squared-error gradient over n samples accumulated into grad (device,
// fp32, MLP_NPARAMS); divides by `denom`; adds the loss sum to *loss_sum.
void mlp_accumulate_grad(const float *w, const float *x, const float *t, int64_t n, double denom, float *grad,
                         double *loss_sum, cudaStream_t s);
void mlp_adam_step(float *w, float *m, float *v, float *grad, int64_t step, float lr, cudaStream_t s);
// y (n x 2) = forward(x) with fp16 weights wh and fp32 accumulation.
void mlp_predict(const __half *wh, const float *x, int64_t n, float *y, cudaStream_t s);
void mlp_to_half(const float *w, __half *wh, cudaStream_t s);

}  // namespace ct

struct ct_predictor {
    int device = 0;
    float *w = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    __half *wh = nullptr;
    int64_t step = 0;
    // feature and target standardisation (fitted on the training set)
    float fmean[ct::MLP_IN] = {0}, fstd[ct::MLP_IN] = {0};
    float tmean[ct::MLP_OUT] = {0}, tstd[ct::MLP_OUT] = {0};
    bool fitted = false;
    // capacity of a row: ceil(predicted degree * (1 + margin)) + pad; overflow
    // arena: arena_frac * (sum of capacities) + arena_min entries
    float margin = 0.5f;
    int32_t pad = 16;
    float arena_frac = 0.25f;
    int64_t arena_min = 65536;
    // walk the groups in order of decreasing predicted walk length (else by
    // decreasing group radius)
    int32_t order_by_work = 1;
};

namespace ct {
void predictor_init(ct_predictor *P, uint64_t seed);
void predictor_release(ct_predictor *P);
// Trains on the tree's exact labels; returns the mean standardised loss of
// the last tenth of the steps.
double predictor_fit(ct_predictor *P, const ct_tree *t, double eps, const ct_fit_opts &o, cudaStream_t s);
// Features of every tree position (raw when P is null, else standardised).
void predictor_features(const ct_tree *t, double eps, const ct_predictor *P, float *x, cudaStream_t s);
void predictor_predict(const ct_predictor *P, const ct_tree *t, double eps, float *pdeg, float *pvisit,
                       cudaStream_t s);
}  // namespace ct
