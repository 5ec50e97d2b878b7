// mlp.cu -- forward, backward and Adam kernels of the degree/work predictor
// (16 -> 64 -> 64 -> 2, ReLU, mean squared error).  The paper has no learned
// component; this predictor sizes the one-pass emit and orders work.
#include "mlp.cuh"

namespace ct {
namespace {

constexpr int SB = 64;  // samples per training block
constexpr int MT = 128; // threads per training block

struct MlpShared {
    float w[MLP_NPARAMS];
    float x[SB][MLP_IN + 1];
    float h1[SB][MLP_HID + 1];
    float h2[SB][MLP_HID + 1];
    float d2[SB][MLP_HID + 1];
    float d1[SB][MLP_HID + 1];
    float dy[SB][MLP_OUT];
    double red[MT / 32];
};

// Per block of 64 samples: forward (thread per sample), backpropagation of
// the squared error (thread per sample), then the parameter gradient summed
// over the block's samples (thread per parameter) and added to grad.
__global__ void __launch_bounds__(MT) k_mlp_grad(const float *__restrict__ w, const float *__restrict__ x,
                                                 const float *__restrict__ t, int64_t n, float inv_denom,
                                                 float *__restrict__ grad, double *__restrict__ loss_sum) {
    extern __shared__ __align__(16) unsigned char raw[];
    MlpShared &S = *reinterpret_cast<MlpShared *>(raw);
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * SB;
    for (int e = tid; e < MLP_NPARAMS; e += MT) S.w[e] = w[e];
    for (int e = tid; e < SB * MLP_IN; e += MT) {
        const int s = e / MLP_IN, k = e - s * MLP_IN;
        S.x[s][k] = base + s < n ? x[(base + s) * MLP_IN + k] : 0.f;
    }
    __syncthreads();
    double l = 0.0;
    if (tid < SB) {
        const int s = tid;
        const bool valid = base + s < n;
        const float *W1 = S.w + P_W1, *b1 = S.w + P_B1, *W2 = S.w + P_W2, *b2 = S.w + P_B2;
        const float *W3 = S.w + P_W3, *b3 = S.w + P_B3;
        for (int i = 0; i < MLP_HID; ++i) {
            float a = b1[i];
#pragma unroll
            for (int k = 0; k < MLP_IN; ++k) a = fmaf(W1[i * MLP_IN + k], S.x[s][k], a);
            S.h1[s][i] = valid ? fmaxf(a, 0.f) : 0.f;
        }
        for (int i = 0; i < MLP_HID; ++i) {
            float a = b2[i];
            for (int j = 0; j < MLP_HID; ++j) a = fmaf(W2[i * MLP_HID + j], S.h1[s][j], a);
            S.h2[s][i] = valid ? fmaxf(a, 0.f) : 0.f;
        }
        for (int o = 0; o < MLP_OUT; ++o) {
            float y = b3[o];
            for (int i = 0; i < MLP_HID; ++i) y = fmaf(W3[o * MLP_HID + i], S.h2[s][i], y);
            const float d = valid ? y - t[(base + s) * MLP_OUT + o] : 0.f;
            S.dy[s][o] = 2.f * d * inv_denom;
            l += (double)d * (double)d;
        }
        __syncwarp();
        for (int i = 0; i < MLP_HID; ++i) {
            float g = 0.f;
            for (int o = 0; o < MLP_OUT; ++o) g = fmaf(W3[o * MLP_HID + i], S.dy[s][o], g);
            S.d2[s][i] = S.h2[s][i] > 0.f ? g : 0.f;
        }
        for (int j = 0; j < MLP_HID; ++j) {
            float g = 0.f;
            for (int i = 0; i < MLP_HID; ++i) g = fmaf(W2[i * MLP_HID + j], S.d2[s][i], g);
            S.d1[s][j] = S.h1[s][j] > 0.f ? g : 0.f;
        }
    }
    __syncthreads();
    for (int e = tid; e < MLP_NPARAMS; e += MT) {
        float acc = 0.f;
        if (e < P_B1) {
            const int i = (e - P_W1) / MLP_IN, k = (e - P_W1) % MLP_IN;
            for (int s = 0; s < SB; ++s) acc = fmaf(S.d1[s][i], S.x[s][k], acc);
        } else if (e < P_W2) {
            const int i = e - P_B1;
            for (int s = 0; s < SB; ++s) acc += S.d1[s][i];
        } else if (e < P_B2) {
            const int i = (e - P_W2) / MLP_HID, j = (e - P_W2) % MLP_HID;
            for (int s = 0; s < SB; ++s) acc = fmaf(S.d2[s][i], S.h1[s][j], acc);
        } else if (e < P_W3) {
            const int i = e - P_B2;
            for (int s = 0; s < SB; ++s) acc += S.d2[s][i];
        } else if (e < P_B3) {
            const int o = (e - P_W3) / MLP_HID, i = (e - P_W3) % MLP_HID;
            for (int s = 0; s < SB; ++s) acc = fmaf(S.dy[s][o], S.h2[s][i], acc);
        } else {
            const int o = e - P_B3;
            for (int s = 0; s < SB; ++s) acc += S.dy[s][o];
        }
        if (acc != 0.f) atomicAdd(grad + e, acc);
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((tid & 31) == 0) S.red[tid >> 5] = l;
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (int i = 0; i < MT / 32; ++i) sum += S.red[i];
        if (loss_sum && sum != 0.0) atomicAdd(loss_sum, sum);
    }
}

// Adam (beta1 0.9, beta2 0.999, eps 1e-8); clears the gradient.
__global__ void k_adam(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v, float *__restrict__ g,
                       float lr, float c1, float c2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= MLP_NPARAMS) return;
    const float gr = g[e];
    const float mm = 0.9f * m[e] + 0.1f * gr;
    const float vv = 0.999f * v[e] + 0.001f * gr * gr;
    m[e] = mm;
    v[e] = vv;
    w[e] -= lr * (mm * c1) / (sqrtf(vv * c2) + 1e-8f);
    g[e] = 0.f;
}

__global__ void k_to_half(const float *__restrict__ w, __half *__restrict__ wh) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < MLP_NPARAMS) wh[e] = __float2half_rn(w[e]);
}

// Inference: thread per sample, fp16 weights in shared memory, fp32 sums.
__global__ void __launch_bounds__(128) k_mlp_predict(const __half *__restrict__ wh, const float *__restrict__ x,
                                                     int64_t n, float *__restrict__ y) {
    __shared__ __half sw[MLP_NPARAMS];
    for (int e = threadIdx.x; e < MLP_NPARAMS; e += blockDim.x) sw[e] = wh[e];
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float xi[MLP_IN], h1[MLP_HID];
#pragma unroll
    for (int k = 0; k < MLP_IN; ++k) xi[k] = x[s * MLP_IN + k];
#pragma unroll
    for (int i = 0; i < MLP_HID; ++i) {
        float a = __half2float(sw[P_B1 + i]);
#pragma unroll
        for (int k = 0; k < MLP_IN; ++k) a = fmaf(__half2float(sw[P_W1 + i * MLP_IN + k]), xi[k], a);
        h1[i] = fmaxf(a, 0.f);
    }
    float y0 = __half2float(sw[P_B3]), y1 = __half2float(sw[P_B3 + 1]);
#pragma unroll 1
    for (int i = 0; i < MLP_HID; ++i) {
        float a = __half2float(sw[P_B2 + i]);
#pragma unroll
        for (int j = 0; j < MLP_HID; ++j) a = fmaf(__half2float(sw[P_W2 + i * MLP_HID + j]), h1[j], a);
        const float h = fmaxf(a, 0.f);
        y0 = fmaf(__half2float(sw[P_W3 + i]), h, y0);
        y1 = fmaf(__half2float(sw[P_W3 + MLP_HID + i]), h, y1);
    }
    y[s * MLP_OUT] = y0;
    y[s * MLP_OUT + 1] = y1;
}

}  // namespace

void mlp_accumulate_grad(const float *w, const float *x, const float *t, int64_t n, double denom, float *grad,
                         double *loss_sum, cudaStream_t s) {
    if (n <= 0) return;
    static bool ready = false;
    if (!ready) {
        CT_CHECK_CUDA(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sizeof(MlpShared)));
        ready = true;
    }
    const int64_t blocks = ceil_div(n, SB);
    k_mlp_grad<<<(unsigned)blocks, MT, sizeof(MlpShared), s>>>(w, x, t, n, (float)(1.0 / denom), grad, loss_sum);
    CT_COUNT_LAUNCH();
    CT_LAUNCH_CHECK();
}

void mlp_adam_step(float *w, float *m, float *v, float *grad, int64_t step, float lr, cudaStream_t s) {
    const double c1 = 1.0 / (1.0 - pow(0.9, (double)step)), c2 = 1.0 / (1.0 - pow(0.999, (double)step));
    k_adam<<<(MLP_NPARAMS + 255) / 256, 256, 0, s>>>(w, m, v, grad, lr, (float)c1, (float)c2);
    CT_COUNT_LAUNCH();
    CT_LAUNCH_CHECK();
}

void mlp_to_half(const float *w, __half *wh, cudaStream_t s) {
    k_to_half<<<(MLP_NPARAMS + 255) / 256, 256, 0, s>>>(w, wh);
    CT_COUNT_LAUNCH();
    CT_LAUNCH_CHECK();
}

void mlp_predict(const __half *wh, const float *x, int64_t n, float *y, cudaStream_t s) {
    if (n <= 0) return;
    k_mlp_predict<<<(unsigned)ceil_div(n, 128), 128, 0, s>>>(wh, x, n, y);
    CT_COUNT_LAUNCH();
    CT_LAUNCH_CHECK();
}

}  // namespace ct
