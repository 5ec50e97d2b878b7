// learned.cu -- the learned form of the query: per-query features, fitting of
// the degree/work predictor on the GPU, and the plan it makes before the
// traversal (row capacities and overflow arena of the one-pass emit; groups
// walked in order of decreasing predicted walk length).  The paper has no
// learned component; the output is the same edge set as the two-pass form
// whatever the predictions are.
#include <atomic>
#include <cmath>
#include <random>
#include <vector>

#include "mlp.cuh"
#include "profile.cuh"
#include "query.cuh"

namespace ct {
namespace {

inline unsigned grid_of(int64_t n, int t) { return (unsigned)ceil_div(n > 0 ? n : 1, t); }

struct Norm {
    float mean[MLP_IN], inv[MLP_IN];
    int d, on;
};

// Position -> query group (groups are runs of positions in increasing order).
__global__ void k_pos_group(int64_t n, int G, const int32_t *__restrict__ group_begin, int32_t *__restrict__ gof) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = G;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (group_begin[mid] <= i) lo = mid; else hi = mid;
    }
    gof[i] = lo;
}

// log1p(r / e) in fp32 with inv_e = fl(1 / e), log_e = fl(log e): the ratio
// carries a relative error below 2^-22, which moves the logarithm by less
// than 2^-22; past 2^100 the ratio takes log r - log e (log1p(q) and log q
// agree far below fp32 resolution there, and fl(r inv_e) may overflow).
__device__ __forceinline__ float rel_log(float r, float inv_e, float log_e) {
    const float q = r * inv_e;
    return q < 0x1p100f ? log1pf(q) : logf(r) - log_e;
}

// The 16 features of the query at tree position i (see
// ct_predictor_features); e = max(eps, 1e-20):
//  0 log1p(d(q, leaf centre)/e)      1 log1p(d(q, group centre)/e) (L2; 0 else)
//  2 log1p(group radius/e)           3 log2(group size)
//  4..11 leaf block and its first three ancestors: log1p(points below),
//        log1p(radius/e)
//  12..15 log1p(points below the lowest ancestor with radius >= e, 2e, 4e, 16e)
__global__ void __launch_bounds__(256) k_features(
    int64_t n, int dp, int l2, const float *__restrict__ pts, const float *__restrict__ dcen,
    const int32_t *__restrict__ leaf_ids, int n_leaves, const int32_t *__restrict__ node_begin,
    const int32_t *__restrict__ node_count, const float *__restrict__ radius, const int32_t *__restrict__ parent,
    const int32_t *__restrict__ group_begin, const int32_t *__restrict__ group_count,
    const float *__restrict__ group_radius, const int32_t *__restrict__ gof, double e, float inv_e, float log_e,
    Norm nm,
    float *__restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = n_leaves;  // leaf block holding position i
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (node_begin[leaf_ids[mid]] <= i) lo = mid; else hi = mid;
    }
    const int leaf = leaf_ids[lo];
    const int g = gof[i];
    float f[MLP_IN];
    f[0] = rel_log(dcen[i], inv_e, log_e);
    f[1] = 0.f;
    if (l2) {
        const float4 *a = reinterpret_cast<const float4 *>(pts + (size_t)i * dp);
        const float4 *b = reinterpret_cast<const float4 *>(pts + (size_t)group_begin[g] * dp);
        float s = 0.f;
        for (int k = 0; k < (dp >> 2); ++k) {
            const float4 u = a[k], v = b[k];
            const float d0 = u.x - v.x, d1 = u.y - v.y, d2 = u.z - v.z, d3 = u.w - v.w;
            s = fmaf(d0, d0, s);
            s = fmaf(d1, d1, s);
            s = fmaf(d2, d2, s);
            s = fmaf(d3, d3, s);
        }
        f[1] = rel_log(sqrtf(s), inv_e, log_e);
    }
    f[2] = rel_log(group_radius[g], inv_e, log_e);
    f[3] = log2f((float)group_count[g]);
    int v = leaf;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        f[4 + 2 * k] = log1pf((float)node_count[v]);
        f[5 + 2 * k] = rel_log(radius[v], inv_e, log_e);
        if (k < 3 && parent[v] >= 0) v = parent[v];
    }
    const double mult[4] = {1.0, 2.0, 4.0, 16.0};
    int found = 0;
    v = leaf;
    for (int guard = 0; guard < 4096 && found < 4; ++guard) {
        const double r = (double)radius[v];
        while (found < 4 && r >= mult[found] * e) f[12 + found++] = log1pf((float)node_count[v]);
        if (parent[v] < 0) break;
        v = parent[v];
    }
    for (; found < 4; ++found) f[12 + found] = log1pf((float)node_count[v]);
    if (nm.on) {
#pragma unroll
        for (int k = 0; k < MLP_IN; ++k) f[k] = (f[k] - nm.mean[k]) * nm.inv[k];
    }
    float4 *out = reinterpret_cast<float4 *>(x + (size_t)i * MLP_IN);
#pragma unroll
    for (int k = 0; k < MLP_IN / 4; ++k) out[k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
}

// Training targets at position i: log1p(degree), log1p(vertices tested by
// the walk of the query's group).
__global__ void k_targets(int64_t n, const int32_t *__restrict__ perm, const int32_t *__restrict__ gof,
                          const int32_t *__restrict__ deg, const int32_t *__restrict__ gvisit, float *__restrict__ t) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    t[2 * i] = log1pf((float)deg[perm[i]]);
    t[2 * i + 1] = log1pf((float)gvisit[gof[i]]);
}

// Column sums and sums of squares of an n x d matrix (d <= 16), in FP64.
__global__ void __launch_bounds__(256) k_moments(const float *__restrict__ x, int64_t n, int d,
                                                 double *__restrict__ acc) {
    double s[MLP_IN], q[MLP_IN];
#pragma unroll
    for (int k = 0; k < MLP_IN; ++k) s[k] = q[k] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < MLP_IN; ++k) {
            if (k < d) {
                const double v = (double)x[i * d + k];
                s[k] += v;
                q[k] += v * v;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < MLP_IN; ++k) {
        if (k >= d) continue;
        for (int o = 16; o > 0; o >>= 1) {
            s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
            q[k] += __shfl_xor_sync(0xffffffffu, q[k], o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(acc + k, s[k]);
            atomicAdd(acc + MLP_IN + k, q[k]);
        }
    }
}

__global__ void k_standardize(float *__restrict__ x, int64_t n, Norm nm) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * nm.d) return;
    const int k = (int)(e % nm.d);
    x[e] = (x[e] - nm.mean[k]) * nm.inv[k];
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {  // splitmix64 finaliser
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Mini-batch of b samples drawn uniformly (with replacement) from n.
__global__ void k_gather_batch(const float *__restrict__ x, const float *__restrict__ t, int64_t n, int b,
                               uint64_t seed, int64_t step, float *__restrict__ xb, float *__restrict__ tb) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= b) return;
    const uint64_t h = mix64(seed ^ mix64(((uint64_t)step << 32) + (uint64_t)j + 0x9e3779b97f4a7c15ull));
    const int64_t i = (int64_t)(h % (uint64_t)n);
    const float4 *src = reinterpret_cast<const float4 *>(x + i * MLP_IN);
    float4 *dst = reinterpret_cast<float4 *>(xb + (int64_t)j * MLP_IN);
#pragma unroll
    for (int k = 0; k < MLP_IN / 4; ++k) dst[k] = src[k];
    tb[2 * j] = t[2 * i];
    tb[2 * j + 1] = t[2 * i + 1];
}

struct TargetNorm {
    float mean[2], std[2];
};

__device__ __forceinline__ float predicted(const float *y, int64_t i, int o, const TargetNorm &tn) {
    const float lg = fmaf(y[2 * i + o], tn.std[o], tn.mean[o]);
    return fmaxf(expm1f(fminf(lg, 80.f)), 0.f);
}

// Row capacity of the point at position i (stored by original id), and the
// predicted values when asked for.
__global__ void k_capacity(int64_t n, const float *__restrict__ y, const int32_t *__restrict__ perm, TargetNorm tn,
                           float margin, int pad, int32_t *__restrict__ cap, float *__restrict__ pdeg,
                           float *__restrict__ pblk) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int o = perm[i];
    const float d = predicted(y, i, 0, tn);
    if (pdeg) pdeg[o] = d;
    if (pblk) pblk[o] = predicted(y, i, 1, tn);
    if (cap) {
        const float want = fminf(ceilf(d * (1.0f + margin)), (float)n);
        int64_t c = (int64_t)fmaxf(want, 0.f) + pad;
        cap[o] = (int32_t)(c < n ? c : n);
    }
}

std::atomic<int64_t> g_capacity_budget{0};

// Capacities scaled by f (the one-pass buffers over their memory budget).
__global__ void k_scale_capacity(int64_t n, double f, int32_t *__restrict__ cap) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cap[i] = (int32_t)floor((double)cap[i] * f);
}

// Traversal order: per group the mean predicted walk length of its queries;
// sort key larger first.
__global__ void k_group_keys(int G, const int32_t *__restrict__ group_begin, const int32_t *__restrict__ group_count,
                             const float *__restrict__ y, TargetNorm tn, int gbase, uint32_t *__restrict__ keys,
                             uint32_t *__restrict__ vals) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const int qb = group_begin[g], qn = group_count[g];
    float s = 0.f;
    for (int q = 0; q < qn; ++q) s += predicted(y, qb + q, 1, tn);
    keys[gbase + g] = ~__float_as_uint(fmaxf(s / (float)max(qn, 1), 0.f));
    vals[gbase + g] = (uint32_t)(gbase + g);
}

Norm make_norm(const float *mean, const float *std_, int d, bool on) {
    Norm nm{};
    nm.d = d;
    nm.on = on;
    for (int k = 0; k < d; ++k) {
        nm.mean[k] = mean[k];
        nm.inv[k] = std_[k] > 0.f ? 1.0f / std_[k] : 1.0f;
    }
    return nm;
}

void moments(const float *x, int64_t n, int d, float *mean, float *std_, cudaStream_t s) {
    DBuf<double> acc(2 * MLP_IN, s);
    CT_CHECK_CUDA(cudaMemsetAsync(acc.p, 0, 2 * MLP_IN * sizeof(double), s));
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), num_sms() * 4));
    k_moments<<<blocks, 256, 0, s>>>(x, n, d, acc.p);
    CT_COUNT_LAUNCH();
    CT_LAUNCH_CHECK();
    double h[2 * MLP_IN];
    to_host(h, acc.p, 2 * MLP_IN, s);
    for (int k = 0; k < d; ++k) {
        const double m = h[k] / (double)n;
        const double var = std::max(0.0, h[MLP_IN + k] / (double)n - m * m);
        mean[k] = (float)m;
        std_[k] = var > 1e-12 ? (float)std::sqrt(var) : 0.f;
    }
}

}  // namespace

// Raw (P == nullptr) or standardised features of every tree position.
void predictor_features(const ct_tree *t, double eps, const ct_predictor *P, float *x, cudaStream_t s) {
    const int64_t n = t->n;
    if (n == 0) return;
    DBuf<int32_t> gof(n, s);
    k_pos_group<<<grid_of(n, 256), 256, 0, s>>>(n, t->n_groups, t->group_begin, gof.p);
    CT_COUNT_LAUNCH();
    const Norm nm = P ? make_norm(P->fmean, P->fstd, MLP_IN, true) : Norm{};
    const double e = eps > 1e-20 ? eps : 1e-20;
    k_features<<<grid_of(n, 256), 256, 0, s>>>(n, t->dp, t->metric == CT_L2_F32, t->pts, t->dcen, t->leaf_ids,
                                               t->n_leaves, t->node_begin, t->node_count, t->radius, t->parent,
                                               t->group_begin, t->group_count, t->group_radius, gof.p, e, (float)(1.0 / e),
                                               (float)std::log(e), nm, x);
    CT_COUNT_LAUNCH();
    CT_LAUNCH_CHECK();
}

void predictor_init(ct_predictor *P, uint64_t seed) {
    std::vector<float> w(MLP_NPARAMS, 0.f);
    std::mt19937_64 gen(seed);
    auto fill = [&](int off, int rows, int cols) {
        std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / cols));
        for (int i = 0; i < rows * cols; ++i) w[off + i] = (float)nd(gen);
    };
    fill(P_W1, MLP_HID, MLP_IN);
    fill(P_W2, MLP_HID, MLP_HID);
    fill(P_W3, MLP_OUT, MLP_HID);
    P->w = (float *)dmalloc(sizeof(float) * MLP_NPARAMS, 0);
    P->m = (float *)dmalloc(sizeof(float) * MLP_NPARAMS, 0);
    P->v = (float *)dmalloc(sizeof(float) * MLP_NPARAMS, 0);
    P->grad = (float *)dmalloc(sizeof(float) * MLP_NPARAMS, 0);
    P->wh = (__half *)dmalloc(sizeof(__half) * MLP_NPARAMS, 0);
    CT_CHECK_CUDA(cudaMemcpyAsync(P->w, w.data(), sizeof(float) * MLP_NPARAMS, cudaMemcpyHostToDevice, 0));
    CT_CHECK_CUDA(cudaMemsetAsync(P->m, 0, sizeof(float) * MLP_NPARAMS, 0));
    CT_CHECK_CUDA(cudaMemsetAsync(P->v, 0, sizeof(float) * MLP_NPARAMS, 0));
    CT_CHECK_CUDA(cudaMemsetAsync(P->grad, 0, sizeof(float) * MLP_NPARAMS, 0));
    mlp_to_half(P->w, P->wh, 0);
    CT_CHECK_CUDA(cudaStreamSynchronize(0));
}

void predictor_release(ct_predictor *P) {
    cudaDeviceSynchronize();
    for (void *p : {(void *)P->w, (void *)P->m, (void *)P->v, (void *)P->grad, (void *)P->wh})
        if (p) cudaFree(p);
}

double predictor_fit(ct_predictor *P, const ct_tree *t, double eps, const ct_fit_opts &o, cudaStream_t s) {
    const int64_t n = t->n;
    const int G = t->n_groups;
    // labels from one traversal and one count pass of the plain query
    const QParams qp = make_qparams(t, eps, o.include_self);
    DBuf<int32_t> deg(n, s), gvisit(G ? G : 1, s), gof(n, s);
    DBuf<float> x(n * MLP_IN, s), y(n * MLP_OUT, s);
    Probe pr;
    pr.deg = deg.p;
    pr.gvisit = gvisit.p;
    QueryOut tmp;
    query_multi(1, &t, &qp, s, &tmp, 0, nullptr, &pr);
    predictor_features(t, eps, nullptr, x.p, s);
    k_pos_group<<<grid_of(n, 256), 256, 0, s>>>(n, G, t->group_begin, gof.p);
    CT_COUNT_LAUNCH();
    k_targets<<<grid_of(n, 256), 256, 0, s>>>(n, t->perm, gof.p, deg.p, gvisit.p, y.p);
    CT_COUNT_LAUNCH();
    CT_LAUNCH_CHECK();
    moments(x.p, n, MLP_IN, P->fmean, P->fstd, s);
    moments(y.p, n, MLP_OUT, P->tmean, P->tstd, s);
    for (int k = 0; k < MLP_OUT; ++k)
        if (!(P->tstd[k] > 0.f)) P->tstd[k] = 1.0f;
    const Norm fx = make_norm(P->fmean, P->fstd, MLP_IN, true), fy = make_norm(P->tmean, P->tstd, MLP_OUT, true);
    k_standardize<<<grid_of(n * MLP_IN, 256), 256, 0, s>>>(x.p, n, fx);
    CT_COUNT_LAUNCH();
    k_standardize<<<grid_of(n * MLP_OUT, 256), 256, 0, s>>>(y.p, n, fy);
    CT_COUNT_LAUNCH();
    CT_LAUNCH_CHECK();

    const int steps = o.steps > 0 ? o.steps : 1500;
    const int batch = o.batch > 0 ? o.batch : 4096;
    const float lr = o.lr > 0.f ? o.lr : 2e-3f;
    DBuf<float> xb((size_t)batch * MLP_IN, s), tb((size_t)batch * MLP_OUT, s);
    DBuf<double> lsum(1, s);
    CT_CHECK_CUDA(cudaMemsetAsync(lsum.p, 0, sizeof(double), s));
    const int tail = std::max(1, steps / 10);
    for (int k = 1; k <= steps; ++k) {
        k_gather_batch<<<grid_of(batch, 256), 256, 0, s>>>(x.p, y.p, n, batch, o.seed, k, xb.p, tb.p);
        CT_COUNT_LAUNCH();
        mlp_accumulate_grad(P->w, xb.p, tb.p, batch, (double)batch, P->grad, k > steps - tail ? lsum.p : nullptr, s);
        const double frac = (double)(k - 1) / (double)steps;
        const float lr_k = (float)(lr * (0.1 + 0.9 * 0.5 * (1.0 + std::cos(3.14159265358979323846 * frac))));
        mlp_adam_step(P->w, P->m, P->v, P->grad, ++P->step, lr_k, s);
    }
    mlp_to_half(P->w, P->wh, s);
    double l = 0.0;
    to_host(&l, lsum.p, 1, s);
    P->fitted = true;
    return l / ((double)batch * tail);
}

// Predicted degree and walk length by original id.
void predictor_predict(const ct_predictor *P, const ct_tree *t, double eps, float *pdeg, float *pvisit,
                       cudaStream_t s) {
    const int64_t n = t->n;
    if (n == 0) return;
    DBuf<float> x(n * MLP_IN, s), y(n * MLP_OUT, s);
    predictor_features(t, eps, P, x.p, s);
    mlp_predict(P->wh, x.p, n, y.p, s);
    TargetNorm tn{{P->tmean[0], P->tmean[1]}, {P->tstd[0], P->tstd[1]}};
    k_capacity<<<grid_of(n, 256), 256, 0, s>>>(n, y.p, t->perm, tn, 0.f, 0, nullptr, pdeg, pvisit);
    CT_COUNT_LAUNCH();
    CT_LAUNCH_CHECK();
}

// The plan of a batch of C clouds (rows and groups concatenated).
void learned_plan(const ct_predictor *P, int C, const ct_tree *const *trees, const QParams *qps,
                  const int64_t *rbase, const int32_t *gbase, cudaStream_t s, LearnedPlan &lp) {
    if (!P->fitted) CT_FAIL(CT_EINVAL, "the predictor has not been fitted");
    const int64_t n = rbase[C];
    const int G = gbase[C];
    DBuf<float> x(n * MLP_IN, s), y(n * MLP_OUT, s);
    for (int c = 0; c < C; ++c) predictor_features(trees[c], qps[c].eps64, P, x.p + rbase[c] * MLP_IN, s);
    mlp_predict(P->wh, x.p, n, y.p, s);
    x.reset();
    const TargetNorm tn{{P->tmean[0], P->tmean[1]}, {P->tstd[0], P->tstd[1]}};
    // row capacities (rows of cloud c from rbase[c]) and their offsets
    DBuf<int32_t> cap(n + 1, s);
    lp.cap_off = DBuf<int64_t>(n + 1, s);
    for (int c = 0; c < C; ++c) {
        const int64_t nc = trees[c]->n;
        if (!nc) continue;
        k_capacity<<<grid_of(nc, 256), 256, 0, s>>>(nc, y.p + MLP_OUT * rbase[c], trees[c]->perm, tn, P->margin,
                                                    P->pad, cap.p + rbase[c], nullptr, nullptr);
        CT_COUNT_LAUNCH();
    }
    CT_LAUNCH_CHECK();
    exclusive_scan_i32_to_i64(cap.p, lp.cap_off.p, n + 1, nullptr, s);
    // groups by decreasing predicted walk length
    if (G > 1 && P->order_by_work) {
        DBuf<uint32_t> keys(G, s), vals(G, s), tk(G, s), tv(G, s);
        for (int c = 0; c < C; ++c) {
            const int Gc = trees[c]->n_groups;
            if (!Gc) continue;
            k_group_keys<<<grid_of(Gc, 256), 256, 0, s>>>(Gc, trees[c]->group_begin, trees[c]->group_count,
                                                          y.p + MLP_OUT * rbase[c], tn, gbase[c], keys.p, vals.p);
            CT_COUNT_LAUNCH();
        }
        CT_LAUNCH_CHECK();
        radix_sort_pairs(keys.p, vals.p, tk.p, tv.p, G, 32, s);
        lp.group_order = DBuf<int32_t>(G, s);
        CT_CHECK_CUDA(cudaMemcpyAsync(lp.group_order.p, vals.p, G * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
    int64_t total = 0;
    to_host(&total, lp.cap_off.p + n, 1, s);
    lp.arena = (int64_t)std::ceil((double)P->arena_frac * (double)total) + P->arena_min;
    // the one-pass buffers (capacities and arena) take at most a third of the
    // free device memory: predictions that ask for more (a predictor far from
    // its training data) are scaled down to that budget -- entries past a
    // row's capacity go to the arena, rows past the arena are emitted again
    // exactly -- and only a budget below the arena's minimum takes the
    // two-pass form
    lp.one_pass = true;
    size_t fr = 0, tot = 0;
    const int64_t fixed = g_capacity_budget.load();
    if (fixed > 0 || cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
        const double budget = fixed > 0 ? (double)fixed : (double)fr / 3.0;
        const double need = (double)total * 8.0 + (double)lp.arena * 16.0;
        if (need > budget) {
            const double room = budget - 16.0 * (double)P->arena_min;
            if (room <= 0.0) {
                lp.one_pass = false;
            } else {
                const double f = room / ((double)total * (8.0 + 16.0 * (double)P->arena_frac));
                k_scale_capacity<<<grid_of(n, 256), 256, 0, s>>>(n, f, cap.p);
                CT_COUNT_LAUNCH();
                CT_LAUNCH_CHECK();
                exclusive_scan_i32_to_i64(cap.p, lp.cap_off.p, n + 1, nullptr, s);
                to_host(&total, lp.cap_off.p + n, 1, s);
                lp.arena = (int64_t)std::ceil((double)P->arena_frac * (double)total) + P->arena_min;
            }
        }
    } else {
        cudaGetLastError();
    }
    lp.cap_total = total;
}

void set_capacity_budget(int64_t bytes) { g_capacity_budget.store(bytes > 0 ? bytes : 0); }

void query_predicted(const ct_tree *t, const QParams &qp, const void *predictor, int precision, cudaStream_t s,
                     QueryOut &out) {
    const ct_predictor *P = static_cast<const ct_predictor *>(predictor);
    if (!P->fitted) CT_FAIL(CT_EINVAL, "the predictor has not been fitted");
    if (P->device != t->device) CT_FAIL(CT_EINVAL, "predictor and tree live on different devices");
    query_multi(1, &t, &qp, s, &out, precision, P, nullptr);
}

}  // namespace ct
