// l2dist.cuh -- the L2 pair decision shared by every kernel that decides or
// re-decides an edge: the canonical fp32 squared distance of a pair (one
// operation order everywhere, so that decisions and stored distances agree
// bit for bit between kernels), the decision from it with its guard band,
// and the pinned FP64 sum that decides inside the band.
#pragma once

#include "query.cuh"

namespace ct {
namespace {

// Edge decision from the canonical fp32 squared distance sv: 1 edge, 0 none,
// -1 the pinned FP64 sum decides.  Mode 0: outside the guard band
// |d - eps| <= 1e-3 eps the fp32 value decides; inside it (counted in band)
// the fp32 value still decides when its rigorous error bound (c_lo, c_hi)
// puts the exact sum -- and so the pinned FP64 sum -- on one side of eps^2.
// Mode 1 (eps = 0): sv > 0 means x != y; sv == 0 can also be an underflowed
// square, so FP64 decides.  Mode 3: every pair.  Mode 2: always FP64.
__device__ __forceinline__ int decide32(const QParams &qp, float sv, unsigned long long &band) {
    if (qp.mode == 0) {
        if (sv < qp.lo2) return 1;
        if (sv > qp.hi2) return 0;
        ++band;
        return sv < qp.c_lo ? 1 : (sv > qp.c_hi ? 0 : -1);
    }
    if (qp.mode == 1) return sv > 0.0f ? 0 : -1;
    if (qp.mode == 3) return 1;
    return -1;
}

// Pinned FP64 sum of squared differences: fp32 inputs widened exactly,
// t = x - y, s = s + t*t in ascending index order, every op rounded to
// nearest and never contracted.
// Rows start on 16-byte boundaries (global or shared memory): the loads go
// four floats at a time, the sum stays in ascending index order.
template <bool INL>
__device__ __forceinline__ double sq_l2_exact4_t(const float4 *x, const float4 *y, int dim);
__device__ __noinline__ double sq_l2_exact4(const float4 *x, const float4 *y, int dim) {
    return sq_l2_exact4_t<true>(x, y, dim);
}
template <bool INL>
__device__ __forceinline__ double sq_l2_exact4_t(const float4 *x, const float4 *y, int dim) {
    double s = 0.0;
    const int n4 = dim >> 2;
#pragma unroll 4
    for (int k = 0; k < n4; ++k) {
        const float4 a = x[k], b = y[k];
        double t = __dsub_rn((double)a.x, (double)b.x);
        s = __dadd_rn(s, __dmul_rn(t, t));
        t = __dsub_rn((double)a.y, (double)b.y);
        s = __dadd_rn(s, __dmul_rn(t, t));
        t = __dsub_rn((double)a.z, (double)b.z);
        s = __dadd_rn(s, __dmul_rn(t, t));
        t = __dsub_rn((double)a.w, (double)b.w);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    const float *xs = reinterpret_cast<const float *>(x), *ys = reinterpret_cast<const float *>(y);
    for (int k = 4 * n4; k < dim; ++k) {
        const double t = __dsub_rn((double)xs[k], (double)ys[k]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}
__device__ __forceinline__ double sq_l2_exact(const float *x, const float *y, int dim) {
    return sq_l2_exact4(reinterpret_cast<const float4 *>(x), reinterpret_cast<const float4 *>(y), dim);
}

// The same squared distance for one pair, scalar, in the same operation order
// as the tiles (per 16 coordinates: x and z terms into one FMA chain, y and w
// into another; chain sums added; chunk sums added into the total), so that
// its decisions equal the tiles' bit for bit.  x may point to shared or
// global memory (generic loads); y is a global row.
__device__ __forceinline__ float pair_sqdist(const float4 *x, const float4 *__restrict__ y, int nq4) {
    float tot = 0.f;
    int k = 0;
    for (; k + 4 <= nq4; k += 4) {
        float lo = 0.f, hi = 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float4 a = x[k + u], b = __ldg(y + k + u);
            const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z, dw = a.w - b.w;
            lo = fmaf(dx, dx, lo);
            hi = fmaf(dy, dy, hi);
            lo = fmaf(dz, dz, lo);
            hi = fmaf(dw, dw, hi);
        }
        tot += lo + hi;
    }
    if (k < nq4) {
        float lo = 0.f, hi = 0.f;
        for (; k < nq4; ++k) {
            const float4 a = x[k], b = __ldg(y + k);
            const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z, dw = a.w - b.w;
            lo = fmaf(dx, dx, lo);
            hi = fmaf(dy, dy, hi);
            lo = fmaf(dz, dz, lo);
            hi = fmaf(dw, dw, hi);
        }
        tot += lo + hi;
    }
    return tot;
}

}  // namespace
}  // namespace ct
