// sweep.cu -- several radii over one tree.  The paper queries each dataset at
// three radii (Table I); the tree does not depend on eps, so it is built once
// and the largest radius is queried in full (Algorithm 3).  Every smaller
// radius is then derived from the CSR of the next larger one: the exact
// graph at eps' <= eps is a subset of the graph at eps, so each entry is
// decided again at eps' and the survivors are compacted, rows staying sorted.
//
// An entry is re-decided from its stored distance when that distance is far
// from both radii (outside the guard band |d - r| <= 1e-3 r of either); the
// stored value is within 1e-6 relative of the exact distance, so the side of
// eps' is certain, and the pair was decided in fp32 at both radii, so the
// stored distance is the one a query at eps' would store.  Entries inside
// either band are evaluated again from the points with the query's own
// decision (canonical fp32 sum, guard band, pinned FP64 sum) and stored
// distance rule.  The output is therefore the CSR that eps_graph_query
// returns at eps', bit for bit.  Edit distances are exact integers: an entry
// survives iff d <= floor(eps').
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "l2dist.cuh"
#include "profile.cuh"
#include "query.cuh"

namespace ct {

namespace {

constexpr int SW_T = 256;  // threads per block (a warp per row)

struct Redecide {
    QParams qp;                // decision at the new radius
    float src_lo, src_hi;      // guard band of the radius the source CSR was made at (in distance)
    float dst_lo, dst_hi;      // guard band of the new radius
    int all;                   // re-evaluate every entry (special radii: 0, tiny, huge)
    int lev;                   // edit distance: integer distances, no re-evaluation
    const float *pts;          // points in tree order
    const int32_t *pos;        // original id -> tree position
    int dp, dim;
};

// Decides entry (row, col) with stored distance d at the new radius; *nd is
// the distance to store.
__device__ __forceinline__ bool redecide(const Redecide &R, int32_t row, int32_t col, float d, float *nd,
                                         unsigned long long &evals, unsigned long long &g64,
                                         unsigned long long &band) {
    if (R.lev) {
        *nd = d;
        return d <= (float)R.qp.lev_k;
    }
    const bool zone = R.all || (d >= R.src_lo && d <= R.src_hi) || (d >= R.dst_lo && d <= R.dst_hi);
    if (!zone) {
        *nd = d;
        return d < R.dst_lo;
    }
    ++evals;
    const float *x = R.pts + (size_t)R.pos[row] * R.dp, *y = R.pts + (size_t)R.pos[col] * R.dp;
    const float sv = pair_sqdist(reinterpret_cast<const float4 *>(x), reinterpret_cast<const float4 *>(y),
                                 R.dp >> 2);
    int e = decide32(R.qp, sv, band);
    if (e < 0) {
        const double s64 = sq_l2_exact(x, y, R.dim);
        ++g64;
        e = s64 <= R.qp.eps2_64;
        *nd = (float)sqrt(s64);
    } else {
        *nd = R.dp <= 128 ? sqrtf(sv) : (float)sqrt(sq_l2_exact(x, y, R.dim));
    }
    return e != 0;
}

__global__ void k_inv_perm(int64_t n, const int32_t *__restrict__ perm, int32_t *__restrict__ pos) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pos[perm[i]] = (int32_t)i;
}

// Warp per row: the number of entries that survive at the new radius.
__global__ void __launch_bounds__(SW_T) k_sweep_count(int64_t n, const int64_t *__restrict__ rp,
                                                       const int32_t *__restrict__ col, const float *__restrict__ dist,
                                                       Redecide R, int32_t *__restrict__ deg,
                                                       unsigned long long *__restrict__ st) {
    const int64_t row = ((int64_t)blockIdx.x * SW_T + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    unsigned long long evals = 0, g64 = 0, band = 0;
    if (row < n) {
        int cnt = 0;
        for (int64_t e = rp[row] + lane; e < rp[row + 1]; e += 32) {
            float nd;
            cnt += redecide(R, (int32_t)row, col[e], dist[e], &nd, evals, g64, band) ? 1 : 0;
        }
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0) deg[row] = cnt;
    }
    for (int o = 16; o > 0; o >>= 1) {
        evals += __shfl_xor_sync(0xffffffffu, evals, o);
        g64 += __shfl_xor_sync(0xffffffffu, g64, o);
        band += __shfl_xor_sync(0xffffffffu, band, o);
    }
    if (lane == 0) {
        if (evals) atomicAdd(st + ST_PAIRS, evals);
        if (g64) atomicAdd(st + ST_GUARD, g64);
        if (band) atomicAdd(st + ST_BAND, band);
    }
}

// Warp per row: the survivors in their order (ballot compaction).
__global__ void __launch_bounds__(SW_T) k_sweep_emit(int64_t n, const int64_t *__restrict__ rp,
                                                      const int32_t *__restrict__ col, const float *__restrict__ dist,
                                                      Redecide R, const int64_t *__restrict__ rp2,
                                                      int32_t *__restrict__ col2, float *__restrict__ dist2,
                                                      int32_t *__restrict__ err) {
    const int64_t row = ((int64_t)blockIdx.x * SW_T + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    unsigned long long evals = 0, g64 = 0, band = 0;
    int64_t at = rp2[row];
    const int64_t end2 = rp2[row + 1];
    for (int64_t b = rp[row]; b < rp[row + 1]; b += 32) {
        const int64_t e = b + lane;
        bool keep = false;
        float nd = 0.f;
        int32_t c = 0;
        if (e < rp[row + 1]) {
            c = col[e];
            keep = redecide(R, (int32_t)row, c, dist[e], &nd, evals, g64, band);
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int64_t w = at + __popc(m & lanemask_lt());
            if (w < end2) {
                col2[w] = c;
                dist2[w] = nd;
            } else {
                atomicOr(err, 8);
            }
        }
        at += __popc(m);
    }
    if (lane == 0 && at != end2) atomicOr(err, 16);
}

inline unsigned grid_rows(int64_t n) { return (unsigned)ceil_div(std::max<int64_t>(n, 1) * 32, SW_T); }

// Guard band of a radius in distance, widened by one part in 10^6 and rounded
// outwards to fp32.
void band_of(const QParams &qp, float &lo, float &hi) {
    const double w = 1e-3 + 1e-6;
    lo = (float)(qp.eps64 * (1.0 - w));
    hi = (float)(qp.eps64 * (1.0 + w));
    if ((double)lo > qp.eps64 * (1.0 - w)) lo = nextafterf(lo, 0.0f);
    if ((double)hi < qp.eps64 * (1.0 + w)) hi = nextafterf(hi, INFINITY);
}

}  // namespace

// The CSR of `t` at radius qd.eps64 from `src`, the CSR at qs.eps64 >= qd.eps64.
void sweep_filter(const ct_tree *t, const QParams &qs, const QParams &qd, const QueryOut &src, cudaStream_t s,
                  QueryOut &out) {
    const int64_t n = t->n;
    DBuf<unsigned long long> st(ST_N, s);
    CT_CHECK_CUDA(cudaMemsetAsync(st.p, 0, ST_N * sizeof(unsigned long long), s));
    int32_t *err = reinterpret_cast<int32_t *>(st.p + ST_ERR);
    Redecide R{};
    R.qp = qd;
    R.lev = t->metric != CT_L2_F32;
    R.pts = t->pts;
    R.dp = t->dp;
    R.dim = t->dim;
    R.all = qs.mode != 0 || qd.mode != 0;
    band_of(qs, R.src_lo, R.src_hi);
    band_of(qd, R.dst_lo, R.dst_hi);
    DBuf<int32_t> pos(R.lev ? 0 : (n ? n : 1), s);
    if (!R.lev && n) {
        k_inv_perm<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(n, t->perm, pos.p);
        CT_COUNT_LAUNCH();
        R.pos = pos.p;
    }
    DBuf<int32_t> deg(n + 1, s);
    CT_CHECK_CUDA(cudaMemsetAsync(deg.p, 0, (n + 1) * sizeof(int32_t), s));
    {
        ProfScope ps("sweep_filter", s);
        if (n) {
            k_sweep_count<<<grid_rows(n), SW_T, 0, s>>>(n, src.row_ptr, src.col, src.dist, R, deg.p, st.p);
            CT_COUNT_LAUNCH();
            CT_LAUNCH_CHECK();
        }
    }
    out.row_ptr = (int64_t *)dmalloc((size_t)(n + 1) * sizeof(int64_t), s);
    exclusive_scan_i32_to_i64(deg.p, out.row_ptr, n + 1, nullptr, s);
    int64_t nnz = 0;
    to_host(&nnz, out.row_ptr + n, 1, s);
    out.nnz = nnz;
    out.col = (int32_t *)dmalloc((size_t)(nnz ? nnz : 1) * sizeof(int32_t), s);
    out.dist = (float *)dmalloc((size_t)(nnz ? nnz : 1) * sizeof(float), s);
    if (n && nnz) {
        ProfScope ps("sweep_emit", s);
        k_sweep_emit<<<grid_rows(n), SW_T, 0, s>>>(n, src.row_ptr, src.col, src.dist, R, out.row_ptr, out.col,
                                                   out.dist, err);
        CT_COUNT_LAUNCH();
        CT_LAUNCH_CHECK();
    }
    unsigned long long hs[ST_N];
    to_host(hs, st.p, ST_N, s);
    prof_flush();
    if (hs[ST_ERR]) CT_FAIL(CT_ECUDA, "internal consistency check failed in the radius sweep (code %llu)", hs[ST_ERR]);
    out.stats = ct_query_stats{};
    out.stats.leaf_pairs = (int64_t)hs[ST_PAIRS];
    out.stats.guard_fp64 = (int64_t)hs[ST_GUARD];
    out.stats.guard_band = (int64_t)hs[ST_BAND];
}

}  // namespace ct
