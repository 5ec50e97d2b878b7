// landmark.cu -- the ε-graph through landmarks on one GPU (Sec. IV-D; the
// paper's Algorithms 5 and 6 with the processors replaced by one batch):
//   1. Voronoi cells of the caller's centres C (each point's nearest centre,
//      the lowest index among equals);
//   2. the ε-ghosts of every cell by Lemma 1: a point p outside cell k whose
//      neighbours could lie in it, d(p, c_k) <= d(p, C) + 2 eps;
//   3. one cover tree per cell over its points and ghosts (Algorithms 1-2),
//      all cells queried in shared launches (the batched query);
//   4. every point's row taken from its own cell's CSR: by Lemma 1 each of
//      its neighbours in another cell is a ghost of its own cell, so the row
//      is complete there.
// The output is the CSR eps_graph_query returns (same entries and stored
// distances: each pair is decided by the same kernels).  A cell's members are
// kept in increasing original id, so the local-to-original map is increasing
// and rows stay sorted.
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "profile.cuh"
#include "query.cuh"

namespace ct {

ct_tree *build_tree(const ct_points *pts, int zeta, int root, cudaStream_t s);
void free_tree(ct_tree *t);
void query_batched(int n_clouds, const ct_tree *const *trees, const QParams *qps, const ct_query_opts *opts,
                   cudaStream_t s, QueryOut *outs);

namespace {

constexpr int LM_T = 256;

// Distances of the Voronoi step: fp32 direct differences (L2; the ghost test
// below carries a margin far above their error) or exact popcounts (Hamming).
__device__ __forceinline__ float lm_dist_l2(const float *__restrict__ x, const float *__restrict__ c, int dim) {
    float acc = 0.f;
    for (int k = 0; k < dim; ++k) {
        const float d = x[k] - c[k];
        acc = fmaf(d, d, acc);
    }
    return sqrtf(acc);
}
__device__ __forceinline__ int lm_dist_ham(const uint8_t *__restrict__ a, const uint8_t *__restrict__ b, int dim) {
    const int nb = (dim + 7) >> 3;
    int d = 0;
    for (int i = 0; i < nb; ++i) {
        uint32_t x = (uint32_t)(a[i] ^ b[i]);
        if (8 * i + 8 > dim) x &= (1u << (dim - 8 * i)) - 1u;  // bits past dim are not part of the row
        d += __popc(x);
    }
    return d;
}

struct LmInput {
    int metric, dim;
    const float *X;      // L2: n x dim
    const uint8_t *B;    // Hamming: n x ceil(dim/8)
    const int64_t *cid;  // m centre ids
    int m;
};

__device__ __forceinline__ float lm_dist(const LmInput &in, int64_t p, int k) {
    const int64_t c = in.cid[k];
    if (in.metric == CT_L2_F32) return lm_dist_l2(in.X + p * in.dim, in.X + c * in.dim, in.dim);
    const int nb = (in.dim + 7) >> 3;
    return (float)lm_dist_ham(in.B + p * nb, in.B + c * nb, in.dim);
}

// Lemma 1's ghost test of point p (nearest-centre distance dmin) for cell k:
// exact for Hamming (integers); for L2 with a relative margin of 2^-10 over
// fp32 distances whose error is below 2^-17 (more ghosts never change rows).
__device__ __forceinline__ bool lm_ghost(const LmInput &in, float d, float dmin, float eps_up, int lev_k) {
    if (in.metric == CT_HAMMING_B1) return d <= dmin + 2.0f * (float)lev_k;
    return d <= fmaf(dmin + eps_up, 1.0f + 0x1p-10f, eps_up) + 0x1p-60f;
}

__global__ void k_lm_nearest(LmInput in, int64_t n, int32_t *__restrict__ cell, float *__restrict__ dmin) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int best = 0;
    float bd = lm_dist(in, p, 0);
    for (int k = 1; k < in.m; ++k) {
        const float d = lm_dist(in, p, k);
        if (d < bd) {
            bd = d;
            best = k;
        }
    }
    cell[p] = best;
    dmin[p] = bd;
}

// Memberships of point p: its own cell and the cells it is a ghost of
// (count pass: keys == nullptr; fill pass: keys (cell << 32 | p) at moff[p]).
__global__ void k_lm_members(LmInput in, int64_t n, const int32_t *__restrict__ cell, const float *__restrict__ dmin,
                             float eps_up, int lev_k, int32_t *__restrict__ mcount, const int64_t *__restrict__ moff,
                             uint64_t *__restrict__ keys) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int own = cell[p];
    const float dm = dmin[p];
    int64_t at = keys ? moff[p] : 0;
    int c = 0;
    for (int k = 0; k < in.m; ++k) {
        const bool mem = k == own || lm_ghost(in, lm_dist(in, p, k), dm, eps_up, lev_k);
        if (!mem) continue;
        if (keys) keys[at++] = ((uint64_t)k << 32) | (uint64_t)p;
        ++c;
    }
    if (!keys) mcount[p] = c;
}

__global__ void k_lm_cell_counts(const uint64_t *__restrict__ keys, int64_t M, int32_t *__restrict__ cnt) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < M) atomicAdd(&cnt[(int)(keys[j] >> 32)], 1);
}

// Rows of the members, cell by cell, in member order.
__global__ void k_lm_gather_l2(const uint64_t *__restrict__ keys, int64_t M, const float *__restrict__ X, int dim,
                               float *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * dim) return;
    const int64_t j = i / dim;
    const int k = (int)(i - j * dim);
    out[i] = X[(int64_t)(uint32_t)keys[j] * dim + k];
}
__global__ void k_lm_gather_bytes(const uint64_t *__restrict__ keys, int64_t M, const uint8_t *__restrict__ B, int nb,
                                  uint8_t *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * nb) return;
    const int64_t j = i / nb;
    const int k = (int)(i - j * nb);
    out[i] = B[(int64_t)(uint32_t)keys[j] * nb + k];
}

// Per cell: its CSR (local row offsets, columns as local member indices).
struct CellCsr {
    const int64_t *const *rp;
    const int32_t *const *col;
    const float *const *dist;
};

// Degree of each point: the length of its row in its own cell.
__global__ void k_lm_degrees(const uint64_t *__restrict__ keys, int64_t M, const int64_t *__restrict__ cell_off,
                             const int32_t *__restrict__ cell, CellCsr cc, int32_t *__restrict__ deg) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const int k = (int)(keys[j] >> 32);
    const int64_t p = (int64_t)(uint32_t)keys[j];
    if (cell[p] != k) return;  // a ghost here
    const int64_t l = j - cell_off[k];
    deg[p] = (int32_t)(cc.rp[k][l + 1] - cc.rp[k][l]);
}

// Warp per membership of an own point: its row, columns mapped to original ids.
__global__ void k_lm_fill(const uint64_t *__restrict__ keys, int64_t M, const int64_t *__restrict__ cell_off,
                          const int32_t *__restrict__ cell, CellCsr cc, const int64_t *__restrict__ row_ptr,
                          int32_t *__restrict__ col, float *__restrict__ dist) {
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= M) return;
    const int k = (int)(keys[j] >> 32);
    const int64_t p = (int64_t)(uint32_t)keys[j];
    if (cell[p] != k) return;
    const int64_t l = j - cell_off[k];
    const int64_t a = cc.rp[k][l], b = cc.rp[k][l + 1], o = row_ptr[p];
    const uint64_t *mk = keys + cell_off[k];
    for (int64_t e = a + lane; e < b; e += 32) {
        col[o + (e - a)] = (int32_t)(uint32_t)mk[cc.col[k][e]];
        dist[o + (e - a)] = cc.dist[k][e];
    }
}

inline unsigned grid_of(int64_t n, int t) { return (unsigned)ceil_div(n > 0 ? n : 1, t); }

}  // namespace

void landmark_query(const ct_points *pts, const int64_t *centres_h, int m, double eps, int zeta,
                    const ct_query_opts *opts, cudaStream_t s, QueryOut &out, ct_landmark_info *info) {
    const int64_t n = pts->n;
    const bool l2 = pts->metric == CT_L2_F32;
    if (info) *info = ct_landmark_info{};
    if (n == 0) {  // the empty graph
        out.row_ptr = (int64_t *)dmalloc(sizeof(int64_t), s);
        CT_CHECK_CUDA(cudaMemsetAsync(out.row_ptr, 0, sizeof(int64_t), s));
        out.col = (int32_t *)dmalloc(sizeof(int32_t), s);
        out.dist = (float *)dmalloc(sizeof(float), s);
        out.nnz = 0;
        return;
    }
    if (!l2 && pts->metric != CT_HAMMING_B1)
        CT_FAIL(CT_EUNSUPPORTED, "the landmark form takes L2 points or Hamming rows");
    if (m < 1 || (int64_t)m > std::max<int64_t>(n, 1)) CT_FAIL(CT_EINVAL, "m must be in [1, n] (got %d)", m);
    for (int k = 0; k < m; ++k)
        if (centres_h[k] < 0 || centres_h[k] >= n) CT_FAIL(CT_EINVAL, "centre %d out of range", k);
    const int dim = pts->dim, nb = (dim + 7) / 8;
    // QParams of the metric for the ghost bound (an empty tree stands in)
    ct_tree shape;
    shape.metric = pts->metric;
    shape.dp = l2 ? (int)ceil_div(dim, 4) * 4 : 0;
    QParams qp = make_qparams(&shape, eps, opts->include_self);
    qp.half = opts->upper_triangle;
    DBuf<int64_t> cid(m, s);
    CT_CHECK_CUDA(cudaMemcpyAsync(cid.p, centres_h, (size_t)m * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    const LmInput in{pts->metric, dim, l2 ? (const float *)pts->data : nullptr,
                     l2 ? nullptr : (const uint8_t *)pts->data, cid.p, m};
    // 1. Voronoi cells, 2. memberships (own cell and ghost cells), cell-major and id-minor
    DBuf<int32_t> cell(n, s), mcount(n + 1, s);
    DBuf<float> dmin(n, s);
    DBuf<int64_t> moff(n + 1, s);
    k_lm_nearest<<<grid_of(n, LM_T), LM_T, 0, s>>>(in, n, cell.p, dmin.p);
    CT_COUNT_LAUNCH();
    CT_CHECK_CUDA(cudaMemsetAsync(mcount.p + n, 0, sizeof(int32_t), s));
    k_lm_members<<<grid_of(n, LM_T), LM_T, 0, s>>>(in, n, cell.p, dmin.p, qp.eps_up, qp.lev_k, mcount.p, nullptr,
                                                   nullptr);
    CT_COUNT_LAUNCH();
    exclusive_scan_i32_to_i64(mcount.p, moff.p, n + 1, nullptr, s);
    int64_t M = 0;
    to_host(&M, moff.p + n, 1, s);
    DBuf<uint64_t> keys(M, s), tk(M, s);
    DBuf<uint32_t> vals(M, s), tv(M, s);
    k_lm_members<<<grid_of(n, LM_T), LM_T, 0, s>>>(in, n, cell.p, dmin.p, qp.eps_up, qp.lev_k, mcount.p, moff.p,
                                                   keys.p);
    CT_COUNT_LAUNCH();
    CT_CHECK_CUDA(cudaMemsetAsync(vals.p, 0, (size_t)M * sizeof(uint32_t), s));
    int bits = 32;
    while ((int64_t(1) << (bits - 32)) < m) ++bits;
    radix_sort_pairs64(keys.p, vals.p, tk.p, tv.p, M, bits, s);
    tk.reset();
    tv.reset();
    vals.reset();
    DBuf<int32_t> ccnt(m + 1, s);
    DBuf<int64_t> coff(m + 1, s);
    CT_CHECK_CUDA(cudaMemsetAsync(ccnt.p, 0, (size_t)(m + 1) * sizeof(int32_t), s));
    k_lm_cell_counts<<<grid_of(M, LM_T), LM_T, 0, s>>>(keys.p, M, ccnt.p);
    CT_COUNT_LAUNCH();
    exclusive_scan_i32_to_i64(ccnt.p, coff.p, m + 1, nullptr, s);
    std::vector<int64_t> hoff(m + 1);
    to_host(hoff.data(), coff.p, m + 1, s);
    // 3. member rows gathered cell by cell; a tree per cell
    DBuf<float> gx(l2 ? (size_t)M * dim : 0, s);
    DBuf<uint8_t> gb(l2 ? 0 : (size_t)M * nb, s);
    if (l2) {
        k_lm_gather_l2<<<grid_of(M * dim, LM_T), LM_T, 0, s>>>(keys.p, M, (const float *)pts->data, dim, gx.p);
    } else {
        k_lm_gather_bytes<<<grid_of(M * nb, LM_T), LM_T, 0, s>>>(keys.p, M, (const uint8_t *)pts->data, nb, gb.p);
    }
    CT_COUNT_LAUNCH();
    CT_LAUNCH_CHECK();
    struct Trees {
        std::vector<ct_tree *> t;
        ~Trees() {
            for (ct_tree *x : t) free_tree(x);
        }
    } trees;
    std::vector<QueryOut> outs((size_t)m);
    struct OutsGuard {
        std::vector<QueryOut> &o;
        cudaStream_t s;
        ~OutsGuard() {
            for (auto &q : o) {
                if (!q.shared) {
                    dfree(q.row_ptr, s);
                    dfree(q.col, s);
                    dfree(q.dist, s);
                }
                q = QueryOut();
            }
        }
    } og{outs, s};
    int64_t largest = 0;
    {
        ProfScope ps("landmark_build", s);
        for (int k = 0; k < m; ++k) {
            ct_points cp{};
            cp.metric = pts->metric;
            cp.dim = dim;
            cp.n = hoff[k + 1] - hoff[k];
            cp.data = l2 ? (const void *)(gx.p + hoff[k] * dim) : (const void *)(gb.p + hoff[k] * nb);
            largest = std::max(largest, cp.n);
            trees.t.push_back(build_tree(&cp, zeta, 0, s));
        }
    }
    std::vector<QParams> qps((size_t)m, qp);
    {
        ProfScope ps("landmark_query", s);
        query_batched(m, trees.t.data(), qps.data(), opts, s, outs.data());
    }
    // 4. rows of the own points from their cells
    DBuf<const int64_t *> prp(m, s);
    DBuf<const int32_t *> pcol(m, s);
    DBuf<const float *> pdist(m, s);
    {
        std::vector<const int64_t *> a((size_t)m);
        std::vector<const int32_t *> b((size_t)m);
        std::vector<const float *> c((size_t)m);
        for (int k = 0; k < m; ++k) {
            a[k] = outs[k].row_ptr;
            b[k] = outs[k].col;
            c[k] = outs[k].dist;
        }
        CT_CHECK_CUDA(cudaMemcpyAsync(prp.p, a.data(), (size_t)m * sizeof(void *), cudaMemcpyHostToDevice, s));
        CT_CHECK_CUDA(cudaMemcpyAsync(pcol.p, b.data(), (size_t)m * sizeof(void *), cudaMemcpyHostToDevice, s));
        CT_CHECK_CUDA(cudaMemcpyAsync(pdist.p, c.data(), (size_t)m * sizeof(void *), cudaMemcpyHostToDevice, s));
        CT_CHECK_CUDA(cudaStreamSynchronize(s));  // the host arrays above are on the stack
    }
    const CellCsr cc{prp.p, pcol.p, pdist.p};
    DBuf<int32_t> deg(n + 1, s);
    CT_CHECK_CUDA(cudaMemsetAsync(deg.p, 0, (size_t)(n + 1) * sizeof(int32_t), s));
    k_lm_degrees<<<grid_of(M, LM_T), LM_T, 0, s>>>(keys.p, M, coff.p, cell.p, cc, deg.p);
    CT_COUNT_LAUNCH();
    out.row_ptr = (int64_t *)dmalloc((size_t)(n + 1) * sizeof(int64_t), s);
    exclusive_scan_i32_to_i64(deg.p, out.row_ptr, n + 1, nullptr, s);
    int64_t nnz = 0;
    to_host(&nnz, out.row_ptr + n, 1, s);
    out.nnz = nnz;
    out.col = (int32_t *)dmalloc((size_t)(nnz ? nnz : 1) * sizeof(int32_t), s);
    out.dist = (float *)dmalloc((size_t)(nnz ? nnz : 1) * sizeof(float), s);
    k_lm_fill<<<grid_of(M * 32, LM_T), LM_T, 0, s>>>(keys.p, M, coff.p, cell.p, cc, out.row_ptr, out.col, out.dist);
    CT_COUNT_LAUNCH();
    CT_LAUNCH_CHECK();
    CT_CHECK_CUDA(cudaStreamSynchronize(s));
    prof_flush();
    out.stats = ct_query_stats{};
    // the batches' counters (every CSR of an L2 batch carries that batch's;
    // Hamming cells are queried one at a time)
    for (int k = 0; k < m; k += l2 ? kBatchClouds : 1) {
        const ct_query_stats &b = outs[k].stats;
        out.stats.traversal_evals += b.traversal_evals;
        out.stats.leaf_pairs += b.leaf_pairs;
        out.stats.guard_fp64 += b.guard_fp64;
        out.stats.recheck_fp32 += b.recheck_fp32;
        out.stats.candidates += b.candidates;
        out.stats.leaf_rows += b.leaf_rows;
        out.stats.guard_band += b.guard_band;
    }
    if (info) {
        info->members = M;
        info->ghosts = M - n;
        info->largest_cell = largest;
        info->cells = m;
    }
}

}  // namespace ct
