// build.cu -- cover-tree construction on the GPU (Algorithm 1 SplitVertex and
// Algorithm 2 BuildLevel of the paper, Sec. IV-A).
//
// All hubs created in one round are split together.  One split iteration is
// two launches over every hub of the round:
//   k_hub_step      -- per hub: take the farthest point found by the previous
//                      pass (largest D, lowest position on ties, as the strict
//                      comparison of Algorithm 1 in scan order); stop the hub
//                      once it lies within 2^(l-1), else make it the next centre;
//   k_dist_update   -- per point of an active hub: d = d(p, newest centre);
//                      if d < D[p] then D[p] = d, L[p] = new label (strict <);
//                      then the hub's argmax of D by a packed 64-bit atomicMax.
// When every hub has stopped, the round's points are partitioned by
// (hub, label) with a stable radix sort; each child's centre is moved to the
// front of its range, its radius is the max of D over its range, and a child
// with more than zeta points and positive radius becomes a hub of the next
// round at level ceil(log2 r) (levels with a single nested child are skipped);
// the others become leaf blocks.  Radii are stored rounded up so that they
// bound every descendant's exact distance.
//
// Distances are fp32 for L2 (direct differences) and exact integers for edit
// distance (bit-parallel, lev.cuh).
#include <climits>
#include <cstdio>
#include <memory>
#include <mutex>
#include <vector>
#include <algorithm>

#include "common.cuh"
#include "lev.cuh"
#include "profile.cuh"

namespace ct {

namespace {

constexpr int BT = 256;  // threads per block in the build kernels
constexpr int32_t kNone = 0x7f7f7f7f;  // byte-fill 0x7f: "no position yet"

// ceil(log2 r) for finite r > 0 (exact at powers of two).
__device__ __forceinline__ int ceil_log2f(float r) {
    int e;
    float m = frexpf(r, &e);  // r = m * 2^e, m in [0.5, 1)
    return m == 0.5f ? e - 1 : e;
}

// Rounded-up radius: bounds the exact distance of every point whose fp32
// distance was at most r (fp32 relative error of the distance sums here is
// below 2^-17 for rows up to 4096 floats; absolute slack covers underflow).
__device__ __forceinline__ float round_radius_up(float r, int metric) {
    if (metric != CT_L2_F32) return r;
    if (r == 0.0f) return 0.0f;
    float t = __fmul_ru(r, 1.0f + 0x1p-16f);
    return __fadd_ru(t, 0x1p-64f);
}

// ---- L2 distance of a point row to a centre row held in shared memory.
// TPD threads cooperate on one distance; lane j reads float4s j, j+TPD, ...
// The shuffles name only the TPD lanes of the caller's group, so groups of
// one warp may take different branches around the call.
template <int TPD>
__device__ __forceinline__ float group_sqdist(const float4 *__restrict__ row, const float4 *cen,
                                              int nq, int j) {
    float acc = 0.f;
#pragma unroll 4
    for (int k = j; k < nq; k += TPD) {
        float4 a = __ldg(row + k);
        float4 b = cen[k];
        float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z, dw = a.w - b.w;
        acc = fmaf(dx, dx, acc);
        acc = fmaf(dy, dy, acc);
        acc = fmaf(dz, dz, acc);
        acc = fmaf(dw, dw, acc);
    }
    const unsigned mask = TPD == 32 ? 0xffffffffu : (((1u << TPD) - 1u) << ((threadIdx.x & 31) & ~(TPD - 1)));
#pragma unroll
    for (int o = TPD / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(mask, acc, o, TPD);
    return acc;
}

constexpr int UPD_PASSES = 8;  // passes of a block over its chunk in k_dist_update_l2

// The same distance with the row staged in shared memory by the calling lane
// (lane j copied float4s j, j + TPD, ... and reads only those): the same
// operations in the same order, so the same value.
template <int TPD>
__device__ __forceinline__ float group_sqdist_staged(const float4 *row, const float4 *cen, int nq, int j) {
    float acc = 0.f;
#pragma unroll 4
    for (int k = j; k < nq; k += TPD) {
        float4 a = row[k];
        float4 b = cen[k];
        float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z, dw = a.w - b.w;
        acc = fmaf(dx, dx, acc);
        acc = fmaf(dy, dy, acc);
        acc = fmaf(dz, dz, acc);
        acc = fmaf(dw, dw, acc);
    }
    const unsigned mask = TPD == 32 ? 0xffffffffu : (((1u << TPD) - 1u) << ((threadIdx.x & 31) & ~(TPD - 1)));
#pragma unroll
    for (int o = TPD / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(mask, acc, o, TPD);
    return acc;
}
__device__ __forceinline__ void stage_copy16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void stage_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }
// Staged passes keep UPD_STAGES buffers of G rows in shared memory: the rows
// of passes p + 1 and p + 2 are in flight while pass p is computed.
constexpr int UPD_STAGES = 3;
constexpr int UPD_STAGE_F4 = 1024;  // float4s of one buffer (G rows of nq float4s) that allow staging

struct Hubs {
    int32_t *begin, *count, *node, *nc, *cur, *done, *level;
    int32_t *flat;     // 1: the split stopped early and every child is a leaf block
    int32_t *covered;  // points within the split threshold after the last pass (L2)
    float *thr;
    unsigned long long *key;
};

// A split that has taken FLAT_MIN_CENTRES centres while they cover on average
// fewer than 1 + 1/8 points each is making almost every point its own child
// (in high-dimensional data where all distances lie above the threshold):
// the triangle inequality can then prune nothing below this hub, and the
// farthest-first iterations would grow quadratically with its size.  Such a
// hub keeps the centres taken so far (a net of its own: separated, within
// 2^l of the hub's centre) and its children become leaf blocks whatever their
// size; their stored radii keep the query exact.
constexpr int FLAT_MIN_CENTRES = 256;
__device__ __forceinline__ bool flat_split(int nc, int covered) {
    return nc >= FLAT_MIN_CENTRES && covered <= nc + (nc >> 3);
}

// The next split step of a hub, taken inside the update pass by the hub's
// last block to finish (its arrival completes the hub's count in `arrive`;
// every other block of the hub has written its distances and its key by
// then): k_hub_step for that hub, then k_centre_dists for its new centre.
// One launch per split iteration instead of three; nothing waits -- the
// blocks only count their arrivals.
struct Step {
    int32_t *arrive;      // per hub: blocks of the pass that have finished (reset by the last)
    int32_t *active_out;  // hubs that took a new centre
    int32_t *cpos;        // centre positions per hub label
    float *dcc;           // distances of the new centre to the hub's centres (read by the pass, then rewritten)
};

template <int TPD>
__device__ __noinline__ void step_tail(const float *__restrict__ X, int dp, const int32_t *__restrict__ ids,
                                       Hubs hb, int h, float4 *cen, Step st) {
    __shared__ int s_act, s_nc, s_cur;
    if (threadIdx.x == 0) {
        const unsigned long long k = atomicAdd(&hb.key[h], 0ull);  // every block's maximum has landed
        const float v = key_value(k);
        const int covered = atomicExch(&hb.covered[h], 0);           // every block's count has landed
        s_act = 0;
        if (k == 0ull || !(v > hb.thr[h])) {
            hb.done[h] = 1;
        } else if (flat_split(hb.nc[h], covered)) {
            hb.done[h] = 1;
            hb.flat[h] = 1;
        } else {
            const int b = hb.begin[h], nc = hb.nc[h];
            const int cur = (int32_t)key_pos(k);
            hb.cur[h] = cur;
            st.cpos[b] = b;  // label 0: the hub's own centre
            st.cpos[b + nc] = cur;
            hb.nc[h] = nc + 1;
            hb.key[h] = 0ull;
            atomicAdd(st.active_out, 1);
            s_act = 1;
            s_nc = nc + 1;
            s_cur = cur;
        }
        st.arrive[h] = 0;
    }
    __syncthreads();
    if (!s_act) return;
    const int b = hb.begin[h], nc = s_nc, nq = dp >> 2;
    const float4 *crow = reinterpret_cast<const float4 *>(X + (size_t)ids[s_cur] * dp);
    for (int i = threadIdx.x; i < nq; i += blockDim.x) cen[i] = crow[i];
    __syncthreads();
    constexpr int G = BT / TPD;
    const int g = threadIdx.x / TPD, j = threadIdx.x % TPD;
    // the row of label L (its centre's point id), the next step's loaded
    // while this step's distance is computed
    auto row_of = [&](int L) { return ids[st.cpos[b + (L < nc ? L : 0)]]; };
    int rid = row_of(g);
    for (int L0 = 0; L0 < nc; L0 += G) {  // every group runs the same number of steps
        const int L = L0 + g;
        const int nrid = L0 + G < nc ? row_of(L + G) : 0;
        const float dd = sqrtf(group_sqdist<TPD>(reinterpret_cast<const float4 *>(X + (size_t)rid * dp), cen, nq, j));
        if (L < nc && j == 0) st.dcc[b + L] = dd;
        rid = nrid;
    }
}

// Pruning (L2): a point labelled L cannot come closer to the new centre c
// than D when d(c, centre L) >= 2 D (triangle inequality); such points keep D
// and L without reading their row.  dcc[begin + L] = d(c, centre L) of the
// hub (nullptr: no pruning).  STAGE: the rows of the chunk's passes are
// copied into shared memory two passes ahead (cp.async), so that a group's
// eight passes do not wait on memory one after another; otherwise each pass
// reads its rows from global memory.
template <int TPD, bool STAGE>
__global__ void __launch_bounds__(BT, 4) k_dist_update_l2(
    const float *__restrict__ X, int dp, const int32_t *__restrict__ ids, float *__restrict__ D,
    int32_t *__restrict__ lab, const int32_t *__restrict__ chunk_hub,
    const int32_t *__restrict__ chunk_start, int chunk_len, Hubs hb, const float *dcc, Step st) {
    extern __shared__ float4 cen[];
    int c = blockIdx.x;
    int h = chunk_hub[c];
    if (hb.done[h]) return;
    int start = chunk_start[c];
    const int hbeg = hb.begin[h];
    int end = min(start + chunk_len, hbeg + hb.count[h]);
    int cpos = hb.cur[h];
    int lbl = hb.nc[h] - 1;
    int nq = dp >> 2;
    const float4 *crow = reinterpret_cast<const float4 *>(X + (size_t)ids[cpos] * dp);
    for (int i = threadIdx.x; i < nq; i += blockDim.x) cen[i] = crow[i];
    constexpr int G = BT / TPD;
    int g = threadIdx.x / TPD, j = threadIdx.x % TPD;
    // the chunk's passes (chunk_len = UPD_PASSES * G): distances, labels and
    // ids of every pass first, then the pruning test, then the distances --
    // three round trips to memory per chunk instead of three per pass
    float cur[UPD_PASSES];
    int lb[UPD_PASSES], pid[UPD_PASSES];
    bool far[UPD_PASSES];
#pragma unroll
    for (int p = 0; p < UPD_PASSES; ++p) {
        const int pos = start + p * G + g;
        const bool valid = pos < end;
        cur[p] = valid ? D[pos] : 0.f;
        lb[p] = valid ? lab[pos] : 0;
        pid[p] = valid ? ids[pos] : 0;
        far[p] = !valid;
    }
    if (dcc) {
#pragma unroll
        for (int p = 0; p < UPD_PASSES; ++p)
            if (!far[p]) far[p] = dcc[hbeg + lb[p]] >= 2.0f * cur[p] * (1.0f + 0x1p-12f) + 0x1p-60f;
    }
    // STAGE: buffer b holds G rows of nq float4s after the centre row; a lane
    // copies (and later reads) only its own float4s of its group's row
    float4 *stage = cen + nq;
    auto issue = [&](int p) {
        if (p < UPD_PASSES && !far[p]) {
            const float4 *row = reinterpret_cast<const float4 *>(X + (size_t)pid[p] * dp);
            float4 *dst = stage + ((size_t)(p % UPD_STAGES) * G + g) * nq;
            for (int k = j; k < nq; k += TPD) stage_copy16(dst + k, row + k);
        }
        stage_commit();
    };
    if (STAGE) {
        issue(0);
        issue(1);
    }
    __syncthreads();  // the centre row
    unsigned long long best = 0ull;
#pragma unroll
    for (int p = 0; p < UPD_PASSES; ++p) {
        const int pos = start + p * G + g;
        if (STAGE) issue(p + 2);
        if (!far[p]) {  // the same for the group's TPD lanes
            float s;
            if (STAGE) {
                stage_wait<UPD_STAGES - 1>();  // this lane's copies of pass p have landed
                s = group_sqdist_staged<TPD>(stage + ((size_t)(p % UPD_STAGES) * G + g) * nq, cen, nq, j);
            } else {
                s = group_sqdist<TPD>(reinterpret_cast<const float4 *>(X + (size_t)pid[p] * dp), cen, nq, j);
            }
            if (j == 0) {
                float d = sqrtf(s);
                if (d < cur[p]) {
                    D[pos] = d;
                    lab[pos] = lbl;
                    cur[p] = d;
                }
            }
        }
        if (pos < end && j == 0) {
            unsigned long long k = pack_max_key(cur[p], (uint32_t)pos);
            best = k > best ? k : best;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
        best = v > best ? v : best;
    }
    // points now within the split threshold (the flat-split test)
    const float thr = hb.thr[h];
    int cov = 0;
#pragma unroll
    for (int p = 0; p < UPD_PASSES; ++p) cov += (j == 0 && start + p * G + g < end && cur[p] <= thr) ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) cov += __shfl_xor_sync(0xffffffffu, cov, o);
    // the block's maximum key and count go to the hub in one atomic each (a
    // block's chunk lies in one hub); then, with pruning, the block arrives
    // and the hub's last block takes its next step
    __shared__ unsigned long long s_best[BT / 32];
    __shared__ int s_cov[BT / 32];
    __shared__ int s_last;
    if ((threadIdx.x & 31) == 0) {
        s_best[threadIdx.x >> 5] = best;
        s_cov[threadIdx.x >> 5] = cov;
    }
    if (st.arrive) __threadfence();  // this thread's D and lab writes, before the block's arrival
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long bk = 0ull;
        int bc = 0;
#pragma unroll
        for (int w = 0; w < BT / 32; ++w) {
            bk = s_best[w] > bk ? s_best[w] : bk;
            bc += s_cov[w];
        }
        if (bk) atomicMax(&hb.key[h], bk);
        if (bc) atomicAdd(&hb.covered[h], bc);
        if (st.arrive) {
            __threadfence();  // the key and the count, before the arrival
            const int blocks = (hb.count[h] + chunk_len - 1) / chunk_len;  // all of the hub's chunks run
            s_last = atomicAdd(&st.arrive[h], 1) == blocks - 1;
        }
    }
    if (st.arrive) {
        __syncthreads();
        if (s_last) {
            __threadfence();
            step_tail<TPD>(X, dp, ids, hb, h, cen, st);
        }
    }
}

// The hub step's decision in the hub's last block (thread 0; every block's
// key and count have landed): the next centre from the hub's largest key, or
// the hub is done (nothing above the split threshold, or a flat split where
// `flat_check`).  The same decision as k_hub_step.
__device__ __forceinline__ void step_decide(Hubs hb, int h, Step st, bool flat_check) {
    const unsigned long long k = atomicAdd(&hb.key[h], 0ull);
    const float v = key_value(k);
    const int covered = atomicExch(&hb.covered[h], 0);
    if (k == 0ull || !(v > hb.thr[h])) {
        hb.done[h] = 1;
    } else if (flat_check && flat_split(hb.nc[h], covered)) {
        hb.done[h] = 1;
        hb.flat[h] = 1;
    } else {
        hb.cur[h] = (int32_t)key_pos(k);
        hb.nc[h] += 1;
        hb.key[h] = 0ull;
        atomicAdd(st.active_out, 1);
    }
    st.arrive[h] = 0;
}

// A block's arrival at the end of an update pass (its writes and atomics
// fenced first): true in every thread of the hub's last block to arrive.
__device__ __forceinline__ bool last_to_arrive(Step st, int h, int blocks) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&st.arrive[h], 1) == blocks - 1;
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

// Edit distance: one thread per point; the newest centre is the pattern of
// the bit-parallel recurrence, its match masks in shared memory.
template <int W>
__global__ void __launch_bounds__(BT) k_dist_update_lev(
    const uint8_t *__restrict__ S, const int64_t *__restrict__ off, const int32_t *__restrict__ ids,
    float *__restrict__ D, int32_t *__restrict__ lab, const int32_t *__restrict__ chunk_hub,
    const int32_t *__restrict__ chunk_start, int chunk_len, Hubs hb, Step st) {
    __shared__ uint64_t peq[256 * W];
    int c = blockIdx.x;
    int h = chunk_hub[c];
    if (hb.done[h]) return;
    int start = chunk_start[c];
    int end = min(start + chunk_len, hb.begin[h] + hb.count[h]);
    int cid = ids[hb.cur[h]];
    int lbl = hb.nc[h] - 1;
    const uint8_t *pat = S + off[cid];
    int m = (int)(off[cid + 1] - off[cid]);
    lev_build_peq<W>(peq, pat, m);
    __syncthreads();
    unsigned long long best = 0ull;
    for (int base = start; base < end; base += blockDim.x) {
        int pos = base + threadIdx.x;
        if (pos < end) {
            int id = ids[pos];
            const uint8_t *txt = S + off[id];
            int n = (int)(off[id + 1] - off[id]);
            float cur = D[pos];
            int cutoff = isinf(cur) ? INT_MAX / 2 : (int)cur - 1;
            int d = lev_myers<W>(peq, m, txt, n, cutoff);
            if (d <= cutoff && (float)d < cur) {
                D[pos] = (float)d;
                lab[pos] = lbl;
                cur = (float)d;
            }
            unsigned long long k = pack_max_key(cur, (uint32_t)pos);
            best = k > best ? k : best;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
        best = v > best ? v : best;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(&hb.key[h], best);
    if (st.arrive) {  // the hub's last block takes its next step (no flat-split test: no counts here)
        const int blocks = (hb.count[h] + chunk_len - 1) / chunk_len;  // all of the hub's chunks run
        if (last_to_arrive(st, h, blocks) && threadIdx.x == 0) step_decide(hb, h, st, false);
    }
}

// ---- Hamming distance: rows of wp 32-bit words (wp a multiple of 4),
// compared four words at a time.
__device__ __forceinline__ int ham_dist4(const uint4 *__restrict__ a, const uint4 *b, int nq) {
    int d = 0;
    for (int k = 0; k < nq; ++k) {
        const uint4 x = a[k], y = b[k];
        d += __popc(x.x ^ y.x) + __popc(x.y ^ y.y) + __popc(x.z ^ y.z) + __popc(x.w ^ y.w);
    }
    return d;
}

// Input rows of ceil(dim/8) bytes (bit j = bit j % 8 of byte j / 8) into
// words of 32 bits (bit j = bit j % 32 of word j / 32); bits past dim cleared.
__global__ void k_pack_bits(const uint8_t *__restrict__ src, int64_t n, int dim, int wp, uint32_t *__restrict__ dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * wp) return;
    const int64_t r = i / wp;
    const int w = (int)(i - r * wp);
    const int nbytes = (dim + 7) >> 3;
    uint32_t v = 0u;
    for (int b = 0; b < 4; ++b) {
        const int byte = 4 * w + b;
        if (byte < nbytes) v |= (uint32_t)src[r * nbytes + byte] << (8 * b);
    }
    const int lo = 32 * w;
    if (lo >= dim) v = 0u;
    else if (dim - lo < 32) v &= (1u << (dim - lo)) - 1u;
    dst[i] = v;
}

// Hamming: one thread per point against the newest centre (its row in shared
// memory); also counts the hub's points within the split threshold.
__global__ void __launch_bounds__(BT) k_dist_update_ham(
    const uint32_t *__restrict__ X, int wp, const int32_t *__restrict__ ids, float *__restrict__ D,
    int32_t *__restrict__ lab, const int32_t *__restrict__ chunk_hub, const int32_t *__restrict__ chunk_start,
    int chunk_len, Hubs hb, Step st) {
    extern __shared__ uint4 hcen[];
    const int c = blockIdx.x;
    const int h = chunk_hub[c];
    if (hb.done[h]) return;
    const int start = chunk_start[c];
    const int end = min(start + chunk_len, hb.begin[h] + hb.count[h]);
    const int nq = wp >> 2;
    const uint4 *crow = reinterpret_cast<const uint4 *>(X + (size_t)ids[hb.cur[h]] * wp);
    for (int i = threadIdx.x; i < nq; i += blockDim.x) hcen[i] = crow[i];
    __syncthreads();
    const int lbl = hb.nc[h] - 1;
    const float thr = hb.thr[h];
    unsigned long long best = 0ull;
    int cov = 0;
    for (int base = start; base < end; base += blockDim.x) {
        const int pos = base + threadIdx.x;
        if (pos < end) {
            float cur = D[pos];
            const int d = ham_dist4(reinterpret_cast<const uint4 *>(X + (size_t)ids[pos] * wp), hcen, nq);
            if ((float)d < cur) {
                D[pos] = (float)d;
                lab[pos] = lbl;
                cur = (float)d;
            }
            cov += cur <= thr;
            const unsigned long long k = pack_max_key(cur, (uint32_t)pos);
            best = k > best ? k : best;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
        best = v > best ? v : best;
        cov += __shfl_xor_sync(0xffffffffu, cov, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (best) atomicMax(&hb.key[h], best);
        if (cov) atomicAdd(&hb.covered[h], cov);
    }
    if (st.arrive) {  // the hub's last block takes its next step
        const int blocks = (hb.count[h] + chunk_len - 1) / chunk_len;  // all of the hub's chunks run
        if (last_to_arrive(st, h, blocks) && threadIdx.x == 0) step_decide(hb, h, st, true);
    }
}

__global__ void k_gather_bits(const uint32_t *__restrict__ Xb, int wp, const int32_t *__restrict__ perm, int64_t n,
                              uint32_t *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nq = wp >> 2;
    if (i >= n * nq) return;
    const int64_t r = i / nq;
    const int k = (int)(i - r * nq);
    reinterpret_cast<uint4 *>(out)[r * nq + k] = reinterpret_cast<const uint4 *>(Xb)[(int64_t)perm[r] * nq + k];
}

// Radius of each query group (Hamming): warp per group, lane per point.
__global__ void k_group_radius_ham(int ng, const int32_t *__restrict__ gbeg, const int32_t *__restrict__ gcnt,
                                   const uint32_t *__restrict__ bits, int wp, float *__restrict__ grad) {
    const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (g >= ng) return;
    const int nq = wp >> 2;
    const uint4 *c = reinterpret_cast<const uint4 *>(bits + (size_t)gbeg[g] * wp);
    int r = 0;
    for (int i = lane; i < gcnt[g]; i += 32)
        r = max(r, ham_dist4(reinterpret_cast<const uint4 *>(bits + (size_t)(gbeg[g] + i) * wp), c, nq));
    for (int o = 16; o > 0; o >>= 1) r = max(r, __shfl_xor_sync(0xffffffffu, r, o));
    if (lane == 0) grad[g] = (float)r;
}

// One thread per hub: decide termination or choose the next centre (its
// position goes to cpos[begin + label] when cpos is given).
__global__ void k_hub_step(int nh, const int32_t *__restrict__ hlist, Hubs hb, int32_t *__restrict__ active_out,
                           int32_t *__restrict__ cpos, int flat_check) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int h = i < nh && hlist ? hlist[i] : i;
    int act = 0;
    if (i < nh && !hb.done[h]) {
        unsigned long long k = hb.key[h];
        float v = key_value(k);
        const int covered = hb.covered[h];
        hb.covered[h] = 0;
        if (k == 0ull || !(v > hb.thr[h])) {
            hb.done[h] = 1;
        } else if (flat_check && flat_split(hb.nc[h], covered)) {
            hb.done[h] = 1;
            hb.flat[h] = 1;
        } else {
            hb.cur[h] = (int32_t)key_pos(k);
            if (cpos) {
                cpos[hb.begin[h]] = hb.begin[h];  // label 0: the hub's own centre
                cpos[hb.begin[h] + hb.nc[h]] = hb.cur[h];
            }
            hb.nc[h] += 1;
            hb.key[h] = 0ull;
            act = 1;
        }
    }
    unsigned b = __ballot_sync(0xffffffffu, act);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(active_out, __popc(b));
}

// Per hub that took a new centre: its distance to each of the hub's centres
// (TPD lanes per distance, warps over the labels).
template <int TPD>
__global__ void __launch_bounds__(BT) k_centre_dists(const float *__restrict__ X, int dp,
                                                     const int32_t *__restrict__ ids, Hubs hb,
                                                     const int32_t *__restrict__ hlist,
                                                     const int32_t *__restrict__ cpos, float *__restrict__ dcc) {
    const int h = hlist ? hlist[blockIdx.x] : blockIdx.x;
    if (hb.done[h]) return;
    const int b = hb.begin[h], nc = hb.nc[h], nq = dp >> 2;
    const float4 *crow = reinterpret_cast<const float4 *>(X + (size_t)ids[hb.cur[h]] * dp);
    constexpr int G = BT / TPD;
    const int g = threadIdx.x / TPD, j = threadIdx.x % TPD;
    for (int L0 = 0; L0 < nc; L0 += G) {  // every group runs the same number of steps
        const int L = L0 + g;
        const int pos = cpos[b + (L < nc ? L : 0)];
        const float dd = sqrtf(group_sqdist<TPD>(reinterpret_cast<const float4 *>(X + (size_t)ids[pos] * dp), crow,
                                                 nq, j));
        if (L < nc && j == 0) dcc[b + L] = dd;
    }
}

// Chunk table of a round: chunk -> (hub, first position).
__global__ void k_chunk_counts(int nh, const int32_t *__restrict__ count, int chunk_len,
                               int32_t *__restrict__ out) {
    int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h < nh) out[h] = (count[h] + chunk_len - 1) / chunk_len;
}
// The whole split (Algorithm 1) of one small hub (at most SPLIT_SMALL points)
// in one CTA: the iterations of k_hub_step, k_centre_dists and
// k_dist_update_l2 for that hub (the same steps and pruning; TPD lanes per
// distance, four 16-byte loads each, so that a pass has many rows in
// flight), its distances, labels and centres in shared memory, and no
// launch per iteration.  One CTA per hub of the round (larger hubs exit);
// the distances, labels and the number of children go back to global memory.
constexpr int SPLIT_SMALL = 512;
template <int TPD>
__global__ void __launch_bounds__(BT) k_split_small(const float *__restrict__ X, int dp,
                                                    const int32_t *__restrict__ ids, float *__restrict__ D,
                                                    int32_t *__restrict__ lab, Hubs hb, int32_t *__restrict__ err) {
    __shared__ float Ds[SPLIT_SMALL], dccs[SPLIT_SMALL];
    __shared__ int32_t labs[SPLIT_SMALL], cposs[SPLIT_SMALL];
    __shared__ float4 cen[32];  // dp <= 128 (TPD is chosen for it)
    __shared__ unsigned long long red[BT / 32];
    __shared__ int s_nc, s_done;
    __shared__ unsigned long long s_key;
    const int h = blockIdx.x;
    if (hb.done[h] || hb.count[h] > SPLIT_SMALL) return;  // a large hub: the level-wide iterations
    const int b = hb.begin[h], cnt = hb.count[h], nq = dp >> 2;
    const float thr = hb.thr[h];
    for (int i = threadIdx.x; i < cnt; i += BT) {
        Ds[i] = D[b + i];
        labs[i] = lab[b + i];
    }
    if (threadIdx.x == 0) {
        s_nc = hb.nc[h];
        s_key = hb.key[h];
        cposs[0] = b;  // label 0: the hub's own centre
    }
    __syncthreads();
    constexpr int G = BT / TPD;
    const int g = threadIdx.x / TPD, j = threadIdx.x % TPD;
    for (;;) {
        // k_hub_step: done, or the farthest point becomes the next centre
        if (threadIdx.x == 0) {
            const unsigned long long k = s_key;
            const float v = key_value(k);
            if (k == 0ull || !(v > thr) || s_nc >= cnt + 1) {
                if (k != 0ull && v > thr) atomicOr(err, 4);  // cannot happen: every centre is a distinct point
                s_done = 1;
            } else {
                cposs[s_nc] = (int32_t)key_pos(k);
                s_nc += 1;
                s_done = 0;
            }
            s_key = 0ull;
        }
        __syncthreads();
        if (s_done) break;
        const int nc = s_nc, cur = cposs[nc - 1];
        const float4 *crow = reinterpret_cast<const float4 *>(X + (size_t)ids[cur] * dp);
        for (int i = threadIdx.x; i < nq; i += BT) cen[i] = crow[i];
        __syncthreads();
        // k_centre_dists: the new centre against every centre of the hub
        for (int L0 = 0; L0 < nc; L0 += G) {
            const int L = L0 + g;
            const int pos = cposs[L < nc ? L : 0];
            const float dd = sqrtf(group_sqdist<TPD>(reinterpret_cast<const float4 *>(X + (size_t)ids[pos] * dp), cen,
                                                     nq, j));
            if (L < nc && j == 0) dccs[L] = dd;
        }
        __syncthreads();
        // k_dist_update_l2 over the hub's points, with the same pruning
        unsigned long long best = 0ull;
        for (int base = 0; base < cnt; base += G) {
            const int i = base + g;
            const bool valid = i < cnt;
            float curd = valid ? Ds[i] : 0.f;
            bool far = !valid;
            if (valid) far = dccs[labs[i]] >= 2.0f * curd * (1.0f + 0x1p-12f) + 0x1p-60f;
            if (!far) {
                const float sq = group_sqdist<TPD>(reinterpret_cast<const float4 *>(X + (size_t)ids[b + i] * dp), cen,
                                                   nq, j);
                if (j == 0) {
                    const float d = sqrtf(sq);
                    if (d < curd) {
                        Ds[i] = d;
                        labs[i] = nc - 1;
                        curd = d;
                    }
                }
            }
            if (valid && j == 0) {
                const unsigned long long k = pack_max_key(curd, (uint32_t)(b + i));
                best = k > best ? k : best;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
            best = v > best ? v : best;
        }
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long m = 0ull;
            for (int w = 0; w < BT / 32; ++w) m = red[w] > m ? red[w] : m;
            s_key = m;
        }
        // the next pass's reads of Ds / labs follow the barrier at its top
    }
    for (int i = threadIdx.x; i < cnt; i += BT) {
        D[b + i] = Ds[i];
        lab[b + i] = labs[i];
    }
    if (threadIdx.x == 0) {
        hb.nc[h] = s_nc;
        hb.done[h] = 1;
        hb.key[h] = 0ull;
    }
}

// Hubs not yet done, and the chunks of those hubs (from the current chunk
// list), for the next burst of split iterations: late iterations touch only
// the few hubs still splitting.  The order within the lists is immaterial
// (every hub and point is updated independently; keys combine by max).
__global__ void k_active_hubs(int nh, const int32_t *__restrict__ done, int32_t *__restrict__ hlist,
                              int32_t *__restrict__ cnt) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    const bool a = h < nh && !done[h];
    const unsigned m = __ballot_sync(0xffffffffu, a);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(cnt, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (a) hlist[base + __popc(m & ((1u << lane) - 1u))] = h;
}
__global__ void k_active_chunks(int64_t nchunks, const int32_t *__restrict__ chub, const int32_t *__restrict__ cst,
                                const int32_t *__restrict__ done, int32_t *__restrict__ chub2,
                                int32_t *__restrict__ cst2, int32_t *__restrict__ cnt) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool a = c < nchunks && !done[chub[c]];
    const unsigned m = __ballot_sync(0xffffffffu, a);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(cnt, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (a) {
        const int k = base + __popc(m & ((1u << lane) - 1u));
        chub2[k] = chub[c];
        cst2[k] = cst[c];
    }
}

// Chunk table of a round, one thread per chunk: its hub is the last one whose
// chunk offset is at most the chunk's index (hubs without chunks share an
// offset with the next hub and are skipped by the search).
__global__ void k_chunk_fill(int64_t nchunks, int nh, const int32_t *__restrict__ begin,
                             const int64_t *__restrict__ coff, int chunk_len,
                             int32_t *__restrict__ chunk_hub, int32_t *__restrict__ chunk_start) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nchunks) return;
    int lo = 0, hi = nh;  // coff[lo] <= c, and c < coff[hi] unless hi = nh
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(coff + mid) <= c) lo = mid; else hi = mid;
    }
    chunk_hub[c] = lo;
    chunk_start[c] = begin[lo] + (int)(c - coff[lo]) * chunk_len;
}

// Partition keys for the round: key = child_base[hub] + label, value = round
// index.  One thread per point of the round; its hub is the last one whose
// round offset is at most the index (hubs without points share an offset with
// the next hub and are skipped by the search).
__global__ void k_part_keys(int64_t R, int nh, const int32_t *__restrict__ begin,
                            const int64_t *__restrict__ round_off, const int64_t *__restrict__ child_base,
                            const int32_t *__restrict__ lab, uint32_t *__restrict__ keys,
                            uint32_t *__restrict__ vals, int32_t *__restrict__ rpos) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    int lo = 0, hi = nh;  // round_off[lo] <= r, and r < round_off[hi] unless hi = nh
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(round_off + mid) <= r) lo = mid; else hi = mid;
    }
    const int pos = begin[lo] + (int)(r - round_off[lo]);
    keys[r] = (uint32_t)(child_base[lo] + lab[pos]);
    vals[r] = (uint32_t)r;
    rpos[r] = pos;
}

// Gather the round in sorted order into temporaries; per child: count, first
// position, first zero-distance position (its centre or a duplicate of it).
// The sorted keys put each child's points in one run, so a warp combines its
// lanes of the same run (their destinations increase along the run) and one
// lane per run updates the child's count, first position and zero point.
__global__ void k_part_gather(int64_t R, const uint32_t *__restrict__ skeys, const uint32_t *__restrict__ svals,
                              const int32_t *__restrict__ rpos, const int32_t *__restrict__ ids,
                              const float *__restrict__ D, int32_t *__restrict__ tids,
                              float *__restrict__ tD, int32_t *__restrict__ ccount,
                              int32_t *__restrict__ cbegin, int32_t *__restrict__ czero) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < R;
    uint32_t gc = 0xffffffffu;
    int dst = 0;
    int zero = INT_MAX;
    if (valid) {
        const int src = rpos[svals[i]];
        dst = rpos[i];
        gc = skeys[i];
        const float d = D[src];
        tids[i] = ids[src];
        tD[i] = d;
        if (d == 0.0f) zero = dst;
    }
    const unsigned same = __match_any_sync(0xffffffffu, gc);
    const int lane = threadIdx.x & 31;
    const int zmin = __reduce_min_sync(same, (unsigned)zero);
    if (valid && lane == __ffs(same) - 1) {  // the run's first lane: the smallest destination
        atomicAdd(&ccount[gc], __popc(same));
        atomicMin(&cbegin[gc], dst);
        if (zmin != INT_MAX) atomicMin(&czero[gc], zmin);
    }
}

// Writes the sorted round back; every point starts the next round labelled 0
// (the centre of the child it now belongs to).
__global__ void k_part_scatter(int64_t R, const int32_t *__restrict__ rpos, const int32_t *__restrict__ tids,
                               const float *__restrict__ tD, int32_t *__restrict__ ids,
                               float *__restrict__ D, int32_t *__restrict__ lab) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R) return;
    int dst = rpos[i];
    ids[dst] = tids[i];
    D[dst] = tD[i];
    lab[dst] = 0;
}

// Move each child's centre to the front of its range.
__global__ void k_centre_front(int64_t T, const int32_t *__restrict__ cbegin, const int32_t *__restrict__ czero,
                               int32_t *__restrict__ ids, float *__restrict__ D, int32_t *__restrict__ err) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= T) return;
    int b = cbegin[c], z = czero[c];
    if (z == kNone) { atomicOr(err, 1); return; }
    if (z != b) {
        int ti = ids[b]; ids[b] = ids[z]; ids[z] = ti;
        float td = D[b]; D[b] = D[z]; D[z] = td;
    }
}

// Per child, the largest (distance, position) key: a prefix maximum along each
// run of equal keys in the warp, then one atomic per run (its last lane).
__global__ void k_child_keys(int64_t R, const uint32_t *__restrict__ skeys, const int32_t *__restrict__ rpos,
                             const float *__restrict__ D, unsigned long long *__restrict__ ckey) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < R;
    const int lane = threadIdx.x & 31;
    uint32_t gc = 0xffffffffu;
    unsigned long long v = 0ull;
    if (valid) {
        const int pos = rpos[i];
        gc = skeys[i];
        v = pack_max_key(D[pos], (uint32_t)pos);
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long ov = __shfl_up_sync(0xffffffffu, v, o);
        const uint32_t og = __shfl_up_sync(0xffffffffu, gc, o);
        if (lane >= o && og == gc && ov > v) v = ov;
    }
    const uint32_t next = __shfl_down_sync(0xffffffffu, gc, 1);
    if (valid && (lane == 31 || next != gc)) atomicMax(&ckey[gc], v);
}

// Link every hub to its children (consecutive node ids).
__global__ void k_link_children(int nh, Hubs hb, const int64_t *__restrict__ child_base, int node_base,
                                int32_t *__restrict__ child_begin, int32_t *__restrict__ child_count,
                                int32_t *__restrict__ node_level, int32_t *__restrict__ parent,
                                int32_t *__restrict__ leafy) {
    int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= nh) return;
    int u = hb.node[h];
    int first = node_base + (int32_t)child_base[h];
    child_begin[u] = first;
    child_count[u] = hb.nc[h];
    node_level[u] = hb.level[h];
    const int fl = hb.flat[h];
    for (int c = 0; c < hb.nc[h]; ++c) {
        parent[first + c] = u;
        leafy[child_base[h] + c] = fl;
    }
}

// New vertices of the round; flags children that become next-round hubs.
__global__ void k_make_nodes(int64_t T, int node_base, int zeta, int metric,
                             const int32_t *__restrict__ cbegin, const int32_t *__restrict__ ccount,
                             const unsigned long long *__restrict__ ckey, int32_t *__restrict__ node_begin,
                             int32_t *__restrict__ node_count, int32_t *__restrict__ child_begin,
                             int32_t *__restrict__ child_count, float *__restrict__ radius,
                             int32_t *__restrict__ level, const int32_t *__restrict__ leafy,
                             int32_t *__restrict__ is_hub) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= T) return;
    int v = node_base + (int)c;
    float r = key_value(ckey[c]);
    node_begin[v] = cbegin[c];
    node_count[v] = ccount[c];
    child_begin[v] = 0;
    child_count[v] = 0;
    radius[v] = round_radius_up(r, metric);
    level[v] = r > 0.0f ? ceil_log2f(r) : INT_MIN;
    is_hub[c] = (ccount[c] > zeta && r > 0.0f && !leafy[c]) ? 1 : 0;
}

// Next round's hubs from the flagged children (order preserved).
__global__ void k_next_hubs(int64_t T, int node_base, const int32_t *__restrict__ is_hub,
                            const int64_t *__restrict__ hub_off, const int32_t *__restrict__ cbegin,
                            const int32_t *__restrict__ ccount, const unsigned long long *__restrict__ ckey,
                            const int32_t *__restrict__ level, Hubs nh) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= T || !is_hub[c]) return;
    int64_t h = hub_off[c];
    int v = node_base + (int)c;
    nh.begin[h] = cbegin[c];
    nh.count[h] = ccount[c];
    nh.node[h] = v;
    nh.nc[h] = 1;
    nh.cur[h] = cbegin[c];
    nh.done[h] = 0;
    nh.flat[h] = 0;
    nh.covered[h] = 0;
    nh.key[h] = ckey[c];
    int l = level[v];
    nh.level[h] = l;
    nh.thr[h] = ldexpf(1.0f, l - 1);
}

__global__ void k_root_init(int64_t n, int root, int32_t *__restrict__ ids, float *__restrict__ D,
                            int32_t *__restrict__ lab) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    ids[i] = i == 0 ? root : (i <= root ? (int32_t)i - 1 : (int32_t)i);
    D[i] = INFINITY;
    lab[i] = 0;
}

__global__ void k_root_node(int64_t n, int zeta, int metric, const unsigned long long *__restrict__ key,
                            int32_t *__restrict__ node_begin, int32_t *__restrict__ node_count,
                            int32_t *__restrict__ child_begin, int32_t *__restrict__ child_count,
                            float *__restrict__ radius, int32_t *__restrict__ level, Hubs hb,
                            int32_t *__restrict__ is_hub) {
    float r = key_value(key[0]);
    node_begin[0] = 0;
    node_count[0] = (int32_t)n;
    child_begin[0] = 0;
    child_count[0] = 0;
    radius[0] = round_radius_up(r, metric);
    int l = r > 0.0f ? ceil_log2f(r) : INT_MIN;
    level[0] = l;
    int hub = (n > zeta && r > 0.0f) ? 1 : 0;
    *is_hub = hub;
    // the root hub for the first round
    hb.begin[0] = 0;
    hb.count[0] = (int32_t)n;
    hb.node[0] = 0;
    hb.nc[0] = 1;
    hb.cur[0] = 0;
    hb.done[0] = 0;
    hb.flat[0] = 0;
    hb.covered[0] = 0;
    hb.key[0] = key[0];
    hb.level[0] = l;
    hb.thr[0] = hub ? ldexpf(1.0f, l - 1) : 0.0f;
}

// Rows already of dp = dim floats (dim a multiple of 4, 16-byte aligned
// source): a float4 copy with the same coordinate-range check.
__global__ void k_copy_rows4(const float4 *__restrict__ src, int64_t nq, float4 *__restrict__ dst,
                             int32_t *__restrict__ bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    const float4 v = src[i];
    if (!(fabsf(v.x) <= 0x1p50f && fabsf(v.y) <= 0x1p50f && fabsf(v.z) <= 0x1p50f && fabsf(v.w) <= 0x1p50f))
        atomicOr(bad, 1);
    dst[i] = v;
}

// Pad rows to dp floats (original order) and check the coordinate range.
__global__ void k_pad_rows(const float *__restrict__ src, int64_t n, int dim, int dp,
                           float *__restrict__ dst, int32_t *__restrict__ bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * dp) return;
    int64_t r = i / dp;
    int k = (int)(i - r * dp);
    float v = k < dim ? src[r * dim + k] : 0.0f;
    if (!(fabsf(v) <= 0x1p50f)) atomicOr(bad, 1);
    dst[i] = v;
}

__global__ void k_gather_rows(const float *__restrict__ Xp, int dp, const int32_t *__restrict__ perm,
                              int64_t n, float *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int nq = dp >> 2;
    if (i >= n * nq) return;
    int64_t r = i / nq;
    int k = (int)(i - r * nq);
    reinterpret_cast<float4 *>(out)[i] = reinterpret_cast<const float4 *>(Xp + (size_t)perm[r] * dp)[k];
}

__global__ void k_node_centres(int nn, const int32_t *__restrict__ node_begin, const float *__restrict__ pts,
                               int dp, float *__restrict__ ctr) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int nq = dp >> 2;
    if (i >= (int64_t)nn * nq) return;
    int64_t v = i / nq;
    int k = (int)(i - v * nq);
    reinterpret_cast<float4 *>(ctr)[i] =
        reinterpret_cast<const float4 *>(pts + (size_t)node_begin[v] * dp)[k];
}

__global__ void k_leaf_keys(int nn, const int32_t *__restrict__ child_count, const int32_t *__restrict__ node_begin,
                            const int32_t *__restrict__ node_count, uint32_t *__restrict__ keys,
                            uint32_t *__restrict__ vals, int32_t *__restrict__ nleaf,
                            int32_t *__restrict__ maxcnt) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nn || child_count[v] != 0) return;
    int slot = atomicAdd(nleaf, 1);
    keys[slot] = (uint32_t)node_begin[v];
    vals[slot] = (uint32_t)v;
    atomicMax(maxcnt, node_count[v]);
}

__global__ void k_string_lengths(int64_t n, const int32_t *__restrict__ perm, const int64_t *__restrict__ off,
                                 int64_t *__restrict__ len_out, int32_t *__restrict__ maxlen) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t id = perm ? perm[i] : i;
    int64_t l = off[id + 1] - off[id];
    len_out[i] = l;
    atomicMax(maxlen, (int32_t)(l < INT_MAX ? l : INT_MAX));
}

__global__ void k_gather_strings(int64_t n, const int32_t *__restrict__ perm, const uint8_t *__restrict__ S,
                                 const int64_t *__restrict__ off, const int64_t *__restrict__ noff,
                                 uint8_t *__restrict__ out) {
    int64_t i = blockIdx.x;
    if (i >= n) return;
    int64_t id = perm[i];
    int64_t b = off[id], l = off[id + 1] - b, o = noff[i];
    for (int64_t k = threadIdx.x; k < l; k += blockDim.x) out[o + k] = S[b + k];
}

// Query groups: greedy runs of consecutive sibling leaf blocks of at most
// kGroupSize points in total; a larger block is cut into groups of kGroupSize
// consecutive points (the last one shorter) that hold no other block.  The
// leaf blocks are in position order; k_group_prep lays out each block's size
// and parent in that order, a run of siblings starts where the parent
// changes, and one thread walks each run (sequential reads), marking how many
// groups start at each block and recording the size of a merged group there.
__global__ void k_group_prep(int L, const int32_t *__restrict__ leaf_ids, const int32_t *__restrict__ node_count,
                             const int32_t *__restrict__ parent, int32_t *__restrict__ lcount,
                             int32_t *__restrict__ lpar) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L) return;
    const int v = leaf_ids[i];
    lcount[i] = node_count[v];
    lpar[i] = parent[v];
}

__global__ void k_group_marks(int L, const int32_t *__restrict__ lcount, const int32_t *__restrict__ lpar,
                              int32_t *__restrict__ gstart, int32_t *__restrict__ gsize,
                              unsigned long long *__restrict__ maxc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L) return;
    const int p = lpar[i];
    if (i > 0 && lpar[i - 1] == p) return;  // not the first block of its sibling run
    int first = -1, acc = 0, big = 0;
    for (int j = i; j < L && lpar[j] == p; ++j) {
        const int c = lcount[j];
        if (c > kGroupSize) {  // groups of its own
            if (first >= 0) gsize[first] = acc;
            gstart[j] = (c + kGroupSize - 1) / kGroupSize;
            gsize[j] = c;
            big = kGroupSize;
            first = -1;
            acc = 0;
        } else if (first >= 0 && acc + c <= kGroupSize) {
            acc += c;
            gstart[j] = 0;
        } else {
            if (first >= 0) gsize[first] = acc;
            big = max(big, acc);
            first = j;
            acc = c;
            gstart[j] = 1;
        }
    }
    if (first >= 0) gsize[first] = acc;
    big = max(big, acc);
    atomicMax(maxc, (unsigned long long)big);
}

__global__ void k_group_scatter(int L, const int32_t *__restrict__ leaf_ids, const int32_t *__restrict__ node_begin,
                                const int32_t *__restrict__ gstart, const int32_t *__restrict__ gsize,
                                const int64_t *__restrict__ gidx, int32_t *__restrict__ group_begin,
                                int32_t *__restrict__ group_count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L || !gstart[i]) return;
    const int64_t g = gidx[i];
    const int b = node_begin[leaf_ids[i]], c = gsize[i];
    for (int k = 0; k < gstart[i]; ++k) {  // one group, or the cuts of a large block
        group_begin[g + k] = b + k * kGroupSize;
        group_count[g + k] = min(kGroupSize, c - k * kGroupSize);
    }
}

// Sort keys putting larger radii first (radii are non-negative floats).
__global__ void k_radius_desc_keys(int ng, const float *__restrict__ r, uint32_t *__restrict__ keys,
                                   uint32_t *__restrict__ vals) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    keys[g] = 0xFFFFFFFFu - __float_as_uint(r[g]);
    vals[g] = (uint32_t)g;
}

// Radius of each query group: max distance from its first point (rounded up).
// One warp per group, one lane per point.
__global__ void k_group_radius_l2(int ng, const int32_t *__restrict__ gbeg, const int32_t *__restrict__ gcnt,
                                  const float *__restrict__ pts, int dp, float *__restrict__ grad) {
    int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (g >= ng) return;
    const float4 *c = reinterpret_cast<const float4 *>(pts + (size_t)gbeg[g] * dp);
    float r = 0.f;
    for (int i = lane; i < gcnt[g]; i += 32) {
        const float4 *p = reinterpret_cast<const float4 *>(pts + (size_t)(gbeg[g] + i) * dp);
        float acc = 0.f;
        for (int k = 0; k < dp / 4; ++k) {
            float4 a = __ldg(c + k), b = __ldg(p + k);
            float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z, dw = a.w - b.w;
            acc = fmaf(dx, dx, acc); acc = fmaf(dy, dy, acc); acc = fmaf(dz, dz, acc); acc = fmaf(dw, dw, acc);
        }
        r = fmaxf(r, sqrtf(acc));
    }
    for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    if (lane == 0) grad[g] = round_radius_up(r, CT_L2_F32);
}

template <int W>
__global__ void __launch_bounds__(32) k_group_radius_lev(int ng, const int32_t *__restrict__ gbeg,
                                                         const int32_t *__restrict__ gcnt,
                                                         const uint8_t *__restrict__ S,
                                                         const int64_t *__restrict__ off, float *__restrict__ grad) {
    __shared__ uint64_t peq[256 * W];
    int g = blockIdx.x;
    if (g >= ng) return;
    int cpos = gbeg[g];
    const uint8_t *pat = S + off[cpos];
    int m = (int)(off[cpos + 1] - off[cpos]);
    lev_build_peq<W>(peq, pat, m);
    __syncthreads();
    int r = 0;
    for (int i = threadIdx.x; i < gcnt[g]; i += 32) {
        int p = cpos + i;
        int d = lev_myers<W>(peq, m, S + off[p], (int)(off[p + 1] - off[p]), INT_MAX / 2);
        r = max(r, d);
    }
    for (int o = 16; o > 0; o >>= 1) r = max(r, __shfl_xor_sync(0xffffffffu, r, o));
    if (threadIdx.x == 0) grad[g] = (float)r;
}

inline unsigned grid_for(int64_t n, int t = BT) { return (unsigned)ceil_div(n > 0 ? n : 1, t); }

int bits_for(int64_t v) {
    int b = 0;
    while ((int64_t(1) << b) <= v && b < 62) ++b;
    return b;
}

}  // namespace

// Builds the tree; on failure throws ct::Error after freeing what it allocated.
void free_tree(ct_tree *t);

namespace {
struct TreeGuard {
    ct_tree *t;
    ~TreeGuard() { if (t) free_tree(t); }
};
}  // namespace

ct_tree *build_tree(const ct_points *pts, int zeta, int root, cudaStream_t s) {
    const int64_t n = pts->n;
    TreeGuard tg{new ct_tree()};
    ct_tree *t = tg.t;
    struct Flush { ~Flush() { prof_flush(); } } flush_at_exit;
    ProfScope prof_all("build", s);
    t->metric = pts->metric;
    t->n = n;
    t->leaf_size = zeta;
    t->stream = s;
    CT_CHECK_CUDA(cudaGetDevice(&t->device));
    const bool l2 = pts->metric == CT_L2_F32;
    const bool ham = pts->metric == CT_HAMMING_B1;
    const bool lev = pts->metric == CT_LEVENSHTEIN_U8;
    t->dim = l2 || ham ? pts->dim : 0;
    t->dp = l2 ? (int)ceil_div(pts->dim, 4) * 4 : 0;
    t->wp = ham ? (int)ceil_div(pts->dim, 128) * 4 : 0;
    const int dp = t->dp, wp = t->wp;

    DBuf<int32_t> err(2, s);
    CT_CHECK_CUDA(cudaMemsetAsync(err.p, 0, 2 * sizeof(int32_t), s));

    // padded copy of the input (original order) / string lengths
    DBuf<float> Xp;
    DBuf<uint32_t> Xb;
    int W = 1;
    if (ham) {
        Xb = DBuf<uint32_t>((size_t)(n ? n : 1) * wp, s);
        if (n) {
            k_pack_bits<<<grid_for(n * wp), BT, 0, s>>>((const uint8_t *)pts->data, n, pts->dim, wp, Xb.p);
            CT_COUNT_LAUNCH();
        }
    } else if (l2) {
        Xp = DBuf<float>((size_t)n * dp, s);
        if (n && dp == pts->dim && (reinterpret_cast<uintptr_t>(pts->data) & 15) == 0) {
            const int64_t nq = n * dp / 4;
            k_copy_rows4<<<grid_for(nq), BT, 0, s>>>((const float4 *)pts->data, nq, (float4 *)Xp.p, err.p);
            CT_COUNT_LAUNCH();
        } else if (n) {
            k_pad_rows<<<grid_for(n * dp), BT, 0, s>>>((const float *)pts->data, n, pts->dim, dp, Xp.p, err.p);
            CT_COUNT_LAUNCH();
        }
    } else {
        DBuf<int64_t> lens(n > 0 ? n : 1, s);
        if (n) {
            k_string_lengths<<<grid_for(n), BT, 0, s>>>(n, nullptr, pts->offsets, lens.p, err.p + 1);
            CT_COUNT_LAUNCH();
        }
    }
    CT_LAUNCH_CHECK();
    int32_t herr[2] = {0, 0};
    to_host(herr, err.p, 2, s);
    if (herr[0]) CT_FAIL(CT_EUNSUPPORTED, "coordinates must be finite with |x| <= 2^50");
    if (lev) {
        if (herr[1] > CT_MAX_STRING_LEN)
            CT_FAIL(CT_EUNSUPPORTED, "string of length %d above the limit %d", herr[1], CT_MAX_STRING_LEN);
        t->max_len = herr[1];
        W = lev_words_for(t->max_len);
    }

    // tree arrays: a tree whose internal vertices have >= 2 children has < 2n vertices
    const int64_t cap = 2 * n + 1;
    DBuf<int32_t> nb(cap, s), ncnt(cap, s), cbeg(cap, s), ccnt(cap, s), lvl(cap, s), par(cap, s);
    CT_CHECK_CUDA(cudaMemsetAsync(par.p, 0xff, cap * sizeof(int32_t), s));
    DBuf<float> rad(cap, s);
    DBuf<int32_t> ids(n ? n : 1, s), lab(n ? n : 1, s);
    DBuf<float> D(n ? n : 1, s);

    int n_nodes = 0, depth = 0;
    if (n > 0) {
        if (root < 0 || root >= n) CT_FAIL(CT_EINVAL, "root %d out of range", root);
        // ---- round 0: distances to the root
        const int64_t cap_h = n;  // hubs per round never exceed n / (zeta+1) + 1
        DBuf<int32_t> hbuf(9 * (cap_h + 1), s);
        DBuf<float> hthr(cap_h + 1, s);
        DBuf<unsigned long long> hkey(cap_h + 1, s);
        DBuf<int32_t> hbuf2(9 * (cap_h + 1), s);
        DBuf<float> hthr2(cap_h + 1, s);
        DBuf<unsigned long long> hkey2(cap_h + 1, s);
        auto make_hubs = [&](DBuf<int32_t> &b, DBuf<float> &th, DBuf<unsigned long long> &k) {
            Hubs h;
            int64_t st = cap_h + 1;
            h.begin = b.p; h.count = b.p + st; h.node = b.p + 2 * st; h.nc = b.p + 3 * st;
            h.cur = b.p + 4 * st; h.done = b.p + 5 * st; h.level = b.p + 6 * st;
            h.flat = b.p + 7 * st; h.covered = b.p + 8 * st;
            h.thr = th.p; h.key = k.p;
            return h;
        };
        Hubs H = make_hubs(hbuf, hthr, hkey), H2 = make_hubs(hbuf2, hthr2, hkey2);

        k_root_init<<<grid_for(n), BT, 0, s>>>(n, root, ids.p, D.p, lab.p);
        CT_COUNT_LAUNCH();
        // one pass of the update kernel with the root as the only centre
        // lanes per distance: four 16-byte loads each (a pass has many rows in
        // flight); a chunk is eight passes of a block
        int tpd = 1;  // a power of two
        while (l2 && tpd < 32 && 2 * tpd * 16 <= dp) tpd *= 2;
        // points per block of an update pass: L2, eight passes of the block's
        // groups; Hamming, four per thread; edit distance, one per thread (a
        // long recurrence each: more blocks share a pass)
        const int chunk_len = l2 ? UPD_PASSES * (BT / tpd) : ham ? 4 * BT : BT;
        // staged update passes where the buffers fit (a pass's rows: BT / tpd
        // rows of dp / 4 float4s), with their shared memory allowed once
        const bool stage = l2 && (int64_t)(BT / tpd) * (dp / 4) <= UPD_STAGE_F4;
        const size_t stage_sm = ((size_t)dp / 4 + (size_t)UPD_STAGES * (BT / tpd) * (dp / 4)) * sizeof(float4);
        if (stage) {
            static std::once_flag once[6];
            auto allow = [&](int k, const void *fn) {
                std::call_once(once[k], [&] {
                    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(float4) * (1 + UPD_STAGES) * UPD_STAGE_F4));
                });
            };
            switch (tpd) {
                case 1: allow(0, (const void *)k_dist_update_l2<1, true>); break;
                case 2: allow(1, (const void *)k_dist_update_l2<2, true>); break;
                case 4: allow(2, (const void *)k_dist_update_l2<4, true>); break;
                case 8: allow(3, (const void *)k_dist_update_l2<8, true>); break;
                case 16: allow(4, (const void *)k_dist_update_l2<16, true>); break;
                case 32: allow(5, (const void *)k_dist_update_l2<32, true>); break;
            }
            CT_CHECK_CUDA(cudaGetLastError());
        }
        // pruned updates (L2): centre positions and centre-to-new-centre distances per hub label
        DBuf<int32_t> cpos(l2 ? n : 1, s);
        DBuf<float> dcc(l2 ? n : 1, s);
        bool prune = false;  // off for the root's first pass (no labels yet)
        auto update = [&](Hubs &hb, int64_t nchunks, const int32_t *chub, const int32_t *cst, Step st) {
            if (!nchunks) return;
            if (l2) {
                if (stage) {
                    switch (tpd) {
#define CT_UPD(T) case T: k_dist_update_l2<T, true><<<(unsigned)nchunks, BT, stage_sm, s>>>(Xp.p, dp, ids.p, D.p, lab.p, chub, cst, chunk_len, hb, prune ? dcc.p : nullptr, st); break;
                        CT_UPD(1) CT_UPD(2) CT_UPD(4) CT_UPD(8) CT_UPD(16) CT_UPD(32)
#undef CT_UPD
                    }
                } else {
                    const size_t sm = (size_t)dp * sizeof(float);
                    switch (tpd) {
#define CT_UPD(T) case T: k_dist_update_l2<T, false><<<(unsigned)nchunks, BT, sm, s>>>(Xp.p, dp, ids.p, D.p, lab.p, chub, cst, chunk_len, hb, prune ? dcc.p : nullptr, st); break;
                        CT_UPD(1) CT_UPD(2) CT_UPD(4) CT_UPD(8) CT_UPD(16) CT_UPD(32)
#undef CT_UPD
                    }
                }
            } else if (ham) {
                k_dist_update_ham<<<(unsigned)nchunks, BT, (size_t)wp * sizeof(uint32_t), s>>>(
                    Xb.p, wp, ids.p, D.p, lab.p, chub, cst, chunk_len, hb, st);
            } else {
                const uint8_t *S = (const uint8_t *)pts->data;
                switch (W) {
#define CT_UPDL(WW) case WW: k_dist_update_lev<WW><<<(unsigned)nchunks, BT, 0, s>>>(S, pts->offsets, ids.p, D.p, lab.p, chub, cst, chunk_len, hb, st); break;
                    CT_UPDL(1) CT_UPDL(2) CT_UPDL(4) CT_UPDL(8) CT_UPDL(16)
#undef CT_UPDL
                }
            }
            CT_COUNT_LAUNCH();
            CT_LAUNCH_CHECK();
        };
        // root hub state for the initial pass: centre = position 0, label 0
        {
            int32_t one = 1;
            int32_t zero = 0;
            unsigned long long z = 0;
            CT_CHECK_CUDA(cudaMemcpyAsync(H.begin, &zero, 4, cudaMemcpyHostToDevice, s));
            int32_t cnt = (int32_t)n;
            CT_CHECK_CUDA(cudaMemcpyAsync(H.count, &cnt, 4, cudaMemcpyHostToDevice, s));
            CT_CHECK_CUDA(cudaMemcpyAsync(H.nc, &one, 4, cudaMemcpyHostToDevice, s));
            CT_CHECK_CUDA(cudaMemcpyAsync(H.cur, &zero, 4, cudaMemcpyHostToDevice, s));
            CT_CHECK_CUDA(cudaMemcpyAsync(H.done, &zero, 4, cudaMemcpyHostToDevice, s));
            CT_CHECK_CUDA(cudaMemcpyAsync(H.flat, &zero, 4, cudaMemcpyHostToDevice, s));
            CT_CHECK_CUDA(cudaMemcpyAsync(H.covered, &zero, 4, cudaMemcpyHostToDevice, s));
            CT_CHECK_CUDA(cudaMemcpyAsync(H.key, &z, 8, cudaMemcpyHostToDevice, s));
            CT_CHECK_CUDA(cudaStreamSynchronize(s));  // host values above are on the stack
        }
        int64_t nchunks0 = ceil_div(n, chunk_len);
        DBuf<int32_t> chub(nchunks0, s), cst(nchunks0, s);
        {
            DBuf<int64_t> coff(1, s);
            CT_CHECK_CUDA(cudaMemsetAsync(coff.p, 0, sizeof(int64_t), s));
            k_chunk_fill<<<grid_for(nchunks0), BT, 0, s>>>(nchunks0, 1, H.begin, coff.p, chunk_len, chub.p, cst.p);
            CT_COUNT_LAUNCH();
            update(H, nchunks0, chub.p, cst.p, Step{});
        }
        DBuf<int32_t> is_root_hub(1, s);
        k_root_node<<<1, 1, 0, s>>>(n, zeta, pts->metric, H.key, nb.p, ncnt.p, cbeg.p, ccnt.p, rad.p, lvl.p, H,
                                    is_root_hub.p);
        CT_COUNT_LAUNCH();
        CT_LAUNCH_CHECK();
        int32_t root_hub = 0;
        to_host(&root_hub, is_root_hub.p, 1, s);
        n_nodes = 1;
        int64_t nh = root_hub ? 1 : 0;

        // scratch for partitioning
        DBuf<uint32_t> pk(n, s), pv(n, s), tk(n, s), tv(n, s);
        DBuf<int32_t> rpos(n, s), tids(n, s);
        DBuf<float> tD(n, s);
        DBuf<int32_t> active(3, s);  // hub activations of a burst, active hubs, active chunks
        DBuf<int32_t> hlist(n, s), chub2(nchunks0, s), cst2(nchunks0, s);
        DBuf<int32_t> arrive(cap_h + 1, s);  // per hub: finished blocks of an update pass
        DBuf<int64_t> i64tmp(2, s);

        while (nh > 0) {
            ++depth;
            // chunk table of this round
            DBuf<int32_t> ccounts(nh, s);
            DBuf<int64_t> coff(nh, s);
            k_chunk_counts<<<grid_for(nh), BT, 0, s>>>((int)nh, H.count, chunk_len, ccounts.p);
            CT_COUNT_LAUNCH();
            exclusive_scan_i32_to_i64(ccounts.p, coff.p, nh, i64tmp.p, s);
            int64_t nchunks = 0;
            to_host(&nchunks, i64tmp.p, 1, s);
            chub.grow(nchunks);
            cst.grow(nchunks);
            chub2.grow(nchunks);
            cst2.grow(nchunks);
            k_chunk_fill<<<grid_for(nchunks), BT, 0, s>>>(nchunks, (int)nh, H.begin, coff.p, chunk_len, chub.p, cst.p);
            CT_COUNT_LAUNCH();
            CT_LAUNCH_CHECK();

            // split iterations (Algorithm 1) for every hub of the round
            {
                ProfScope prof_split("build_split", s);
                int burst = 1;
                int64_t iters = 0;
                bool first_step = true;
                // the hubs and chunks a burst visits: all at first, then those
                // of the hubs still splitting after the previous burst
                const int32_t *hl = nullptr;
                int64_t nl = nh, nck = nchunks;
                int32_t *cb = chub.p, *cs = cst.p, *cb2 = chub2.p, *cs2 = cst2.p;
                if (l2 && dp <= 128 && prune) {
                    // small hubs split whole in one CTA each; the loop below takes the rest
                    switch (tpd) {
#define CT_SS(T) case T: k_split_small<T><<<(unsigned)nh, BT, 0, s>>>(Xp.p, dp, ids.p, D.p, lab.p, H, err.p); break;
                        CT_SS(1) CT_SS(2) CT_SS(4) CT_SS(8) CT_SS(16) CT_SS(32)
#undef CT_SS
                    }
                    CT_COUNT_LAUNCH();
                    CT_CHECK_CUDA(cudaMemsetAsync(active.p, 0, 3 * sizeof(int32_t), s));
                    k_active_hubs<<<grid_for(nh), BT, 0, s>>>((int)nh, H.done, hlist.p, active.p + 1);
                    CT_COUNT_LAUNCH();
                    k_active_chunks<<<grid_for(nck), BT, 0, s>>>(nck, cb, cs, H.done, cb2, cs2, active.p + 2);
                    CT_COUNT_LAUNCH();
                    CT_LAUNCH_CHECK();
                    int32_t cnt3[3] = {0, 0, 0};
                    to_host(cnt3, active.p, 3, s);
                    hl = hlist.p;
                    nl = cnt3[1];
                    nck = cnt3[2];
                    std::swap(cb, cb2);
                    std::swap(cs, cs2);
                }
                for (; nl > 0;) {
                    // every iteration adds a distinct centre to some hub, so
                    // no hub is active after n + 1 of them; a burst of up to
                    // 16 may run past the last useful iteration
                    if (iters > n + 2 + 16) CT_FAIL(CT_ECUDA, "split loop did not terminate");
                    iters += burst;
                    CT_CHECK_CUDA(cudaMemsetAsync(active.p, 0, 3 * sizeof(int32_t), s));
                    if (l2) {
                        // the level's first step by its own kernels; every later
                        // step is taken inside the update pass by each hub's last block
                        if (first_step) {
                            CT_CHECK_CUDA(cudaMemsetAsync(arrive.p, 0, nh * sizeof(int32_t), s));
                            k_hub_step<<<grid_for(nl), BT, 0, s>>>((int)nl, hl, H, active.p, cpos.p, 1);
                            CT_COUNT_LAUNCH();
                            switch (tpd) {
#define CT_CD(T) case T: k_centre_dists<T><<<(unsigned)nl, BT, 0, s>>>(Xp.p, dp, ids.p, H, hl, cpos.p, dcc.p); break;
                                CT_CD(1) CT_CD(2) CT_CD(4) CT_CD(8) CT_CD(16) CT_CD(32)
#undef CT_CD
                            }
                            CT_COUNT_LAUNCH();
                            prune = true;
                            first_step = false;
                        }
                        const Step st{arrive.p, active.p, cpos.p, dcc.p};
                        for (int it = 0; it < burst; ++it) update(H, nck, cb, cs, st);
                    } else {
                        // the level's first step by k_hub_step; every later step
                        // is taken inside the update pass by each hub's last block
                        if (first_step) {
                            CT_CHECK_CUDA(cudaMemsetAsync(arrive.p, 0, nh * sizeof(int32_t), s));
                            k_hub_step<<<grid_for(nl), BT, 0, s>>>((int)nl, hl, H, active.p, nullptr, ham ? 1 : 0);
                            CT_COUNT_LAUNCH();
                            first_step = false;
                        }
                        const Step st{arrive.p, active.p, nullptr, nullptr};
                        for (int it = 0; it < burst; ++it) update(H, nck, cb, cs, st);
                    }
                    k_active_hubs<<<grid_for(nh), BT, 0, s>>>((int)nh, H.done, hlist.p, active.p + 1);
                    CT_COUNT_LAUNCH();
                    if (nck) {
                        k_active_chunks<<<grid_for(nck), BT, 0, s>>>(nck, cb, cs, H.done, cb2, cs2, active.p + 2);
                        CT_COUNT_LAUNCH();
                    }
                    CT_LAUNCH_CHECK();
                    int32_t act[3] = {0, 0, 0};
                    to_host(act, active.p, 3, s);
                    if (act[0] == 0) break;
                    hl = hlist.p;
                    nl = act[1];
                    nck = act[2];
                    std::swap(cb, cb2);
                    std::swap(cs, cs2);
                    if (nl == 0) break;
                    burst = burst < 16 ? burst * 2 : 16;
                }
            }

            // partition the round's points by (hub, label)
            DBuf<int32_t> ncs(nh, s);
            DBuf<int64_t> child_base(nh, s), round_off(nh, s);
            CT_CHECK_CUDA(cudaMemcpyAsync(ncs.p, H.nc, nh * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
            exclusive_scan_i32_to_i64(ncs.p, child_base.p, nh, i64tmp.p, s);
            exclusive_scan_i32_to_i64(H.count, round_off.p, nh, i64tmp.p + 1, s);
            int64_t tot[2];
            to_host(tot, i64tmp.p, 2, s);
            const int64_t T = tot[0], R = tot[1];
            if (n_nodes + T > cap) CT_FAIL(CT_ECUDA, "vertex capacity exceeded");
            k_part_keys<<<grid_for(R), BT, 0, s>>>(R, (int)nh, H.begin, round_off.p, child_base.p, lab.p, pk.p,
                                                   pv.p, rpos.p);
            CT_COUNT_LAUNCH();
            radix_sort_pairs(pk.p, pv.p, tk.p, tv.p, R, bits_for(T), s);
            DBuf<int32_t> ccount(T, s), cbegin(T, s), czero(T, s), is_hub(T, s), leafy(T, s);
            DBuf<unsigned long long> ckey(T, s);
            CT_CHECK_CUDA(cudaMemsetAsync(ccount.p, 0, T * sizeof(int32_t), s));
            CT_CHECK_CUDA(cudaMemsetAsync(cbegin.p, 0x7f, T * sizeof(int32_t), s));
            CT_CHECK_CUDA(cudaMemsetAsync(czero.p, 0x7f, T * sizeof(int32_t), s));
            CT_CHECK_CUDA(cudaMemsetAsync(ckey.p, 0, T * sizeof(unsigned long long), s));
            k_part_gather<<<grid_for(R), BT, 0, s>>>(R, pk.p, pv.p, rpos.p, ids.p, D.p, tids.p, tD.p, ccount.p,
                                                     cbegin.p, czero.p);
            CT_COUNT_LAUNCH();
            k_part_scatter<<<grid_for(R), BT, 0, s>>>(R, rpos.p, tids.p, tD.p, ids.p, D.p, lab.p);
            CT_COUNT_LAUNCH();
            k_centre_front<<<grid_for(T), BT, 0, s>>>(T, cbegin.p, czero.p, ids.p, D.p, err.p);
            CT_COUNT_LAUNCH();
            k_child_keys<<<grid_for(R), BT, 0, s>>>(R, pk.p, rpos.p, D.p, ckey.p);
            CT_COUNT_LAUNCH();
            k_link_children<<<grid_for(nh), BT, 0, s>>>((int)nh, H, child_base.p, n_nodes, cbeg.p, ccnt.p, lvl.p, par.p,
                                                         leafy.p);
            CT_COUNT_LAUNCH();
            k_make_nodes<<<grid_for(T), BT, 0, s>>>(T, n_nodes, zeta, pts->metric, cbegin.p, ccount.p, ckey.p,
                                                    nb.p, ncnt.p, cbeg.p, ccnt.p, rad.p, lvl.p, leafy.p, is_hub.p);
            CT_COUNT_LAUNCH();
            DBuf<int64_t> hub_off(T, s);
            exclusive_scan_i32_to_i64(is_hub.p, hub_off.p, T, i64tmp.p, s);
            int64_t nh2 = 0;
            to_host(&nh2, i64tmp.p, 1, s);
            if (nh2 > cap_h) CT_FAIL(CT_ECUDA, "hub capacity exceeded");
            k_next_hubs<<<grid_for(T), BT, 0, s>>>(T, n_nodes, is_hub.p, hub_off.p, cbegin.p, ccount.p, ckey.p, lvl.p,
                                                   H2);
            CT_COUNT_LAUNCH();
            CT_LAUNCH_CHECK();
            n_nodes += (int)T;
            std::swap(H, H2);
            nh = nh2;
        }
        int32_t e2 = 0;
        to_host(&e2, err.p, 1, s);
        if (e2) CT_FAIL(CT_ECUDA, "internal: a child without a zero-distance centre");
    }

    // ---- final layout
    t->n_nodes = n_nodes;
    t->depth = depth;
    t->perm = ids.release();
    t->dcen = D.release();
    lab.reset();
    if (n == 0) {
        // empty tree: keep valid (non-null) small allocations
        t->perm = (int32_t *)dmalloc(sizeof(int32_t), s);
        t->dcen = (float *)dmalloc(sizeof(float), s);
    }
    if (l2) {
        t->pts = (float *)dmalloc((size_t)(n ? n : 1) * dp * sizeof(float) + 16, s);
        if (n) {
            k_gather_rows<<<grid_for(n * (dp / 4)), BT, 0, s>>>(Xp.p, dp, t->perm, n, t->pts);
            CT_COUNT_LAUNCH();
        }
        Xp.reset();
    } else if (ham) {
        t->bits = (uint32_t *)dmalloc((size_t)(n ? n : 1) * wp * sizeof(uint32_t) + 16, s);
        if (n) {
            k_gather_bits<<<grid_for(n * (wp / 4)), BT, 0, s>>>(Xb.p, wp, t->perm, n, t->bits);
            CT_COUNT_LAUNCH();
        }
        Xb.reset();
    } else {
        DBuf<int64_t> lens(n + 1, s);
        DBuf<int32_t> ml(1, s);
        CT_CHECK_CUDA(cudaMemsetAsync(ml.p, 0, sizeof(int32_t), s));
        if (n) {
            k_string_lengths<<<grid_for(n), BT, 0, s>>>(n, t->perm, pts->offsets, lens.p, ml.p);
            CT_COUNT_LAUNCH();
        }
        t->soff = (int64_t *)dmalloc((size_t)(n + 1) * sizeof(int64_t), s);
        DBuf<int64_t> tot(1, s);
        exclusive_scan_i64(lens.p, t->soff, n, tot.p, s);
        CT_CHECK_CUDA(cudaMemcpyAsync(t->soff + n, tot.p, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
        int64_t total = 0;
        to_host(&total, tot.p, 1, s);
        t->sbytes = total;
        t->sdata = (uint8_t *)dmalloc((size_t)total + 16, s);
        if (n) {
            k_gather_strings<<<(unsigned)n, 128, 0, s>>>(n, t->perm, (const uint8_t *)pts->data, pts->offsets,
                                                         t->soff, t->sdata);
            CT_COUNT_LAUNCH();
        }
    }
    // shrink vertex arrays to n_nodes
    auto shrink_i = [&](DBuf<int32_t> &b) {
        int32_t *p = (int32_t *)dmalloc(sizeof(int32_t) * (size_t)(n_nodes ? n_nodes : 1), s);
        if (n_nodes) CT_CHECK_CUDA(cudaMemcpyAsync(p, b.p, sizeof(int32_t) * n_nodes, cudaMemcpyDeviceToDevice, s));
        b.reset();
        return p;
    };
    t->node_begin = shrink_i(nb);
    t->node_count = shrink_i(ncnt);
    t->child_begin = shrink_i(cbeg);
    t->child_count = shrink_i(ccnt);
    t->level = shrink_i(lvl);
    t->parent = shrink_i(par);
    t->radius = (float *)dmalloc(sizeof(float) * (size_t)(n_nodes ? n_nodes : 1), s);
    if (n_nodes) CT_CHECK_CUDA(cudaMemcpyAsync(t->radius, rad.p, sizeof(float) * n_nodes, cudaMemcpyDeviceToDevice, s));
    rad.reset();
    if (l2) {
        t->node_ctr = (float *)dmalloc(sizeof(float) * (size_t)(n_nodes ? n_nodes : 1) * dp + 16, s);
        if (n_nodes) {
            k_node_centres<<<grid_for((int64_t)n_nodes * (dp / 4)), BT, 0, s>>>(n_nodes, t->node_begin, t->pts, dp,
                                                                               t->node_ctr);
            CT_COUNT_LAUNCH();
        }
    }
    // leaf blocks in position order
    {
        int64_t nn = n_nodes ? n_nodes : 1;
        DBuf<uint32_t> k1(nn, s), v1(nn, s), k2(nn, s), v2(nn, s);
        DBuf<int32_t> cnts(2, s);
        CT_CHECK_CUDA(cudaMemsetAsync(cnts.p, 0, 2 * sizeof(int32_t), s));
        if (n_nodes) {
            k_leaf_keys<<<grid_for(n_nodes), BT, 0, s>>>(n_nodes, t->child_count, t->node_begin, t->node_count, k1.p,
                                                         v1.p, cnts.p, cnts.p + 1);
            CT_COUNT_LAUNCH();
        }
        int32_t hc[2];
        to_host(hc, cnts.p, 2, s);
        t->n_leaves = hc[0];
        t->max_leaf_count = hc[1];
        radix_sort_pairs(k1.p, v1.p, k2.p, v2.p, hc[0], bits_for(n), s);
        t->leaf_ids = (int32_t *)dmalloc(sizeof(int32_t) * (size_t)(hc[0] ? hc[0] : 1), s);
        if (hc[0]) CT_CHECK_CUDA(cudaMemcpyAsync(t->leaf_ids, v1.p, sizeof(int32_t) * hc[0], cudaMemcpyDeviceToDevice, s));
    }
    // query groups: greedy runs of consecutive sibling leaf blocks (k_group_marks)
    {
        const int L = t->n_leaves;
        DBuf<int32_t> gstart(L ? L : 1, s), gsize(L ? L : 1, s), lcount(L ? L : 1, s), lpar(L ? L : 1, s);
        DBuf<int64_t> gidx(L ? L : 1, s), tot(2, s);  // tot: group count, largest group
        CT_CHECK_CUDA(cudaMemsetAsync(tot.p, 0, 2 * sizeof(int64_t), s));
        if (L) {
            k_group_prep<<<grid_for(L), BT, 0, s>>>(L, t->leaf_ids, t->node_count, t->parent, lcount.p, lpar.p);
            CT_COUNT_LAUNCH();
            k_group_marks<<<grid_for(L), BT, 0, s>>>(L, lcount.p, lpar.p, gstart.p, gsize.p,
                                                     reinterpret_cast<unsigned long long *>(tot.p + 1));
            CT_COUNT_LAUNCH();
            exclusive_scan_i32_to_i64(gstart.p, gidx.p, L, tot.p, s);
        }
        int64_t gh[2] = {0, 0};
        to_host(gh, tot.p, 2, s);
        const int G = (int)gh[0];
        t->n_groups = G;
        t->max_group_count = (int)gh[1];
        t->group_begin = (int32_t *)dmalloc(sizeof(int32_t) * (size_t)(G ? G : 1), s);
        t->group_count = (int32_t *)dmalloc(sizeof(int32_t) * (size_t)(G ? G : 1), s);
        if (G) {
            k_group_scatter<<<grid_for(L), BT, 0, s>>>(L, t->leaf_ids, t->node_begin, gstart.p, gsize.p, gidx.p,
                                                       t->group_begin, t->group_count);
            CT_COUNT_LAUNCH();
        }
        t->group_radius = (float *)dmalloc(sizeof(float) * (size_t)(G ? G : 1), s);
        if (G) {
            if (ham) {
                k_group_radius_ham<<<grid_for((int64_t)G * 32), BT, 0, s>>>(G, t->group_begin, t->group_count,
                                                                           t->bits, wp, t->group_radius);
            } else if (l2) {
                k_group_radius_l2<<<grid_for((int64_t)G * 32), BT, 0, s>>>(G, t->group_begin, t->group_count, t->pts,
                                                                          dp, t->group_radius);
            } else {
                switch (W) {
#define CT_GR(WW) case WW: k_group_radius_lev<WW><<<G, 32, 0, s>>>(G, t->group_begin, t->group_count, t->sdata, t->soff, t->group_radius); break;
                    CT_GR(1) CT_GR(2) CT_GR(4) CT_GR(8) CT_GR(16)
#undef CT_GR
                }
            }
            CT_COUNT_LAUNCH();
        }
        // traversal order: groups with larger balls walk more of the tree; taking
        // them first shortens the tail of the dynamically scheduled walk
        t->group_order = (int32_t *)dmalloc(sizeof(int32_t) * (size_t)(G ? G : 1), s);
        if (G) {
            DBuf<uint32_t> ok(G, s), ov(G, s), tk2(G, s), tv2(G, s);
            k_radius_desc_keys<<<grid_for(G), BT, 0, s>>>(G, t->group_radius, ok.p, ov.p);
            CT_COUNT_LAUNCH();
            radix_sort_pairs(ok.p, ov.p, tk2.p, tv2.p, G, 32, s);
            CT_CHECK_CUDA(cudaMemcpyAsync(t->group_order, ov.p, sizeof(int32_t) * G, cudaMemcpyDeviceToDevice, s));
        }
    }
    CT_LAUNCH_CHECK();
    CT_CHECK_CUDA(cudaStreamSynchronize(s));
    tg.t = nullptr;
    return t;
}

void free_tree(ct_tree *t) {
    if (!t) return;
    cudaStream_t s = t->stream;
    void *ptrs[] = {t->pts, t->bits, t->sdata, t->soff, t->perm, t->dcen, t->node_begin, t->node_count,
                    t->child_begin, t->child_count, t->radius, t->level, t->node_ctr, t->leaf_ids,
                    t->parent, t->group_begin, t->group_count, t->group_radius, t->group_order};
    for (void *p : ptrs)
        if (p) cudaFreeAsync(p, s);
    cudaStreamSynchronize(s);
    delete t;
}

}  // namespace ct
