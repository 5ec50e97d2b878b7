// query.cu -- the batched ε query (Algorithm 3 with the batching of Sec. IV-B)
// as a two-pass count -> scan -> emit pipeline, plus the CSR row sort.
//
// Query groups are the tree's leaf blocks (<= zeta points, contiguous in tree
// order, centre c_g, radius r_g).  Stages:
//   1. traversal (k_traverse_*): one warp per group walks the tree from the
//      root with a stack of sibling ranges; 32 vertices are tested at a time,
//      one per lane.  A vertex v survives iff d(c_g, v) <= r(v) + eps + r_g
//      (every query q of the group has d(q, c_g) <= r_g, so no descendant of a
//      pruned v is within eps of any q: triangle inequality).  Survivors are
//      compacted with ballots: leaf blocks are candidates, internal vertices
//      push their child range.  Run twice: count, then fill a CSR of
//      candidates per group.
//   2. leaf tiles (k_leaf_*): one CTA per group evaluates every (query,
//      candidate point) pair and decides d(q, p) <= eps exactly (see QParams).
//      Count pass: per-query degree, and a flag on every candidate block that
//      produced an edge.  Emit pass: flagged blocks only; writes col/dist at
//      the row offsets.
//   3. scan of degrees to row_ptr (int64), then a per-row sort by column.
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstring>
#include <cuda.h>
#include <mutex>

#include "lev.cuh"
#include "profile.cuh"
#include "query.cuh"
#include "tc.cuh"
#include "l2dist.cuh"

namespace ct {

namespace {

constexpr int TRAV_WARPS = 4;              // warps per traversal block
constexpr int LEAF_T = 128;                // threads per leaf-tile block
constexpr int KC = 128;                    // floats per K chunk of a tile
constexpr int KS4 = KC / 4 + 1;            // padded row stride in float4
constexpr uint32_t FLAG = 0x80000000u;     // candidate produced an edge
constexpr float PRUNE_REL = 1.0f + 0x1p-10f;
constexpr float PRUNE_ABS = 0x1p-60f;


// Diagnostic (off unless a test sets it): the CSR rows of both ends of every
// pair a count pass decides by the FP64 sum, appended to a caller's buffer.
__device__ int32_t *g_guard_rows = nullptr;
__device__ unsigned long long *g_guard_n = nullptr;
__device__ long long g_guard_cap = 0;

__device__ __forceinline__ void note_guard_rows(int32_t a, int32_t b) {
    int32_t *r = g_guard_rows;
    if (!r) return;
    const unsigned long long k = atomicAdd(g_guard_n, 2ull);
    if ((long long)k + 1 < g_guard_cap) {
        r[k] = a;
        r[k + 1] = b;
    }
}

__device__ __forceinline__ void stat_add(unsigned long long *st, int slot, unsigned long long v) {
    if (v) atomicAdd(st + slot, v);
}

struct TreeView {
    const float *pts, *node_ctr, *radius, *dcen, *group_radius;
    const uint32_t *bits;  // Hamming rows (wp words each)
    const int32_t *perm, *node_begin, *node_count, *child_begin, *child_count, *leaf_ids;
    const int32_t *group_begin, *group_count, *group_order;
    const uint8_t *sdata;
    const int64_t *soff;
    int dp, dim, n_leaves, n_groups, wp;
};

TreeView view_of(const ct_tree *t) {
    TreeView v;
    v.pts = t->pts; v.node_ctr = t->node_ctr; v.radius = t->radius; v.dcen = t->dcen;
    v.perm = t->perm; v.node_begin = t->node_begin; v.node_count = t->node_count;
    v.child_begin = t->child_begin; v.child_count = t->child_count; v.leaf_ids = t->leaf_ids;
    v.sdata = t->sdata; v.soff = t->soff; v.dp = t->dp; v.dim = t->dim; v.n_leaves = t->n_leaves;
    v.group_begin = t->group_begin; v.group_count = t->group_count; v.group_radius = t->group_radius;
    v.group_order = t->group_order;
    v.n_groups = t->n_groups;
    v.bits = t->bits;
    v.wp = t->wp;
    return v;
}

// Up to kMaxClouds trees queried by the same launches (in the kernel parameter
// bank): global group gg of cloud c is gbase[c] + g, global row rbase[c] + o.
// A single query is the case nc = 1.
constexpr int kMaxClouds = kBatchClouds;
struct Views {
    int nc;
    int32_t gbase[kMaxClouds + 1];
    int64_t rbase[kMaxClouds + 1];
    TreeView tv[kMaxClouds];
    QParams qp[kMaxClouds];
    int16_t item_len[kMaxClouds];  // candidate blocks per work item
    uint8_t use_tc[kMaxClouds];    // leaf kernel of the count pass: tensor-core tiles (1) or FP32 tiles (0)
    // tensor-core filter rows: the fp16 rows, a TMA map of them, their squared norms, {s, s eps_up}
    const uint4 *h16[kMaxClouds];
    const float *n16[kMaxClouds];
    const float *s16[kMaxClouds];
    CUtensorMap tmap[kMaxClouds];  // (a 128-byte aligned type)
};
static_assert(sizeof(Views) <= 32000, "Views exceeds the kernel parameter space");
__device__ __forceinline__ int cloud_of_group(const Views &V, int gg) {
    int lo = 0, hi = V.nc;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (V.gbase[mid] <= gg) lo = mid; else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------ traversal
//
// One pass: every warp appends the candidate leaf blocks of its groups to
// private chunks of a shared pool; a group's candidates form one or more
// segments (group, pool offset, count).  If the pool runs out, the host reruns
// the pass with the exact size.

constexpr int POOL_CHUNK = 2048;

struct Pool {
    uint32_t *data;
    int64_t cap;
    unsigned long long *next;  // chunk allocator
    int32_t *seg_group, *seg_count;
    int64_t *seg_begin;
    int32_t *nseg;
    int64_t seg_cap;
    unsigned long long *total;  // candidates of all groups
    int32_t *overflow;
};

// Walks stopped at a step limit leave their stack's ranges here, as items
// (global group, first vertex, count, -) that the next round walks.
struct Spill {
    int4 *items;
    int32_t *count;  // may exceed cap: ranges past cap were not stored
    int cap;
    int limit;       // steps before a walk stops
};
constexpr int TRAV_ROUNDS = 4;     // rounds after the groups' round; the last one has no step limit
constexpr int TRAV_LIMIT0 = 256;   // step limit of the groups' round
constexpr int TRAV_LIMIT = 128;    // step limit of the next rounds
// edit distance: a step (32 bit-parallel recurrences) costs about a hundred
// L2 steps, so its walks stop much sooner
constexpr int TRAV_LIMIT0_LEV = 8, TRAV_LIMIT_LEV = 8;

// Warp-uniform write cursor: current chunk, its fill, the open segment.
struct PoolCursor {
    int64_t cur;
    int fill;
    int64_t seg_begin;
    int seg_count;
};

__device__ __forceinline__ void pool_close(const Pool &P, int g, PoolCursor &pc) {
    if (pc.seg_count > 0 && (threadIdx.x & 31) == 0) {
        int idx = atomicAdd(P.nseg, 1);
        if (idx < P.seg_cap) {
            P.seg_group[idx] = g;
            P.seg_begin[idx] = pc.seg_begin;
            P.seg_count[idx] = pc.seg_count;
        } else {
            atomicOr(P.overflow, 1);
        }
    }
    pc.seg_count = 0;
}

// Appends the values of the lanes with `flag` set, in lane order.
__device__ __forceinline__ void pool_append(const Pool &P, int g, PoolCursor &pc, bool flag, uint32_t v) {
    const int lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    const int n = __popc(m);
    if (!n) return;
    const int rank = __popc(m & lanemask_lt());
    const int room = pc.cur >= 0 ? POOL_CHUNK - pc.fill : 0;
    if (n <= room) {
        if (flag) P.data[pc.cur + pc.fill + rank] = v;
        pc.fill += n;
        pc.seg_count += n;
        return;
    }
    if (flag && rank < room) P.data[pc.cur + pc.fill + rank] = v;
    pc.seg_count += room;
    pool_close(P, g, pc);
    unsigned long long c = 0ull;
    if (lane == 0) c = atomicAdd(P.next, (unsigned long long)POOL_CHUNK);
    c = __shfl_sync(0xffffffffu, c, 0);
    if ((int64_t)c + POOL_CHUNK > P.cap) {  // out of pool: keep counting, write nothing
        if (lane == 0) atomicOr(P.overflow, 1);
        pc.cur = -1;
        pc.fill = POOL_CHUNK;
        pc.seg_begin = 0;
        pc.seg_count = 0;
        return;
    }
    pc.cur = (int64_t)c;
    pc.fill = n - room;
    pc.seg_begin = pc.cur;
    pc.seg_count = n - room;
    if (flag && rank >= room) P.data[pc.cur + rank - room] = v;
}

// DFS over ranges of sibling vertices from `start` (count 0: the root's
// children): up to 32 vertices are tested per step, vertex i of the step by
// lane i (`tester(v, n)` returns the keep flag of the lane's vertex v, for
// lanes below n); a top range shorter than 32 is completed from the range
// below it, so that fewer lanes idle; survivors are
// compacted with ballots -- leaf blocks are appended to the pool, internal
// vertices push their child range.  The vertices' child ranges are loaded
// before the test, so that their loads overlap the test's.  With `sp`, a walk
// that reaches sp->limit steps stores the ranges left on its stack in
// sp->items and stops (if they do not fit it goes on).
template <class Tester>
__device__ __forceinline__ int walk_group(const TreeView &tv, int2 *__restrict__ stack, int cap, int g, int2 start,
                                          const Pool &P, PoolCursor &pc, unsigned long long &evals,
                                          int32_t *__restrict__ err, const Spill *sp, Tester tester) {
    const int lane = threadIdx.x & 31;
    int n_cand = 0;
    pc.seg_begin = pc.cur + pc.fill;
    pc.seg_count = 0;
    if (start.y == 0 && tv.child_count[0] == 0) {  // the root is a leaf block: it is the only candidate
        pool_append(P, g, pc, lane == 0, 0u);
        n_cand = 1;
    } else {
        int top = 0;
        if (lane == 0) stack[0] = start.y ? start : make_int2(tv.child_begin[0], tv.child_count[0]);
        top = 1;
        __syncwarp();
        int limit = sp ? sp->limit : INT_MAX;
        for (int steps = 0; top > 0; ++steps) {
            if (steps >= limit) {
                int base = 0;
                if (lane == 0) base = atomicAdd(sp->count, top);
                base = __shfl_sync(0xffffffffu, base, 0);
                if (base + top <= sp->cap) {
                    for (int i = lane; i < top; i += 32) {
                        const int2 r = stack[i];
                        sp->items[base + i] = make_int4(g, r.x, r.y, 0);
                    }
                    break;
                }
                // no room: the slots reserved below the end hold empty ranges
                // (count 0, skipped), and the walk is finished here
                for (int i = base + lane; i < sp->cap; i += 32) sp->items[i] = make_int4(g, 0, 0, 0);
                limit = INT_MAX;
            }
            // the step's vertices: the top ranges of the stack, newest first,
            // until the 32 lanes are filled (lane i reads the i-th range from
            // the top; ranges are never empty); the last range drawn on may be
            // taken in part and keeps its rest on the stack.  A step reaches an
            // older block of ranges only when the newer ones are used up, so
            // the least deep vertex of each block on the stack is deeper than
            // the block below's: at most depth + 1 blocks of at most 32 ranges.
            const int nr = top < 32 ? top : 32;
            const int2 ri = lane < nr ? stack[top - 1 - lane] : make_int2(0, 0);
            int incl = ri.y;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int excl = incl - ri.y;
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            const int n = total < 32 ? total : 32;
            const int nfull = __popc(__ballot_sync(0xffffffffu, lane < nr && incl <= 32));
            // the first lane of each range drawn on, then each lane's range
            const unsigned smask = __reduce_or_sync(0xffffffffu, (lane < nr && excl < 32) ? 1u << excl : 0u);
            const int k = __popc(smask & (0xffffffffu >> (31 - lane))) - 1;
            const int kx = __shfl_sync(0xffffffffu, ri.x, k);
            const int ke = __shfl_sync(0xffffffffu, excl, k);
            const int px = __shfl_sync(0xffffffffu, ri.x, nfull & 31), py = __shfl_sync(0xffffffffu, ri.y, nfull & 31);
            const int pe = __shfl_sync(0xffffffffu, excl, nfull & 31);
            __syncwarp();
            top -= nfull;
            if (nfull < nr && pe < 32 && lane == 0) stack[top - 1] = make_int2(px + (32 - pe), py - (32 - pe));
            if (lane < n) ++evals;
            const int v = lane < n ? kx + (lane - ke) : 0;
            int ccount = 0, cbegin = 0;
            if (lane < n) {
                ccount = tv.child_count[v];
                cbegin = tv.child_begin[v];
            }
            const bool keep = tester(v, n);
            const bool leaf = keep && ccount == 0;
            pool_append(P, g, pc, keep && leaf, (uint32_t)v);
            n_cand += __popc(__ballot_sync(0xffffffffu, keep && leaf));
            const unsigned mi = __ballot_sync(0xffffffffu, keep && !leaf);
            const int np = __popc(mi);
            if (top + np > cap) {  // cannot happen for a stack of 32 * (depth + 2) ranges (above)
                if (lane == 0) atomicOr(err, 2);
                return -1;
            }
            if (keep && !leaf) {
                // reverse lane order so the lowest lane's children are on top (DFS order)
                int slot = top + __popc(mi & ~lanemask_lt() & ~(1u << lane));
                stack[slot] = make_int2(cbegin, ccount);
            }
            top += np;
            __syncwarp();
        }
    }
    pool_close(P, g, pc);
    if (lane == 0) atomicAdd(P.total, (unsigned long long)n_cand);
    return 0;
}

// Vertices the warp tested for group g (for fitting the predictor; the rounds
// of one group's walk add up).
__device__ __forceinline__ void group_visits(int32_t *gvisit, int g, unsigned long long mine) {
    unsigned long long v = mine;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(gvisit + g, (int32_t)(v < 0x7fffffffull ? v : 0x7fffffffull));
}

// L2 test of `take` consecutive vertices against the group centre (shared
// memory): TPD lanes share one vertex and read its centre row in coalesced
// 16-byte pieces; the partial sums are reduced by shuffles and lane i gets
// vertex i's squared distance.  Keep v unless d > (r(v) + eps + r_g)(1 + 2^-10).
template <int TPD>
__device__ __forceinline__ bool l2_keep(const TreeView &tv, const float4 *cen, int nq4, int vid, int take,
                                        float add) {
    constexpr int NPR = 32 / TPD;  // vertices per round; TPD rounds cover a step of 32
    const int lane = threadIdx.x & 31, sub = lane / TPD, j = lane % TPD;
    const float rad = lane < take ? tv.radius[vid] : 0.f;  // issued with the centre rows
    // all rounds' partial sums first (their loads overlap), then the reductions
    float part[TPD];
#pragma unroll
    for (int u = 0; u < TPD; ++u) {
        const int i = u * NPR + sub;
        const int vi = __shfl_sync(0xffffffffu, vid, i);  // vertex of lane i
        float acc = 0.f;
        if (u * NPR < take && i < take) {
            const float4 *row = reinterpret_cast<const float4 *>(tv.node_ctr) + (size_t)vi * nq4;
#pragma unroll 4
            for (int k = j; k < nq4; k += TPD) {
                const float4 a = cen[k], b = __ldg(row + k);
                const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z, dw = a.w - b.w;
                acc = fmaf(dx, dx, acc);
                acc = fmaf(dy, dy, acc);
                acc = fmaf(dz, dz, acc);
                acc = fmaf(dw, dw, acc);
            }
        }
        part[u] = acc;
    }
    float mine = 0.f;
#pragma unroll
    for (int u = 0; u < TPD; ++u) {
        if (u * NPR >= take) break;  // warp-uniform
        float acc = part[u];
#pragma unroll
        for (int o = TPD / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        const int r0 = u * NPR;
        const int src = ((lane - r0) & (NPR - 1)) * TPD;
        const float v = __shfl_sync(0xffffffffu, acc, src);
        if (lane >= r0 && lane < r0 + NPR) mine = v;
    }
    if (lane >= take) return false;
    const float bound = fmaf(rad + add, PRUNE_REL, PRUNE_ABS);
    return !(sqrtf(mine) > bound);
}

// Warp per group over all clouds' groups, taken dynamically in `order`
// (global group ids), or -- in the later rounds -- per stored range of a
// walk that reached the step limit; the lanes per vertex test follow the
// cloud's row length.  Walks stop at out.limit steps (no limit without
// out.items) and store the rest of their stack in `out`.
__global__ void __launch_bounds__(TRAV_WARPS * 32, 8) k_traverse_l2(
    const __grid_constant__ Views V, const int32_t *__restrict__ order, int n_order,
    const int4 *__restrict__ in_items, const int32_t *__restrict__ in_count, int in_cap, Spill out, Pool P,
    longlong2 *__restrict__ cursors, int2 *__restrict__ stacks, int cap, unsigned long long *__restrict__ st,
    int32_t *__restrict__ err, int32_t *__restrict__ next_group, int32_t *__restrict__ gvisit, int max_nq4) {
    extern __shared__ float4 sc[];  // TRAV_WARPS x (largest dp / 4)
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4 *cen = sc + wib * max_nq4;
    const int gw = blockIdx.x * TRAV_WARPS + wib;
    int2 *stack = stacks + (int64_t)gw * cap;
    unsigned long long evals = 0;
    // the warp's pool chunk carries over from the previous round
    PoolCursor pc{-1, POOL_CHUNK, 0, 0};
    if (in_items) {
        const longlong2 c = cursors[gw];
        pc.cur = c.x;
        pc.fill = (int)c.y;
    }
    const int n_work = in_items ? min(*in_count, in_cap) : n_order;
    const Spill *sp = out.items ? &out : nullptr;
    for (;;) {
        // work is taken dynamically: walks differ widely in length
        int gi = 0;
        if (lane == 0) gi = atomicAdd(next_group, 1);
        gi = __shfl_sync(0xffffffffu, gi, 0);
        if (gi >= n_work) break;
        int gg;
        int2 start = make_int2(0, 0);
        if (in_items) {
            const int4 w = in_items[gi];
            if (w.z <= 0) continue;  // an empty range (a stop that did not fit)
            gg = w.x;
            start = make_int2(w.y, w.z);
        } else {
            gg = order[gi];
        }
        const int c = cloud_of_group(V, gg);
        const TreeView &tv = V.tv[c];
        const int g = gg - V.gbase[c];
        const int nq4 = tv.dp >> 2;
        const int tpd = nq4 >= 16 ? 8 : nq4 >= 8 ? 4 : nq4 >= 4 ? 2 : 1;
        const float4 *crow = reinterpret_cast<const float4 *>(tv.pts + (size_t)tv.group_begin[g] * tv.dp);
        for (int k = lane; k < nq4; k += 32) cen[k] = crow[k];
        __syncwarp();
        const float add = V.qp[c].eps_up + tv.group_radius[g];
        auto tester = [&](int v, int take) {
            switch (tpd) {
                case 8: return l2_keep<8>(tv, cen, nq4, v, take, add);
                case 4: return l2_keep<4>(tv, cen, nq4, v, take, add);
                case 2: return l2_keep<2>(tv, cen, nq4, v, take, add);
                default: return l2_keep<1>(tv, cen, nq4, v, take, add);
            }
        };
        const unsigned long long e0 = evals;
        if (walk_group(tv, stack, cap, gg, start, P, pc, evals, err, sp, tester) < 0) return;
        if (gvisit) group_visits(gvisit, gg, evals - e0);
        __syncwarp();
    }
    if (lane == 0) cursors[gw] = make_longlong2(pc.cur, pc.fill);
    for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(0xffffffffu, evals, o);
    if (lane == 0) stat_add(st, ST_TRAV, evals);
}

// Edit distance: a vertex survives iff lev(c_g, v) <= r(v) + eps + r_g
// (integers, exact).  One warp per block; the group centre's match masks are
// in shared memory.
template <int W>
__global__ void __launch_bounds__(32) k_traverse_lev(
    TreeView tv, QParams qp, const int4 *__restrict__ in_items, const int32_t *__restrict__ in_count, int in_cap,
    Spill out, Pool P, longlong2 *__restrict__ cursors, int2 *__restrict__ stacks, int cap,
    unsigned long long *__restrict__ st, int32_t *__restrict__ err, int32_t *__restrict__ next_group,
    int32_t *__restrict__ gvisit) {
    __shared__ uint64_t peq[256 * W];
    const int lane = threadIdx.x;
    int2 *stack = stacks + (int64_t)blockIdx.x * cap;
    unsigned long long evals = 0;
    // the warp's pool chunk carries over from the previous round
    PoolCursor pc{-1, POOL_CHUNK, 0, 0};
    if (in_items) {
        const longlong2 c = cursors[blockIdx.x];
        pc.cur = c.x;
        pc.fill = (int)c.y;
    }
    const int n_work = in_items ? min(*in_count, in_cap) : tv.n_groups;
    const Spill *sp = out.items ? &out : nullptr;
    for (;;) {
        int gi = 0;
        if (lane == 0) gi = atomicAdd(next_group, 1);
        gi = __shfl_sync(0xffffffffu, gi, 0);
        if (gi >= n_work) break;
        int g;
        int2 start = make_int2(0, 0);
        if (in_items) {
            const int4 w = in_items[gi];
            if (w.z <= 0) continue;  // an empty range (a stop that did not fit)
            g = w.x;
            start = make_int2(w.y, w.z);
        } else {
            g = tv.group_order[gi];
        }
        int cpos = tv.group_begin[g];
        const uint8_t *pat = tv.sdata + tv.soff[cpos];
        int m = (int)(tv.soff[cpos + 1] - tv.soff[cpos]);
        __syncwarp();
        lev_build_peq<W>(peq, pat, m);
        __syncwarp();
        const int add = qp.lev_k + (int)tv.group_radius[g];
        auto tester = [&](int v, int take) {
            if (lane >= take) return false;
            const int vp = tv.node_begin[v];
            const int k = add + (int)tv.radius[v];
            const uint8_t *txt = tv.sdata + tv.soff[vp];
            const int n = (int)(tv.soff[vp + 1] - tv.soff[vp]);
            return lev_myers<W>(peq, m, txt, n, k) <= k;
        };
        const unsigned long long e0 = evals;
        if (walk_group(tv, stack, cap, g, start, P, pc, evals, err, sp, tester) < 0) return;
        if (gvisit) group_visits(gvisit, g, evals - e0);
        __syncwarp();
    }
    if (lane == 0) cursors[blockIdx.x] = make_longlong2(pc.cur, pc.fill);
    for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(0xffffffffu, evals, o);
    if (lane == 0) stat_add(st, ST_TRAV, evals);
}

// Hamming: a vertex survives iff ham(c_g, v) <= r(v) + eps + r_g (integers,
// exact).  One warp per block, lane i tests vertex i of a step against the
// group centre's row in shared memory.
// Distance of a row in shared memory (a) to a row in global memory (b, read
// through the read-only path).
__device__ __forceinline__ int ham_rows(const uint4 *a, const uint4 *__restrict__ b, int nq) {
    int d = 0;
    for (int k = 0; k < nq; ++k) {
        const uint4 x = a[k], y = __ldg(b + k);
        d += __popc(x.x ^ y.x) + __popc(x.y ^ y.y) + __popc(x.z ^ y.z) + __popc(x.w ^ y.w);
    }
    return d;
}
// Both rows in shared memory (plain loads).
__device__ __forceinline__ int ham_rows_smem(const uint4 *a, const uint4 *b, int nq) {
    int d = 0;
    for (int k = 0; k < nq; ++k) {
        const uint4 x = a[k], y = b[k];
        d += __popc(x.x ^ y.x) + __popc(x.y ^ y.y) + __popc(x.z ^ y.z) + __popc(x.w ^ y.w);
    }
    return d;
}

__global__ void __launch_bounds__(32) k_traverse_ham(
    TreeView tv, QParams qp, const int4 *__restrict__ in_items, const int32_t *__restrict__ in_count, int in_cap,
    Spill out, Pool P, longlong2 *__restrict__ cursors, int2 *__restrict__ stacks, int cap,
    unsigned long long *__restrict__ st, int32_t *__restrict__ err, int32_t *__restrict__ next_group,
    int32_t *__restrict__ gvisit) {
    __shared__ uint4 cen[32];  // up to 4096 bits
    const int lane = threadIdx.x;
    const int nq = tv.wp >> 2;
    int2 *stack = stacks + (int64_t)blockIdx.x * cap;
    unsigned long long evals = 0;
    // the warp's pool chunk carries over from the previous round
    PoolCursor pc{-1, POOL_CHUNK, 0, 0};
    if (in_items) {
        const longlong2 c = cursors[blockIdx.x];
        pc.cur = c.x;
        pc.fill = (int)c.y;
    }
    const int n_work = in_items ? min(*in_count, in_cap) : tv.n_groups;
    const Spill *sp = out.items ? &out : nullptr;
    for (;;) {
        int gi = 0;
        if (lane == 0) gi = atomicAdd(next_group, 1);
        gi = __shfl_sync(0xffffffffu, gi, 0);
        if (gi >= n_work) break;
        int g;
        int2 start = make_int2(0, 0);
        if (in_items) {
            const int4 w = in_items[gi];
            if (w.z <= 0) continue;  // an empty range (a stop that did not fit)
            g = w.x;
            start = make_int2(w.y, w.z);
        } else {
            g = tv.group_order[gi];
        }
        const uint4 *crow = reinterpret_cast<const uint4 *>(tv.bits + (size_t)tv.group_begin[g] * tv.wp);
        __syncwarp();
        for (int k = lane; k < nq; k += 32) cen[k] = crow[k];
        __syncwarp();
        const int add = qp.lev_k + (int)tv.group_radius[g];
        auto tester = [&](int v, int take) {
            if (lane >= take) return false;
            const int k = add + (int)tv.radius[v];
            const uint4 *row = reinterpret_cast<const uint4 *>(tv.bits + (size_t)tv.node_begin[v] * tv.wp);
            return ham_rows(cen, row, nq) <= k;
        };
        const unsigned long long e0 = evals;
        if (walk_group(tv, stack, cap, g, start, P, pc, evals, err, sp, tester) < 0) return;
        if (gvisit) group_visits(gvisit, g, evals - e0);
        __syncwarp();
    }
    if (lane == 0) cursors[blockIdx.x] = make_longlong2(pc.cur, pc.fill);
    for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(0xffffffffu, evals, o);
    if (lane == 0) stat_add(st, ST_TRAV, evals);
}

// ------------------------------------------------------------ leaf tiles

// Packs the next run of candidate points into a tile of up to 32 rows.  The
// candidates of a group are leaf blocks of a few points each; rows of
// consecutive candidates are concatenated so that every tile is full.
// Called by warp 0; (s_ci, s_off) is the cursor: candidate index and the number
// of its points already consumed.  In the emit pass, candidates without the
// "produced an edge" flag are skipped.
__device__ __forceinline__ void fill_tile(const TreeView &tv, const uint32_t *__restrict__ cand, int64_t c1,
                                          bool flagged_only, int64_t *s_ci, int *s_off, int *s_rows,
                                          int *tpos, int64_t *tcand) {
    const int lane = threadIdx.x & 31;
    const int64_t ci = *s_ci;
    const int off = *s_off;
    const int64_t c = ci + lane;
    int beg = 0, cnt = 0;
    if (c < c1) {
        uint32_t e = cand[c];
        if (!flagged_only || (e & FLAG)) {
            int v = (int)(e & ~FLAG);
            beg = tv.node_begin[v];
            cnt = tv.node_count[v];
        }
    }
    if (lane == 0) {
        beg += off;
        cnt -= off;
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int excl = incl - cnt;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int rows = total < 32 ? total : 32;
    // owner of row r = lane: number of candidates whose inclusive end is <= r
    int L = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
        int probe = __shfl_sync(0xffffffffu, incl, L + step - 1);
        if (probe <= lane) L += step;
    }
    const int bl = __shfl_sync(0xffffffffu, beg, L);
    const int el = __shfl_sync(0xffffffffu, excl, L);
    if (lane < rows) {
        tpos[lane] = bl + (lane - el);
        tcand[lane] = ci + L;
    }
    const int L31 = __shfl_sync(0xffffffffu, L, 31);
    const int e31 = __shfl_sync(0xffffffffu, excl, L31);
    const int n31 = __shfl_sync(0xffffffffu, cnt, L31);
    if (lane == 0) {
        if (total <= 32) {
            int64_t nx = ci + 32;
            *s_ci = nx < c1 ? nx : c1;
            *s_off = 0;
        } else {
            int used = 32 - e31;
            if (used == n31) {
                *s_ci = ci + L31 + 1;
                *s_off = 0;
            } else {
                *s_ci = ci + L31;
                *s_off = (L31 == 0 ? off : 0) + used;
            }
        }
        *s_rows = rows;
    }
}

// Loads rows (K chunk kc0 .. kc0 + 4 kq floats) into a padded shared tile;
// row r comes from position pos[r] (or first + r when pos is null); rows
// beyond `rows` are zero.
__device__ __forceinline__ void load_rows(float4 *__restrict__ tile, const float *__restrict__ pts, int dp,
                                          const int *pos, int first, int rows, int kc0, int kq) {
    for (int i = threadIdx.x; i < 32 * kq; i += LEAF_T) {
        int r = i / kq, k = i - r * kq;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < rows) {
            int p = pos ? pos[r] : first + r;
            v = __ldg(reinterpret_cast<const float4 *>(pts + (size_t)p * dp + kc0) + k);
        }
        tile[r * KS4 + k] = v;
    }
}

constexpr int NB = 128;       // candidate leaf blocks per batch
constexpr int GQ_CAP = 1088;  // guard-band queue: <= 63 carried + 1024 from one tile
constexpr int RCAP = 512;     // packed rows mapped to positions at a time

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    int n = valid ? 16 : 0;  // 0: the 16 bytes are zero-filled, nothing is read
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(n));
}
// 4-byte copy through L1 (cp.async.cg takes 16-byte copies only)
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Packed fp32 pairs (sm_100+ f32x2 instructions): two independent IEEE
// round-to-nearest operations per instruction.
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_sqacc(unsigned long long d, unsigned long long acc) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(r) : "l"(d), "l"(acc));
    return r;
}
__device__ __forceinline__ float f2_sum(unsigned long long v) {
    return __uint_as_float((uint32_t)v) + __uint_as_float((uint32_t)(v >> 32));
}

// Squared distances of the 2 x 4 pairs owned by this thread: queries qi and
// qi + 16 of the Q tile against rows pj, pj+8, pj+16, pj+24 of the P tile,
// whose positions are prow[0..npr).  Coordinates are summed in chunks of 16
// (FMA per term) and the chunk sums added into the total.  Contains barriers;
// every thread of the block calls it.  On return the P tile is loaded and
// every thread is past its last read of Qs/Ps for this call.
__device__ __forceinline__ void tile_accumulate(const float4 *Qs, const float4 *Ps, int kq, float (&tot)[2][4]);

__device__ __forceinline__ void tile_sqdist(const TreeView &tv, float4 *Qs, float4 *Ps, const int *prow, int npr,
                                            int qfirst, int nqr, int nkc, float (&tot)[2][4]) {
    const int dp = tv.dp;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) tot[i][j] = 0.f;
    for (int kc = 0; kc < nkc; ++kc) {
        const int k0 = kc * KC;
        const int kq = min(KC, dp - k0) >> 2;
        if (kc > 0) __syncthreads();
        if (nkc > 1) load_rows(Qs, tv.pts, dp, nullptr, qfirst, nqr, k0, kq);
        load_rows(Ps, tv.pts, dp, prow, 0, npr, k0, kq);
        __syncthreads();
        tile_accumulate(Qs, Ps, kq, tot);  // KC is a multiple of 16: chunks line up across K chunks
    }
}

// 2 x 4 micro-tile from tiles already in shared memory (rows of kq float4).
// Per chunk of 16 coordinates two packed partial sums of 8 terms each (even
// and odd coordinates) are formed with FMA, added, and the chunk sum is added
// into the running total: fp32 error of the squared distance <= ~19 u for
// rows of 128 floats (u = 2^-24).
__device__ __forceinline__ void tile_accumulate(const float4 *Qs, const float4 *Ps, int kq, float (&tot)[2][4]) {
    const int tid = threadIdx.x, qi = tid >> 3, pj = tid & 7;
    const ulonglong2 *qa[2] = {reinterpret_cast<const ulonglong2 *>(Qs + qi * KS4),
                               reinterpret_cast<const ulonglong2 *>(Qs + (qi + 16) * KS4)};
    const ulonglong2 *pr[4] = {reinterpret_cast<const ulonglong2 *>(Ps + pj * KS4),
                               reinterpret_cast<const ulonglong2 *>(Ps + (pj + 8) * KS4),
                               reinterpret_cast<const ulonglong2 *>(Ps + (pj + 16) * KS4),
                               reinterpret_cast<const ulonglong2 *>(Ps + (pj + 24) * KS4)};
    int k4 = 0;
    for (; k4 + 4 <= kq; k4 += 4) {
        unsigned long long acc[2][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0ull;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const ulonglong2 a0 = qa[0][k4 + u], a1 = qa[1][k4 + u];
            const ulonglong2 b[4] = {pr[0][k4 + u], pr[1][k4 + u], pr[2][k4 + u], pr[3][k4 + u]};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                acc[0][j] = f2_sqacc(f2_sub(a0.x, b[j].x), acc[0][j]);
                acc[0][j] = f2_sqacc(f2_sub(a0.y, b[j].y), acc[0][j]);
                acc[1][j] = f2_sqacc(f2_sub(a1.x, b[j].x), acc[1][j]);
                acc[1][j] = f2_sqacc(f2_sub(a1.y, b[j].y), acc[1][j]);
            }
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) tot[i][j] += f2_sum(acc[i][j]);
    }
    if (k4 < kq) {  // rows whose length is not a multiple of 16 floats
        unsigned long long acc[2][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0ull;
        for (int k = k4; k < kq; ++k) {
            const ulonglong2 a0 = qa[0][k], a1 = qa[1][k];
            const ulonglong2 b[4] = {pr[0][k], pr[1][k], pr[2][k], pr[3][k]};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                acc[0][j] = f2_sqacc(f2_sub(a0.x, b[j].x), acc[0][j]);
                acc[0][j] = f2_sqacc(f2_sub(a0.y, b[j].y), acc[0][j]);
                acc[1][j] = f2_sqacc(f2_sub(a1.x, b[j].x), acc[1][j]);
                acc[1][j] = f2_sqacc(f2_sub(a1.y, b[j].y), acc[1][j]);
            }
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) tot[i][j] += f2_sum(acc[i][j]);
    }
}

__device__ __forceinline__ void tile_sqdist_smem(const float4 *Qs, const float4 *Ps, int kq, float (&tot)[2][4]) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) tot[i][j] = 0.f;
    tile_accumulate(Qs, Ps, kq, tot);
}

// pair_sqdist with both rows in shared memory (plain loads).
__device__ __forceinline__ float pair_sqdist_smem(const float4 *x, const float4 *y, int nq4) {
    float tot = 0.f;
    int k = 0;
    for (; k + 4 <= nq4; k += 4) {
        float lo = 0.f, hi = 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float4 a = x[k + u], b = y[k + u];
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
            const float4 a = x[k], b = y[k];
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

struct LeafShared {
    float4 Qs[32 * KS4];
    float4 Ps[2][32 * KS4];
    int bbeg[NB], bcnt[NB], bpre[NB + 1];
    uint32_t bmask[NB], bem[NB];
    float brad[NB];
    int64_t bci[NB];
    int rpos[RCAP];
    uint8_t rli[RCAP];
    int64_t rowb[32], rowe[32];
    int cursor[32], qcnt[32];
    int gpos[GQ_CAP];
    uint8_t gq[GQ_CAP], gb[GQ_CAP];
    int gn, nb_fill, scan_tmp[LEAF_T / 32];
    uint32_t selm;
    int64_t next_ci;
    int tpre[33];  // emit pass: pairs per row of the current tile (exclusive prefix)
};
constexpr size_t kLeafSmem = sizeof(LeafShared);

// One CTA per query group; queries in chunks of 32 (Q tile), candidate leaf
// blocks in batches of NB.  Per batch:
//  stage 1 (count pass) -- Algorithm 3's own test per query,
//             d(q, c_v) <= r(v) + eps, for every (query, candidate block) pair,
//             as dense 32 x 32 tiles of query rows against block centres; it
//             gives each block the mask of queries that still need it (a
//             pruned pair cannot hold an edge);
//  stage 2 -- the points of blocks with a non-empty mask, packed into 32-row
//             tiles (double buffered with cp.async); pairs outside the block's
//             mask are skipped.
// The emit pass skips stage 1: the count pass leaves, per candidate block,
// the mask of queries that found an edge in it, and the emit pass batches only
// blocks whose mask is non-empty.  Pairs that the fp32 value cannot decide
// (decide32) are queued and decided in FP64 by whole warps.
// A work item: a slice of at most kItem candidate blocks of one query group.
// Heavy groups (large candidate lists) are spread over several CTAs.
constexpr int kItem = 512;
constexpr int kItemTC = 1024;  // the tensor-core leaf kernel's work items (precision 1)
struct Items {
    const int32_t *group;
    const int64_t *begin, *end;
    const int32_t *count;  // device: number of items
};

// One-pass emit (learned form): the count pass also writes every edge into a
// per-row capacity region sized from the predicted degree.  A row's entries
// past its capacity go to an overflow arena as (row, slot, col, dist); once
// the arena is full the row is marked lost and re-emitted exactly later.
// off == nullptr: plain count pass.
struct CapOut {
    const int64_t *off;      // n + 1 capacity offsets by original id
    int32_t *fill;           // entries produced per row (ends equal to the degree)
    int32_t *col;
    float *dist;             // capacity region
    int32_t *ovf_row, *ovf_slot, *ovf_col;
    float *ovf_dist;
    unsigned long long *ovf_n;
    int64_t ovf_cap;
    uint8_t *lost;
};

// Writes entry `slot` of row o: in the row's capacity, else in the arena.
__device__ __forceinline__ void cap_place(const CapOut &co, int o, int slot, int32_t c, float d) {
    const int64_t b = co.off[o];
    if (slot < co.off[o + 1] - b) {
        co.col[b + slot] = c;
        co.dist[b + slot] = d;
        return;
    }
    const unsigned long long k = atomicAdd(co.ovf_n, 1ull);
    if ((int64_t)k < co.ovf_cap) {
        co.ovf_row[k] = o;
        co.ovf_slot[k] = slot;
        co.ovf_col[k] = c;
        co.ovf_dist[k] = d;
    } else {
        co.lost[o] = 1;
    }
}

__device__ __forceinline__ void cap_put(const CapOut &co, int o, int32_t c, float d) {
    cap_place(co, o, atomicAdd(&co.fill[o], 1), c, d);
}

// One work item of the FP32 tiles (count or emit pass), by the whole CTA.
template <bool EMIT>
__device__ __forceinline__ void leaf_l2_item(
    const Views &V, const Items &items, const int it, const uint32_t *__restrict__ cand,
    uint32_t *__restrict__ emask, int32_t *__restrict__ deg, const int64_t *__restrict__ row_ptr,
    int32_t *__restrict__ rowcur, int32_t *__restrict__ col, float *__restrict__ dist,
    unsigned long long *__restrict__ st, int32_t *__restrict__ err, const CapOut &co,
    const uint8_t *__restrict__ rowsel, LeafShared &S) {
    if (it >= *items.count) return;
    const int gg = items.group[it];
    const int cloud = cloud_of_group(V, gg);
    const TreeView &tv = V.tv[cloud];
    const QParams &qp = V.qp[cloud];
    const int g = gg - V.gbase[cloud];
    const int64_t rbase = V.rbase[cloud];  // CSR rows of this cloud start here
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int qi = tid >> 3, pj = tid & 7;
    const int dp = tv.dp, dim = tv.dim;
    const int nkc = (dp + KC - 1) / KC;
    const int kq = dp >> 2;  // float4 per row when nkc == 1
    const bool fp32_dist_ok = dp <= 128;
    const int qb = tv.group_begin[g], qn = tv.group_count[g];
    const int qe = qb + qn;       // the group's positions: [qb, qe)
    const bool half = qp.half != 0;
    const int64_t c0 = items.begin[it], c1 = items.end[it];
    unsigned long long pairs = 0, s1evals = 0, guard = 0, band = 0, rows_ld = 0;  // rows_ld: thread 0
    // upper-triangle form: an edge (q, p) with p in a later group is also the
    // edge (p, q) of p's row -- its degree (count pass, with the one-pass
    // emit's entry) or its entry (emit pass; only a selected row when rows
    // are emitted again)
    auto mirror = [&](int qpos, int ppos, float d) {
        const int64_t o = rbase + tv.perm[ppos];
        if (!EMIT) {
            atomicAdd(&deg[o], 1);
            if (co.off) cap_put(co, (int)o, tv.perm[qpos], d);
        } else {
            if (rowsel && !rowsel[o]) return;
            const int slot = atomicAdd(&rowcur[o], 1);
            const int64_t at = row_ptr[o] + slot;
            if (at < row_ptr[o + 1]) {
                col[at] = tv.perm[qpos];
                dist[at] = d;
            } else {
                atomicOr(err, 4);
            }
        }
    };

    for (int q0 = 0; q0 < qn; q0 += 32) {
        const int nqr = min(32, qn - q0);
        const int qfirst = qb + q0;
        __syncthreads();
        if (tid < 32) {
            S.qcnt[tid] = 0;
            bool sel = false;
            if (tid < nqr) {
                const int64_t o = rbase + tv.perm[qfirst + tid];
                S.cursor[tid] = (int)o;  // row of the query in the (concatenated) CSR
                if (EMIT) {
                    S.rowb[tid] = row_ptr[o];
                    S.rowe[tid] = row_ptr[o + 1];
                    sel = rowsel == nullptr || rowsel[o] != 0;
                }
            }
            // emit pass: queries whose rows are written (all, or the selected ones)
            const unsigned sm = __ballot_sync(0xffffffffu, sel);
            if (tid == 0) S.selm = sm;
        }
        if (tid == 0) S.gn = 0;
        int cnt0 = 0, cnt1 = 0;
        if (nkc == 1) load_rows(S.Qs, tv.pts, dp, nullptr, qfirst, nqr, 0, kq);

        // decides the queued guard-band pairs; `all` drains everything, else
        // whole warps' worth and keeps the rest
        auto drain = [&](bool all) {
            __syncthreads();
            const int n = S.gn;
            const int m = all ? n : (n & ~31);
            for (int i = tid; i < m; i += LEAF_T) {
                const int q = S.gq[i], ppos = S.gpos[i], li = S.gb[i];
                if (!EMIT) {
                    ++guard;
                    note_guard_rows(S.cursor[q], (int32_t)(rbase + tv.perm[ppos]));
                }
                double s64 = sq_l2_exact(tv.pts + (size_t)(qfirst + q) * dp, tv.pts + (size_t)ppos * dp, dim);
                if (s64 <= qp.eps2_64) {
                    if (half && ppos >= qe) mirror(qfirst + q, ppos, (float)sqrt(s64));
                    if (!EMIT) {
                        atomicAdd(&S.qcnt[q], 1);
                        atomicOr(&S.bem[li], 1u << q);
                        if (co.off) cap_put(co, S.cursor[q], tv.perm[ppos], (float)sqrt(s64));
                    } else if ((S.selm >> q) & 1u) {
                        int slot = atomicAdd(&rowcur[S.cursor[q]], 1);
                        int64_t at = S.rowb[q] + slot;
                        if (at < S.rowe[q]) {
                            col[at] = tv.perm[ppos];
                            dist[at] = (float)sqrt(s64);
                        } else {
                            atomicOr(err, 4);
                        }
                    }
                }
            }
            __syncthreads();
            const int rest = n - m;
            int rp = 0, rq = 0, rb = 0;
            if (tid < rest) {
                rp = S.gpos[m + tid];
                rq = S.gq[m + tid];
                rb = S.gb[m + tid];
            }
            __syncthreads();
            if (tid < rest) {
                S.gpos[tid] = rp;
                S.gq[tid] = (uint8_t)rq;
                S.gb[tid] = (uint8_t)rb;
            }
            if (tid == 0) S.gn = rest;
            __syncthreads();
        };

        // issues the cp.async copies of tile t (rows rowsrc[32t ..]) into buffer buf
        auto issue = [&](int t, int buf, const int *rowsrc, int nrows) {
            if (nkc != 1) return;
            const int r0 = 32 * t;
            const int rows = min(32, nrows - r0);
            float4 *dst = S.Ps[buf];
            for (int i = tid; i < 32 * kq; i += LEAF_T) {
                const int r = i / kq, k = i - r * kq;
                const bool valid = r < rows;
                const int pos = valid ? rowsrc[r0 + r] : qfirst;
                cp_async16(dst + r * KS4 + k, tv.pts + (size_t)pos * dp + 4 * k, valid);
            }
            cp_async_commit();
        };
        auto compute = [&](int t, int buf, const int *rowsrc, int nrows, float (&tot)[2][4]) {
            if (nkc == 1) {
                tile_sqdist_smem(S.Qs, S.Ps[buf], kq, tot);
            } else {
                const int r0 = 32 * t;
                tile_sqdist(tv, S.Qs, S.Ps[0], rowsrc + r0, min(32, nrows - r0), qfirst, nqr, nkc, tot);
            }
        };

        int64_t ci = c0;
        while (ci < c1) {
            // ---- batch of candidate blocks
            int bn;
            if (EMIT) {
                __syncthreads();
                if (tid == 0) S.nb_fill = 0;
                __syncthreads();
                for (;;) {
                    const int nf = S.nb_fill;
                    if (nf >= NB || ci >= c1) break;
                    const int64_t idx = ci + tid;
                    // (rows emitted again in the upper-triangle form: every query, as a
                    // selected row can be the mirror of another query's edge)
                    const uint32_t m = idx < c1 ? (emask[idx] & (half && rowsel ? 0xffffffffu : S.selm)) : 0u;
                    const bool f = m != 0u;
                    const unsigned bal = __ballot_sync(0xffffffffu, f);
                    if (lane == 0) S.scan_tmp[warp] = __popc(bal);
                    __syncthreads();
                    int off = 0, tot = 0;
#pragma unroll
                    for (int w = 0; w < LEAF_T / 32; ++w) {
                        if (w < warp) off += S.scan_tmp[w];
                        tot += S.scan_tmp[w];
                    }
                    const int rank = off + __popc(bal & lanemask_lt());
                    const int room = NB - nf;
                    if (f && rank < room) {
                        S.bci[nf + rank] = idx;
                        S.bmask[nf + rank] = m;
                    }
                    if (f && rank == room) S.next_ci = idx;
                    __syncthreads();
                    if (tot <= room) ci = ci + LEAF_T < c1 ? ci + LEAF_T : c1;
                    else ci = S.next_ci;
                    if (tid == 0) S.nb_fill = nf + (tot < room ? tot : room);
                    __syncthreads();
                }
                bn = S.nb_fill;
                if (bn == 0) break;
            } else {
                bn = (int)((c1 - ci) < NB ? (c1 - ci) : NB);
                if (tid < NB) S.bci[tid] = ci + tid;
                ci += bn;
            }
            __syncthreads();
            for (int i = tid; i < bn; i += LEAF_T) {
                const int v = (int)cand[S.bci[i]];
                S.bbeg[i] = tv.node_begin[v];
                S.bcnt[i] = tv.node_count[v];
                S.brad[i] = tv.radius[v];
                if (!EMIT) S.bmask[i] = 0u;
                S.bem[i] = 0u;
            }
            __syncthreads();

            // ---- stage 1 (count pass): per-query test against the block centres
            if (!EMIT) {
                const int nt = (bn + 31) >> 5;
                if (tid == 0) rows_ld += bn;
                issue(0, 0, S.bbeg, bn);
                for (int t = 0; t < nt; ++t) {
                    if (t + 1 < nt) {
                        issue(t + 1, (t + 1) & 1, S.bbeg, bn);
                        cp_async_wait<1>();
                    } else {
                        cp_async_wait<0>();
                    }
                    __syncthreads();
                    float tot[2][4];
                    compute(t, t & 1, S.bbeg, bn, tot);
                    const int rows = min(32, bn - 32 * t);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int p = pj + 8 * j;
                        if (p >= rows) continue;
                        const int li = 32 * t + p;
                        const float bound = fmaf(S.brad[li] + qp.eps_up, PRUNE_REL, PRUNE_ABS);
                        uint32_t m = 0u;
#pragma unroll
                        for (int i = 0; i < 2; ++i) {
                            const int q = qi + 16 * i;
                            if (q >= nqr) continue;
                            ++s1evals;
                            if (!(sqrtf(tot[i][j]) > bound)) m |= 1u << q;
                        }
                        if (m) atomicOr(&S.bmask[li], m);
                    }
                    __syncthreads();
                }
            }

            // ---- prefix over the batch (warp 0): count pass -- points of the
            // surviving blocks; emit pass -- (query, point) pairs to evaluate
            const uint32_t qvalid = nqr >= 32 ? 0xffffffffu : ((1u << nqr) - 1u);
            if (warp == 0) {
                int loc[4], sum = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int i = 4 * lane + k;
                    if (EMIT && nkc > 1) loc[k] = i < bn ? __popc(S.bmask[i] & qvalid) * S.bcnt[i] : 0;
                    else loc[k] = (i < bn && (S.bmask[i] & qvalid) != 0u) ? S.bcnt[i] : 0;
                    sum += loc[k];
                }
                int incl = sum;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                int run = incl - sum;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    S.bpre[4 * lane + k] = run;
                    run += loc[k];
                }
                if (lane == 31) S.bpre[NB] = incl;
            }
            __syncthreads();
            const int T = S.bpre[NB];

            // ---- emit pass: one thread per (query, point) pair of the blocks in
            // which the query found an edge; same arithmetic as the tiles;
            // undecided pairs go through the FP64 queue
            if (EMIT && nkc > 1) {
                for (int r0 = 0; r0 < T; r0 += LEAF_T) {
                    const int r = r0 + tid;
                    if (r < T) {
                        int lo = 0, hi = NB;
                        while (hi - lo > 1) {
                            const int mid = (lo + hi) >> 1;
                            if (S.bpre[mid] <= r) lo = mid; else hi = mid;
                        }
                        const int idx = r - S.bpre[lo], cnt = S.bcnt[lo];
                        const int qr = idx / cnt, pidx = idx - qr * cnt;
                        const int q = (int)__fns(S.bmask[lo] & qvalid, 0u, qr + 1);
                        const int qpos = qfirst + q, ppos = S.bbeg[lo] + pidx;
                        if ((qpos != ppos || qp.include_self) && !(half && ppos < qb)) {
                            ++pairs;
                            const float4 *qrow = reinterpret_cast<const float4 *>(tv.pts + (size_t)qpos * dp);
                            const float sv = pair_sqdist(qrow, reinterpret_cast<const float4 *>(tv.pts + (size_t)ppos * dp),
                                                         dp >> 2);
                            const int edge = decide32(qp, sv, band);
                            if (edge < 0) {
                                const int slot = atomicAdd(&S.gn, 1);
                                S.gpos[slot] = ppos;
                                S.gq[slot] = (uint8_t)q;
                                S.gb[slot] = (uint8_t)lo;
                            } else if (edge) {
                                const float d = fp32_dist_ok ? sqrtf(sv)
                                                             : (float)sqrt(sq_l2_exact(tv.pts + (size_t)qpos * dp,
                                                                                       tv.pts + (size_t)ppos * dp, dim));
                                if (half && ppos >= qe) mirror(qpos, ppos, d);
                                if ((S.selm >> q) & 1u) {
                                    const int slot = atomicAdd(&rowcur[S.cursor[q]], 1);
                                    const int64_t at = S.rowb[q] + slot;
                                    if (at < S.rowe[q]) {
                                        col[at] = tv.perm[ppos];
                                        dist[at] = d;
                                    } else {
                                        atomicOr(err, 4);
                                    }
                                }
                            }
                        }
                    }
                    __syncthreads();
                    if (S.gn >= 64) drain(false);
                }
            }

            // ---- stage 2: packed points of the surviving blocks (count pass: dense
            // 32 x 32 tiles; emit pass: only the (query, row) pairs of each tile
            // whose block holds an edge of the query)
            for (int R0 = 0; (!EMIT || nkc == 1) && R0 < T; R0 += RCAP) {
                const int RN = min(RCAP, T - R0);
                if (!EMIT && tid == 0) rows_ld += RN;
                __syncthreads();
                for (int r = tid; r < RN; r += LEAF_T) {
                    const int R = R0 + r;
                    int lo = 0, hi = NB;  // last li with bpre[li] <= R (and a non-empty block)
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (S.bpre[mid] <= R) lo = mid; else hi = mid;
                    }
                    S.rpos[r] = S.bbeg[lo] + (R - S.bpre[lo]);
                    S.rli[r] = (uint8_t)lo;
                }
                __syncthreads();
                const int nt = (RN + 31) >> 5;
                issue(0, 0, S.rpos, RN);
                for (int t = 0; t < nt; ++t) {
                    if (t + 1 < nt) {
                        issue(t + 1, (t + 1) & 1, S.rpos, RN);
                        cp_async_wait<1>();
                    } else {
                        cp_async_wait<0>();
                    }
                    __syncthreads();
                    const int npr = min(32, RN - 32 * t);
                    if (EMIT) {
                        // pairs of this tile: row r pairs with the queries of its block's mask
                        if (warp == 0) {
                            const int c = lane < npr ? __popc(S.bmask[S.rli[32 * t + lane]] & qvalid) : 0;
                            int incl = c;
#pragma unroll
                            for (int o = 1; o < 32; o <<= 1) {
                                int y = __shfl_up_sync(0xffffffffu, incl, o);
                                if (lane >= o) incl += y;
                            }
                            S.tpre[lane] = incl - c;
                            if (lane == 31) S.tpre[32] = incl;
                        }
                        __syncthreads();
                        const int TP = S.tpre[32];
                        const float4 *Pb = S.Ps[t & 1];
                        for (int pi = tid; pi < TP; pi += LEAF_T) {
                            int lo = 0, hi = 32;
                            while (hi - lo > 1) {
                                const int mid = (lo + hi) >> 1;
                                if (S.tpre[mid] <= pi) lo = mid; else hi = mid;
                            }
                            const int r = 32 * t + lo;
                            const int li = S.rli[r];
                            const int q = (int)__fns(S.bmask[li] & qvalid, 0u, pi - S.tpre[lo] + 1);
                            const int qpos = qfirst + q, ppos = S.rpos[r];
                            if (qpos == ppos && !qp.include_self) continue;
                            if (half && ppos < qb) continue;
                            ++pairs;
                            const float sv = pair_sqdist_smem(S.Qs + q * KS4, Pb + lo * KS4, kq);
                            const int edge = decide32(qp, sv, band);
                            if (edge < 0) {
                                const int slot = atomicAdd(&S.gn, 1);
                                S.gpos[slot] = ppos;
                                S.gq[slot] = (uint8_t)q;
                                S.gb[slot] = (uint8_t)li;
                            } else if (edge) {
                                if (half && ppos >= qe) mirror(qpos, ppos, sqrtf(sv));
                                if ((S.selm >> q) & 1u) {
                                    const int slot = atomicAdd(&rowcur[S.cursor[q]], 1);
                                    const int64_t at = S.rowb[q] + slot;
                                    if (at < S.rowe[q]) {
                                        col[at] = tv.perm[ppos];
                                        dist[at] = sqrtf(sv);
                                    } else {
                                        atomicOr(err, 4);
                                    }
                                }
                            }
                        }
                        __syncthreads();
                        if (S.gn >= 64) drain(false);
                        continue;
                    }
                    float tot[2][4];
                    compute(t, t & 1, S.rpos, RN, tot);
                    uint32_t hitrow = 0u;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int p = pj + 8 * j;
                        if (p >= npr) continue;
                        const int r = 32 * t + p;
                        const int li = S.rli[r];
                        const uint32_t mask = S.bmask[li];
                        const int ppos = S.rpos[r];
#pragma unroll
                        for (int i = 0; i < 2; ++i) {
                            const int q = qi + 16 * i;
                            if (q >= nqr || !((mask >> q) & 1u)) continue;
                            const int qpos = qfirst + q;
                            if (qpos == ppos && !qp.include_self) continue;
                            if (half && ppos < qb) continue;
                            if (!EMIT) ++pairs;
                            const float sv = tot[i][j];
                            const int edge = decide32(qp, sv, band);
                            if (edge < 0) {  // undecided in fp32: queue for the FP64 decision
                                const int slot = atomicAdd(&S.gn, 1);
                                S.gpos[slot] = ppos;
                                S.gq[slot] = (uint8_t)q;
                                S.gb[slot] = (uint8_t)li;
                                continue;
                            }
                            if (!edge) continue;
                            const bool want_d = co.off || EMIT || (half && ppos >= qe);
                            const float d = !want_d ? 0.f
                                            : fp32_dist_ok ? sqrtf(sv)
                                                           : (float)sqrt(sq_l2_exact(tv.pts + (size_t)qpos * dp,
                                                                                     tv.pts + (size_t)ppos * dp, dim));
                            if (half && ppos >= qe) mirror(qpos, ppos, d);
                            if (!EMIT) {
                                if (i == 0) ++cnt0; else ++cnt1;
                                hitrow |= 1u << (4 * j + i);
                                if (co.off) cap_put(co, S.cursor[q], tv.perm[ppos], d);
                            } else if ((S.selm >> q) & 1u) {
                                const int slot = atomicAdd(&rowcur[S.cursor[q]], 1);
                                const int64_t at = S.rowb[q] + slot;
                                if (at < S.rowe[q]) {
                                    col[at] = tv.perm[ppos];
                                    dist[at] = d;
                                } else {
                                    atomicOr(err, 4);
                                }
                            }
                        }
                    }
                    if (!EMIT && hitrow) {
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const uint32_t qm = (hitrow >> (4 * j)) & 3u;
                            if (!qm) continue;
                            uint32_t bits = 0u;
                            if (qm & 1u) bits |= 1u << qi;
                            if (qm & 2u) bits |= 1u << (qi + 16);
                            atomicOr(&S.bem[S.rli[32 * t + pj + 8 * j]], bits);
                        }
                    }
                    __syncthreads();
                    if (S.gn >= 64) drain(false);
                }
            }
            drain(true);
            // count pass: queries that found an edge in each block (all queries
            // for a group above 32 points), read by the emit pass
            if (!EMIT && emask) {
                for (int i = tid; i < bn; i += LEAF_T) emask[S.bci[i]] = qn <= 32 ? S.bem[i] : ~0u;
            }
        }
        if (!EMIT) {
            for (int o = 1; o < 8; o <<= 1) {
                cnt0 += __shfl_xor_sync(0xffffffffu, cnt0, o);
                cnt1 += __shfl_xor_sync(0xffffffffu, cnt1, o);
            }
            __syncthreads();
            if (pj == 0) {
                if (qi < nqr && cnt0 + S.qcnt[qi]) atomicAdd(&deg[S.cursor[qi]], cnt0 + S.qcnt[qi]);
                if (qi + 16 < nqr && cnt1 + S.qcnt[qi + 16])
                    atomicAdd(&deg[S.cursor[qi + 16]], cnt1 + S.qcnt[qi + 16]);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
        s1evals += __shfl_xor_sync(0xffffffffu, s1evals, o);
        guard += __shfl_xor_sync(0xffffffffu, guard, o);
        band += __shfl_xor_sync(0xffffffffu, band, o);
    }
    if ((tid & 31) == 0) {
        if (!EMIT) {
            stat_add(st, ST_PAIRS, pairs);
            stat_add(st, ST_TRAV, s1evals);
            stat_add(st, ST_GUARD, guard);
            stat_add(st, ST_BAND, band);
            if (tid == 0) stat_add(st, ST_ROWS, rows_ld);
        } else {
            stat_add(st, ST_EMIT, pairs);
        }
    }
}

// One CTA per work item.
template <bool EMIT>
__global__ void __launch_bounds__(LEAF_T, 3) k_leaf_l2(
    const __grid_constant__ Views V, Items items, const uint32_t *__restrict__ cand,
    uint32_t *__restrict__ emask, int32_t *__restrict__ deg, const int64_t *__restrict__ row_ptr,
    int32_t *__restrict__ rowcur, int32_t *__restrict__ col, float *__restrict__ dist,
    unsigned long long *__restrict__ st, int32_t *__restrict__ err, CapOut co, const uint8_t *__restrict__ rowsel) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    leaf_l2_item<EMIT>(V, items, blockIdx.x, cand, emask, deg, row_ptr, rowcur, col, dist, st, err, co, rowsel,
                       *reinterpret_cast<LeafShared *>(smem_raw));
}

// Work items: every pool segment split into slices of at most kItem blocks.
// The walk rounds leave a group's candidates in several pool segments; these
// copy them into one contiguous range per group (longer work items, fewer
// CTAs in the leaf pass): counts per group, then a warp per segment copies it
// to its group's range at a place taken from the group's fill counter.
__global__ void k_group_cand_counts(int nseg, const int32_t *__restrict__ seg_group,
                                    const int32_t *__restrict__ seg_count, int32_t *__restrict__ gcnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nseg && seg_count[i] > 0) atomicAdd(gcnt + seg_group[i], seg_count[i]);
}
__global__ void k_group_cand_copy(int nseg, const int32_t *__restrict__ seg_group,
                                  const int64_t *__restrict__ seg_begin, const int32_t *__restrict__ seg_count,
                                  const int64_t *__restrict__ goff, int32_t *__restrict__ gfill,
                                  const uint32_t *__restrict__ pool, uint32_t *__restrict__ gcand) {
    const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (i >= nseg) return;
    const int g = seg_group[i], c = seg_count[i];
    int64_t base = 0;
    if (lane == 0) base = goff[g] + atomicAdd(gfill + g, c);
    base = __shfl_sync(0xffffffffu, base, 0);
    const uint32_t *src = pool + seg_begin[i];
    for (int k = lane; k < c; k += 32) gcand[base + k] = src[k];
}
// The copy in the upper-triangle form: a group keeps the candidate blocks
// that reach its first position or beyond (the pairs with earlier points are
// evaluated by their own groups); each warp ballots a segment's blocks 32 at
// a time and appends the kept ones, so a group's kept count ends in gfill.
// With nseg_dev (a plan) the segment count is read on the device and the
// destinations are checked against cand_cap.
__global__ void k_group_cand_copy_half(const __grid_constant__ Views V, int nseg, const int32_t *__restrict__ nseg_dev,
                                       int64_t seg_cap, const int32_t *__restrict__ seg_group,
                                       const int64_t *__restrict__ seg_begin, const int32_t *__restrict__ seg_count,
                                       const int64_t *__restrict__ goff, int32_t *__restrict__ gfill,
                                       const uint32_t *__restrict__ pool, uint32_t *__restrict__ gcand,
                                       int64_t cand_cap, int32_t *__restrict__ err) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t ns = nseg_dev ? min((int64_t)*nseg_dev, seg_cap) : (int64_t)nseg;
    if (i >= ns) return;
    const int gg = seg_group[i], c = seg_count[i];
    const int cl = cloud_of_group(V, gg);
    const TreeView &tv = V.tv[cl];
    const bool half = V.qp[cl].half != 0;
    const int qb = tv.group_begin[gg - V.gbase[cl]];
    const uint32_t *src = pool + seg_begin[i];
    for (int k0 = 0; k0 < c; k0 += 32) {
        const int k = k0 + lane;
        uint32_t v = 0u;
        bool keep = false;
        if (k < c) {
            v = src[k];
            keep = !half || tv.node_begin[v] + tv.node_count[v] > qb;
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        int64_t base = 0;
        if (lane == 0 && m) base = goff[gg] + atomicAdd(gfill + gg, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base + __popc(m) > cand_cap) {  // a plan's overflow (reported; the producer skips the group)
            if (lane == 0) atomicOr(err, 128);
            return;
        }
        if (keep) gcand[base + __popc(m & lanemask_lt())] = v;
    }
}

__global__ void k_iota(int n, int32_t *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = i;
}

__global__ void k_item_counts(const __grid_constant__ Views V, int nseg, const int32_t *__restrict__ seg_group,
                              const int32_t *__restrict__ seg_count, int32_t *__restrict__ icnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nseg) return;
    const int len = V.item_len[cloud_of_group(V, seg_group[i])];
    icnt[i] = (seg_count[i] + len - 1) / len;
}
__global__ void k_item_fill(const __grid_constant__ Views V, int nseg, const int32_t *__restrict__ seg_group,
                            const int64_t *__restrict__ seg_begin, const int32_t *__restrict__ seg_count,
                            const int64_t *__restrict__ ioff, int32_t *__restrict__ ig, int64_t *__restrict__ ib,
                            int64_t *__restrict__ ie, int32_t *__restrict__ nitems) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *nitems = (int32_t)ioff[nseg];
    if (i >= nseg) return;
    const int len = V.item_len[cloud_of_group(V, seg_group[i])];
    const int64_t a = seg_begin[i], b = a + seg_count[i];
    int64_t k = ioff[i];
    for (int64_t c = a; c < b; c += len, ++k) {
        ig[k] = seg_group[i];
        ib[k] = c;
        ie[k] = c + len < b ? c + len : b;
    }
}
// Splits the items between the two count kernels by their cloud's choice.
__global__ void k_item_split(const __grid_constant__ Views V, Items all, int32_t *__restrict__ tg,
                             int64_t *__restrict__ tb, int64_t *__restrict__ te, int32_t *__restrict__ tn,
                             int32_t *__restrict__ fg, int64_t *__restrict__ fb, int64_t *__restrict__ fe,
                             int32_t *__restrict__ fn) {
    const int it = blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= *all.count) return;
    const int gg = all.group[it];
    if (V.use_tc[cloud_of_group(V, gg)]) {
        const int k = atomicAdd(tn, 1);
        tg[k] = gg;
        tb[k] = all.begin[it];
        te[k] = all.end[it];
    } else {
        const int k = atomicAdd(fn, 1);
        fg[k] = gg;
        fb[k] = all.begin[it];
        fe[k] = all.end[it];
    }
}
__global__ void k_check_rows(int64_t n, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ rowcur,
                             int32_t *__restrict__ err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && row_ptr[i] + rowcur[i] != row_ptr[i + 1]) atomicOr(err, 8);
}
// rowsel != nullptr: only the selected rows were written.
__global__ void k_check_rows_sel(int64_t n, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ rowcur,
                                 const uint8_t *__restrict__ rowsel, int32_t *__restrict__ err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && rowsel[i] && row_ptr[i] + rowcur[i] != row_ptr[i + 1]) atomicOr(err, 8);
}

// One-pass emit, after the count pass: every row's produced entries must
// equal its degree; counts rows past their capacity (cnt[0]) and lost rows
// (cnt[1]).
__global__ void k_cap_rows(int64_t n, const int64_t *__restrict__ row_ptr, const int64_t *__restrict__ off,
                           const int32_t *__restrict__ fill, const uint8_t *__restrict__ lost,
                           unsigned long long *__restrict__ cnt, int32_t *__restrict__ err) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool ov = false, ls = false;
    if (o < n) {
        const int64_t deg = row_ptr[o + 1] - row_ptr[o];
        if ((int64_t)fill[o] != deg) atomicOr(err, 64);
        ov = deg > off[o + 1] - off[o];
        ls = lost[o] != 0;
    }
    const unsigned a = __ballot_sync(0xffffffffu, ov), b = __ballot_sync(0xffffffffu, ls);
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicAdd(cnt, (unsigned long long)__popc(a));
        if (b) atomicAdd(cnt + 1, (unsigned long long)__popc(b));
    }
}

// Copies each kept row's capacity-region entries into the CSR (warp per row).
__global__ void k_compact(int64_t n, const int64_t *__restrict__ row_ptr, const int64_t *__restrict__ off,
                          const uint8_t *__restrict__ lost, const int32_t *__restrict__ ccol,
                          const float *__restrict__ cdist, int32_t *__restrict__ col, float *__restrict__ dist) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n || lost[w]) return;
    const int64_t b = off[w], cap = off[w + 1] - b, d0 = row_ptr[w], deg = row_ptr[w + 1] - d0;
    const int64_t m = deg < cap ? deg : cap;
    for (int64_t j = lane; j < m; j += 32) {
        col[d0 + j] = ccol[b + j];
        dist[d0 + j] = cdist[b + j];
    }
}

// Places the overflow arena's entries of kept rows at their slots.
__global__ void k_ovf_scatter(int64_t used, const int32_t *__restrict__ orow, const int32_t *__restrict__ oslot,
                              const int32_t *__restrict__ ocol, const float *__restrict__ odist,
                              const uint8_t *__restrict__ lost, const int64_t *__restrict__ row_ptr,
                              int32_t *__restrict__ col, float *__restrict__ dist, int32_t *__restrict__ err) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= used) return;
    const int r = orow[k];
    if (lost[r]) return;
    const int64_t at = row_ptr[r] + oslot[k];
    if (at >= row_ptr[r + 1]) {
        atomicOr(err, 128);
        return;
    }
    col[at] = ocol[k];
    dist[at] = odist[k];
}

// ---------------------------------------------------------------------------
// Precision 1: tensor-core filter, FP32 recheck, FP64 guard band.
//
// Count pass per work item: the group's queries (B, N = 32) and 128-row tiles
// of packed candidate points (A, M = 128), both as fp16 rows prepared once per
// query (below), are multiplied by tcgen05 MMAs (K = 16 per instruction) into a
// 128 x 32 fp32 accumulator in tensor memory.  The accumulator, the rows'
// squared norms and a rigorous bound on the fp16 and fp32 rounding give a
// filter that keeps every edge; kept pairs are decided like the FP32 path: the
// canonical fp32 direct-difference sum of the original rows (decide32), the
// pinned FP64 sum where that cannot decide.  The emit pass is the FP32 path's,
// driven by the same per-block edge masks.
constexpr int TC_ROWS = 128;
constexpr int TC_NB = kItemTC;          // candidate blocks of one item
constexpr uint32_t TC_WAIT = 1u << 22;  // mbarrier polls before a wait gives up
constexpr uint32_t TC_HINT = 1u << 16;  // ns a suspended poll may sleep (woken by the phase)
constexpr uint32_t TC_SLEEPS = 1u << 14;  // suspended polls before a wait gives up (about a second)
constexpr int TC_KL = 1024;             // kept pairs rechecked per round

// ---------------------------------------------------------------------------
// FP16 rows for the tensor-core filter.  Each cloud's points are stored once
// per query as x^ = fp16(s fl(x - m)) (m: the column means, s: a power of two
// with s |x_k - m_k| < 2^14), rows of kp = 64 ceil(dp / 64) halves, zero
// padded, with n^ = the fp32 sum of their squares.  Rounding to nearest gives
// |x^_k - s (x_k - m_k)| <= 2^-11 (1 + 2^-10) |x^_k| + 2^-25 (the last for
// subnormal halves), so with |x^| <= sqrt(n^) (1 + 2^-16) =: a_x
//   ||x^ - y^|| <= s d(x, y) + rel (a_x + a_y) + 2^-20,  rel = 2^-11 (1 + 2^-8).
// d^2 = n^_x + n^_y - 2 x^.y^ is formed from exact fp16 products with fp32
// sums: the MMA's accumulation (K <= 128 terms, below 2^-17 (n^_x + n^_y)),
// the norms (2^-17 each) and the formula (2^-22) stay below 2^-15.9 (n^_x +
// n^_y).  A pair is kept iff
//   d^2 <= (s eps + rel (a_x + a_y) + 2^-20)^2 + 2^-14 (a_x^2 + a_y^2) + 2^-60,
// which keeps every edge with a 4x margin on the fp32 terms.  The slack
// relative to eps grows with |x - m| / eps (about 2^-10 of it); rows are
// copied into the MMA's layout unchanged, so the count pass converts nothing.
constexpr int H16_MB = 1024;  // blocks of the column-mean partial sums
constexpr float H16_REL = 0x1.01p-11f, H16_ABS = 0x1p-20f, H16_ABS2 = 0x1p-14f;
constexpr float H16_NORM_UP = 1.0f + 0x1p-16f;

// Partial column sums: block b adds points b, b + H16_MB, ...; thread k is
// coordinate k (dp <= 128).
__global__ void k_col_partial(const float *__restrict__ pts, int64_t n, int dp, float *__restrict__ partial) {
    const int k = threadIdx.x;
    if (k >= dp) return;
    float acc = 0.f;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) acc += __ldg(pts + i * dp + k);
    partial[(size_t)blockIdx.x * dp + k] = acc;
}

// Column means (partials added in block order) and the scale: every point is
// within r_root of the root centre, so |x_k - m_k| <= |x - m| <= 2 r_root;
// s = 2^(14 - e) with max(2 r_root, eps) < 2^e.  scal = {s, s eps_up}.
__global__ void k_col_final(const float *__restrict__ partial, int dp, int64_t n, const float *__restrict__ radius,
                            float eps_up, float *__restrict__ mean, float *__restrict__ scal) {
    const int k = threadIdx.x;
    if (k < dp) {
        double acc = 0.0;
        for (int b = 0; b < H16_MB; ++b) acc += (double)partial[(size_t)b * dp + k];
        mean[k] = n ? (float)(acc / (double)n) : 0.f;
    }
    if (k == 0) {
        const float M = fmaxf(2.0f * radius[0] * (1.0f + 0x1p-10f), eps_up);
        float s = 0x1p-100f;
        if (M <= 0x1p100f) {
            int e;
            frexpf(fmaxf(M, 0x1p-100f), &e);  // M < 2^e
            s = ldexpf(1.0f, 14 - e);
        }
        scal[0] = s;
        scal[1] = s * eps_up;
    }
}

// Rows in tree order -> fp16 rows and their squared norms; sixteen lanes per
// row, lane j converts halves 8j .. 8j + 7 (one 16-byte chunk).
__global__ void k_to_h16(const float *__restrict__ pts, int64_t n, int dp, int kp, const float *__restrict__ mean,
                         const float *__restrict__ scal, uint4 *__restrict__ h16, float *__restrict__ n16) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = gid >> 4;
    const int j = (int)(gid & 15), kc = kp >> 3;
    const float s = scal[0];
    float sq = 0.f;
    if (row < n && j < kc) {
        float v[8];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = 8 * j + 4 * h;
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f), m = x;
            if (k < dp) {  // dp is a multiple of 4
                x = __ldg(reinterpret_cast<const float4 *>(pts + row * dp + k));
                m = __ldg(reinterpret_cast<const float4 *>(mean + k));
            }
            v[4 * h + 0] = (x.x - m.x) * s;
            v[4 * h + 1] = (x.y - m.y) * s;
            v[4 * h + 2] = (x.z - m.z) * s;
            v[4 * h + 3] = (x.w - m.w) * s;
        }
        uint32_t w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const __half2 hh = __floats2half2_rn(v[2 * u], v[2 * u + 1]);
            w[u] = *reinterpret_cast<const uint32_t *>(&hh);
            const float2 f = __half22float2(hh);
            sq = fmaf(f.x, f.x, sq);
            sq = fmaf(f.y, f.y, sq);
        }
        h16[row * kc + j] = make_uint4(w[0], w[1], w[2], w[3]);
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o, 16);
    if (j == 0 && row < n) n16[row] = sq;
}

constexpr int TC_T = 256;   // threads per CTA (two CTAs per SM)
constexpr int TC_EB = 768;  // edge buffer entries (one-pass emit)
constexpr int TC_ISSUER = TC_T - 32;  // lane 0 of the last warp: issues the tiles' MMAs, tracks the query rows' load
struct __align__(1024) TcShared {
    unsigned char A[2][2][TC_ROWS * 128];  // fp16 candidate rows: buffer, K half (64 halves), 128-byte swizzle
    unsigned char B[2][32 * 128];          // fp16 query rows, the same layout
    float pn[4][TC_ROWS];                  // squared norms of the rows, per map slot
    int pos[4][TC_ROWS];                   // map slots of tiles t .. t + 3 (slot t & 3): tree positions
    uint16_t li[4][TC_ROWS];               //   and candidate blocks
    uint16_t kl[TC_KL];                    // kept pairs of the tile: (query << 7) | row
    int ecol[TC_EB];
    float edist[TC_EB];
    uint16_t erank[TC_EB];
    uint8_t eq[TC_EB];
    float2 qhg[32];                        // per query: threshold terms (h_q, g_q) of the filter
    int bbeg[TC_NB], bpre[TC_NB + 1];
    uint32_t bem[TC_NB];
    int qcnt[32], orig[32], qfill[32], qbase[32];
    int wsum[TC_T / 32];
    int kn[2], en;
    uint32_t tslot;
    uint64_t mbar[2], bbar;                // MMAs (per buffer), query rows
};
constexpr size_t kTcSmem = sizeof(TcShared) + 1024;
static_assert(2 * (kTcSmem + 1024) <= 228 * 1024, "k_leaf_tc: two CTAs per SM");
static_assert(TC_NB % TC_T == 0, "block prefix takes TC_NB / TC_T candidate blocks per thread");

// Count pass (and one-pass emit) with the FP16 filter.  One CTA of 8 warps per
// work item, two CTAs per SM (one's setup and drain overlap the other's
// tiles).  Candidate rows arrive by 16-byte cp.async copies of every thread
// (half a row each), written in the MMA's 128-byte swizzled operand layout,
// two tiles ahead; the 32 query rows by TMA gathers.  One thread issues the
// MMA of tile t + 1 (second accumulator) as the iteration of tile t begins, so
// that it runs while tile t is filtered and rechecked.  Rechecks read the
// original fp32 rows from global memory, eight lanes per pair.
__global__ void __launch_bounds__(TC_T, 2) k_leaf_tc(const __grid_constant__ Views V, Items items,
                                                     const uint32_t *__restrict__ cand, uint32_t *__restrict__ emask,
                                                     int32_t *__restrict__ deg, unsigned long long *__restrict__ st,
                                                     int32_t *__restrict__ err, CapOut co) {
    extern __shared__ unsigned char tc_raw[];
    TcShared &S = *reinterpret_cast<TcShared *>(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    const int it = blockIdx.x;
    if (it >= *items.count) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gg = items.group[it];
    const int cloud = cloud_of_group(V, gg);
    const TreeView &tv = V.tv[cloud];
    const QParams &qp = V.qp[cloud];
    const void *tmap = &V.tmap[cloud];
    const uint4 *h16 = V.h16[cloud];
    const float *n16 = V.n16[cloud];
    const int g = gg - V.gbase[cloud];
    const int64_t rbase = V.rbase[cloud];  // CSR rows of this cloud start here
    const int dp = tv.dp, dim = tv.dim, dp4 = dp >> 2;
    const float4 *pts4 = reinterpret_cast<const float4 *>(tv.pts);
    const int halves = (dp + 63) >> 6;               // 64-half K blocks of an fp16 row (1 or 2)
    const int ksteps = 4 * halves;                   // MMA K steps of 16
    const int kc = 8 * halves;                       // 16-byte chunks of an fp16 row
    const uint32_t q_bytes = (uint32_t)(32 * 128 * halves);
    const int qb = tv.group_begin[g], qn = tv.group_count[g];
    const int qe = qb + qn;  // the group's positions; upper-triangle form: rows before qb are skipped, edges
                             // with rows from qe on are mirrored into those rows
    const int64_t c0 = items.begin[it];
    const int nb = (int)(items.end[it] - c0);        // <= TC_NB
    uint32_t pairs = 0, kept = 0, guard = 0, band = 0, rows_ld = 0;  // rows_ld, kept: thread 0
    bool failed = false;
    // next phase parity of each barrier (bit b: buffer b): mph in every thread
    // (warp 0 waits), bph in the issuing thread (it waits), which also tracks
    // what is in flight, for a clean exit after a failure
    uint32_t mph = 0u, bph = 0u, mpend = 0u, bpend = 0u;
    bool tok = true;  // the issuing thread (TC_ISSUER): its own waits succeeded

    if (warp == 0) tc::tmem_alloc(&S.tslot, 64);
    if (tid == 0) {
        tc::mbar_init(&S.mbar[0], 1);
        tc::mbar_init(&S.mbar[1], 1);
        tc::mbar_init(&S.bbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    // candidate blocks of the item and their row prefix (TC_NB / TC_T blocks per thread)
    {
        constexpr int BPT = TC_NB / TC_T;
        int loc[BPT], sum = 0;
#pragma unroll
        for (int k = 0; k < BPT; ++k) {
            const int i = BPT * tid + k;
            int beg = 0, cnt = 0;
            if (i < nb) {
                const int v = (int)cand[c0 + i];
                beg = tv.node_begin[v];
                cnt = tv.node_count[v];
            }
            S.bbeg[i] = beg;
            S.bem[i] = 0u;
            loc[k] = cnt;
            sum += cnt;
        }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) S.wsum[warp] = incl;
        __syncthreads();
        int base = 0;
#pragma unroll
        for (int w = 0; w < TC_T / 32; ++w)
            if (w < warp) base += S.wsum[w];
        int run = base + incl - sum;
#pragma unroll
        for (int k = 0; k < BPT; ++k) {
            S.bpre[BPT * tid + k] = run;
            run += loc[k];
        }
        if (tid == TC_T - 1) S.bpre[TC_NB] = run;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = S.tslot;
    const int T = S.bpre[TC_NB];
    const int ntiles = (T + TC_ROWS - 1) / TC_ROWS;
    const float s_eps = V.s16[cloud][1];  // s eps_up

    // rows of tile t -> (position, block) in map slot t & 3 and the rows'
    // norms (4-byte copies; each thread commits one copy group per call).
    // Warp w in 1..4 maps rows 32 (w - 1) .. + 31 of the tile: the block b0
    // holding the window's first row R0 comes from two 32-wide ballot
    // searches over the block prefix (the largest b0 with bpre[b0] <= R0);
    // blocks b0 + 1 .. b0 + 31 start inside the window or after it, and a
    // row's block is b0 plus the number of block starts in (R0, R].
    auto prep_map = [&](int t) {
        const int wq = warp - 1, R0 = t * TC_ROWS + 32 * wq;
        if (t < ntiles && wq >= 0 && wq < 4 && R0 < T) {  // warp-uniform
            const unsigned mc = __ballot_sync(0xffffffffu, S.bpre[32 * lane] <= R0);  // bit 0 set: bpre[0] = 0
            const int c = 31 - __clz(mc);
            const unsigned mf = __ballot_sync(0xffffffffu, S.bpre[32 * c + lane] <= R0);
            const int b0 = 32 * c + 31 - __clz(mf);
            const int j = b0 + 1 + lane;
            const int v = j <= TC_NB ? S.bpre[j] : INT_MAX;
            const unsigned m = __reduce_or_sync(0xffffffffu, v < R0 + 32 ? 1u << (v - R0) : 0u);  // v > R0
            const int R = R0 + lane;
            if (R < T) {
                const int blk = b0 + __popc(m & (0xffffffffu >> (31 - lane)));
                const int pos = S.bbeg[blk] + (R - S.bpre[blk]);
                const int r = 32 * wq + lane;
                S.pos[t & 3][r] = pos;
                S.li[t & 3][r] = (uint16_t)blk;
                cp_async4(&S.pn[t & 3][r], n16 + pos);
            }
        }
        cp_async_commit();
    };
    // every thread: rows of tile t (past the last row of a short tile: row 0
    // again) into buffer t & 1 by 16-byte copies, consecutive threads taking
    // consecutive chunks of a row (a warp's copy covers 2 or 4 whole rows), in
    // the MMA's 128-byte swizzled K-major layout (chunk j of row r at chunk
    // j ^ (r % 8) of the row's 128 bytes; 1024-byte atoms of 8 rows).
    // Completed by the copy group wait, a proxy fence and the barrier at the
    // top of the next iteration, before the MMA that reads them is issued.
    auto load_tile = [&](int t) {
        const int rows = min(TC_ROWS, T - t * TC_ROWS), sl = t & 3, bf = t & 1;
        const int lkc = 2 + halves;  // log2 of kc (8 or 16 chunks per row)
        for (int g = tid; g < TC_ROWS * kc; g += TC_T) {
            const int r = g >> lkc, ch = g & (kc - 1), h = ch >> 3, j = ch & 7;
            const int pos = S.pos[sl][r < rows ? r : 0];
            cp_async16(S.A[bf][h] + r * 128 + ((j ^ (r & 7)) << 4), h16 + (size_t)pos * kc + ch, true);
        }
    };
    // the issuing thread: tile t's MMA chain into accumulator columns 32 (t & 1)
    auto mma_tile = [&](int t) {
        const int bf = t & 1;
        constexpr uint32_t idesc = tc::idesc_f16_f32(TC_ROWS, 32);
        for (int ks = 0; ks < ksteps; ++ks) {
            const int h = ks >> 2, j = ks & 3;  // K half, 16-half step inside it (32 bytes)
            const uint64_t ad = tc::smem_desc_sw128(tc::smem_u32(S.A[bf][h]) + 32 * j);
            const uint64_t bd = tc::smem_desc_sw128(tc::smem_u32(S.B[h]) + 32 * j);
            tc::mma_f16(tmem + (uint32_t)(32 * bf), ad, bd, idesc, ks > 0);
        }
        tc::mma_commit(&S.mbar[bf]);
        mpend |= 1u << bf;
    };

    for (int q0 = 0; q0 < qn && !failed; q0 += 32) {
        const int nqr = min(32, qn - q0);
        const int qfirst = qb + q0;
        __syncthreads();
        if (tid < 32) {
            S.qcnt[tid] = 0;
            S.qfill[tid] = 0;
            S.orig[tid] = tid < nqr ? (int)(rbase + tv.perm[qfirst + tid]) : 0;
            // filter test per query (see the filter)
            const float qn2 = tid < nqr ? __ldg(n16 + qfirst + tid) : 0.f;
            const float qa = sqrtf(qn2) * H16_NORM_UP;
            const float E = fmaf(H16_REL, qa, s_eps) + H16_ABS;
            const float h = 0.5f * (qn2 - fmaf(E, E, fmaf(H16_ABS2 * qa, qa, 0x1p-60f))) - 0x1p-20f * (E * E);
            S.qhg[tid] = make_float2(h, -H16_REL * E);
        }
        for (int i = tid; i < nb; i += TC_T) S.bem[i] = 0u;
        if (tid == 0) {
            S.en = 0;
            S.kn[0] = S.kn[1] = 0;
        }
        prep_map(0);
        prep_map(1);
        prep_map(2);
        if (tid == TC_ISSUER) {  // the expectation before any gather of the query rows is issued
            tc::mbar_arrive_expect_tx(&S.bbar, q_bytes);
            bpend = 1u;
        }
        __syncthreads();
        // query rows (past the group's queries: its last query again) and tiles 0, 1
        if (warp == 0 && lane < 8) {
            const int q = 4 * lane;
            const int r0 = qfirst + min(q, nqr - 1), r1 = qfirst + min(q + 1, nqr - 1);
            const int r2 = qfirst + min(q + 2, nqr - 1), r3 = qfirst + min(q + 3, nqr - 1);
            for (int h = 0; h < halves; ++h) tc::tma_gather4(S.B[h] + q * 128, tmap, 64 * h, r0, r1, r2, r3, &S.bbar);
        }
        for (int t = 0; t < 2 && t < ntiles; ++t) load_tile(t);
        cp_async_commit();
        cp_async_wait<0>();
        tc::fence_smem_to_async();
        __syncthreads();
        if (tid == TC_ISSUER) {  // the issuing thread alone tracks the query rows' barrier phase
            const bool okb = tok && tc::mbar_wait_sleep(&S.bbar, bph, TC_SLEEPS, TC_HINT);
            if (okb) {
                bpend = 0u;
                bph ^= 1u;
                if (ntiles > 0) {
                    tc::fence_after_sync();
                    mma_tile(0);
                }
            }
            tok = okb;
        }

        auto flush = [&]() {
            if (tid < 32 && S.qfill[tid]) S.qbase[tid] = atomicAdd(&co.fill[S.orig[tid]], S.qfill[tid]);
            __syncthreads();
            const int n = min(S.en, TC_EB);
            for (int i = tid; i < n; i += TC_T) {
                const int q = S.eq[i];
                if (q & 0x80)  // an edge mirrored into the row of tree position ecol (upper triangle)
                    cap_put(co, (int)(rbase + tv.perm[S.ecol[i]]), tv.perm[qfirst + (q & 31)], S.edist[i]);
                else
                    cap_place(co, S.orig[q], S.qbase[q] + S.erank[i], tv.perm[S.ecol[i]], S.edist[i]);
            }
            __syncthreads();
            if (tid < 32) S.qfill[tid] = 0;
            if (tid == 0) S.en = 0;
        };
        // pair e = (query << 7) | row in map slot sl, by the eight lanes of an
        // octet: lane j sums coordinate chunk j (16 floats of both original
        // rows) in the canonical order, the chunk sums are added in ascending
        // order -- the canonical fp32 sum; the octet's first lane decides (FP64
        // where fp32 cannot) and records the edge
        auto recheck8 = [&](int e, int sl) {
            const int q = e >> 7, r = e & 127, sub = lane & 7;
            const unsigned omask = 0xffu << (lane & 24);
            const int ppos = S.pos[sl][r];
            const float4 *prow = pts4 + (size_t)ppos * dp4;
            const float4 *qrow = pts4 + (size_t)(qfirst + q) * dp4;
            const int k0 = 4 * sub;
            float lo = 0.f, hi = 0.f;
            if (k0 < dp4) {
                float4 a[4], b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const bool in = k0 + u < dp4;
                    a[u] = in ? qrow[k0 + u] : make_float4(0.f, 0.f, 0.f, 0.f);
                    b[u] = in ? __ldg(prow + k0 + u) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (k0 + u < dp4) {
                        const float dx = a[u].x - b[u].x, dy = a[u].y - b[u].y, dz = a[u].z - b[u].z,
                                    dw = a[u].w - b[u].w;
                        lo = fmaf(dx, dx, lo);
                        hi = fmaf(dy, dy, hi);
                        lo = fmaf(dz, dz, lo);
                        hi = fmaf(dw, dw, hi);
                    }
            }
            const float chunk = lo + hi;
            const int nch = (dp4 + 3) >> 2;
            float sv = __shfl_sync(omask, chunk, 0, 8);
#pragma unroll
            for (int j = 1; j < 8; ++j) {
                const float cj = __shfl_sync(omask, chunk, j, 8);
                if (j < nch) sv += cj;
            }
            if (sub) return;
            unsigned long long in_band = 0;
            const int edge = decide32(qp, sv, in_band);
            band += (uint32_t)in_band;
            bool is_edge;
            float d;
            if (edge < 0) {
                ++guard;
                note_guard_rows(S.orig[q], (int32_t)(rbase + tv.perm[ppos]));
                const double s64 = sq_l2_exact4(qrow, prow, dim);
                is_edge = s64 <= qp.eps2_64;
                d = (float)sqrt(s64);
            } else {
                is_edge = edge != 0;
                d = sqrtf(sv);
            }
            if (is_edge) {
                if (qp.half && ppos >= qe) {
                    const int64_t o = rbase + tv.perm[ppos];
                    atomicAdd(&deg[o], 1);
                    if (co.off) {  // its slot is taken at the flush, off the recheck's path
                        const int slot = atomicAdd(&S.en, 1);
                        if (slot < TC_EB) {
                            S.eq[slot] = (uint8_t)(0x80 | q);
                            S.ecol[slot] = ppos;
                            S.edist[slot] = d;
                        } else {
                            cap_put(co, (int)o, tv.perm[qfirst + q], d);
                        }
                    }
                }
                atomicAdd(&S.qcnt[q], 1);
                atomicOr(&S.bem[S.li[sl][r]], 1u << q);
                if (co.off) {
                    const int slot = atomicAdd(&S.en, 1);
                    if (slot < TC_EB) {
                        S.eq[slot] = (uint8_t)q;
                        S.ecol[slot] = ppos;  // tree position; the original id is looked up at the flush
                        S.edist[slot] = d;
                        S.erank[slot] = (uint16_t)atomicAdd(&S.qfill[q], 1);
                    } else {
                        cap_put(co, S.orig[q], tv.perm[ppos], d);
                    }
                }
            }
        };

        for (int t = 0; t < ntiles; ++t) {
            const int sl = t & 3, bf = t & 1;
            const int rows = min(TC_ROWS, T - t * TC_ROWS);
            if (tid == 0) rows_ld += rows;
            // tile t's MMA has completed (warp 0 waits); the rows of tile t + 1
            // (copied an iteration ago) and the norms have landed
            cp_async_wait<0>();
            tc::fence_smem_to_async();
            bool ok = tid != TC_ISSUER || tok;  // the issuing thread's own waits so far
            if (warp == 0) ok = tc::mbar_wait_sleep(&S.mbar[bf], (mph >> bf) & 1u, TC_SLEEPS, TC_HINT);
            if (!__syncthreads_and(ok)) {
                if (tid == 0) atomicOr(err, 32);
                failed = true;
                break;
            }
            mph ^= 1u << bf;
            if (tid == TC_ISSUER) mpend &= ~(1u << bf);
            tc::fence_after_sync();
            if (co.off && S.en >= TC_EB / 2) flush();  // tile t - 1's rechecks are done
            // the issuing thread: tile t + 1's MMA into the other accumulator now,
            // so that it runs while tile t is filtered and rechecked (its rows
            // were copied an iteration ago; its columns were last read by tile
            // t - 1's filter, before the barrier above)
            if (t + 1 < ntiles && tid == TC_ISSUER && tok) mma_tile(t + 1);
            if (t + 2 < ntiles) load_tile(t + 2);  // buffer bf: tile t's MMA has completed
            prep_map(t + 3);                       // commits the group (tile t + 2's rows, t + 3's norms)
            // epilogue, filter: warp w reads rows 32 (w % 4) .. + 31, queries
            // 16 (w / 4) .. + 15; kept pairs go to the tile's list
            uint32_t keepm = 0u;
            int kb = 0;
            {
                const int quarter = warp & 3, qh = warp >> 2;
                float dot[16];
                tc::tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(32 * bf + 16 * qh), dot);
                const int r = 32 * quarter + lane;
                if (r < rows) {
                    // kept iff d^2 = n^_q + n^_p - 2 dot <= (E_q + rel |p^|)^2 + abs2 (|q^|^2 + |p^|^2)
                    // + 2^-60 with E_q = s eps + rel |q^| + 2^-20, i.e. iff dot >= h_q + g_q |p^| + w_p
                    // with h_q = (n^_q - E_q^2 - abs2 |q^|^2 - 2^-60) / 2, g_q = -rel E_q,
                    // w_p = (n^_p - (rel^2 + abs2) |p^|^2) / 2.  The rounding of this form stays
                    // below 2^-21 (n^_q + n^_p + 2 E_q^2): the first part is inside the abs2
                    // term's slack over the other fp32 errors, the second is covered by the
                    // 2^-20 E_q^2 taken off h_q.  NaN keeps the pair.
                    const int ppos = S.pos[sl][r];
                    const float pn = S.pn[sl][r];
                    const float pa = sqrtf(pn) * H16_NORM_UP;
                    const float wp = 0.5f * fmaf(-(H16_REL * H16_REL + H16_ABS2) * pa, pa, pn);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float2 hg = S.qhg[16 * qh + j];
                        if (!(dot[j] < fmaf(hg.y, pa, hg.x) + wp)) keepm |= 1u << j;
                    }
                    uint32_t validm = (nqr >= 16 * qh + 16 ? 0xffffu : (1u << max(nqr - 16 * qh, 0)) - 1u);
                    const int self = ppos - qfirst - 16 * qh;
                    if (!qp.include_self && (unsigned)self < 16u) validm &= ~(1u << self);
                    if (qp.half && ppos < qb) validm = 0u;
                    keepm &= validm;
                    pairs += __popc(validm);
                }
                const int c = __popc(keepm);
                int incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                int base = 0;
                if (lane == 31 && incl) base = atomicAdd(&S.kn[bf], incl);
                kb = __shfl_sync(0xffffffffu, base, 31) + incl - c;
                uint32_t m = keepm;
                for (int idx = kb; m && idx < TC_KL; ++idx) {
                    const int j = __ffs(m) - 1;
                    m &= m - 1u;
                    S.kl[idx] = (uint16_t)(((16 * qh + j) << 7) | r);
                }
            }
            tc::fence_before_sync();
            __syncthreads();
            const int n = S.kn[bf];
            if (tid == 0) {
                kept += n;
                S.kn[bf ^ 1] = 0;  // tile t + 1's list (filled after the next barrier)
            }
            // recheck: the kept pairs spread over the lane octets, one pair per
            // octet, TC_KL at a time (pairs past the list are re-derived from
            // the filter's masks)
            for (int i = tid >> 3; i < min(n, TC_KL); i += TC_T / 8) recheck8(S.kl[i], sl);
            for (int lo = TC_KL; lo < n; lo += TC_KL) {
                __syncthreads();
                uint32_t m = keepm;
                const int qc = 16 * (warp >> 2), r = 32 * (warp & 3) + lane;
                for (int idx = kb; m && idx < lo + TC_KL; ++idx) {
                    const int j = __ffs(m) - 1;
                    m &= m - 1u;
                    if (idx >= lo) S.kl[idx - lo] = (uint16_t)(((qc + j) << 7) | r);
                }
                __syncthreads();
                for (int i = tid >> 3; i < min(n - lo, TC_KL); i += TC_T / 8) recheck8(S.kl[i], sl);
            }
        }
        if (failed) break;
        __syncthreads();
        if (co.off) flush();
        __syncthreads();
        if (tid < nqr && S.qcnt[tid]) atomicAdd(&deg[S.orig[tid]], S.qcnt[tid]);
    }
    if (!failed && emask)
        for (int i = tid; i < nb; i += TC_T) emask[c0 + i] = qn <= 32 ? S.bem[i] : ~0u;
    unsigned long long pairs64 = pairs, kept64 = kept, guard64 = guard, band64 = band;
    for (int o = 16; o > 0; o >>= 1) {
        pairs64 += __shfl_xor_sync(0xffffffffu, pairs64, o);
        kept64 += __shfl_xor_sync(0xffffffffu, kept64, o);
        guard64 += __shfl_xor_sync(0xffffffffu, guard64, o);
        band64 += __shfl_xor_sync(0xffffffffu, band64, o);
    }
    if (lane == 0) {
        stat_add(st, ST_PAIRS, pairs64);
        stat_add(st, ST_RECHECK, kept64);
        stat_add(st, ST_GUARD, guard64);
        stat_add(st, ST_BAND, band64);
        if (tid == 0) stat_add(st, ST_ROWS, rows_ld);
    }
    cp_async_wait<0>();  // no copy into this CTA's shared memory outlives it
    if (tid == TC_ISSUER) {  // after a failure: let the query rows' gathers and MMAs in flight finish (bounded)
        for (int b = 0; b < 2; ++b)
            if (mpend >> b & 1u) tc::mbar_wait(&S.mbar[b], (mph >> b) & 1u, TC_WAIT);
        if (bpend) tc::mbar_wait_sleep(&S.bbar, bph, TC_SLEEPS, TC_HINT);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 64);
}


// Dynamic shared memory of the L2 leaf kernel (set once per process).
void leaf_l2_prepare() {
    static bool done = false;
    if (done) return;
    CT_CHECK_CUDA(cudaFuncSetAttribute(k_leaf_l2<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLeafSmem));
    CT_CHECK_CUDA(cudaFuncSetAttribute(k_leaf_l2<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLeafSmem));
    done = true;
}

// Upper-triangle form, integer metrics (one cloud): the edge (q, p) with p in
// a later group is also the edge (p, q) of p's row: its degree and one-pass
// entry (count pass) or its entry (emit pass; a selected row only when rows
// are emitted again).
__device__ __forceinline__ void mirror_int(const TreeView &tv, int32_t *deg, const int64_t *row_ptr, int32_t *rowcur,
                                           int32_t *col, float *dist, int32_t *err, const CapOut &co,
                                           const uint8_t *rowsel, bool emit, int qpos, int ppos, int d) {
    const int o = tv.perm[ppos];
    if (!emit) {
        atomicAdd(&deg[o], 1);
        if (co.off) cap_put(co, o, tv.perm[qpos], (float)d);
        return;
    }
    if (rowsel && !rowsel[o]) return;
    const int slot = atomicAdd(&rowcur[o], 1);
    const int64_t at = row_ptr[o] + slot;
    if (at < row_ptr[o + 1]) {
        col[at] = tv.perm[qpos];
        dist[at] = (float)d;
    } else {
        atomicOr(err, 4);
    }
}

// Edit distance of one (pattern, text) pair over alphabet-mapped symbols;
// the distance if <= k, else k + 1.
template <int W>
__device__ __forceinline__ int lev_mapped(const uint64_t *__restrict__ pq, const uint8_t *__restrict__ amap, int m,
                                          const uint8_t *__restrict__ txt, int n, int k,
                                          unsigned long long &cols) {
    if (k < 0) return (m == 0 && n == 0) ? 0 : k + 1;
    if ((m > n ? m - n : n - m) > k) return k + 1;
    if (m == 0) return n;
    if (n == 0) return m;
    const int nw = (m + 63) >> 6, hw = (m - 1) >> 6;
    const uint64_t hbit = 1ull << ((m - 1) & 63);
    uint64_t Pv[W], Mv[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        Pv[w] = ~0ull;
        Mv[w] = 0ull;
    }
    int score = m;
    for (int j = 0; j < n; ++j) {
        const uint64_t *eqr = pq + (int)amap[txt[j]] * W;
        uint64_t carry = 0ull, hp_in = 1ull, hn_in = 0ull;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            if (w < nw) {
                uint64_t Eq = eqr[w], pv = Pv[w], mv = Mv[w];
                uint64_t Xv = Eq | mv, tt = Eq & pv;
                uint64_t s1 = tt + pv, c1b = s1 < tt ? 1ull : 0ull;
                uint64_t s2 = s1 + carry, c2b = s2 < s1 ? 1ull : 0ull;
                carry = c1b | c2b;
                uint64_t Xh = (s2 ^ pv) | Eq;
                uint64_t Ph = mv | ~(Xh | pv), Mh = pv & Xh;
                if (w == hw) {
                    if (Ph & hbit) ++score;
                    else if (Mh & hbit) --score;
                }
                uint64_t po = Ph >> 63, mo = Mh >> 63;
                Ph = (Ph << 1) | hp_in;
                Mh = (Mh << 1) | hn_in;
                hp_in = po;
                hn_in = mo;
                Pv[w] = Mh | ~(Xv | Ph);
                Mv[w] = Ph & Xv;
            }
        }
        if (score - (n - 1 - j) > k) {
            cols += (unsigned long long)(j + 1) * nw;
            return k + 1;
        }
    }
    cols += (unsigned long long)n * nw;
    return score;
}

// Edit distance leaf stage: one CTA per group; packed candidate tiles as in
// the L2 kernel; each thread decides (query, candidate point) pairs with the
// query as the bit-parallel pattern.  The queries' match masks cover only the
// bytes that occur in the data (alphabet map amap, A symbols).
template <bool EMIT, int W>
__global__ void __launch_bounds__(LEAF_T) k_leaf_lev(
    TreeView tv, QParams qp, const uint8_t *__restrict__ amap_g, int A, int qchunk, Items items,
    uint32_t *__restrict__ cand, int32_t *__restrict__ deg, const int64_t *__restrict__ row_ptr,
    int32_t *__restrict__ rowcur, int32_t *__restrict__ col, float *__restrict__ dist,
    unsigned long long *__restrict__ st, int32_t *__restrict__ err, CapOut co, const uint8_t *__restrict__ rowsel) {
    extern __shared__ uint64_t speq[];  // qchunk x A x W
    __shared__ uint8_t amap[256];
    __shared__ int cnt[32], cursor[32], qlen[32], sel[32];
    __shared__ int64_t rowb[32], rowe[32];
    __shared__ int tpos[32];
    __shared__ int64_t tcand[32];
    __shared__ int64_t s_ci;
    __shared__ int s_off, s_rows;
    __shared__ unsigned s_hit;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int it = blockIdx.x;
    if (it >= *items.count) return;
    const int g = items.group[it];
    const int qb = tv.group_begin[g], qn = tv.group_count[g], qe = qb + qn;
    const int64_t c0 = items.begin[it], c1 = items.end[it];
    const int k = qp.lev_k;
    for (int i = tid; i < 256; i += LEAF_T) amap[i] = amap_g[i];
    unsigned long long pairs = 0, cols = 0;
    for (int q0 = 0; q0 < qn; q0 += qchunk) {
        const int nqr = min(qchunk, qn - q0);
        __syncthreads();
        for (int i = tid; i < qchunk * A * W; i += LEAF_T) speq[i] = 0ull;
        if (tid < 32) {
            cnt[tid] = 0;
            if (tid < nqr) {
                int qpos = qb + q0 + tid;
                qlen[tid] = (int)(tv.soff[qpos + 1] - tv.soff[qpos]);
                int o = tv.perm[qpos];
                cursor[tid] = o;  // original id of the query (row of the CSR)
                sel[tid] = rowsel == nullptr || rowsel[o] != 0;
                if (EMIT) {
                    rowb[tid] = row_ptr[o];
                    rowe[tid] = row_ptr[o + 1];
                }
            }
        }
        if (tid == 0) {
            s_ci = c0;
            s_off = 0;
            s_hit = 0u;
        }
        __syncthreads();
        for (int q = 0; q < nqr; ++q) {
            int qpos = qb + q0 + q;
            const uint8_t *sq = tv.sdata + tv.soff[qpos];
            int m = qlen[q];
            for (int j = tid; j < m; j += LEAF_T)
                atomicOr((unsigned long long *)&speq[((size_t)q * A + amap[sq[j]]) * W + (j >> 6)], 1ull << (j & 63));
        }
        for (;;) {
            __syncthreads();
            if (warp == 0) fill_tile(tv, cand, c1, EMIT, &s_ci, &s_off, &s_rows, tpos, tcand);
            __syncthreads();
            const int npr = s_rows;
            const bool last = s_ci >= c1;
            if (npr > 0) {
                unsigned hit = 0u;
                for (int t = tid; t < nqr * npr; t += LEAF_T) {
                    int q = t / npr, p = t - q * npr;
                    int qpos = qb + q0 + q, ppos = tpos[p];
                    if (qpos == ppos && !qp.include_self) continue;
                    if (qp.half && ppos < qb) continue;
                    const bool mir = qp.half && ppos >= qe;
                    if (EMIT && !sel[q] && !(mir && rowsel)) continue;
                    if (!EMIT) ++pairs;
                    const uint8_t *txt = tv.sdata + tv.soff[ppos];
                    int n = (int)(tv.soff[ppos + 1] - tv.soff[ppos]);
                    int d = lev_mapped<W>(speq + (size_t)q * A * W, amap, qlen[q], txt, n, k, cols);
                    if (d > k) continue;
                    if (mir) mirror_int(tv, deg, row_ptr, rowcur, col, dist, err, co, rowsel, EMIT, qpos, ppos, d);
                    if (!EMIT) {
                        hit |= 1u << p;
                        atomicAdd(&cnt[q], 1);
                        if (co.off) cap_put(co, cursor[q], tv.perm[ppos], (float)d);
                    } else if (sel[q]) {
                        int slot = atomicAdd(&rowcur[cursor[q]], 1);
                        int64_t at = rowb[q] + slot;
                        if (at < rowe[q]) {
                            col[at] = tv.perm[ppos];
                            dist[at] = (float)d;
                        } else {
                            atomicOr(err, 4);
                        }
                    }
                }
                if (!EMIT) {
                    if (hit) atomicOr(&s_hit, hit);
                    __syncthreads();
                    if (tid < npr && ((s_hit >> tid) & 1u)) atomicOr(&cand[tcand[tid]], FLAG);
                    __syncthreads();
                    if (tid == 0) s_hit = 0u;
                }
            }
            if (last) break;
        }
        __syncthreads();
        if (!EMIT && tid < nqr && cnt[tid]) atomicAdd(&deg[cursor[tid]], cnt[tid]);
    }
    if (!EMIT) {
        for (int o = 16; o > 0; o >>= 1) {
            pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
            cols += __shfl_xor_sync(0xffffffffu, cols, o);
        }
        if ((tid & 31) == 0) {
            stat_add(st, ST_PAIRS, pairs);
            stat_add(st, ST_COLS, cols);
        }
    }
}

// Hamming leaf stage: one CTA per work item; the group's query rows and each
// tile of up to 32 candidate rows in shared memory; thread t takes pairs
// t, t + LEAF_T, ... of the tile (query-major), integer distances.
template <bool EMIT>
__global__ void __launch_bounds__(LEAF_T) k_leaf_ham(
    TreeView tv, QParams qp, Items items, uint32_t *__restrict__ cand, int32_t *__restrict__ deg,
    const int64_t *__restrict__ row_ptr, int32_t *__restrict__ rowcur, int32_t *__restrict__ col,
    float *__restrict__ dist, unsigned long long *__restrict__ st, int32_t *__restrict__ err, CapOut co,
    const uint8_t *__restrict__ rowsel) {
    extern __shared__ uint4 hsm[];  // 32 query rows, then 32 candidate rows (wp / 4 uint4 each)
    __shared__ int cnt[32], cursor[32], sel[32];
    __shared__ int64_t rowb[32], rowe[32];
    __shared__ int tpos[32];
    __shared__ int64_t tcand[32];
    __shared__ int64_t s_ci;
    __shared__ int s_off, s_rows;
    __shared__ unsigned s_hit;
    const int tid = threadIdx.x;
    const int it = blockIdx.x;
    if (it >= *items.count) return;
    const int g = items.group[it];
    const int qb = tv.group_begin[g], qn = tv.group_count[g], qe = qb + qn;  // at most 32 queries
    const int64_t c0 = items.begin[it], c1 = items.end[it];
    const int k = qp.lev_k, nq = tv.wp >> 2;
    uint4 *Qs = hsm, *Ps = hsm + 32 * nq;
    unsigned long long pairs = 0;
    if (tid < 32) {
        cnt[tid] = 0;
        if (tid < qn) {
            const int o = tv.perm[qb + tid];
            cursor[tid] = o;
            sel[tid] = rowsel == nullptr || rowsel[o] != 0;
            if (EMIT) {
                rowb[tid] = row_ptr[o];
                rowe[tid] = row_ptr[o + 1];
            }
        }
    }
    for (int i = tid; i < qn * nq; i += LEAF_T)
        Qs[i] = reinterpret_cast<const uint4 *>(tv.bits)[(size_t)(qb + i / nq) * nq + i % nq];
    if (tid == 0) {
        s_ci = c0;
        s_off = 0;
        s_hit = 0u;
    }
    for (;;) {
        __syncthreads();
        if (tid < 32) fill_tile(tv, cand, c1, EMIT, &s_ci, &s_off, &s_rows, tpos, tcand);
        __syncthreads();
        const int npr = s_rows;
        const bool last = s_ci >= c1;
        for (int i = tid; i < npr * nq; i += LEAF_T)
            Ps[i] = reinterpret_cast<const uint4 *>(tv.bits)[(size_t)tpos[i / nq] * nq + i % nq];
        __syncthreads();
        if (npr > 0) {
            unsigned hit = 0u;
            for (int t = tid; t < qn * npr; t += LEAF_T) {
                const int q = t / npr, p = t - q * npr;
                const int qpos = qb + q, ppos = tpos[p];
                if (qpos == ppos && !qp.include_self) continue;
                if (qp.half && ppos < qb) continue;
                const bool mir = qp.half && ppos >= qe;
                if (EMIT && !sel[q] && !(mir && rowsel)) continue;
                if (!EMIT) ++pairs;
                const int d = ham_rows_smem(Qs + q * nq, Ps + p * nq, nq);
                if (d > k) continue;
                if (mir) mirror_int(tv, deg, row_ptr, rowcur, col, dist, err, co, rowsel, EMIT, qpos, ppos, d);
                if (!EMIT) {
                    hit |= 1u << p;
                    atomicAdd(&cnt[q], 1);
                    if (co.off) cap_put(co, cursor[q], tv.perm[ppos], (float)d);
                } else if (sel[q]) {
                    const int slot = atomicAdd(&rowcur[cursor[q]], 1);
                    const int64_t at = rowb[q] + slot;
                    if (at < rowe[q]) {
                        col[at] = tv.perm[ppos];
                        dist[at] = (float)d;
                    } else {
                        atomicOr(err, 4);
                    }
                }
            }
            if (!EMIT) {
                if (hit) atomicOr(&s_hit, hit);
                __syncthreads();
                if (tid < npr && ((s_hit >> tid) & 1u)) atomicOr(&cand[tcand[tid]], FLAG);
                __syncthreads();
                if (tid == 0) s_hit = 0u;
            }
        }
        if (last) break;
    }
    __syncthreads();
    if (!EMIT && tid < qn && cnt[tid]) atomicAdd(&deg[cursor[tid]], cnt[tid]);
    if (!EMIT) {
        for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
        if ((tid & 31) == 0) stat_add(st, ST_PAIRS, pairs);
    }
}

__global__ void k_alphabet(const uint8_t *__restrict__ s, int64_t nbytes, int32_t *__restrict__ present) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nbytes) present[s[i]] = 1;
}

// ------------------------------------------------------------- row sort

constexpr int SORT_MID = 4096;  // rows up to this length are sorted in one CTA

// Row classes by length: 0 <= 32, 1 <= 64, 2 <= 128, 3 <= 256, 4 <= 512 (one
// warp per row), 5 <= 1024, 6 <= 2048, 7 <= SORT_MID (one CTA per row), 8 longer.
constexpr int kSortClasses = 9;
__global__ void k_row_classes(const int64_t *__restrict__ row_ptr, int64_t n, int32_t *__restrict__ lists,
                              int32_t *__restrict__ counts) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t len = row_ptr[i + 1] - row_ptr[i];
    if (len <= 1) return;
    int cls = kSortClasses - 1;
    for (int c = 0; c < kSortClasses - 1; ++c)
        if (len <= (int64_t)32 << c) {
            cls = c;
            break;
        }
    // one atomic per class present in the warp (the lanes still here)
    const unsigned peers = __match_any_sync(__activemask(), cls);
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&counts[cls], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    lists[(int64_t)cls * n + base + __popc(peers & ((1u << lane) - 1))] = (int32_t)i;
}

// Bitonic network over the 32 lanes of a warp: (key, val) pairs ascending by
// key, lane i ending with the i-th smallest.
__device__ __forceinline__ void warp_sort32(int &key, float &val, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int ok = __shfl_xor_sync(0xffffffffu, key, j);
            const float ov = __shfl_xor_sync(0xffffffffu, val, j);
            const bool up = (lane & k) == 0, lower = (lane & j) == 0;
            if ((lower == up) ? (ok < key) : (ok > key)) {
                key = ok;
                val = ov;
            }
        }
    }
}

// A warp's 32 E entries in the blocked layout: lane l holds entries l E ..
// l E + E - 1 in registers.  In shared memory entry i sits at swz<E>(i), its
// low bits XORed with bits 5.., so that a warp's striped access (entries
// c 32 + lane, coalesced in global memory) and its blocked access (entries
// lane E + e) both hit 32 distinct banks.
template <int E>
__device__ __forceinline__ int swz(int i) {
    return i ^ ((i >> 5) & (E - 1));
}

// Bitonic sorting network over 32 E (key, val) pairs in the blocked layout,
// ascending by key.  Exchanges at distances below E pair entries of one lane
// (registers only); the others pair lane l with lane l ^ (distance / E) at
// the same register (one shuffle of key and of val).  The low distances,
// which the network visits most often, are thus the register ones.
template <int E>
__device__ __forceinline__ void warp_sort_blocked(int (&key)[E], float (&val)[E], int lane) {
    constexpr int N = 32 * E;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j < E) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if (e & j) continue;
                    const int f = e | j;
                    const bool up = ((lane * E + e) & k) == 0;
                    // selects, not a branch: lanes disagree on the swap
                    const int a = key[e], c = key[f];
                    const float va = val[e], vc = val[f];
                    const bool sw = (a > c) == up;
                    key[e] = sw ? c : a;
                    key[f] = sw ? a : c;
                    val[e] = sw ? vc : va;
                    val[f] = sw ? va : vc;
                }
            } else {
                const int lj = j / E;
                const bool keep_min = (((lane * E) & k) == 0) == ((lane & lj) == 0);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int ok = __shfl_xor_sync(0xffffffffu, key[e], lj);
                    const float ov = __shfl_xor_sync(0xffffffffu, val[e], lj);
                    const bool take = (ok < key[e]) == keep_min;  // equal keys: padding only
                    key[e] = take ? ok : key[e];
                    val[e] = take ? ov : val[e];
                }
            }
        }
    }
}

// One warp's blocked registers from / to its swizzled shared slice sh
// (entries at or past len read as INT_MAX keys).
template <int E>
__device__ __forceinline__ void take_blocked(const int *sh, const float *sv, int len, int lane, int (&key)[E],
                                             float (&val)[E]) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = lane * E + e;
        key[e] = i < len ? sh[swz<E>(i)] : INT_MAX;
        val[e] = i < len ? sv[swz<E>(i)] : 0.f;
    }
}
template <int E>
__device__ __forceinline__ void put_blocked(int *sh, float *sv, int lane, const int (&key)[E], const float (&val)[E]) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
        sh[swz<E>(lane * E + e)] = key[e];
        sv[swz<E>(lane * E + e)] = val[e];
    }
}

constexpr int SORT_WARPS = 8;  // warps per CTA of k_sort_warp

// Warp per row of 16 E + 1 .. 32 E entries (E = 2 .. 16): the row is read
// coalesced into the warp's shared slice (all its loads issued before the
// first store), taken into registers in the blocked layout, sorted by
// warp_sort_blocked and written back the same way.
template <int E>
__global__ void __launch_bounds__(32 * SORT_WARPS, 3) k_sort_warp(const int32_t *__restrict__ rows,
                                                               const int32_t *__restrict__ count,
                                                               const int64_t *__restrict__ row_ptr,
                                                               int32_t *__restrict__ col, float *__restrict__ dist) {
    __shared__ int s_key[SORT_WARPS][32 * E];
    __shared__ float s_val[SORT_WARPS][32 * E];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int *sk = s_key[wib];
    float *sv = s_val[wib];
    const int nrows = *count;
    for (int w = blockIdx.x * SORT_WARPS + wib; w < nrows; w += gridDim.x * SORT_WARPS) {
        const int r = rows[w];
        const int64_t b = row_ptr[r];
        const int len = (int)min(row_ptr[r + 1] - b, (int64_t)(32 * E));  // rows of this class fit
        int key[E];
        float val[E];
#pragma unroll
        for (int c = 0; c < E; ++c) {
            const int i = c * 32 + lane;
            key[c] = i < len ? col[b + i] : 0;
            val[c] = i < len ? dist[b + i] : 0.f;
        }
        __syncwarp();  // the previous row's write-back has read the slice
#pragma unroll
        for (int c = 0; c < E; ++c) {
            const int i = c * 32 + lane;
            if (i < len) {
                sk[swz<E>(i)] = key[c];
                sv[swz<E>(i)] = val[c];
            }
        }
        __syncwarp();
        take_blocked<E>(sk, sv, len, lane, key, val);
        warp_sort_blocked<E>(key, val, lane);
        __syncwarp();
        put_blocked<E>(sk, sv, lane, key, val);
        __syncwarp();
#pragma unroll
        for (int c = 0; c < E; ++c) {
            const int i = c * 32 + lane;
            if (i < len) {
                col[b + i] = sk[swz<E>(i)];
                dist[b + i] = sv[swz<E>(i)];
            }
        }
    }
}

// One merge round of a row's sorted runs of length run >= 512 (the last may
// be shorter or alone): the pair (A, B) = runs 2 m, 2 m + 1 goes to the
// outputs [2 m run, ...) of buffers (kn, vn).  Thread tid writes the SEG = 16
// outputs from 16 tid: one binary search along its diagonal finds how many of
// them come from A (merge path), then it merges them one by one.  Every
// buffer holds entry i at swz<16>(i) (runs start at multiples of 512, so a
// run's entry x sits at its start + swz<16>(x)): the warp's stores of its
// 16 consecutive outputs then hit 32 distinct banks.
template <int SEG>
__device__ __forceinline__ void merge_round(const int *__restrict__ kc, const float *__restrict__ vc,
                                            int *__restrict__ kn, float *__restrict__ vn, int len, int run,
                                            int tid) {
    const int o = tid * SEG;
    if (o >= len) return;
    const int s0 = o & ~(2 * run - 1);
    const int na = min(run, len - s0), nb = max(0, min(run, len - s0 - run));
    const int *A = kc + s0, *B = A + run;
    const float *Av = vc + s0, *Bv = Av + run;
    auto at = [](int i) { return swz<16>(i); };
    const int d = o - s0;  // outputs of the pair before this thread's
    int lo = max(0, d - nb), hi = min(d, na);
    while (lo < hi) {  // entries of A among the pair's d smallest
        const int mid = (lo + hi) >> 1;
        if (A[at(mid)] < B[at(d - 1 - mid)]) lo = mid + 1; else hi = mid;
    }
    // An exhausted run's head reads INT_MAX, above every column, so the other
    // run is taken; each step selects, no branch.
    int ia = lo, ib = d - lo;
    int ka = ia < na ? A[at(ia)] : INT_MAX, kb = ib < nb ? B[at(ib)] : INT_MAX;
    const int cnt = min(SEG, len - o);
#pragma unroll 4
    for (int t = 0; t < cnt; ++t) {
        const bool ta = ka < kb;
        kn[swz<16>(o + t)] = ta ? ka : kb;
        vn[swz<16>(o + t)] = ta ? Av[at(ia)] : Bv[at(ib)];
        ia += ta;
        ib += !ta;
        const int nx = ta ? ia : ib;
        const int nk = nx < (ta ? na : nb) ? (ta ? A : B)[at(nx)] : INT_MAX;
        ka = ta ? nk : ka;
        kb = ta ? kb : nk;
    }
}

// CTA of P = CAP / 16 threads per row of 513 .. CAP entries (16 CAP bytes of
// dynamic shared memory: keys and values, two buffers each).  Each warp sorts
// one 512-entry run in registers (warp_sort_blocked<16>) and leaves it in the
// swizzled layout (swz<16>, which every buffer keeps); then runs merge in
// pairs (merge_round) until one is left.
// The columns of a row are distinct, so the merged order is unique.
template <int CAP>
__global__ void __launch_bounds__(CAP / 16, 12288 / CAP) k_sort_merge(const int32_t *__restrict__ rows,
                                                                      const int32_t *__restrict__ count,
                                                                      const int64_t *__restrict__ row_ptr,
                                                                      int32_t *__restrict__ col,
                                                                      float *__restrict__ dist) {
    constexpr int P = CAP / 16, SEG = 16, RUN = 512;
    extern __shared__ int sort_smem[];
    int (*sk)[CAP] = reinterpret_cast<int (*)[CAP]>(sort_smem);
    float (*sv)[CAP] = reinterpret_cast<float (*)[CAP]>(sort_smem + 2 * CAP);
    const int tid = threadIdx.x, lane = tid & 31;
    const int nrows = *count;
    for (int w = blockIdx.x; w < nrows; w += gridDim.x) {
        const int r = rows[w];
        const int64_t b = row_ptr[r];
        const int len = (int)min(row_ptr[r + 1] - b, (int64_t)CAP);  // rows of this class fit
        {  // coalesced read: SEG loads a thread, then the stores
            int key[SEG];
            float val[SEG];
#pragma unroll
            for (int c = 0; c < SEG; ++c) {
                const int i = c * P + tid;
                key[c] = i < len ? col[b + i] : 0;
                val[c] = i < len ? dist[b + i] : 0.f;
            }
            __syncthreads();  // the previous row's write-back has read sk / sv
#pragma unroll
            for (int c = 0; c < SEG; ++c) {
                const int i = c * P + tid;
                if (i < len) {
                    sk[0][swz<16>(i)] = key[c];
                    sv[0][swz<16>(i)] = val[c];
                }
            }
        }
        __syncthreads();
        const int base = (tid >> 5) * RUN;
        if (base < len) {  // the warp's run, sorted in place
            int key[16];
            float val[16];
            take_blocked<16>(sk[0] + base, sv[0] + base, len - base, lane, key, val);
            warp_sort_blocked<16>(key, val, lane);
            __syncwarp();
            put_blocked<16>(sk[0] + base, sv[0] + base, lane, key, val);
        }
        __syncthreads();
        int cur = 0;
        for (int run = RUN; run < len; run <<= 1) {
            merge_round<SEG>(sk[cur], sv[cur], sk[cur ^ 1], sv[cur ^ 1], len, run, tid);
            __syncthreads();
            cur ^= 1;
        }
#pragma unroll
        for (int c = 0; c < SEG; ++c) {
            const int i = c * P + tid;
            if (i < len) {
                col[b + i] = sk[cur][swz<16>(i)];
                dist[b + i] = sv[cur][swz<16>(i)];
            }
        }
    }
}

// Rows of a graph with fewer than 2^20 columns sort one 32-bit key per
// entry, (column << PACK_BITS) | (the entry's position in the row, below
// SORT_MID): a row's keys are distinct and order as its columns do, so the
// network moves keys alone (min / max, no selects of values) and each value
// is fetched by its position once the keys are sorted.
constexpr int PACK_BITS = 12;
constexpr uint32_t PACK_POS = (1u << PACK_BITS) - 1;
constexpr int64_t PACK_MAX_COLS = int64_t(1) << (32 - PACK_BITS);  // packed when n (columns < n) is below
static_assert(SORT_MID <= (1 << PACK_BITS), "positions must fit the packed keys");

// Sorting network over 32 E packed keys in the blocked layout (padding:
// 0xffffffff, above every key): bitonic merges in the form whose first step
// of each merge compares entry i with its mirror i ^ (k - 1) in the block of
// k, the rest comparing i with i ^ j -- every comparator puts the minimum at
// the lower index, so a pair in one lane costs one min and one max.  Across
// lanes (distances of E and more) each lane keeps the minimum or the maximum
// of its key and its partner's, shuffled over.
template <int E>
__device__ __forceinline__ void warp_sort_keys(uint32_t (&key)[E], int lane) {
    constexpr int N = 32 * E;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
        if (k <= E) {  // the mirror step inside a lane
#pragma unroll
            for (int e = 0; e < E; ++e) {
                if (e & (k >> 1)) continue;
                const int f = e ^ (k - 1);
                const uint32_t lo = min(key[e], key[f]), hi = max(key[e], key[f]);
                key[e] = lo;
                key[f] = hi;
            }
        } else {  // mirror partner: lane ^ (k / E - 1), register E - 1 - e
            const int m = k / E - 1;
            const bool keep_min = (lane & (k / (2 * E))) == 0;
#pragma unroll
            for (int t = 0; t < E / 2; ++t) {
                const uint32_t o1 = __shfl_xor_sync(0xffffffffu, key[E - 1 - t], m);
                const uint32_t o2 = __shfl_xor_sync(0xffffffffu, key[t], m);
                key[t] = keep_min ? min(key[t], o1) : max(key[t], o1);
                key[E - 1 - t] = keep_min ? min(key[E - 1 - t], o2) : max(key[E - 1 - t], o2);
            }
        }
#pragma unroll
        for (int j = k >> 2; j > 0; j >>= 1) {
            if (j < E) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if (e & j) continue;
                    const int f = e | j;
                    const uint32_t lo = min(key[e], key[f]), hi = max(key[e], key[f]);
                    key[e] = lo;
                    key[f] = hi;
                }
            } else {
                const int lj = j / E;
                const bool keep_min = (lane & lj) == 0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const uint32_t o = __shfl_xor_sync(0xffffffffu, key[e], lj);
                    key[e] = keep_min ? min(key[e], o) : max(key[e], o);
                }
            }
        }
    }
}

// merge_round on packed keys alone.
template <int SEG>
__device__ __forceinline__ void merge_round_keys(const uint32_t *__restrict__ kc, uint32_t *__restrict__ kn,
                                                 int len, int run, int tid) {
    const int o = tid * SEG;
    if (o >= len) return;
    const int s0 = o & ~(2 * run - 1);
    const int na = min(run, len - s0), nb = max(0, min(run, len - s0 - run));
    const uint32_t *A = kc + s0, *B = A + run;
    auto at = [](int i) { return swz<16>(i); };
    const int d = o - s0;
    int lo = max(0, d - nb), hi = min(d, na);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (A[at(mid)] < B[at(d - 1 - mid)]) lo = mid + 1; else hi = mid;
    }
    int ia = lo, ib = d - lo;
    uint32_t ka = ia < na ? A[at(ia)] : 0xffffffffu, kb = ib < nb ? B[at(ib)] : 0xffffffffu;
    const int cnt = min(SEG, len - o);
#pragma unroll 4
    for (int t = 0; t < cnt; ++t) {
        const bool ta = ka < kb;
        kn[swz<16>(o + t)] = min(ka, kb);
        ia += ta;
        ib += !ta;
        const int nx = ta ? ia : ib;
        const uint32_t nk = nx < (ta ? na : nb) ? (ta ? A : B)[at(nx)] : 0xffffffffu;
        ka = ta ? nk : ka;
        kb = ta ? kb : nk;
    }
}

// k_sort_warp on packed keys: the values wait in shared memory in row order.
template <int E>
__global__ void __launch_bounds__(32 * SORT_WARPS, 4) k_sort_warp_packed(const int32_t *__restrict__ rows,
                                                                         const int32_t *__restrict__ count,
                                                                         const int64_t *__restrict__ row_ptr,
                                                                         int32_t *__restrict__ col,
                                                                         float *__restrict__ dist) {
    __shared__ uint32_t s_key[SORT_WARPS][32 * E];
    __shared__ float s_val[SORT_WARPS][32 * E];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t *sk = s_key[wib];
    float *sv = s_val[wib];
    const int nrows = *count;
    for (int w = blockIdx.x * SORT_WARPS + wib; w < nrows; w += gridDim.x * SORT_WARPS) {
        const int r = rows[w];
        const int64_t b = row_ptr[r];
        const int len = (int)min(row_ptr[r + 1] - b, (int64_t)(32 * E));  // rows of this class fit
        uint32_t key[E];
        float val[E];
#pragma unroll
        for (int c = 0; c < E; ++c) {
            const int i = c * 32 + lane;
            key[c] = i < len ? ((uint32_t)col[b + i] << PACK_BITS) | (uint32_t)i : 0u;
            val[c] = i < len ? dist[b + i] : 0.f;
        }
        __syncwarp();  // the previous row's write-back has read the slice
#pragma unroll
        for (int c = 0; c < E; ++c) {
            const int i = c * 32 + lane;
            if (i < len) {
                sk[swz<E>(i)] = key[c];
                sv[i] = val[c];
            }
        }
        __syncwarp();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = lane * E + e;
            key[e] = i < len ? sk[swz<E>(i)] : 0xffffffffu;
        }
        warp_sort_keys<E>(key, lane);
        __syncwarp();
#pragma unroll
        for (int e = 0; e < E; ++e) sk[swz<E>(lane * E + e)] = key[e];
        __syncwarp();
#pragma unroll
        for (int c = 0; c < E; ++c) {
            const int i = c * 32 + lane;
            if (i < len) {
                const uint32_t kk = sk[swz<E>(i)];
                col[b + i] = (int32_t)(kk >> PACK_BITS);
                dist[b + i] = sv[kk & PACK_POS];
            }
        }
    }
}

// k_sort_merge on packed keys (12 CAP bytes of dynamic shared memory: two
// key buffers and the values in row order).
template <int CAP>
__global__ void __launch_bounds__(CAP / 16, 16384 / CAP) k_sort_merge_packed(const int32_t *__restrict__ rows,
                                                                             const int32_t *__restrict__ count,
                                                                             const int64_t *__restrict__ row_ptr,
                                                                             int32_t *__restrict__ col,
                                                                             float *__restrict__ dist) {
    constexpr int P = CAP / 16, SEG = 16, RUN = 512;
    extern __shared__ uint32_t sort_smem_packed[];
    uint32_t (*sk)[CAP] = reinterpret_cast<uint32_t (*)[CAP]>(sort_smem_packed);
    float *sv = reinterpret_cast<float *>(sort_smem_packed + 2 * CAP);
    const int tid = threadIdx.x, lane = tid & 31;
    const int nrows = *count;
    for (int w = blockIdx.x; w < nrows; w += gridDim.x) {
        const int r = rows[w];
        const int64_t b = row_ptr[r];
        const int len = (int)min(row_ptr[r + 1] - b, (int64_t)CAP);  // rows of this class fit
        {
            uint32_t key[SEG];
            float val[SEG];
#pragma unroll
            for (int c = 0; c < SEG; ++c) {
                const int i = c * P + tid;
                key[c] = i < len ? ((uint32_t)col[b + i] << PACK_BITS) | (uint32_t)i : 0u;
                val[c] = i < len ? dist[b + i] : 0.f;
            }
            __syncthreads();  // the previous row's write-back has read sk / sv
#pragma unroll
            for (int c = 0; c < SEG; ++c) {
                const int i = c * P + tid;
                if (i < len) {
                    sk[0][swz<16>(i)] = key[c];
                    sv[i] = val[c];
                }
            }
        }
        __syncthreads();
        const int base = (tid >> 5) * RUN;
        if (base < len) {
            uint32_t key[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int i = lane * 16 + e;
                key[e] = base + i < len ? sk[0][base + swz<16>(i)] : 0xffffffffu;
            }
            warp_sort_keys<16>(key, lane);
            __syncwarp();
#pragma unroll
            for (int e = 0; e < 16; ++e) sk[0][base + swz<16>(lane * 16 + e)] = key[e];
        }
        __syncthreads();
        int cur = 0;
        for (int run = RUN; run < len; run <<= 1) {
            merge_round_keys<SEG>(sk[cur], sk[cur ^ 1], len, run, tid);
            __syncthreads();
            cur ^= 1;
        }
#pragma unroll
        for (int c = 0; c < SEG; ++c) {
            const int i = c * P + tid;
            if (i < len) {
                const uint32_t kk = sk[cur][swz<16>(i)];
                col[b + i] = (int32_t)(kk >> PACK_BITS);
                dist[b + i] = sv[kk & PACK_POS];
            }
        }
    }
}

// Warp per row, <= 32 entries: bitonic network across lanes.
__global__ void k_sort_small(const int32_t *__restrict__ rows, const int32_t *__restrict__ count,
                             const int64_t *__restrict__ row_ptr, int32_t *__restrict__ col,
                             float *__restrict__ dist) {
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= *count) return;
    int r = rows[w];
    int64_t b = row_ptr[r];
    int len = (int)(row_ptr[r + 1] - b);
    int key = lane < len ? col[b + lane] : INT_MAX;
    float val = lane < len ? dist[b + lane] : 0.f;
    warp_sort32(key, val, lane);
    if (lane < len) {
        col[b + lane] = key;
        dist[b + lane] = val;
    }
}
// Long rows: gather (row rank, col) keys and sort them globally.
__global__ void k_big_gather(const int32_t *__restrict__ rows, int nbig, const int64_t *__restrict__ row_ptr,
                             const int64_t *__restrict__ big_off, const int32_t *__restrict__ col,
                             uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    int w = blockIdx.x;
    if (w >= nbig) return;
    int r = rows[w];
    int64_t b = row_ptr[r], len = row_ptr[r + 1] - b, o = big_off[w];
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
        keys[o + i] = ((uint64_t)w << 32) | (uint32_t)col[b + i];
        vals[o + i] = (uint32_t)i;
    }
}
__global__ void k_big_apply(const int32_t *__restrict__ rows, int nbig, const int64_t *__restrict__ row_ptr,
                            const int64_t *__restrict__ big_off, const uint64_t *__restrict__ keys,
                            const uint32_t *__restrict__ vals, int32_t *__restrict__ col, float *__restrict__ dist,
                            float *__restrict__ tmpd) {
    int w = blockIdx.x;
    if (w >= nbig) return;
    int r = rows[w];
    int64_t b = row_ptr[r], len = row_ptr[r + 1] - b, o = big_off[w];
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) tmpd[o + i] = dist[b + vals[o + i]];
    __syncthreads();
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
        col[b + i] = (int32_t)(uint32_t)(keys[o + i] & 0xffffffffull);
        dist[b + i] = tmpd[o + i];
    }
}
__global__ void k_big_lengths(const int32_t *__restrict__ rows, int nbig, const int64_t *__restrict__ row_ptr,
                              int64_t *__restrict__ lens) {
    int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w < nbig) lens[w] = row_ptr[rows[w] + 1] - row_ptr[rows[w]];
}

inline unsigned grid_for(int64_t n, int t) { return (unsigned)ceil_div(n > 0 ? n : 1, t); }

// Row-sort kernels: dynamic shared memory allowed and CTAs resident per SM,
// found once (before any capture) and kept.  [0]: (key, value) kernels, [1]:
// packed keys.
struct SortGrids {
    int warp_per_sm[2][5] = {};   // k_sort_warp<2 .. 16> for classes 1 .. 4
    int merge_per_sm[2][8] = {};  // k_sort_merge for classes 5 .. 7
};
const SortGrids &sort_grids() {
    static const SortGrids g = [] {
        SortGrids r;
        auto warp = [&](int pk, int c, auto kern) {
            CT_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r.warp_per_sm[pk][c], kern,
                                                                        32 * SORT_WARPS, 0));
            r.warp_per_sm[pk][c] = std::max(r.warp_per_sm[pk][c], 1);
        };
        auto merge = [&](int pk, int c, auto kern, int cap) {
            const int smem = (pk ? 12 : 16) * cap;
            if (smem > 48 * 1024)
                CT_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            CT_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r.merge_per_sm[pk][c], kern, cap / 16, smem));
            r.merge_per_sm[pk][c] = std::max(r.merge_per_sm[pk][c], 1);
        };
        warp(0, 1, k_sort_warp<2>);
        warp(0, 2, k_sort_warp<4>);
        warp(0, 3, k_sort_warp<8>);
        warp(0, 4, k_sort_warp<16>);
        merge(0, 5, k_sort_merge<1024>, 1024);
        merge(0, 6, k_sort_merge<2048>, 2048);
        merge(0, 7, k_sort_merge<SORT_MID>, SORT_MID);
        warp(1, 1, k_sort_warp_packed<2>);
        warp(1, 2, k_sort_warp_packed<4>);
        warp(1, 3, k_sort_warp_packed<8>);
        warp(1, 4, k_sort_warp_packed<16>);
        merge(1, 5, k_sort_merge_packed<1024>, 1024);
        merge(1, 6, k_sort_merge_packed<2048>, 2048);
        merge(1, 7, k_sort_merge_packed<SORT_MID>, SORT_MID);
        return r;
    }();
    return g;
}

// The sorts of the rows in classes 0 .. kSortClasses - 2 (class lists of
// stride n, their counts on the device) of a graph whose columns are below
// ncols.  hc: the same counts on the host -- classes without rows are skipped
// and grids sized to the rows; null: every class launched on a full grid (the
// kernels loop over the rows the device counted).
void launch_class_sorts(const int32_t *lists, const int32_t *counts, const int32_t *hc, int64_t n, int64_t ncols,
                        const int64_t *row_ptr, int32_t *col, float *dist, cudaStream_t s) {
    const SortGrids &g = sort_grids();
    const int pk = ncols < PACK_MAX_COLS ? 1 : 0;
    if (!hc || hc[0]) {
        k_sort_small<<<grid_for((hc ? hc[0] : n) * 32, 256), 256, 0, s>>>(lists, counts, row_ptr, col, dist);
        CT_COUNT_LAUNCH();
    }
    auto launch = [&](int c, auto kern, int threads, int smem, int per_sm, int rows_per_cta) {
        if (hc && !hc[c]) return;
        const int64_t full = (int64_t)num_sms() * per_sm;
        const int64_t blocks = hc ? std::min<int64_t>(ceil_div((int64_t)hc[c], rows_per_cta), full) : full;
        kern<<<(unsigned)blocks, threads, smem, s>>>(lists + (int64_t)c * n, counts + c, row_ptr, col, dist);
        CT_COUNT_LAUNCH();
    };
    constexpr int WT = 32 * SORT_WARPS;
    if (pk) {
        launch(1, k_sort_warp_packed<2>, WT, 0, g.warp_per_sm[1][1], SORT_WARPS);
        launch(2, k_sort_warp_packed<4>, WT, 0, g.warp_per_sm[1][2], SORT_WARPS);
        launch(3, k_sort_warp_packed<8>, WT, 0, g.warp_per_sm[1][3], SORT_WARPS);
        launch(4, k_sort_warp_packed<16>, WT, 0, g.warp_per_sm[1][4], SORT_WARPS);
        launch(5, k_sort_merge_packed<1024>, 1024 / 16, 12 * 1024, g.merge_per_sm[1][5], 1);
        launch(6, k_sort_merge_packed<2048>, 2048 / 16, 12 * 2048, g.merge_per_sm[1][6], 1);
        launch(7, k_sort_merge_packed<SORT_MID>, SORT_MID / 16, 12 * SORT_MID, g.merge_per_sm[1][7], 1);
    } else {
        launch(1, k_sort_warp<2>, WT, 0, g.warp_per_sm[0][1], SORT_WARPS);
        launch(2, k_sort_warp<4>, WT, 0, g.warp_per_sm[0][2], SORT_WARPS);
        launch(3, k_sort_warp<8>, WT, 0, g.warp_per_sm[0][3], SORT_WARPS);
        launch(4, k_sort_warp<16>, WT, 0, g.warp_per_sm[0][4], SORT_WARPS);
        launch(5, k_sort_merge<1024>, 1024 / 16, 16 * 1024, g.merge_per_sm[0][5], 1);
        launch(6, k_sort_merge<2048>, 2048 / 16, 16 * 2048, g.merge_per_sm[0][6], 1);
        launch(7, k_sort_merge<SORT_MID>, SORT_MID / 16, 16 * SORT_MID, g.merge_per_sm[0][7], 1);
    }
}

}  // namespace

void sort_rows(const int64_t *row_ptr, int64_t n, int64_t ncols, int32_t *col, float *dist, int64_t nnz,
               cudaStream_t s) {
    if (n <= 0 || nnz <= 0) return;
    DBuf<int32_t> lists(kSortClasses * n, s), counts(kSortClasses, s);
    CT_CHECK_CUDA(cudaMemsetAsync(counts.p, 0, kSortClasses * sizeof(int32_t), s));
    k_row_classes<<<grid_for(n, 256), 256, 0, s>>>(row_ptr, n, lists.p, counts.p);
    CT_COUNT_LAUNCH();
    int32_t hc[kSortClasses];
    to_host(hc, counts.p, kSortClasses, s);
    launch_class_sorts(lists.p, counts.p, hc, n, ncols, row_ptr, col, dist, s);
    constexpr int BIG = kSortClasses - 1;
    if (hc[BIG]) {
        int nb = hc[BIG];
        const int32_t *big = lists.p + BIG * n;
        DBuf<int64_t> lens(nb, s), off(nb, s), tot(1, s);
        k_big_lengths<<<grid_for(nb, 256), 256, 0, s>>>(big, nb, row_ptr, lens.p);
        CT_COUNT_LAUNCH();
        exclusive_scan_i64(lens.p, off.p, nb, tot.p, s);
        int64_t total = 0;
        to_host(&total, tot.p, 1, s);
        DBuf<uint64_t> k1(total, s), k2(total, s);
        DBuf<uint32_t> v1(total, s), v2(total, s);
        DBuf<float> td(total, s);
        k_big_gather<<<nb, 256, 0, s>>>(big, nb, row_ptr, off.p, col, k1.p, v1.p);
        CT_COUNT_LAUNCH();
        int bits = 32;
        while ((int64_t(1) << (bits - 32)) < nb) ++bits;
        radix_sort_pairs64(k1.p, v1.p, k2.p, v2.p, total, bits, s);
        k_big_apply<<<nb, 256, 0, s>>>(big, nb, row_ptr, off.p, k1.p, v1.p, col, dist, td.p);
        CT_COUNT_LAUNCH();
    }
    CT_LAUNCH_CHECK();
}

QParams make_qparams(const ct_tree *t, double eps, int include_self) {
    QParams q;
    q.eps64 = eps;
    q.eps2_64 = eps * eps;
    q.include_self = include_self;
    float ef = (float)eps;
    if ((double)ef < eps) ef = nextafterf(ef, INFINITY);
    q.eps_up = ef;
    if (t->metric == CT_LEVENSHTEIN_U8 || t->metric == CT_HAMMING_B1) {
        double fl = floor(eps);
        q.lev_k = fl > 1e9 ? 1000000000 : (int)fl;
        return q;
    }
    const double e2 = q.eps2_64;
    if (eps == 0.0) {
        q.mode = 1;
    } else if (e2 >= 0x1p115) {
        q.mode = 3;
    } else if (e2 < 0x1p-100 || e2 > 0x1p100) {
        q.mode = 2;
    } else {
        q.mode = 0;
        double lo = eps * (1.0 - 1e-3), hi = eps * (1.0 + 1e-3);
        double lo2 = lo * lo, hi2 = hi * hi;
        float l = (float)lo2, h = (float)hi2;
        if ((double)l > lo2) l = nextafterf(l, 0.0f);
        if ((double)h < hi2) h = nextafterf(h, INFINITY);
        q.lo2 = l;
        q.hi2 = h;
        // error bound of the canonical fp32 sum: one rounding per FMA of a
        // 16-float chunk (8), the chunk sum, one per chunk of the running
        // total, the rounded differences; doubled
        const double m = 2.0 * ((double)(t->dp / 16) + 16.0) * 0x1p-24;
        const double cl = e2 * (1.0 - m), ch = e2 * (1.0 + m);
        float a = (float)cl, b = (float)ch;
        if ((double)a > cl) a = nextafterf(a, 0.0f);
        if ((double)b < ch) b = nextafterf(b, INFINITY);
        q.c_lo = a;
        q.c_hi = b;
    }
    return q;
}

// Traversal launch shape: L2 uses blocks of TRAV_WARPS warps, edit distance
// one warp per block; both are capped at a resident-sized grid.
struct TravLaunch {
    int blocks, warps;
};
TravLaunch trav_launch_config(bool l2, int64_t G) {
    TravLaunch tl;
    if (l2) {
        tl.blocks = (int)std::min<int64_t>(ceil_div(G, TRAV_WARPS), (int64_t)num_sms() * 8);
        tl.blocks = std::max(tl.blocks, 1);
        tl.warps = tl.blocks * TRAV_WARPS;
    } else {
        // a warp per block, as many as an SM holds: the later rounds' stored
        // ranges can outnumber the groups
        tl.blocks = (int)std::max<int64_t>(1, (int64_t)num_sms() * 32);
        tl.warps = tl.blocks;
    }
    return tl;
}

// First pool size: 256 candidate blocks per point (or 512 per group), at most
// a quarter of the free device memory, plus one chunk per warp.
int64_t pool_capacity_guess(int64_t n, int64_t G, const TravLaunch &tl) {
    int64_t want = std::max<int64_t>(256 * n, G * 512);
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
        int64_t lim = (int64_t)(fr / 4 / sizeof(uint32_t));
        if (lim > 0 && want > lim) want = lim;
    } else {
        cudaGetLastError();
    }
    return want + (int64_t)(tl.warps + 1) * POOL_CHUNK;
}

// Clears the pool counters and launches the traversal over `order` (global
// group ids; allocates nothing).  L2: a round over the groups with a step
// limit, then TRAV_ROUNDS rounds over the ranges the previous round stored
// (`spill`: two buffers of spill_cap items and two counters; the last round
// has no limit), so that no single long walk sets the time.  Each warp's
// pool chunk carries over between rounds (`cursors`: one per warp of the
// grid).  Hamming and edit distance: a single cloud, the same rounds (one
// warp per block; edit-distance walks stop sooner: their steps cost more).
void launch_traversal(const Views &V, int64_t G, int max_dp, int max_len, bool l2, const int32_t *order,
                      const Pool &P, int2 *stacks, int cap, const TravLaunch &tl, unsigned long long *st,
                      int32_t *err, int32_t *next_group, int4 *const spill[2], int32_t *spill_cnt, int spill_cap,
                      longlong2 *cursors, cudaStream_t s, int32_t *gvisit = nullptr) {
    // P.next .. P.overflow are the four 64-bit words of one counter block
    CT_CHECK_CUDA(cudaMemsetAsync(next_group, 0, sizeof(int32_t), s));
    CT_CHECK_CUDA(cudaMemsetAsync(P.next, 0, 4 * sizeof(unsigned long long), s));
    if (gvisit && G > 0) CT_CHECK_CUDA(cudaMemsetAsync(gvisit, 0, (size_t)G * sizeof(int32_t), s));
    if (G == 0) return;
    if (l2) {
        const size_t tsm = (size_t)TRAV_WARPS * max_dp * sizeof(float);
        if (tsm > 48 * 1024)
            CT_CHECK_CUDA(cudaFuncSetAttribute(k_traverse_l2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm));
        CT_CHECK_CUDA(cudaMemsetAsync(spill_cnt, 0, 2 * sizeof(int32_t), s));
        for (int r = 0; r <= TRAV_ROUNDS; ++r) {
            const int4 *in = r ? spill[(r - 1) & 1] : nullptr;
            const int32_t *in_cnt = r ? spill_cnt + ((r - 1) & 1) : nullptr;
            Spill out{nullptr, spill_cnt + (r & 1), spill_cap, INT_MAX};
            if (r < TRAV_ROUNDS) {
                out.items = spill[r & 1];
                out.limit = r ? TRAV_LIMIT : TRAV_LIMIT0;
            }
            if (r) {
                CT_CHECK_CUDA(cudaMemsetAsync(next_group, 0, sizeof(int32_t), s));
                CT_CHECK_CUDA(cudaMemsetAsync(spill_cnt + (r & 1), 0, sizeof(int32_t), s));
            }
            k_traverse_l2<<<tl.blocks, TRAV_WARPS * 32, tsm, s>>>(V, order, (int)G, in, in_cnt, spill_cap, out, P,
                                                                   cursors, stacks, cap, st, err, next_group,
                                                                   gvisit, max_dp >> 2);
            CT_COUNT_LAUNCH();
            CT_LAUNCH_CHECK();
        }
    } else {  // Hamming or edit distance: one cloud, the same rounds (a warp per block)
        TreeView tv = V.tv[0];
        tv.group_order = order;
        const bool ham = tv.wp != 0;
        CT_CHECK_CUDA(cudaMemsetAsync(spill_cnt, 0, 2 * sizeof(int32_t), s));
        for (int r = 0; r <= TRAV_ROUNDS; ++r) {
            const int4 *in = r ? spill[(r - 1) & 1] : nullptr;
            const int32_t *in_cnt = r ? spill_cnt + ((r - 1) & 1) : nullptr;
            Spill out{nullptr, spill_cnt + (r & 1), spill_cap, INT_MAX};
            if (r < TRAV_ROUNDS) {
                out.items = spill[r & 1];
                out.limit = ham ? (r ? TRAV_LIMIT : TRAV_LIMIT0) : (r ? TRAV_LIMIT_LEV : TRAV_LIMIT0_LEV);
            }
            if (r) {
                CT_CHECK_CUDA(cudaMemsetAsync(next_group, 0, sizeof(int32_t), s));
                CT_CHECK_CUDA(cudaMemsetAsync(spill_cnt + (r & 1), 0, sizeof(int32_t), s));
            }
            if (ham) {
                k_traverse_ham<<<tl.blocks, 32, 0, s>>>(tv, V.qp[0], in, in_cnt, spill_cap, out, P, cursors, stacks,
                                                        cap, st, err, next_group, gvisit);
            } else {
                switch (lev_words_for(max_len)) {
#define CT_TL(WW) \
    case WW: k_traverse_lev<WW><<<tl.blocks, 32, 0, s>>>(tv, V.qp[0], in, in_cnt, spill_cap, out, P, cursors, stacks, cap, st, err, next_group, gvisit); break;
                    CT_TL(1) CT_TL(2) CT_TL(4) CT_TL(8) CT_TL(16)
#undef CT_TL
                }
            }
            CT_COUNT_LAUNCH();
            CT_LAUNCH_CHECK();
        }
    }
}

// Leaf kernel and item length per cloud.  precision 0: FP32 tiles; 1: tensor-
// core tiles where the rows allow (L2, at most 128 floats); 2: the autotuned
// choice of the cloud's row-length class (a default until tuned).
std::mutex g_tune_mu;
LeafChoice g_tune[kDpClasses] = {{-1, kItem}, {-1, kItem}, {-1, kItem}, {-1, kItem}, {-1, kItem}, {-1, kItem}};

int dp_class(int dp) { return dp <= 4 ? 0 : dp <= 16 ? 1 : dp <= 32 ? 2 : dp <= 64 ? 3 : dp <= 128 ? 4 : 5; }

LeafChoice tuned_choice(int dp) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    LeafChoice e = g_tune[dp_class(dp)];
    if (e.use_tc < 0) e.use_tc = dp >= 32;
    return e;
}
void tune_set(int cls, LeafChoice c) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[cls] = c;
}
void tune_reset() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &e : g_tune) e = LeafChoice{-1, kItem};
}
LeafChoice leaf_choice(const ct_tree *t, int precision) {
    if (t->metric != CT_L2_F32 || t->dp > 128 || precision == 0) return LeafChoice{0, kItem};
    if (precision == 1) return LeafChoice{1, kItemTC};
    LeafChoice c = tuned_choice(t->dp);
    if (c.item_len < 32 || c.item_len > kItem) c.item_len = kItem;
    return c;
}

// Global walk order of several clouds: groups by decreasing radius relative
// to their cloud's eps.
__global__ void k_radius_keys(int G, const float *__restrict__ group_radius, float inv_eps, int gbase,
                              uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    keys[gbase + g] = ~__float_as_uint(fmaxf(group_radius[g] * inv_eps, 0.f));
    vals[gbase + g] = (uint32_t)(gbase + g);
}

// Relative row_ptr of one cloud from the concatenated one.
__global__ void k_rel_rows(int64_t n1, const int64_t *__restrict__ grow, int64_t *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n1) out[i] = grow[i] - grow[0];
}

// TMA map of n fp16 rows of kp halves (kp a multiple of 64): boxes of 64
// halves x 1 row (gathered four rows at a time), 128-byte swizzle.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
void encode_rows_f16(CUtensorMap *m, const void *rows, int64_t n, int kp) {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        CT_CHECK_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !p) CT_FAIL(CT_ECUDA, "cuTensorMapEncodeTiled is not available");
        fn = (EncodeTiledFn)p;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
    const cuuint32_t box[2] = {64, 1}, estr[2] = {1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(rows), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) CT_FAIL(CT_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
}

void query_multi(int C, const ct_tree *const *trees, const QParams *qps, cudaStream_t s, QueryOut *outs,
                 int precision, const ct_predictor *pred, Probe *probe) {
    if (C < 1 || C > kMaxClouds) CT_FAIL(CT_EINVAL, "between 1 and %d clouds per batch", kMaxClouds);
    const bool l2 = trees[0]->metric == CT_L2_F32;
    const bool ham = trees[0]->metric == CT_HAMMING_B1;
    if (C > 1 && !l2) CT_FAIL(CT_EINVAL, "edit-distance and Hamming trees are queried one at a time");
    // the clouds' groups and rows, concatenated
    Views V;
    std::memset(&V, 0, sizeof(V));
    V.nc = C;
    int max_dp = 4, max_depth = 0, max_len = 0, min_len = kItemTC;
    bool any_tc = false, any_fp = false, any_half = false;
    for (int c = 0; c < C; ++c) {
        const ct_tree *tc = trees[c];
        if ((tc->metric == CT_L2_F32) != l2) CT_FAIL(CT_EINVAL, "a batch mixes metrics");
        V.tv[c] = view_of(tc);
        V.qp[c] = qps[c];
        any_half |= qps[c].half != 0;
        const LeafChoice ch = leaf_choice(tc, precision);
        V.use_tc[c] = (uint8_t)ch.use_tc;
        V.item_len[c] = (int16_t)ch.item_len;
        any_tc |= ch.use_tc != 0;
        any_fp |= ch.use_tc == 0;
        min_len = std::min(min_len, ch.item_len);
        V.gbase[c + 1] = V.gbase[c] + tc->n_groups;
        V.rbase[c + 1] = V.rbase[c] + tc->n;
        max_dp = std::max(max_dp, tc->dp);
        max_depth = std::max(max_depth, tc->depth);
        max_len = std::max(max_len, tc->max_len);
    }
    if (V.rbase[C] >= 0x7fffffffLL) CT_FAIL(CT_EOVERFLOW, "a batch above 2^31 points");
    // fp16 rows of the clouds that take the tensor-core filter
    std::vector<DBuf<uint4>> h16s;
    std::vector<DBuf<float>> f16s;
    if (any_tc) {
        ProfScope ps("rows_f16", s);
        DBuf<float> partial;
        for (int c = 0; c < C; ++c) {
            if (!V.use_tc[c]) continue;
            const ct_tree *tc = trees[c];
            const int64_t nc = tc->n;
            if (nc == 0) continue;  // no work items
            const int dp = tc->dp, kp = 64 * ((dp + 63) / 64);  // rows of 64-half K blocks
            h16s.emplace_back((size_t)nc * (kp / 8), s);
            f16s.emplace_back((size_t)dp + 4 + nc, s);  // means (dp: a multiple of 4), {s, s eps_up}, norms
            float *mean = f16s.back().p, *scal = mean + dp, *nrm = scal + 4;
            partial.grow((size_t)H16_MB * dp);
            k_col_partial<<<H16_MB, 128, 0, s>>>(tc->pts, nc, dp, partial.p);
            CT_COUNT_LAUNCH();
            CT_LAUNCH_CHECK();
            k_col_final<<<1, 128, 0, s>>>(partial.p, dp, nc, tc->radius, V.qp[c].eps_up, mean, scal);
            CT_COUNT_LAUNCH();
            CT_LAUNCH_CHECK();
            k_to_h16<<<grid_for(nc * 16, 256), 256, 0, s>>>(tc->pts, nc, dp, kp, mean, scal, h16s.back().p, nrm);
            CT_COUNT_LAUNCH();
            CT_LAUNCH_CHECK();
            encode_rows_f16(&V.tmap[c], h16s.back().p, nc, kp);
            V.h16[c] = h16s.back().p;
            V.n16[c] = nrm;
            V.s16[c] = scal;
        }
    }
    const int64_t n = V.rbase[C];
    const int G = V.gbase[C];
    const ct_tree *t = trees[0];  // edit distance: the only cloud
    DBuf<unsigned long long> st(ST_N, s);
    CT_CHECK_CUDA(cudaMemsetAsync(st.p, 0, ST_N * sizeof(unsigned long long), s));
    int32_t *err = reinterpret_cast<int32_t *>(st.p + ST_ERR);
    QueryOut all;  // the concatenated CSR of all clouds
    struct AllGuard {  // releases its arrays unless they were handed to the caller
        QueryOut &q;
        cudaStream_t s;
        bool armed = true;
        ~AllGuard() {
            if (!armed) return;
            dfree(q.row_ptr, s);
            dfree(q.col, s);
            dfree(q.dist, s);
        }
    } all_guard{all, s};

    // learned form: row capacities and the traversal order from the predictor
    LearnedPlan lp;
    if (pred && !probe && n > 0) {
        ProfScope ps("predict", s);
        learned_plan(pred, C, trees, qps, V.rbase, V.gbase, s, lp);
    }
    // walk order: predicted walk length, else decreasing radius (relative to eps)
    DBuf<uint32_t> okeys, ovals;
    const int32_t *order = lp.group_order.p;
    if (!order && C == 1) order = t->group_order;
    if (!order && G > 0) {
        okeys = DBuf<uint32_t>(G, s);
        ovals = DBuf<uint32_t>(G, s);
        for (int c = 0; c < C; ++c) {
            const int Gc = trees[c]->n_groups;
            if (!Gc) continue;
            k_radius_keys<<<grid_for(Gc, 256), 256, 0, s>>>(Gc, trees[c]->group_radius,
                                                            (float)(1.0 / std::max(qps[c].eps64, 1e-30)),
                                                            V.gbase[c], okeys.p, ovals.p);
            CT_COUNT_LAUNCH();
        }
        DBuf<uint32_t> tk(G, s), tvv(G, s);
        radix_sort_pairs(okeys.p, ovals.p, tk.p, tvv.p, G, 32, s);
        order = reinterpret_cast<const int32_t *>(ovals.p);
    }
    int32_t *gvisit = probe ? probe->gvisit : nullptr;

    const int W = l2 || ham ? 1 : lev_words_for(t->max_len);
    // 1. traversal: one pass into the candidate pool (rerun once if it overflows)
    const int cap = 32 * (max_depth + 2);
    TravLaunch tl = trav_launch_config(l2, G);
    DBuf<int2> stacks((size_t)tl.warps * cap, s);
    DBuf<unsigned long long> ctr(4, s);
    DBuf<int32_t> next_group(1, s);
    // ranges of step-limited walks: two buffers and their counters
    const int spill_cap = (int)std::min<int64_t>(std::max<int64_t>(4 * G, 1 << 16), 1 << 20);
    DBuf<int4> spill_a(spill_cap, s), spill_b(spill_cap, s);
    DBuf<int32_t> spill_cnt(2, s);
    int4 *const spills[2] = {spill_a.p, spill_b.p};
    DBuf<longlong2> cursors(tl.warps, s);
    int64_t pool_cap = pool_capacity_guess(n, G, tl);
    DBuf<uint32_t> pool;
    DBuf<int32_t> seg_group, seg_count;
    DBuf<int64_t> seg_begin;
    unsigned long long hc[4] = {0, 0, 0, 0};
    Pool P{};
    for (int attempt = 0;; ++attempt) {
        // a segment per walk (groups, stored ranges) and per chunk a walk crosses
        const int64_t seg_cap = G + (int64_t)TRAV_ROUNDS * spill_cap + pool_cap / POOL_CHUNK + tl.warps + 16;
        pool = DBuf<uint32_t>(pool_cap, s);
        seg_group = DBuf<int32_t>(seg_cap, s);
        seg_count = DBuf<int32_t>(seg_cap, s);
        seg_begin = DBuf<int64_t>(seg_cap, s);
        P = Pool{pool.p, pool_cap, ctr.p, seg_group.p, seg_count.p, seg_begin.p,
                 reinterpret_cast<int32_t *>(ctr.p + 1), seg_cap, ctr.p + 2, reinterpret_cast<int32_t *>(ctr.p + 3)};
        {
            ProfScope ps("traverse", s);
            launch_traversal(V, G, max_dp, max_len, l2, order, P, stacks.p, cap, tl, st.p, err, next_group.p, spills,
                             spill_cnt.p, spill_cap, cursors.p, s, gvisit);
        }
        to_host(hc, ctr.p, 4, s);
        if (!(uint32_t)hc[3]) break;
        if (attempt >= 1) CT_FAIL(CT_ECUDA, "candidate pool overflowed twice");
        pool_cap = (int64_t)hc[2] + 2LL * tl.warps * POOL_CHUNK + POOL_CHUNK;
        CT_CHECK_CUDA(cudaMemsetAsync(st.p, 0, ST_N * sizeof(unsigned long long), s));
    }
    stacks.reset();
    const int64_t n_cand = (int64_t)hc[2];
    int nseg = (int)(uint32_t)hc[1];
    // each group's candidates in one range (segments become one per group)
    DBuf<uint32_t> gcand(n_cand ? n_cand : 1, s);
    DBuf<int32_t> gseg_group, gseg_count;
    DBuf<int64_t> gseg_begin;
    if (nseg && G) {
        gseg_group = DBuf<int32_t>(G, s);
        gseg_count = DBuf<int32_t>(G, s);
        gseg_begin = DBuf<int64_t>(G + 1, s);
        DBuf<int32_t> gfill(G, s);
        CT_CHECK_CUDA(cudaMemsetAsync(gseg_count.p, 0, G * sizeof(int32_t), s));
        CT_CHECK_CUDA(cudaMemsetAsync(gfill.p, 0, G * sizeof(int32_t), s));
        k_group_cand_counts<<<grid_for(nseg, 256), 256, 0, s>>>(nseg, seg_group.p, seg_count.p, gseg_count.p);
        CT_COUNT_LAUNCH();
        exclusive_scan_i32_to_i64(gseg_count.p, gseg_begin.p, G, gseg_begin.p + G, s);
        if (any_half)
            k_group_cand_copy_half<<<grid_for((int64_t)nseg * 32, 256), 256, 0, s>>>(
                V, nseg, nullptr, 0, seg_group.p, seg_begin.p, seg_count.p, gseg_begin.p, gfill.p, pool.p, gcand.p,
                INT64_MAX, err);
        else
            k_group_cand_copy<<<grid_for((int64_t)nseg * 32, 256), 256, 0, s>>>(nseg, seg_group.p, seg_begin.p,
                                                                              seg_count.p, gseg_begin.p, gfill.p,
                                                                              pool.p, gcand.p);
        CT_COUNT_LAUNCH();
        k_iota<<<grid_for(G, 256), 256, 0, s>>>(G, gseg_group.p);
        CT_COUNT_LAUNCH();
        if (any_half)  // the groups' kept counts
            CT_CHECK_CUDA(cudaMemcpyAsync(gseg_count.p, gfill.p, G * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        CT_LAUNCH_CHECK();
        nseg = G;
    }
    pool.reset();
    seg_group.reset();
    seg_count.reset();
    seg_begin.reset();
    DBuf<uint32_t> emask(l2 ? (n_cand ? n_cand : 1) : 0, s);
    // work items: the groups' candidate ranges in slices of the clouds' item lengths
    const int64_t max_items = nseg + n_cand / min_len + 1;
    DBuf<int32_t> icnt(nseg + 1, s), igroup(max_items, s), nitems(1, s);
    DBuf<int64_t> ioff(nseg + 1, s), ibeg(max_items, s), iend(max_items, s);
    Items items{igroup.p, ibeg.p, iend.p, nitems.p};
    CT_CHECK_CUDA(cudaMemsetAsync(nitems.p, 0, sizeof(int32_t), s));
    if (nseg) {
        k_item_counts<<<grid_for(nseg, 256), 256, 0, s>>>(V, nseg, gseg_group.p, gseg_count.p, icnt.p);
        CT_COUNT_LAUNCH();
        exclusive_scan_i32_to_i64(icnt.p, ioff.p, nseg, ioff.p + nseg, s);
        k_item_fill<<<grid_for(nseg, 256), 256, 0, s>>>(V, nseg, gseg_group.p, gseg_begin.p, gseg_count.p, ioff.p,
                                                       igroup.p, ibeg.p, iend.p, nitems.p);
        CT_COUNT_LAUNCH();
        CT_LAUNCH_CHECK();
    }
    DBuf<int32_t> rowcur(n + 1, s);
    uint32_t *cand_p = gcand.p;

    // alphabet of the strings (edit distance)
    DBuf<uint8_t> amap;
    int A = 0, qchunk = 32;
    if (!l2 && !ham) {
        DBuf<int32_t> present(256, s);
        CT_CHECK_CUDA(cudaMemsetAsync(present.p, 0, 256 * sizeof(int32_t), s));
        if (t->sbytes) {
            k_alphabet<<<grid_for(t->sbytes, 256), 256, 0, s>>>(t->sdata, t->sbytes, present.p);
            CT_COUNT_LAUNCH();
        }
        int32_t hp[256];
        to_host(hp, present.p, 256, s);
        uint8_t hm[256];
        for (int c = 0; c < 256; ++c) hm[c] = 0;
        int a = 1;  // slot 0: bytes absent from the data (never matched)
        for (int c = 0; c < 256; ++c)
            if (hp[c]) hm[c] = (uint8_t)std::min(a++, 255);
        A = std::min(a, 256);
        if (a > 256) {  // every byte value occurs: identity map
            for (int c = 0; c < 256; ++c) hm[c] = (uint8_t)c;
            A = 256;
        }
        amap = DBuf<uint8_t>(256, s);
        CT_CHECK_CUDA(cudaMemcpyAsync(amap.p, hm, 256, cudaMemcpyHostToDevice, s));
        CT_CHECK_CUDA(cudaStreamSynchronize(s));
        size_t per_q = (size_t)A * W * sizeof(uint64_t);
        qchunk = (int)std::max<size_t>(1, std::min<size_t>(32, (96 * 1024) / per_q));
    }
    size_t lsm = l2 || ham ? 0 : (size_t)qchunk * A * W * sizeof(uint64_t);

    // one-pass emit: capacity region and overflow arena
    const bool capmode = pred && !probe && lp.one_pass;
    CapOut co{};
    DBuf<int32_t> c_fill, c_col, o_row, o_slot, o_col;
    DBuf<float> c_dist, o_dist;
    DBuf<unsigned long long> o_n;
    DBuf<uint8_t> lost;
    if (capmode) {
        const int64_t ct = lp.cap_total > 0 ? lp.cap_total : 1, oc = lp.arena > 0 ? lp.arena : 1;
        c_fill = DBuf<int32_t>(n + 1, s);
        c_col = DBuf<int32_t>(ct, s);
        c_dist = DBuf<float>(ct, s);
        o_row = DBuf<int32_t>(oc, s);
        o_slot = DBuf<int32_t>(oc, s);
        o_col = DBuf<int32_t>(oc, s);
        o_dist = DBuf<float>(oc, s);
        o_n = DBuf<unsigned long long>(3, s);
        lost = DBuf<uint8_t>(n + 1, s);
        CT_CHECK_CUDA(cudaMemsetAsync(c_fill.p, 0, (n + 1) * sizeof(int32_t), s));
        CT_CHECK_CUDA(cudaMemsetAsync(o_n.p, 0, 3 * sizeof(unsigned long long), s));
        CT_CHECK_CUDA(cudaMemsetAsync(lost.p, 0, n + 1, s));
        co = CapOut{lp.cap_off.p, c_fill.p, c_col.p, c_dist.p, o_row.p, o_slot.p, o_col.p, o_dist.p,
                    o_n.p, lp.arena > 0 ? lp.arena : 0, lost.p};
    }

    // 2. count pass
    DBuf<int32_t> deg(n + 1, s);
    CT_CHECK_CUDA(cudaMemsetAsync(deg.p, 0, (n + 1) * sizeof(int32_t), s));
    auto leaf = [&](bool emit, int64_t *row_ptr, int32_t *col, float *dist, const uint8_t *rowsel,
                    const Items &items) {
        if (G == 0 || nseg == 0) return;
        const CapOut cw = emit ? CapOut{} : co;
        if (l2) {
            leaf_l2_prepare();
            if (emit)
                k_leaf_l2<true><<<(unsigned)max_items, LEAF_T, kLeafSmem, s>>>(V, items, cand_p, emask.p, deg.p, row_ptr, rowcur.p, col, dist, st.p, err, cw, rowsel);
            else
                k_leaf_l2<false><<<(unsigned)max_items, LEAF_T, kLeafSmem, s>>>(V, items, cand_p, emask.p, deg.p, row_ptr, rowcur.p, col, dist, st.p, err, cw, rowsel);
        } else if (ham) {
            const size_t hsm = (size_t)64 * (t->wp / 4) * sizeof(uint4);  // 32 query rows + 32 candidate rows
            if (emit)
                k_leaf_ham<true><<<(unsigned)max_items, LEAF_T, hsm, s>>>(V.tv[0], V.qp[0], items, cand_p, deg.p, row_ptr, rowcur.p, col, dist, st.p, err, cw, rowsel);
            else
                k_leaf_ham<false><<<(unsigned)max_items, LEAF_T, hsm, s>>>(V.tv[0], V.qp[0], items, cand_p, deg.p, row_ptr, rowcur.p, col, dist, st.p, err, cw, rowsel);
        } else {
            switch (W) {
#define CT_LL(WW)                                                                                                      \
    case WW:                                                                                                           \
        if (lsm > 48 * 1024) {                                                                                         \
            CT_CHECK_CUDA(cudaFuncSetAttribute(k_leaf_lev<true, WW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm)); \
            CT_CHECK_CUDA(cudaFuncSetAttribute(k_leaf_lev<false, WW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm)); \
        }                                                                                                              \
        if (emit) k_leaf_lev<true, WW><<<(unsigned)max_items, LEAF_T, lsm, s>>>(V.tv[0], V.qp[0], amap.p, A, qchunk, items, cand_p, deg.p, row_ptr, rowcur.p, col, dist, st.p, err, cw, rowsel); \
        else k_leaf_lev<false, WW><<<(unsigned)max_items, LEAF_T, lsm, s>>>(V.tv[0], V.qp[0], amap.p, A, qchunk, items, cand_p, deg.p, row_ptr, rowcur.p, col, dist, st.p, err, cw, rowsel);    \
        break;
                CT_LL(1) CT_LL(2) CT_LL(4) CT_LL(8) CT_LL(16)
#undef CT_LL
            }
        }
        CT_COUNT_LAUNCH();
        CT_LAUNCH_CHECK();
    };
    // each cloud's count kernel: tensor-core tiles (L2 rows of at most 128
    // floats) or FP32 tiles -- the same output; a mixed batch splits its work
    // items between the two launches
    auto count_tc = [&](const Items &its) {
        ProfScope ps("leaf_count_tc", s);
        static bool tc_ready = false;
        if (!tc_ready) {
            CT_CHECK_CUDA(cudaFuncSetAttribute(k_leaf_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
            tc_ready = true;
        }
        if (G && nseg) {
            k_leaf_tc<<<(unsigned)max_items, TC_T, kTcSmem, s>>>(V, its, cand_p, emask.p, deg.p, st.p, err, co);
            CT_COUNT_LAUNCH();
            CT_LAUNCH_CHECK();
        }
    };
    if (!l2 || !any_tc) {
        ProfScope ps("leaf_count", s);
        leaf(false, nullptr, nullptr, nullptr, nullptr, items);
    } else if (!any_fp) {
        count_tc(items);
    } else {
        DBuf<int32_t> tg(max_items, s), fg(max_items, s), cnt2(2, s);
        DBuf<int64_t> tb(max_items, s), te(max_items, s), fb(max_items, s), fe(max_items, s);
        CT_CHECK_CUDA(cudaMemsetAsync(cnt2.p, 0, 2 * sizeof(int32_t), s));
        if (nseg) {
            k_item_split<<<grid_for(max_items, 256), 256, 0, s>>>(V, items, tg.p, tb.p, te.p, cnt2.p, fg.p, fb.p, fe.p,
                                                                   cnt2.p + 1);
            CT_COUNT_LAUNCH();
            CT_LAUNCH_CHECK();
        }
        count_tc(Items{tg.p, tb.p, te.p, cnt2.p});
        ProfScope ps("leaf_count", s);
        leaf(false, nullptr, nullptr, nullptr, nullptr, Items{fg.p, fb.p, fe.p, cnt2.p + 1});
    }

    auto finish_stats = [&]() {
        unsigned long long hs[ST_N];
        to_host(hs, st.p, ST_N, s);
        prof_flush();
        if (hs[ST_ERR] & 32)
            CT_FAIL(CT_ETIMEOUT, "a bounded wait of the tensor-core leaf kernel gave up (code %llu)", hs[ST_ERR]);
        if (hs[ST_ERR]) CT_FAIL(CT_ECUDA, "internal consistency check failed in the query (code %llu)", hs[ST_ERR]);
        all.stats.traversal_evals = (int64_t)hs[ST_TRAV];
        all.stats.leaf_pairs = (int64_t)hs[ST_PAIRS];
        all.stats.guard_fp64 = (int64_t)hs[ST_GUARD];
        all.stats.recheck_fp32 = (int64_t)hs[ST_RECHECK];
        all.stats.emit_pairs = (int64_t)hs[ST_EMIT];
        all.stats.leaf_rows = (int64_t)hs[ST_ROWS];
        all.stats.guard_band = (int64_t)hs[ST_BAND];
        all.stats.lev_columns = (int64_t)hs[ST_COLS];
        all.stats.candidates = n_cand;
    };

    if (probe) {  // labels for fitting the predictor
        if (n && probe->deg) CT_CHECK_CUDA(cudaMemcpyAsync(probe->deg, deg.p, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        finish_stats();
        return;
    }

    // 3. scan -> row_ptr, then emit
    int64_t *row_ptr = (int64_t *)dmalloc((size_t)(n + 1) * sizeof(int64_t), s);
    all.row_ptr = row_ptr;
    exclusive_scan_i32_to_i64(deg.p, row_ptr, n + 1, nullptr, s);
    int64_t nnz = 0;
    to_host(&nnz, row_ptr + n, 1, s);
    all.nnz = nnz;
    all.col = (int32_t *)dmalloc((size_t)(nnz ? nnz : 1) * sizeof(int32_t), s);
    all.dist = (float *)dmalloc((size_t)(nnz ? nnz : 1) * sizeof(float), s);
    if (capmode) {
        // one-pass emit: move the capacity region and the arena into the CSR;
        // rows that lost entries are emitted again, exactly
        unsigned long long hv[3] = {0, 0, 0};
        {
            ProfScope ps("compact", s);
            if (n) {
                k_cap_rows<<<grid_for(n, 256), 256, 0, s>>>(n, row_ptr, lp.cap_off.p, c_fill.p, lost.p, o_n.p + 1, err);
                CT_COUNT_LAUNCH();
                k_compact<<<grid_for(n * 32, 256), 256, 0, s>>>(n, row_ptr, lp.cap_off.p, lost.p, c_col.p, c_dist.p,
                                                                all.col, all.dist);
                CT_COUNT_LAUNCH();
                CT_LAUNCH_CHECK();
            }
            to_host(hv, o_n.p, 3, s);
            const int64_t used = std::min<int64_t>((int64_t)hv[0], co.ovf_cap);
            if (used > 0) {
                k_ovf_scatter<<<grid_for(used, 256), 256, 0, s>>>(used, o_row.p, o_slot.p, o_col.p, o_dist.p, lost.p,
                                                                  row_ptr, all.col, all.dist, err);
                CT_COUNT_LAUNCH();
                CT_LAUNCH_CHECK();
            }
        }
        all.stats.overflow_rows = (int64_t)hv[1];
        all.stats.reemit_rows = (int64_t)hv[2];
        c_col.reset();
        c_dist.reset();
        if (hv[2]) {
            ProfScope ps("reemit", s);
            CT_CHECK_CUDA(cudaMemsetAsync(rowcur.p, 0, (n + 1) * sizeof(int32_t), s));
            leaf(true, row_ptr, all.col, all.dist, lost.p, items);
            k_check_rows_sel<<<grid_for(n, 256), 256, 0, s>>>(n, row_ptr, rowcur.p, lost.p, err);
            CT_COUNT_LAUNCH();
        }
    } else if (nnz) {
        ProfScope ps("leaf_emit", s);
        CT_CHECK_CUDA(cudaMemsetAsync(rowcur.p, 0, (n + 1) * sizeof(int32_t), s));
        leaf(true, row_ptr, all.col, all.dist, nullptr, items);
        k_check_rows<<<grid_for(n, 256), 256, 0, s>>>(n, row_ptr, rowcur.p, err);
        CT_COUNT_LAUNCH();
    }
    {
        ProfScope ps("row_sort", s);
        int64_t ncols = 0;  // columns index points of their own cloud
        for (int c = 0; c < C; ++c) ncols = std::max<int64_t>(ncols, trees[c]->n);
        sort_rows(row_ptr, n, ncols, all.col, all.dist, nnz, s);
    }
    finish_stats();
    if (C == 1) {
        outs[0] = all;
        all_guard.armed = false;
        return;
    }
    // several clouds: CSRs that view one shared allocation each of row
    // offsets (relative to the cloud), columns and distances
    std::vector<int64_t> hb(C + 1);
    for (int c = 0; c <= C; ++c) to_host_async(&hb[c], row_ptr + V.rbase[c], 1, s);
    CT_CHECK_CUDA(cudaStreamSynchronize(s));
    auto blocks = std::make_shared<SharedBlocks>(s);
    blocks->p[0] = dmalloc((size_t)(n + C) * sizeof(int64_t), s);
    int64_t *rel = (int64_t *)blocks->p[0];
    int32_t *colp = all.col;
    float *distp = all.dist;
    blocks->p[1] = colp;
    blocks->p[2] = distp;
    all.col = nullptr;  // the blocks own them now
    all.dist = nullptr;
    for (int c = 0; c < C; ++c) {
        const int64_t nc1 = trees[c]->n + 1, o = V.rbase[c] + c;
        k_rel_rows<<<grid_for(nc1, 256), 256, 0, s>>>(nc1, row_ptr + V.rbase[c], rel + o);
        CT_COUNT_LAUNCH();
        QueryOut &q = outs[c];
        q.row_ptr = rel + o;
        q.col = colp + hb[c];
        q.dist = distp + hb[c];
        q.nnz = hb[c + 1] - hb[c];
        q.stats = all.stats;
        q.shared = blocks;
    }
    CT_LAUNCH_CHECK();
    all.row_ptr = nullptr;
    all_guard.armed = false;
    dfree(row_ptr, s);  // stream ordered: after the relative copies
}

void query_plain(const ct_tree *t, const QParams &qp, cudaStream_t s, QueryOut &out) {
    query_multi(1, &t, &qp, s, &out, 0, nullptr, nullptr);
}

void query_tc(const ct_tree *t, const QParams &qp, cudaStream_t s, QueryOut &out) {
    query_multi(1, &t, &qp, s, &out, 1, nullptr, nullptr);
}

void set_guard_rows(int32_t *rows, unsigned long long *count, int64_t cap) {
    long long c = rows ? (long long)cap : 0;
    int32_t *r = rows;
    unsigned long long *n = rows ? count : nullptr;
    CT_CHECK_CUDA(cudaDeviceSynchronize());
    CT_CHECK_CUDA(cudaMemcpyToSymbol(g_guard_rows, &r, sizeof(r)));
    CT_CHECK_CUDA(cudaMemcpyToSymbol(g_guard_n, &n, sizeof(n)));
    CT_CHECK_CUDA(cudaMemcpyToSymbol(g_guard_cap, &c, sizeof(c)));
}

// ---------------------------------------------------------------- plans
//
// A batch of L2 clouds queried again and again over the same trees (a served
// set of point clouds): every buffer is sized once, from a sizing query plus
// a margin, so that a run enqueues the whole query -- walk, candidate ranges,
// count pass, scan, emit, row sort -- without reading anything back to the
// host.  A run can therefore be captured in a CUDA graph and replayed.  The
// leaf stage is one persistent launch over every cloud's (cloud, group) work
// items: each CTA first produces the items of a chunk of groups into a device
// work queue (in the walk order, which the predictor sets when one is given),
// then consumes queue slots; a slot is waited for, with a bounded number of
// polls, until its producer has published it.  Sizes that outgrow the plan, a
// wait that gives up, and rows too long for the in-place sorts are reported
// by the run's status word.

namespace {

constexpr int32_t Q_ERR_OVERFLOW = 128;  // a run outgrew one of the plan's capacities
constexpr int32_t Q_ERR_TIMEOUT = 256;   // a queue wait gave up

__device__ __forceinline__ int ld_acquire_i32(const int32_t *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_i32(int32_t *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// The leaf stage's work queue.  Counters: claim (next group chunk to
// produce), tail (slots reserved), head (next slot to consume), published
// (groups whose items are all written).
struct Queue {
    int32_t *claim, *tail, *head, *published;
    int32_t *ready;  // per slot: 1 once its item is written
    int32_t *group;
    int64_t *begin, *end;
    const int32_t *order;   // production order (global group ids)
    const int32_t *gcount;  // candidate blocks per group
    const int64_t *gbegin;  // first candidate of each group
    const int32_t *ctl;     // ctl[0] != 0: producers publish nothing (a test); ctl[1]: polls before a wait gives up
    int64_t cand_cap;       // candidate ranges beyond it were not copied
    int G, cap, produce;
};

// Producer: chunks of LEAF_T groups, one thread per group; a group's items
// are its candidate range cut at its cloud's item length.
__device__ __forceinline__ void queue_produce(const Views &V, const Queue &Q, int32_t *err) {
    __shared__ int s_c0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_c0 = atomicAdd(Q.claim, LEAF_T);
        __syncthreads();
        const int c0 = s_c0;
        if (c0 >= Q.G) break;
        if (Q.ctl[0]) continue;  // withheld: the chunk is taken and nothing is published
        const int i = c0 + threadIdx.x;
        if (i < Q.G) {
            const int gg = Q.order[i];
            const int cnt = Q.gcount[gg];
            const int len = V.item_len[cloud_of_group(V, gg)];
            int k = (cnt + len - 1) / len;
            if (Q.gbegin[gg] + cnt > Q.cand_cap) {  // its range was not copied: no items
                atomicOr(err, Q_ERR_OVERFLOW);
                k = 0;
            }
            if (k > 0) {
                const int base = atomicAdd(Q.tail, k);
                const int64_t b0 = Q.gbegin[gg];
                for (int j = 0; j < k; ++j) {
                    const int slot = base + j;
                    if (slot >= Q.cap) {  // slots past the plan's capacity are never consumed
                        atomicOr(err, Q_ERR_OVERFLOW);
                        break;
                    }
                    Q.group[slot] = gg;
                    Q.begin[slot] = b0 + (int64_t)j * len;
                    Q.end[slot] = min(b0 + (int64_t)(j + 1) * len, b0 + cnt);
                    __threadfence();
                    st_release_i32(Q.ready + slot, 1);
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(Q.published, min(LEAF_T, Q.G - c0));
        }
    }
}

// Consumer: the next slot, once published; -1 when the queue is exhausted
// (or a wait gave up: Q_ERR_TIMEOUT).
__device__ __forceinline__ int queue_next(const Queue &Q, int32_t *err) {
    __shared__ int s_it;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int slot = atomicAdd(Q.head, 1);
        int it = -1;
        if (slot < Q.cap) {
            const unsigned limit = (unsigned)Q.ctl[1];
            for (unsigned poll = 0;; ++poll) {
                if (ld_acquire_i32(Q.ready + slot)) {
                    it = slot;
                    break;
                }
                if (ld_acquire_i32(Q.published) >= Q.G && slot >= ld_acquire_i32(Q.tail)) break;
                if (poll >= limit) {
                    atomicOr(err, Q_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(poll < 64 ? 64 : 1024);
            }
            __threadfence();
        }
        s_it = it;
    }
    __syncthreads();
    return s_it;
}

// The FP32 tiles as one persistent launch over the queue (count pass:
// produce, then consume; emit pass: consume the complete queue again).
template <bool EMIT>
__global__ void __launch_bounds__(LEAF_T, 3) k_leaf_l2_queue(
    const __grid_constant__ Views V, Queue Q, const uint32_t *__restrict__ cand, uint32_t *__restrict__ emask,
    int32_t *__restrict__ deg, const int64_t *__restrict__ row_ptr, int32_t *__restrict__ rowcur,
    int32_t *__restrict__ col, float *__restrict__ dist, unsigned long long *__restrict__ st,
    int32_t *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LeafShared &S = *reinterpret_cast<LeafShared *>(smem_raw);
    if (Q.produce) queue_produce(V, Q, err);
    const Items items{Q.group, Q.begin, Q.end, Q.tail};
    for (;;) {
        const int it = queue_next(Q, err);
        if (it < 0) break;
        leaf_l2_item<EMIT>(V, items, it, cand, emask, deg, row_ptr, rowcur, col, dist, st, err, CapOut{}, nullptr,
                           S);
    }
}

// Candidate ranges per group from the walk's segments (segment count read on
// the device; destinations checked against the plan's capacity).
__global__ void k_plan_cand_counts(const int32_t *__restrict__ nseg_dev, int64_t seg_cap,
                                   const int32_t *__restrict__ seg_group, const int32_t *__restrict__ seg_count,
                                   int32_t *__restrict__ gcnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nseg = min((int64_t)*nseg_dev, seg_cap);
    if (i < nseg && seg_count[i] > 0) atomicAdd(gcnt + seg_group[i], seg_count[i]);
}
__global__ void k_plan_cand_copy(const int32_t *__restrict__ nseg_dev, int64_t seg_cap,
                                 const int32_t *__restrict__ seg_group, const int64_t *__restrict__ seg_begin,
                                 const int32_t *__restrict__ seg_count, const int64_t *__restrict__ goff,
                                 int32_t *__restrict__ gfill, const uint32_t *__restrict__ pool,
                                 uint32_t *__restrict__ gcand, int64_t cand_cap, int32_t *__restrict__ err) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t nseg = min((int64_t)*nseg_dev, seg_cap);
    if (i >= nseg) return;
    const int g = seg_group[i], c = seg_count[i];
    int64_t base = 0;
    if (lane == 0) base = goff[g] + atomicAdd(gfill + g, c);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base + c > cand_cap) {
        if (lane == 0) atomicOr(err, Q_ERR_OVERFLOW);
        return;
    }
    const uint32_t *src = pool + seg_begin[i];
    for (int k = lane; k < c; k += 32) gcand[base + k] = src[k];
}
// The walk's own overflow flag, and the candidate total against the plan.
__global__ void k_plan_walk_check(const int32_t *__restrict__ pool_ovf, const int64_t *__restrict__ total,
                                  int64_t cand_cap, int32_t *__restrict__ err) {
    if (*pool_ovf || *total > cand_cap) atomicOr(err, Q_ERR_OVERFLOW);
}
// Edges above the plan's capacity: flagged, and every row emptied so that the
// emit pass writes nothing.
__global__ void k_plan_nnz_check(const int64_t *__restrict__ row_ptr, int64_t n, int64_t nnz_cap,
                                 int32_t *__restrict__ flag, int32_t *__restrict__ err) {
    if (row_ptr[n] > nnz_cap) {
        *flag = 1;
        atomicOr(err, Q_ERR_OVERFLOW);
    } else {
        *flag = 0;
    }
}
__global__ void k_plan_empty_rows(int64_t n1, const int32_t *__restrict__ flag, int64_t *__restrict__ row_ptr) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n1 && *flag) row_ptr[i] = 0;
}
// Rows longer than the in-place sorts take: their count against the plan,
// their lengths (zero past the count), then (after a scan) their entries
// against the plan's capacity.
__global__ void k_plan_big_lengths(const int32_t *__restrict__ rows, const int32_t *__restrict__ nbig_dev,
                                   int cap_rows, const int64_t *__restrict__ row_ptr, int64_t *__restrict__ lens,
                                   int32_t *__restrict__ err) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const int nbig = *nbig_dev;
    if (w == 0 && nbig > cap_rows) atomicOr(err, Q_ERR_OVERFLOW);
    if (w < cap_rows) lens[w] = w < nbig ? row_ptr[rows[w] + 1] - row_ptr[rows[w]] : 0;
}
__global__ void k_plan_big_check(const int64_t *__restrict__ total, int64_t big_cap, int32_t *__restrict__ err,
                                 int32_t *__restrict__ skip) {
    *skip = *total > big_cap;
    if (*skip) atomicOr(err, Q_ERR_OVERFLOW);
}
// Keys (rank of the row in the list, column) of the long rows, in the
// plan's buffer (prefilled with keys that sort last).
__global__ void k_plan_big_gather(const int32_t *__restrict__ rows, const int32_t *__restrict__ nbig_dev, int cap_rows,
                                  const int32_t *__restrict__ skip, const int64_t *__restrict__ row_ptr,
                                  const int64_t *__restrict__ big_off, const int32_t *__restrict__ col,
                                  uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    const int w = blockIdx.x;
    if (w >= min(*nbig_dev, cap_rows) || *skip) return;
    const int r = rows[w];
    const int64_t b = row_ptr[r], len = row_ptr[r + 1] - b, o = big_off[w];
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
        keys[o + i] = ((uint64_t)w << 32) | (uint32_t)col[b + i];
        vals[o + i] = (uint32_t)i;
    }
}
__global__ void k_plan_big_apply(const int32_t *__restrict__ rows, const int32_t *__restrict__ nbig_dev, int cap_rows,
                                 const int32_t *__restrict__ skip, const int64_t *__restrict__ row_ptr,
                                 const int64_t *__restrict__ big_off, const uint64_t *__restrict__ keys,
                                 const uint32_t *__restrict__ vals, int32_t *__restrict__ col,
                                 float *__restrict__ dist, float *__restrict__ tmpd) {
    const int w = blockIdx.x;
    if (w >= min(*nbig_dev, cap_rows) || *skip) return;
    const int r = rows[w];
    const int64_t b = row_ptr[r], len = row_ptr[r + 1] - b, o = big_off[w];
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) tmpd[o + i] = dist[b + vals[o + i]];
    __syncthreads();
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
        col[b + i] = (int32_t)(uint32_t)(keys[o + i] & 0xffffffffull);
        dist[b + i] = tmpd[o + i];
    }
}

}  // namespace

struct PlanImpl {
    int C = 0;
    std::vector<const ct_tree *> trees;
    Views V;
    int64_t n = 0, max_cols = 0;  // rows of all clouds; points of the largest cloud
    int G = 0;
    int max_dp = 4, cap_stack = 0, spill_cap = 0, leaf_grid = 1;
    TravLaunch tl{1, 1};
    int64_t pool_cap = 0, seg_cap = 0, cand_cap = 0, item_cap = 0, nnz_cap = 0;
    bool any_half = false;  // some cloud is queried in the upper-triangle form
    int big_rows = 0;       // rows above the in-place sorts' length the plan sorts by radix
    int64_t big_cap = 0;    // their entries
    cudaStream_t s0 = 0;
    DBuf<int32_t> order;
    DBuf<unsigned long long> st, ctr;
    DBuf<int32_t> next_group, spill_cnt, ctl, qctr, ready, igroup, gcount, gfill, deg, rowcur, empty_flag;
    DBuf<int2> stacks;
    DBuf<int4> spill_a, spill_b;
    DBuf<longlong2> cursors;
    DBuf<uint32_t> pool, gcand, emask;
    DBuf<int32_t> seg_group, seg_count, col, sort_lists, sort_counts;
    DBuf<int64_t> seg_begin, gbegin, ibeg, iend, sums, row_ptr, rel;
    DBuf<float> dist, big_tmpd;
    DBuf<int64_t> big_lens, big_off;
    DBuf<uint64_t> big_k1, big_k2;
    DBuf<uint32_t> big_v1, big_v2;
    DBuf<int32_t> big_skip;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~PlanImpl() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
};

namespace {
// One run of a plan: every launch on `s`, nothing read back, nothing allocated.
void plan_enqueue(PlanImpl &p, cudaStream_t s) {
    const Views &V = p.V;
    const int64_t n = p.n;
    const int G = p.G;
    unsigned long long *st = p.st.p;
    int32_t *err = reinterpret_cast<int32_t *>(st + ST_ERR);
    CT_CHECK_CUDA(cudaMemsetAsync(st, 0, ST_N * sizeof(unsigned long long), s));
    if (G == 0) {  // empty clouds only
        CT_CHECK_CUDA(cudaMemsetAsync(p.row_ptr.p, 0, (size_t)(n + 1) * sizeof(int64_t), s));
        CT_CHECK_CUDA(cudaMemsetAsync(p.rel.p, 0, (size_t)(n + p.C) * sizeof(int64_t), s));
        return;
    }
    Pool P{p.pool.p, p.pool_cap, p.ctr.p, p.seg_group.p, p.seg_count.p, p.seg_begin.p,
           reinterpret_cast<int32_t *>(p.ctr.p + 1), p.seg_cap, p.ctr.p + 2, reinterpret_cast<int32_t *>(p.ctr.p + 3)};
    int4 *const spills[2] = {p.spill_a.p, p.spill_b.p};
    // 1. the walk over every cloud's groups
    launch_traversal(V, G, p.max_dp, 0, true, p.order.p, P, p.stacks.p, p.cap_stack, p.tl, st, err, p.next_group.p,
                     spills, p.spill_cnt.p, p.spill_cap, p.cursors.p, s);
    k_plan_walk_check<<<1, 1, 0, s>>>(P.overflow, reinterpret_cast<const int64_t *>(P.total), p.cand_cap, err);
    CT_COUNT_LAUNCH();
    // 2. each group's candidates in one range
    CT_CHECK_CUDA(cudaMemsetAsync(p.gcount.p, 0, (size_t)G * sizeof(int32_t), s));
    CT_CHECK_CUDA(cudaMemsetAsync(p.gfill.p, 0, (size_t)G * sizeof(int32_t), s));
    k_plan_cand_counts<<<grid_for(p.seg_cap, 256), 256, 0, s>>>(P.nseg, p.seg_cap, P.seg_group, P.seg_count,
                                                              p.gcount.p);
    CT_COUNT_LAUNCH();
    exclusive_scan_i32_to_i64_into(p.gcount.p, p.gbegin.p, G, p.gbegin.p + G, p.sums.p, s);
    if (p.any_half) {
        k_group_cand_copy_half<<<grid_for(p.seg_cap * 32, 256), 256, 0, s>>>(
            V, 0, P.nseg, p.seg_cap, P.seg_group, P.seg_begin, P.seg_count, p.gbegin.p, p.gfill.p, P.data, p.gcand.p,
            p.cand_cap, err);
        CT_COUNT_LAUNCH();
        // the groups' kept counts (ranges past the plan's capacity are never read: the producer skips them)
        CT_CHECK_CUDA(cudaMemcpyAsync(p.gcount.p, p.gfill.p, (size_t)G * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    } else {
        k_plan_cand_copy<<<grid_for(p.seg_cap * 32, 256), 256, 0, s>>>(P.nseg, p.seg_cap, P.seg_group, P.seg_begin,
                                                                      P.seg_count, p.gbegin.p, p.gfill.p, P.data,
                                                                      p.gcand.p, p.cand_cap, err);
        CT_COUNT_LAUNCH();
    }
    // 3. count pass: one persistent launch producing and consuming the work queue
    CT_CHECK_CUDA(cudaMemsetAsync(p.qctr.p, 0, 4 * sizeof(int32_t), s));
    CT_CHECK_CUDA(cudaMemsetAsync(p.ready.p, 0, (size_t)p.item_cap * sizeof(int32_t), s));
    CT_CHECK_CUDA(cudaMemsetAsync(p.deg.p, 0, (size_t)(n + 1) * sizeof(int32_t), s));
    Queue Q{p.qctr.p, p.qctr.p + 1, p.qctr.p + 2, p.qctr.p + 3, p.ready.p, p.igroup.p, p.ibeg.p, p.iend.p,
            p.order.p, p.gcount.p, p.gbegin.p, p.ctl.p, p.cand_cap, G, (int)p.item_cap, 1};
    k_leaf_l2_queue<false><<<p.leaf_grid, LEAF_T, kLeafSmem, s>>>(V, Q, p.gcand.p, p.emask.p, p.deg.p, nullptr,
                                                                  nullptr, nullptr, nullptr, st, err);
    CT_COUNT_LAUNCH();
    // 4. scan; a run above the plan's edge capacity empties every row
    exclusive_scan_i32_to_i64_into(p.deg.p, p.row_ptr.p, n + 1, nullptr, p.sums.p, s);
    k_plan_nnz_check<<<1, 1, 0, s>>>(p.row_ptr.p, n, p.nnz_cap, p.empty_flag.p, err);
    CT_COUNT_LAUNCH();
    k_plan_empty_rows<<<grid_for(n + 1, 256), 256, 0, s>>>(n + 1, p.empty_flag.p, p.row_ptr.p);
    CT_COUNT_LAUNCH();
    // 5. emit pass over the complete queue
    CT_CHECK_CUDA(cudaMemsetAsync(p.qctr.p + 2, 0, sizeof(int32_t), s));
    CT_CHECK_CUDA(cudaMemsetAsync(p.rowcur.p, 0, (size_t)(n + 1) * sizeof(int32_t), s));
    Q.produce = 0;
    k_leaf_l2_queue<true><<<p.leaf_grid, LEAF_T, kLeafSmem, s>>>(V, Q, p.gcand.p, p.emask.p, p.deg.p, p.row_ptr.p,
                                                                 p.rowcur.p, p.col.p, p.dist.p, st, err);
    CT_COUNT_LAUNCH();
    k_check_rows<<<grid_for(n, 256), 256, 0, s>>>(n, p.row_ptr.p, p.rowcur.p, err);
    CT_COUNT_LAUNCH();
    // 6. rows sorted in place (rows above the in-place sorts' length are reported)
    CT_CHECK_CUDA(cudaMemsetAsync(p.sort_counts.p, 0, kSortClasses * sizeof(int32_t), s));
    k_row_classes<<<grid_for(n, 256), 256, 0, s>>>(p.row_ptr.p, n, p.sort_lists.p, p.sort_counts.p);
    CT_COUNT_LAUNCH();
    launch_class_sorts(p.sort_lists.p, p.sort_counts.p, nullptr, n, p.max_cols, p.row_ptr.p, p.col.p, p.dist.p, s);
    {  // longer rows: one radix sort of (row rank, column) keys over the plan's capacity
        const int32_t *big = p.sort_lists.p + (int64_t)(kSortClasses - 1) * n;
        const int32_t *nbig = p.sort_counts.p + (kSortClasses - 1);
        k_plan_big_lengths<<<grid_for(p.big_rows, 256), 256, 0, s>>>(big, nbig, p.big_rows, p.row_ptr.p,
                                                                     p.big_lens.p, err);
        CT_COUNT_LAUNCH();
        exclusive_scan_i64(p.big_lens.p, p.big_off.p, p.big_rows, p.big_off.p + p.big_rows, s);
        k_plan_big_check<<<1, 1, 0, s>>>(p.big_off.p + p.big_rows, p.big_cap, err, p.big_skip.p);
        CT_COUNT_LAUNCH();
        CT_CHECK_CUDA(cudaMemsetAsync(p.big_k1.p, 0xff, (size_t)p.big_cap * sizeof(uint64_t), s));
        k_plan_big_gather<<<p.big_rows, 256, 0, s>>>(big, nbig, p.big_rows, p.big_skip.p, p.row_ptr.p, p.big_off.p,
                                                     p.col.p, p.big_k1.p, p.big_v1.p);
        CT_COUNT_LAUNCH();
        int bits = 32;
        while ((int64_t(1) << (bits - 32)) < p.big_rows) ++bits;
        radix_sort_pairs64(p.big_k1.p, p.big_v1.p, p.big_k2.p, p.big_v2.p, p.big_cap, bits, s);
        k_plan_big_apply<<<p.big_rows, 256, 0, s>>>(big, nbig, p.big_rows, p.big_skip.p, p.row_ptr.p, p.big_off.p,
                                                    p.big_k1.p, p.big_v1.p, p.col.p, p.dist.p, p.big_tmpd.p);
        CT_COUNT_LAUNCH();
    }
    // 7. each cloud's row offsets relative to its first row
    for (int c = 0; c < p.C; ++c) {
        const int64_t nc1 = p.trees[c]->n + 1;
        k_rel_rows<<<grid_for(nc1, 256), 256, 0, s>>>(nc1, p.row_ptr.p + V.rbase[c], p.rel.p + V.rbase[c] + c);
        CT_COUNT_LAUNCH();
    }
    CT_LAUNCH_CHECK();
}
}  // namespace

PlanImpl *plan_create(int C, const ct_tree *const *trees, const QParams *qps, int precision,
                      const ct_predictor *pred, float margin, bool use_graph, cudaStream_t s) {
    if (C < 1 || C > kMaxClouds) CT_FAIL(CT_EINVAL, "between 1 and %d clouds per plan", kMaxClouds);
    std::unique_ptr<PlanImpl> pp(new PlanImpl());
    PlanImpl &p = *pp;
    p.C = C;
    p.s0 = s;
    std::memset(&p.V, 0, sizeof(p.V));
    p.V.nc = C;
    int max_depth = 0, min_len = kItem;
    for (int c = 0; c < C; ++c) {
        const ct_tree *t = trees[c];
        if (t->metric != CT_L2_F32) CT_FAIL(CT_EINVAL, "plans take L2 trees only");
        p.trees.push_back(t);
        p.V.tv[c] = view_of(t);
        p.V.qp[c] = qps[c];
        p.any_half |= qps[c].half != 0;
        p.V.use_tc[c] = 0;  // the persistent launch runs the FP32 tiles
        const int len = precision == 2 ? leaf_choice(t, 2).item_len : kItem;
        p.V.item_len[c] = (int16_t)len;
        min_len = std::min(min_len, len);
        p.V.gbase[c + 1] = p.V.gbase[c] + t->n_groups;
        p.V.rbase[c + 1] = p.V.rbase[c] + t->n;
        p.max_cols = std::max<int64_t>(p.max_cols, t->n);
        p.max_dp = std::max(p.max_dp, t->dp);
        max_depth = std::max(max_depth, t->depth);
    }
    if (p.V.rbase[C] >= 0x7fffffffLL) CT_FAIL(CT_EOVERFLOW, "a plan above 2^31 points");
    p.n = p.V.rbase[C];
    p.G = p.V.gbase[C];
    const int64_t n = p.n;
    const int G = p.G;
    // sizing query (the batch's own exact query, FP32 tiles)
    std::vector<QueryOut> outs((size_t)C);
    struct OutsGuard {  // the sizing query's CSRs are released on every path
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
    } outs_guard{outs, s};
    query_multi(C, trees, qps, s, outs.data(), 0, pred, nullptr);
    const int64_t n_cand = outs[0].stats.candidates;
    int64_t nnz = 0, nbig = 0, big_entries = 0;
    {
        std::vector<int64_t> hrp;
        for (int c = 0; c < C; ++c) {
            nnz += outs[c].nnz;
            hrp.resize((size_t)trees[c]->n + 1);
            to_host(hrp.data(), outs[c].row_ptr, hrp.size(), s);
            for (size_t i = 0; i + 1 < hrp.size(); ++i) {
                const int64_t len = hrp[i + 1] - hrp[i];
                if (len > SORT_MID) {
                    ++nbig;
                    big_entries += len;
                }
            }
        }
    }
    const double m = std::max(0.0, (double)margin);
    p.big_rows = (int)std::min<int64_t>((int64_t)std::ceil((double)nbig * (1.0 + m)) + 16, 0x7fffffff);
    p.big_cap = (int64_t)std::ceil((double)big_entries * (1.0 + m)) + 4096;
    p.tl = trav_launch_config(true, G);
    p.cap_stack = 32 * (max_depth + 2);
    p.spill_cap = (int)std::min<int64_t>(std::max<int64_t>(4 * (int64_t)G, 1 << 16), 1 << 20);
    p.cand_cap = (int64_t)std::ceil((double)n_cand * (1.0 + m)) + 4096;
    p.pool_cap = p.cand_cap + (int64_t)(p.tl.warps + 1) * POOL_CHUNK;
    p.seg_cap = G + (int64_t)TRAV_ROUNDS * p.spill_cap + p.pool_cap / POOL_CHUNK + p.tl.warps + 16;
    p.item_cap = std::min<int64_t>(G + p.cand_cap / min_len + 1, 0x7fffffff);
    p.nnz_cap = (int64_t)std::ceil((double)nnz * (1.0 + m)) + 4096;
    // walk order: the predictor's (groups by decreasing predicted walk
    // length), else decreasing radius relative to eps
    p.order = DBuf<int32_t>(G ? G : 1, s);
    if (G) {
        LearnedPlan lp;
        if (pred) learned_plan(pred, C, trees, qps, p.V.rbase, p.V.gbase, s, lp);
        if (lp.group_order.p) {
            CT_CHECK_CUDA(cudaMemcpyAsync(p.order.p, lp.group_order.p, (size_t)G * sizeof(int32_t),
                                          cudaMemcpyDeviceToDevice, s));
        } else {
            DBuf<uint32_t> k1(G, s), v1(G, s), k2(G, s), v2(G, s);
            for (int c = 0; c < C; ++c) {
                const int Gc = trees[c]->n_groups;
                if (!Gc) continue;
                k_radius_keys<<<grid_for(Gc, 256), 256, 0, s>>>(Gc, trees[c]->group_radius,
                                                                (float)(1.0 / std::max(qps[c].eps64, 1e-30)),
                                                                p.V.gbase[c], k1.p, v1.p);
                CT_COUNT_LAUNCH();
            }
            radix_sort_pairs(k1.p, v1.p, k2.p, v2.p, G, 32, s);
            CT_CHECK_CUDA(cudaMemcpyAsync(p.order.p, v1.p, (size_t)G * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        }
    }
    // buffers
    p.st = DBuf<unsigned long long>(ST_N, s);
    p.ctr = DBuf<unsigned long long>(4, s);
    p.next_group = DBuf<int32_t>(1, s);
    p.spill_cnt = DBuf<int32_t>(2, s);
    p.ctl = DBuf<int32_t>(2, s);
    p.qctr = DBuf<int32_t>(4, s);
    p.empty_flag = DBuf<int32_t>(1, s);
    p.stacks = DBuf<int2>((size_t)p.tl.warps * p.cap_stack, s);
    p.spill_a = DBuf<int4>(p.spill_cap, s);
    p.spill_b = DBuf<int4>(p.spill_cap, s);
    p.cursors = DBuf<longlong2>(p.tl.warps, s);
    p.pool = DBuf<uint32_t>(p.pool_cap, s);
    p.seg_group = DBuf<int32_t>(p.seg_cap, s);
    p.seg_count = DBuf<int32_t>(p.seg_cap, s);
    p.seg_begin = DBuf<int64_t>(p.seg_cap, s);
    p.gcand = DBuf<uint32_t>(p.cand_cap, s);
    p.emask = DBuf<uint32_t>(p.cand_cap, s);
    p.gcount = DBuf<int32_t>(G ? G : 1, s);
    p.gfill = DBuf<int32_t>(G ? G : 1, s);
    p.gbegin = DBuf<int64_t>(G + 1, s);
    p.sums = DBuf<int64_t>(std::max<int64_t>(scan_scratch_entries(std::max<int64_t>(n + 1, G)), 1), s);
    p.ready = DBuf<int32_t>(p.item_cap, s);
    p.igroup = DBuf<int32_t>(p.item_cap, s);
    p.ibeg = DBuf<int64_t>(p.item_cap, s);
    p.iend = DBuf<int64_t>(p.item_cap, s);
    p.deg = DBuf<int32_t>(n + 1, s);
    p.rowcur = DBuf<int32_t>(n + 1, s);
    p.row_ptr = DBuf<int64_t>(n + 1, s);
    p.rel = DBuf<int64_t>(n + C, s);
    p.col = DBuf<int32_t>(p.nnz_cap, s);
    p.dist = DBuf<float>(p.nnz_cap, s);
    p.sort_lists = DBuf<int32_t>((size_t)kSortClasses * (n ? n : 1), s);
    p.sort_counts = DBuf<int32_t>(kSortClasses, s);
    p.big_lens = DBuf<int64_t>(p.big_rows, s);
    p.big_off = DBuf<int64_t>(p.big_rows + 1, s);
    p.big_k1 = DBuf<uint64_t>(p.big_cap, s);
    p.big_k2 = DBuf<uint64_t>(p.big_cap, s);
    p.big_v1 = DBuf<uint32_t>(p.big_cap, s);
    p.big_v2 = DBuf<uint32_t>(p.big_cap, s);
    p.big_tmpd = DBuf<float>(p.big_cap, s);
    p.big_skip = DBuf<int32_t>(1, s);
    const int32_t ctl0[2] = {0, 1 << 20};  // about a second of polls
    CT_CHECK_CUDA(cudaMemcpyAsync(p.ctl.p, ctl0, sizeof(ctl0), cudaMemcpyHostToDevice, s));
    // persistent grid: the FP32 tiles' resident CTAs on every SM
    leaf_l2_prepare();
    {
        int per_sm = 0;
        CT_CHECK_CUDA(cudaFuncSetAttribute(k_leaf_l2_queue<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kLeafSmem));
        CT_CHECK_CUDA(cudaFuncSetAttribute(k_leaf_l2_queue<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kLeafSmem));
        CT_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_leaf_l2_queue<false>, LEAF_T,
                                                                    kLeafSmem));
        p.leaf_grid = std::max(1, num_sms() * std::max(per_sm, 1));
    }
    {
        const size_t tsm = (size_t)TRAV_WARPS * p.max_dp * sizeof(float);
        if (tsm > 48 * 1024)
            CT_CHECK_CUDA(cudaFuncSetAttribute(k_traverse_l2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm));
        sort_grids();  // row-sort attributes set outside the capture
    }
    CT_CHECK_CUDA(cudaStreamSynchronize(s));
    if (use_graph) {
        // captured on a private stream (the caller's may be the legacy
        // default stream, which cannot be captured); launched on any stream
        cudaStream_t cs = nullptr;
        CT_CHECK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        struct StreamGuard {
            cudaStream_t s;
            ~StreamGuard() { cudaStreamDestroy(s); }
        } sg{cs};
        CT_CHECK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
        try {
            plan_enqueue(p, cs);
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(cs, &g);
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            throw;
        }
        CT_CHECK_CUDA(cudaStreamEndCapture(cs, &p.graph));
        CT_CHECK_CUDA(cudaGraphInstantiate(&p.exec, p.graph, 0));
    }
    return pp.release();
}

void plan_launch(PlanImpl *p, cudaStream_t s) {
    if (p->exec)
        CT_CHECK_CUDA(cudaGraphLaunch(p->exec, s));
    else
        plan_enqueue(*p, s);
}

void plan_set_wait(PlanImpl *p, int withhold, int max_polls) {
    const int32_t v[2] = {withhold ? 1 : 0, max_polls};
    CT_CHECK_CUDA(cudaDeviceSynchronize());  // no run of the plan is in flight
    CT_CHECK_CUDA(cudaMemcpy(p->ctl.p, v, sizeof(v), cudaMemcpyHostToDevice));
}

int plan_clouds(const PlanImpl *p) { return p->C; }
int64_t plan_rows(const PlanImpl *p, int c) { return p->trees[c]->n; }

// Status of the last run (synchronises `s`): CT_OK and the clouds' CSR views
// into the plan's buffers, or the failure.
ct_status plan_result(PlanImpl *p, cudaStream_t s, QueryOut *outs) {
    unsigned long long hs[ST_N];
    to_host(hs, p->st.p, ST_N, s);
    const int32_t e = (int32_t)hs[ST_ERR];
    if (e & Q_ERR_TIMEOUT) {
        set_error("a work-queue wait of the plan's leaf stage gave up (its producer never published)");
        return CT_ETIMEOUT;
    }
    if (e & Q_ERR_OVERFLOW) {
        set_error("the run outgrew the plan's capacities (candidates, work items, edges or row length); "
                  "create a new plan");
        return CT_EOVERFLOW;
    }
    if (e) {
        set_error("internal consistency check failed in the plan's run (code %d)", e);
        return CT_ECUDA;
    }
    std::vector<int64_t> hb((size_t)p->C + 1);
    for (int c = 0; c <= p->C; ++c) to_host_async(&hb[c], p->row_ptr.p + p->V.rbase[c], 1, s);
    CT_CHECK_CUDA(cudaStreamSynchronize(s));
    auto blocks = std::make_shared<SharedBlocks>(s);  // views: the plan keeps the memory
    for (int c = 0; c < p->C; ++c) {
        QueryOut &q = outs[c];
        q.row_ptr = p->rel.p + p->V.rbase[c] + c;
        q.col = p->col.p + hb[c];
        q.dist = p->dist.p + hb[c];
        q.nnz = hb[c + 1] - hb[c];
        q.stats = ct_query_stats{};
        q.stats.traversal_evals = (int64_t)hs[ST_TRAV];
        q.stats.leaf_pairs = (int64_t)hs[ST_PAIRS];
        q.stats.guard_fp64 = (int64_t)hs[ST_GUARD];
        q.stats.emit_pairs = (int64_t)hs[ST_EMIT];
        q.stats.leaf_rows = (int64_t)hs[ST_ROWS];
        q.stats.guard_band = (int64_t)hs[ST_BAND];
        q.shared = blocks;
    }
    return CT_OK;
}

void plan_free(PlanImpl *p) {
    if (!p) return;
    cudaStream_t s = p->s0;
    cudaStreamSynchronize(s);
    delete p;
    cudaStreamSynchronize(s);
}

}  // namespace ct

// ----------------------------------------------------------------------
// Degrees without device allocation.
//
// Some callers cannot let a library allocate device memory: an application
// whose own allocator owns the whole device and hands out fixed budgets, or a
// latency-bound loop where an allocation's implicit synchronisation, or its
// possible failure, is not acceptable.  For them the count pass (tree walk +
// FP32 leaf tiles with the FP64 guard band) also runs with every temporary
// buffer placed in one fixed device array of this translation unit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[CT_NOALLOC_SCRATCH_BYTES];

namespace ct {

namespace {
std::mutex g_noalloc_mu;
void *g_noalloc_addr[64] = {};

// Device address of the fixed array on the current device, looked up once per
// device (the host-side symbol is not a device address).
unsigned char *noalloc_scratch() {
    int dev = 0;
    CT_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) CT_FAIL(CT_EUNSUPPORTED, "device ordinal %d above 63", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            CT_FAIL(CT_ECUDA, "cudaGetSymbolAddress of the fixed scratch failed: %s", cudaGetErrorString(e));
        }
        g_noalloc_addr[dev] = p;
    }
    return (unsigned char *)g_noalloc_addr[dev];
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

void degrees_noalloc(const ct_tree *t, const QParams &qp, int32_t *degrees, cudaStream_t s) {
    if (t->metric != CT_L2_F32) CT_FAIL(CT_EUNSUPPORTED, "the allocation-free degree count supports L2 trees only");
    const int64_t n = t->n;
    if (n == 0) return;
    unsigned char *base = noalloc_scratch();
    const size_t cap_bytes = CT_NOALLOC_SCRATCH_BYTES;
    const int cap = 32 * (t->depth + 2);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char *p = base + off;
        off = align256(off + bytes);
        return p;
    };
    // fixed part: counters, scan tile sums, traversal stacks
    unsigned long long *st = (unsigned long long *)take(ST_N * sizeof(unsigned long long));
    unsigned long long *ctr = (unsigned long long *)take(4 * sizeof(unsigned long long));
    int32_t *next_group = (int32_t *)take(sizeof(int32_t));
    int32_t *nitems = (int32_t *)take(sizeof(int32_t));
    constexpr int kSpillCap = 1 << 15;  // ranges of step-limited walks per round (a full buffer only ends the limit)
    int32_t *spill_cnt = (int32_t *)take(2 * sizeof(int32_t));
    int4 *const spills[2] = {(int4 *)take(kSpillCap * sizeof(int4)), (int4 *)take(kSpillCap * sizeof(int4))};
    TravLaunch tl = trav_launch_config(true, t->n_groups);
    const size_t stack_per_block = (size_t)TRAV_WARPS * cap * sizeof(int2);
    if (off + stack_per_block > cap_bytes / 2)
        CT_FAIL(CT_EUNSUPPORTED, "a tree of depth %d needs more than the fixed %zu-byte scratch", t->depth, cap_bytes);
    // stacks take at most a quarter of the array, and the warps' partly filled
    // pool chunks (POOL_CHUNK entries each) at most a quarter of it: with a
    // 16 MiB array that caps the walk at 64 blocks of TRAV_WARPS warps, fewer
    // than the main path's resident grid (the walk is slower, not different)
    const int64_t chunk_blocks = (int64_t)(cap_bytes / 4 / sizeof(uint32_t)) / ((int64_t)TRAV_WARPS * POOL_CHUNK);
    tl.blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>(std::min<int64_t>(tl.blocks, (cap_bytes / 4) / stack_per_block), chunk_blocks));
    tl.warps = tl.blocks * TRAV_WARPS;
    int2 *stacks = (int2 *)take((size_t)tl.blocks * stack_per_block);
    longlong2 *cursors = (longlong2 *)take((size_t)tl.warps * sizeof(longlong2));
    // the rest: segments (a sixth of it: 16 bytes each, one per walk and per
    // pool chunk a walk crosses) and the pool
    const size_t rest = cap_bytes > off ? cap_bytes - off : 0;
    const int64_t seg_cap = (int64_t)(rest / 6 / (sizeof(int32_t) * 2 + sizeof(int64_t)));
    int32_t *seg_group = (int32_t *)take((size_t)seg_cap * sizeof(int32_t));
    int32_t *seg_count = (int32_t *)take((size_t)seg_cap * sizeof(int32_t));
    int64_t *seg_begin = (int64_t *)take((size_t)seg_cap * sizeof(int64_t));
    if (off >= cap_bytes) CT_FAIL(CT_EUNSUPPORTED, "problem too large for the fixed scratch");
    const int64_t pool_cap = (int64_t)((cap_bytes - off) / sizeof(uint32_t));
    uint32_t *pool = (uint32_t *)take((size_t)pool_cap * sizeof(uint32_t));
    Pool P{pool, pool_cap, ctr, seg_group, seg_count, seg_begin, reinterpret_cast<int32_t *>(ctr + 1), seg_cap,
           ctr + 2, reinterpret_cast<int32_t *>(ctr + 3)};

    Views V;
    std::memset(&V, 0, sizeof(V));
    V.nc = 1;
    V.tv[0] = view_of(t);
    V.qp[0] = qp;
    V.gbase[1] = t->n_groups;
    V.rbase[1] = n;
    V.item_len[0] = kItem;
    int32_t *err = reinterpret_cast<int32_t *>(st + ST_ERR);
    // the array keeps the previous call's contents: clear what must start at zero
    CT_CHECK_CUDA(cudaMemsetAsync(st, 0, ST_N * sizeof(unsigned long long), s));
    launch_traversal(V, t->n_groups, t->dp, 0, true, t->group_order, P, stacks, cap, tl, st, err, next_group, spills,
                     spill_cnt, kSpillCap, cursors, s);
    unsigned long long hc[4] = {0, 0, 0, 0};
    CT_CHECK_CUDA(cudaMemcpyAsync(hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost, s));
    CT_CHECK_CUDA(cudaStreamSynchronize(s));
    if ((uint32_t)hc[3])
        CT_FAIL(CT_EUNSUPPORTED, "%llu candidate blocks do not fit the fixed %zu-byte scratch (room for %lld); use eps_graph_query",
                hc[2], cap_bytes, (long long)pool_cap);
    const int nseg = (int)(uint32_t)hc[1];
    // work items live in the unused tail of the pool
    const int64_t used = (int64_t)hc[0] < pool_cap ? (int64_t)hc[0] : pool_cap;
    const int64_t max_items = nseg + (int64_t)hc[2] / kItem + 1;
    size_t toff = align256((size_t)used * sizeof(uint32_t));
    auto ttake = [&](size_t bytes) {
        unsigned char *p = (unsigned char *)pool + toff;
        toff = align256(toff + bytes);
        return p;
    };
    int32_t *icnt = (int32_t *)ttake((size_t)(nseg + 1) * sizeof(int32_t));
    int64_t *ioff = (int64_t *)ttake((size_t)(nseg + 1) * sizeof(int64_t));
    int64_t *sums = (int64_t *)ttake((size_t)std::max<int64_t>(scan_scratch_entries(nseg), 1) * sizeof(int64_t));
    int32_t *igroup = (int32_t *)ttake((size_t)max_items * sizeof(int32_t));
    int64_t *ibeg = (int64_t *)ttake((size_t)max_items * sizeof(int64_t));
    int64_t *iend = (int64_t *)ttake((size_t)max_items * sizeof(int64_t));
    if (toff > (size_t)pool_cap * sizeof(uint32_t))
        CT_FAIL(CT_EUNSUPPORTED, "work items of %llu candidate blocks do not fit the fixed scratch; use eps_graph_query",
                hc[2]);
    CT_CHECK_CUDA(cudaMemsetAsync(degrees, 0, (size_t)n * sizeof(int32_t), s));
    CT_CHECK_CUDA(cudaMemsetAsync(nitems, 0, sizeof(int32_t), s));
    if (nseg) {
        k_item_counts<<<grid_for(nseg, 256), 256, 0, s>>>(V, nseg, seg_group, seg_count, icnt);
        CT_COUNT_LAUNCH();
        exclusive_scan_i32_to_i64_into(icnt, ioff, nseg, ioff + nseg, sums, s);
        k_item_fill<<<grid_for(nseg, 256), 256, 0, s>>>(V, nseg, seg_group, seg_begin, seg_count, ioff, igroup, ibeg,
                                                       iend, nitems);
        CT_COUNT_LAUNCH();
        Items items{igroup, ibeg, iend, nitems};
        leaf_l2_prepare();
        k_leaf_l2<false><<<(unsigned)max_items, LEAF_T, kLeafSmem, s>>>(V, items, pool, nullptr, degrees, nullptr,
                                                                          nullptr, nullptr, nullptr, st, err, CapOut{},
                                                                          nullptr);
        CT_COUNT_LAUNCH();
    }
    CT_LAUNCH_CHECK();
    unsigned long long e = 0;
    CT_CHECK_CUDA(cudaMemcpyAsync(&e, st + ST_ERR, sizeof(e), cudaMemcpyDeviceToHost, s));
    CT_CHECK_CUDA(cudaStreamSynchronize(s));
    if (e) CT_FAIL(CT_ECUDA, "internal consistency check failed in the degree count (code %llu)", e);
}

}  // namespace ct
