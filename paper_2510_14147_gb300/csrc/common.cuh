// common.cuh -- shared helpers of the CUDA library (status handling, device
// memory, warp utilities, the fp32 distance kernels' building blocks).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/ctgraph.h"

namespace ct {

// ---------------------------------------------------------------- errors

void set_error(const char *fmt, ...);
const char *get_error();

struct Error {
    ct_status st;
};

#define CT_CHECK_CUDA(call)                                                         \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            ::ct::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,              \
                            cudaGetErrorString(e_));                                \
            throw ::ct::Error{e_ == cudaErrorMemoryAllocation ? CT_ENOMEM : CT_ECUDA}; \
        }                                                                           \
    } while (0)

#define CT_LAUNCH_CHECK() CT_CHECK_CUDA(cudaGetLastError())

#define CT_FAIL(code, ...)                 \
    do {                                   \
        ::ct::set_error(__VA_ARGS__);      \
        throw ::ct::Error{code};           \
    } while (0)

// ------------------------------------------------------- device memory

// Stream-ordered device allocation from the device's default pool.  The pool's
// release threshold is raised once per device so freed blocks are reused by the
// next call instead of being returned to the driver.
void *dmalloc(size_t bytes, cudaStream_t s);
void dfree(void *p, cudaStream_t s);
// Test hook: the k-th next dmalloc (k >= 1) fails with CT_ENOMEM; 0 turns it off.
void set_fail_alloc(int64_t k);
// Budget of the learned form's one-pass buffers in bytes (0: a third of the
// free device memory).
void set_capacity_budget(int64_t bytes);

// Owning buffer freed stream-ordered when it goes out of scope.
template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    cudaStream_t s = 0;
    DBuf() = default;
    DBuf(size_t count, cudaStream_t st) : n(count), s(st) {
        p = count ? (T *)dmalloc(count * sizeof(T), st) : nullptr;
    }
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) { reset(); p = o.p; n = o.n; s = o.s; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DBuf() { reset(); }
    void reset() {
        if (p) dfree(p, s);
        p = nullptr;
        n = 0;
    }
    T *release() { T *q = p; p = nullptr; n = 0; return q; }
    void grow(size_t count) {  // reallocate without preserving contents
        if (count <= n) return;
        reset();
        p = (T *)dmalloc(count * sizeof(T), s);
        n = count;
    }
};

template <class T>
inline void to_host(T *h, const T *d, size_t count, cudaStream_t s) {
    if (!count) return;
    CT_CHECK_CUDA(cudaMemcpyAsync(h, d, count * sizeof(T), cudaMemcpyDeviceToHost, s));
    CT_CHECK_CUDA(cudaStreamSynchronize(s));
}
// The copy only; the caller synchronises before reading h.
template <class T>
inline void to_host_async(T *h, const T *d, size_t count, cudaStream_t s) {
    if (count) CT_CHECK_CUDA(cudaMemcpyAsync(h, d, count * sizeof(T), cudaMemcpyDeviceToHost, s));
}

int num_sms();
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Counts kernel launches made by the library on this thread (reported with
// query statistics).
extern thread_local int64_t g_launches;
extern std::atomic<int64_t> g_total_launches;
#define CT_COUNT_LAUNCH() (++::ct::g_launches, ::ct::g_total_launches.fetch_add(1, std::memory_order_relaxed))

// ------------------------------------------------------------- scans

// Exclusive prefix sums (reduce-then-scan, three launches).  `out` may alias
// `in`.  Writes the total to *total_dev when given (device int64).
void exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, int64_t *total_dev,
                               cudaStream_t s);
void exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total_dev,
                        cudaStream_t s);
// The same scan with caller-provided tile sums (scan_scratch_entries(n) int64).
int64_t scan_scratch_entries(int64_t n);
void exclusive_scan_i32_to_i64_into(const int32_t *in, int64_t *out, int64_t n, int64_t *total_dev,
                                    int64_t *tile_sums, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs by the low `key_bits` bits of
// the key.  Sorted output returned in keys/vals (tmp buffers of n entries).
void radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *tmp_keys, uint32_t *tmp_vals,
                      int64_t n, int key_bits, cudaStream_t s);

// Stable sort of 64-bit keys with 32-bit values (used for long CSR rows).
void radix_sort_pairs64(uint64_t *keys, uint32_t *vals, uint64_t *tmp_keys, uint32_t *tmp_vals,
                        int64_t n, int key_bits, cudaStream_t s);

// ------------------------------------------------------- device helpers

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Packs a non-negative float and a position so that a 64-bit max selects the
// largest value and, among equal values, the smallest position.
__device__ __forceinline__ unsigned long long pack_max_key(float v, uint32_t pos) {
    return ((unsigned long long)__float_as_uint(v) << 32) | (unsigned long long)(0xFFFFFFFFu - pos);
}
__device__ __forceinline__ float key_value(unsigned long long k) {
    return __uint_as_float((uint32_t)(k >> 32));
}
__device__ __forceinline__ uint32_t key_pos(unsigned long long k) {
    return 0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFull);
}

}  // namespace ct

// ------------------------------------------------------- the tree

// Device-resident cover tree.  Points are stored in tree order: the points of
// every vertex occupy one contiguous range of positions, and a vertex's centre
// is the first point of its range.
struct ct_tree {
    int32_t metric = CT_L2_F32;
    int32_t dim = 0;     // L2: coordinates per point
    int32_t dp = 0;      // L2: padded row length (multiple of 4 floats)
    int64_t n = 0;
    int32_t leaf_size = 32;
    int device = 0;
    cudaStream_t stream = 0;

    // L2 data in tree order, n x dp fp32, zero padded
    float *pts = nullptr;
    // strings in tree order
    uint8_t *sdata = nullptr;
    int64_t *soff = nullptr;      // n + 1
    int32_t max_len = 0;
    int64_t sbytes = 0;

    // Hamming bit rows in tree order, n x wp 32-bit words (wp a multiple of
    // 4, bits past dim zero); dim is the number of bits
    uint32_t *bits = nullptr;
    int32_t wp = 0;

    int32_t *perm = nullptr;      // position -> original id
    float *dcen = nullptr;        // position -> distance to its leaf block's centre

    // vertices: 0 is the root; children of a vertex are consecutive ids
    int32_t n_nodes = 0, n_leaves = 0, depth = 0;
    int32_t *node_begin = nullptr;   // first position of the vertex's points
    int32_t *node_count = nullptr;   // number of points below the vertex
    int32_t *child_begin = nullptr;  // first child id
    int32_t *child_count = nullptr;  // 0 for a leaf block
    float *radius = nullptr;         // vertex-triple radius, rounded up
    int32_t *level = nullptr;        // split level (INT32_MIN for radius 0)
    float *node_ctr = nullptr;       // L2: n_nodes x dp centre coordinates
    int32_t *leaf_ids = nullptr;     // leaf blocks in position order
    int32_t max_leaf_count = 0;      // largest leaf block
    int32_t *parent = nullptr;       // parent vertex (-1 for the root)

    // query groups: runs of consecutive sibling leaf blocks with at most
    // kGroupSize points in total (a larger leaf block is cut into groups of
    // kGroupSize consecutive points, the last one shorter);
    // centre = first point, radius = max distance to it (rounded up)
    int32_t n_groups = 0, max_group_count = 0;
    int32_t *group_begin = nullptr;
    int32_t *group_count = nullptr;
    float *group_radius = nullptr;
    int32_t *group_order = nullptr;  // groups by decreasing radius (longest walks first)
};

namespace ct {
constexpr int kGroupSize = 32;
}
