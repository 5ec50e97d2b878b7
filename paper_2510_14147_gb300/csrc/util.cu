// util.cu -- errors, device memory, prefix scans and the radix sort used by
// the tree build and the CSR row sort.
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "common.cuh"

namespace ct {

static thread_local char g_err[1024] = "";
thread_local int64_t g_launches = 0;

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
const char *get_error() { return g_err; }

static std::mutex g_pool_mu;
static bool g_pool_ready[64] = {false};

// Test hook: when positive, the allocation that brings it to zero fails as if
// the device were out of memory (host-side fault injection).
static std::atomic<int64_t> g_fail_alloc{0};
void set_fail_alloc(int64_t k) { g_fail_alloc.store(k > 0 ? k : 0); }

void *dmalloc(size_t bytes, cudaStream_t s) {
    int dev = 0;
    CT_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && !g_pool_ready[dev]) {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (!g_pool_ready[dev]) {
            cudaMemPool_t pool;
            CT_CHECK_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
            uint64_t thr = UINT64_MAX;
            CT_CHECK_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
            g_pool_ready[dev] = true;
        }
    }
    void *p = nullptr;
    if (!bytes) return nullptr;
    if (g_fail_alloc.load(std::memory_order_relaxed) > 0 && g_fail_alloc.fetch_sub(1) == 1) {
        set_error("device allocation of %zu bytes failed (injected)", bytes);
        throw Error{CT_ENOMEM};
    }
    cudaError_t e = cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        throw Error{CT_ENOMEM};
    }
    return p;
}

void dfree(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

int num_sms() {
    static int sms[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!sms[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        sms[dev] = v > 0 ? v : 1;
    }
    return sms[dev];
}

// ------------------------------------------------------------------ scans

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class T>
__device__ __forceinline__ int64_t block_reduce_sum(int64_t v, int64_t *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = l < (int)(blockDim.x >> 5) ? sh[l] : 0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    return v;
}

template <class T>
__global__ void k_tile_sums(const T *__restrict__ in, int64_t n, int64_t *__restrict__ sums) {
    __shared__ int64_t sh[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t acc = 0;
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t idx = base + (int64_t)i * SCAN_THREADS + threadIdx.x;
        if (idx < n) acc += (int64_t)in[idx];
    }
    acc = block_reduce_sum<T>(acc, sh);
    if (threadIdx.x == 0) sums[blockIdx.x] = acc;
}

// Block-wide exclusive scan of one value per thread; returns the prefix and
// the block total.
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *sh, int64_t &total) {
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (l >= o) x += y;
    }
    if (l == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        int64_t s = l < nw ? sh[l] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (l >= o) s += y;
        }
        if (l < nw) sh[l] = s;
    }
    __syncthreads();
    int64_t warp_prefix = w ? sh[w - 1] : 0;
    total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

// Single-block exclusive scan over `n` int64 (n up to any size, looped).
__global__ void k_scan_single(int64_t *__restrict__ a, int64_t n, int64_t *__restrict__ total_dev) {
    __shared__ int64_t sh[32];
    int64_t carry = 0;
    for (int64_t base = 0; base < n; base += (int64_t)blockDim.x * SCAN_ITEMS) {
        int64_t v[SCAN_ITEMS];
        int64_t loc = 0;
        int64_t idx0 = base + (int64_t)threadIdx.x * SCAN_ITEMS;
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            v[i] = idx0 + i < n ? a[idx0 + i] : 0;
            loc += v[i];
        }
        int64_t tot;
        int64_t pre = block_exclusive_scan(loc, sh, tot);
        int64_t run = carry + pre;
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            if (idx0 + i < n) a[idx0 + i] = run;
            run += v[i];
        }
        carry += tot;
    }
    if (threadIdx.x == 0 && total_dev) *total_dev = carry;
}

template <class T>
__global__ void k_tile_scan(const T *__restrict__ in, int64_t *__restrict__ out, int64_t n,
                            const int64_t *__restrict__ tile_prefix) {
    __shared__ int64_t sh[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t idx0 = base + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t loc = 0;
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = idx0 + i < n ? (int64_t)in[idx0 + i] : 0;
        loc += v[i];
    }
    int64_t tot;
    int64_t run = tile_prefix[blockIdx.x] + block_exclusive_scan(loc, sh, tot);
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (idx0 + i < n) out[idx0 + i] = run;
        run += v[i];
    }
}

template <class T>
static void exclusive_scan_impl(const T *in, int64_t *out, int64_t n, int64_t *total_dev,
                                cudaStream_t s) {
    if (n <= 0) {
        if (total_dev) CT_CHECK_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(int64_t), s));
        return;
    }
    int64_t tiles = ceil_div(n, SCAN_TILE);
    DBuf<int64_t> sums(tiles, s);
    k_tile_sums<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, sums.p);
    CT_COUNT_LAUNCH();
    k_scan_single<<<1, 1024, 0, s>>>(sums.p, tiles, total_dev);
    CT_COUNT_LAUNCH();
    k_tile_scan<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, sums.p);
    CT_COUNT_LAUNCH();
    CT_LAUNCH_CHECK();
}

void exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, int64_t *total_dev,
                               cudaStream_t s) {
    exclusive_scan_impl<int32_t>(in, out, n, total_dev, s);
}

int64_t scan_scratch_entries(int64_t n) { return n > 0 ? ceil_div(n, SCAN_TILE) : 0; }

void exclusive_scan_i32_to_i64_into(const int32_t *in, int64_t *out, int64_t n, int64_t *total_dev,
                                    int64_t *tile_sums, cudaStream_t s) {
    if (n <= 0) {
        if (total_dev) CT_CHECK_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(int64_t), s));
        return;
    }
    int64_t tiles = ceil_div(n, SCAN_TILE);
    k_tile_sums<int32_t><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, tile_sums);
    CT_COUNT_LAUNCH();
    k_scan_single<<<1, 1024, 0, s>>>(tile_sums, tiles, total_dev);
    CT_COUNT_LAUNCH();
    k_tile_scan<int32_t><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, tile_sums);
    CT_COUNT_LAUNCH();
    CT_LAUNCH_CHECK();
}
void exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total_dev,
                        cudaStream_t s) {
    exclusive_scan_impl<int64_t>(in, out, n, total_dev, s);
}

// ------------------------------------------------------------- radix sort
// LSD radix sort, 8-bit digits, stable.  Per pass: a per-tile digit
// histogram (digit-major layout), a scan of the histograms, and a scatter in
// which each warp ranks its keys with __match_any_sync so equal digits keep
// their input order.

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_IPT = 8;                          // keys per lane
constexpr int RS_TILE = RS_THREADS * RS_IPT;       // 2048 keys per tile
constexpr int RS_WARP_KEYS = 32 * RS_IPT;          // 256 contiguous keys per warp

template <class K>
__global__ void k_rs_hist(const K *__restrict__ keys, int64_t n, int shift,
                          int32_t *__restrict__ hist, int64_t tiles) {
    __shared__ int32_t h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += blockDim.x) {
        int64_t idx = base + i;
        if (idx < n) atomicAdd(&h[(uint32_t)(keys[idx] >> shift) & 255u], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(int64_t)d * tiles + blockIdx.x] = h[d];
}

template <class K>
__global__ void k_rs_scatter(const K *__restrict__ keys, const uint32_t *__restrict__ vals,
                             K *__restrict__ okeys, uint32_t *__restrict__ ovals, int64_t n,
                             int shift, const int64_t *__restrict__ offs, int64_t tiles) {
    __shared__ int32_t wcount[RS_WARPS][256];
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int i = l; i < 256; i += 32) wcount[w][i] = 0;
    __syncwarp();
    int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)w * RS_WARP_KEYS;
    uint32_t dig[RS_IPT];
    int32_t rank[RS_IPT];
    // pass 1: rank within the warp's contiguous sub-tile, in order
    for (int r = 0; r < RS_IPT; ++r) {
        int64_t idx = base + r * 32 + l;
        bool valid = idx < n;
        uint32_t d = valid ? ((uint32_t)(keys[idx] >> shift) & 255u) : 256u + l;
        dig[r] = d;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int before = __popc(peers & lanemask_lt());
        int cnt = __popc(peers);
        int leader = __ffs(peers) - 1;
        int prior = 0;
        if (valid && l == leader) prior = wcount[w][d];
        prior = __shfl_sync(0xffffffffu, prior, leader);
        rank[r] = prior + before;
        __syncwarp();
        if (valid && l == leader) wcount[w][d] = prior + cnt;
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps for each digit
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
        int32_t run = 0;
        for (int ww = 0; ww < RS_WARPS; ++ww) {
            int32_t c = wcount[ww][d];
            wcount[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int r = 0; r < RS_IPT; ++r) {
        int64_t idx = base + r * 32 + l;
        if (idx >= n) continue;
        uint32_t d = dig[r];
        int64_t dst = offs[(int64_t)d * tiles + blockIdx.x] + wcount[w][d] + rank[r];
        okeys[dst] = keys[idx];
        ovals[dst] = vals[idx];
    }
}

template <class K>
static void radix_sort_impl(K *keys, uint32_t *vals, K *tk, uint32_t *tv, int64_t n, int key_bits,
                            cudaStream_t s) {
    if (n <= 1 || key_bits <= 0) return;
    int64_t tiles = ceil_div(n, RS_TILE);
    DBuf<int32_t> hist(256 * tiles, s);
    DBuf<int64_t> offs(256 * tiles, s);
    K *src_k = keys, *dst_k = tk;
    uint32_t *src_v = vals, *dst_v = tv;
    int passes = (key_bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_rs_hist<K><<<(unsigned)tiles, RS_THREADS, 0, s>>>(src_k, n, shift, hist.p, tiles);
        CT_COUNT_LAUNCH();
        exclusive_scan_i32_to_i64(hist.p, offs.p, 256 * tiles, nullptr, s);
        k_rs_scatter<K><<<(unsigned)tiles, RS_THREADS, 0, s>>>(src_k, src_v, dst_k, dst_v, n, shift,
                                                               offs.p, tiles);
        CT_COUNT_LAUNCH();
        CT_LAUNCH_CHECK();
        std::swap(src_k, dst_k);
        std::swap(src_v, dst_v);
    }
    if (src_k != keys) {
        CT_CHECK_CUDA(cudaMemcpyAsync(keys, src_k, n * sizeof(K), cudaMemcpyDeviceToDevice, s));
        CT_CHECK_CUDA(cudaMemcpyAsync(vals, src_v, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
}

void radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *tk, uint32_t *tv, int64_t n,
                      int key_bits, cudaStream_t s) {
    radix_sort_impl<uint32_t>(keys, vals, tk, tv, n, key_bits, s);
}
void radix_sort_pairs64(uint64_t *keys, uint32_t *vals, uint64_t *tk, uint32_t *tv, int64_t n,
                        int key_bits, cudaStream_t s) {
    radix_sort_impl<uint64_t>(keys, vals, tk, tv, n, key_bits, s);
}

}  // namespace ct
