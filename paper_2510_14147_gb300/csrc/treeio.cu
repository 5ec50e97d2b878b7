// treeio.cu -- a cover tree written to a file and read back (the tree does not
// depend on eps, so one build serves every later query: the paper queries each
// dataset at several radii, Table I).
//
// File layout (little-endian, as the host stores it): a fixed header, then
// every device array of the tree in a fixed order, each as raw bytes; then a
// 64-bit FNV-1a checksum of everything before it.  A file whose magic,
// version, sizes or checksum do not match is rejected with CT_EINVAL.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <memory>
#include <vector>

#include "common.cuh"

namespace ct {

namespace {

constexpr char kMagic[8] = {'C', 'T', 'T', 'R', 'E', 'E', '0', '1'};
constexpr uint32_t kVersion = 1;

struct Header {
    char magic[8];
    uint32_t version;
    int32_t metric, dim, dp, leaf_size, max_len;
    int64_t n, sbytes;
    int32_t n_nodes, n_leaves, depth, max_leaf_count, n_groups, max_group_count;
};

struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void *p, size_t k) {
        const unsigned char *b = (const unsigned char *)p;
        for (size_t i = 0; i < k; ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
    }
};

struct FileCloser {
    void operator()(FILE *f) const {
        if (f) fclose(f);
    }
};
using File = std::unique_ptr<FILE, FileCloser>;

// The tree's arrays in file order: (device pointer slot, bytes).
std::vector<std::pair<void **, size_t>> arrays_of(ct_tree *t) {
    const size_t n = (size_t)t->n, N = (size_t)t->n_nodes, L = (size_t)t->n_leaves, G = (size_t)t->n_groups;
    std::vector<std::pair<void **, size_t>> a;
    if (t->metric == CT_L2_F32) {
        a.push_back({(void **)&t->pts, n * (size_t)t->dp * sizeof(float)});
    } else if (t->metric == CT_HAMMING_B1) {
        a.push_back({(void **)&t->bits, n * (size_t)t->wp * sizeof(uint32_t)});
    } else {
        a.push_back({(void **)&t->sdata, (size_t)t->sbytes});
        a.push_back({(void **)&t->soff, (n + 1) * sizeof(int64_t)});
    }
    a.push_back({(void **)&t->perm, n * sizeof(int32_t)});
    a.push_back({(void **)&t->dcen, n * sizeof(float)});
    a.push_back({(void **)&t->node_begin, N * sizeof(int32_t)});
    a.push_back({(void **)&t->node_count, N * sizeof(int32_t)});
    a.push_back({(void **)&t->child_begin, N * sizeof(int32_t)});
    a.push_back({(void **)&t->child_count, N * sizeof(int32_t)});
    a.push_back({(void **)&t->radius, N * sizeof(float)});
    a.push_back({(void **)&t->level, N * sizeof(int32_t)});
    if (t->metric == CT_L2_F32) a.push_back({(void **)&t->node_ctr, N * (size_t)t->dp * sizeof(float)});
    a.push_back({(void **)&t->leaf_ids, L * sizeof(int32_t)});
    a.push_back({(void **)&t->parent, N * sizeof(int32_t)});
    a.push_back({(void **)&t->group_begin, G * sizeof(int32_t)});
    a.push_back({(void **)&t->group_count, G * sizeof(int32_t)});
    a.push_back({(void **)&t->group_radius, G * sizeof(float)});
    a.push_back({(void **)&t->group_order, G * sizeof(int32_t)});
    return a;
}

// Allocation sizes the build uses for each array (a few carry padding the
// kernels may read past the end: the row arrays 16 bytes, and empty arrays
// keep one element).
size_t alloc_bytes(size_t bytes) { return (bytes ? bytes : 8) + 16; }

// Index ranges of a loaded tree: every vertex, leaf, group and permutation
// entry must point inside the arrays it indexes (a file from another writer
// must not send a kernel out of bounds).
__global__ void k_check_loaded(int64_t n, int N, int L, int G, const int32_t *__restrict__ perm,
                               const int32_t *__restrict__ nb, const int32_t *__restrict__ ncnt,
                               const int32_t *__restrict__ cb, const int32_t *__restrict__ cc,
                               const int32_t *__restrict__ leaf_ids, const int32_t *__restrict__ par,
                               const int32_t *__restrict__ gb, const int32_t *__restrict__ gc,
                               const int32_t *__restrict__ go, const int64_t *__restrict__ soff, int64_t sbytes,
                               int max_len, int32_t *__restrict__ bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int b = 0;
    if (soff && i < n) {
        b |= (i == 0 && soff[0] != 0) || soff[i + 1] < soff[i] || soff[i + 1] - soff[i] > max_len;
        b |= i == n - 1 && soff[n] != sbytes;
    }
    if (i < n) b |= perm[i] < 0 || perm[i] >= n;
    if (i < N) {
        b |= nb[i] < 0 || ncnt[i] < 1 || (int64_t)nb[i] + ncnt[i] > n;
        b |= cc[i] < 0 || (cc[i] > 0 && (cb[i] < 1 || (int64_t)cb[i] + cc[i] > N));
        b |= par[i] < -1 || par[i] >= N;
    }
    if (i < L) b |= leaf_ids[i] < 0 || leaf_ids[i] >= N;
    if (i < G) {
        b |= gb[i] < 0 || gc[i] < 1 || (int64_t)gb[i] + gc[i] > n;
        b |= go[i] < 0 || go[i] >= G;
    }
    if (b) atomicOr(bad, 1);
}

}  // namespace

void free_tree(ct_tree *t);

void save_tree(const ct_tree *tc, const char *path) {
    ct_tree *t = const_cast<ct_tree *>(tc);
    File f(fopen(path, "wb"));
    if (!f) CT_FAIL(CT_EINVAL, "cannot open %s for writing", path);
    Header h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kMagic, 8);
    h.version = kVersion;
    h.metric = t->metric;
    h.dim = t->dim;
    h.dp = t->metric == CT_HAMMING_B1 ? t->wp : t->dp;  // Hamming: 32-bit words per row
    h.leaf_size = t->leaf_size;
    h.max_len = t->max_len;
    h.n = t->n;
    h.sbytes = t->sbytes;
    h.n_nodes = t->n_nodes;
    h.n_leaves = t->n_leaves;
    h.depth = t->depth;
    h.max_leaf_count = t->max_leaf_count;
    h.n_groups = t->n_groups;
    h.max_group_count = t->max_group_count;
    Fnv sum;
    sum.add(&h, sizeof(h));
    if (fwrite(&h, sizeof(h), 1, f.get()) != 1) CT_FAIL(CT_EINVAL, "write to %s failed", path);
    CT_CHECK_CUDA(cudaStreamSynchronize(t->stream));
    std::vector<unsigned char> buf;
    for (auto &a : arrays_of(t)) {
        if (!a.second) continue;
        buf.resize(a.second);
        CT_CHECK_CUDA(cudaMemcpy(buf.data(), *a.first, a.second, cudaMemcpyDeviceToHost));
        sum.add(buf.data(), a.second);
        if (fwrite(buf.data(), 1, a.second, f.get()) != a.second) CT_FAIL(CT_EINVAL, "write to %s failed", path);
    }
    if (fwrite(&sum.h, sizeof(sum.h), 1, f.get()) != 1) CT_FAIL(CT_EINVAL, "write to %s failed", path);
    if (fflush(f.get()) != 0) CT_FAIL(CT_EINVAL, "write to %s failed", path);
}

ct_tree *load_tree(const char *path, cudaStream_t s) {
    File f(fopen(path, "rb"));
    if (!f) CT_FAIL(CT_EINVAL, "cannot open %s", path);
    Header h;
    if (fread(&h, sizeof(h), 1, f.get()) != 1) CT_FAIL(CT_EINVAL, "%s: truncated header", path);
    if (std::memcmp(h.magic, kMagic, 8) != 0) CT_FAIL(CT_EINVAL, "%s is not a tree file", path);
    if (h.version != kVersion) CT_FAIL(CT_EINVAL, "%s: version %u, expected %u", path, h.version, kVersion);
    const bool l2 = h.metric == CT_L2_F32, ham = h.metric == CT_HAMMING_B1;
    if ((!l2 && !ham && h.metric != CT_LEVENSHTEIN_U8) || h.n < 0 || h.n >= 0x7f7f7f00LL ||
        h.n_nodes < 0 || h.n_nodes > 2 * h.n + 1 || h.n_leaves < 0 || h.n_leaves > h.n_nodes || h.n_groups < 0 ||
        h.n_groups > h.n || (l2 && (h.dp < 4 || h.dp > 4096 || h.dp % 4 || h.dim < 1 || h.dim > h.dp)) ||
        (ham && (h.dp < 4 || h.dp > 128 || h.dp % 4 || h.dim < 1 || h.dim > 32 * h.dp)) ||
        (!l2 && !ham && (h.sbytes < 0 || h.max_len < 0 || h.max_len > CT_MAX_STRING_LEN)))
        CT_FAIL(CT_EINVAL, "%s: inconsistent header", path);
    Fnv sum;
    sum.add(&h, sizeof(h));
    struct Guard {
        ct_tree *t;
        ~Guard() {
            if (t) free_tree(t);
        }
    } g{new ct_tree()};
    ct_tree *t = g.t;
    t->metric = h.metric;
    t->dim = l2 || ham ? h.dim : 0;
    t->dp = l2 ? h.dp : 0;
    t->wp = ham ? h.dp : 0;
    t->n = h.n;
    t->leaf_size = h.leaf_size;
    t->max_len = h.max_len;
    t->sbytes = h.sbytes;
    t->n_nodes = h.n_nodes;
    t->n_leaves = h.n_leaves;
    t->depth = h.depth;
    t->max_leaf_count = h.max_leaf_count;
    t->n_groups = h.n_groups;
    t->max_group_count = h.max_group_count;
    t->stream = s;
    CT_CHECK_CUDA(cudaGetDevice(&t->device));
    std::vector<unsigned char> buf;
    for (auto &a : arrays_of(t)) {
        *a.first = dmalloc(alloc_bytes(a.second), s);
        CT_CHECK_CUDA(cudaMemsetAsync(*a.first, 0, alloc_bytes(a.second), s));
        if (!a.second) continue;
        buf.resize(a.second);
        if (fread(buf.data(), 1, a.second, f.get()) != a.second) CT_FAIL(CT_EINVAL, "%s: truncated", path);
        sum.add(buf.data(), a.second);
        CT_CHECK_CUDA(cudaMemcpyAsync(*a.first, buf.data(), a.second, cudaMemcpyHostToDevice, s));
        CT_CHECK_CUDA(cudaStreamSynchronize(s));  // buf is reused by the next array
    }
    uint64_t want = 0;
    if (fread(&want, sizeof(want), 1, f.get()) != 1) CT_FAIL(CT_EINVAL, "%s: truncated", path);
    if (want != sum.h) CT_FAIL(CT_EINVAL, "%s: checksum mismatch", path);
    unsigned char extra;
    if (fread(&extra, 1, 1, f.get()) == 1) CT_FAIL(CT_EINVAL, "%s: trailing bytes", path);
    const int64_t span = std::max<int64_t>(std::max<int64_t>(t->n, t->n_nodes), 1);
    DBuf<int32_t> bad(1, s);
    CT_CHECK_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int32_t), s));
    if (t->n > 0) {
        k_check_loaded<<<(unsigned)ceil_div(span, 256), 256, 0, s>>>(
            t->n, t->n_nodes, t->n_leaves, t->n_groups, t->perm, t->node_begin, t->node_count, t->child_begin,
            t->child_count, t->leaf_ids, t->parent, t->group_begin, t->group_count, t->group_order, t->soff,
            t->sbytes, t->max_len, bad.p);
        CT_COUNT_LAUNCH();
        CT_LAUNCH_CHECK();
    }
    int32_t hb = 0;
    to_host(&hb, bad.p, 1, s);
    if (hb) CT_FAIL(CT_EINVAL, "%s: an index of the tree is out of range", path);
    CT_CHECK_CUDA(cudaStreamSynchronize(s));
    g.t = nullptr;
    return t;
}

}  // namespace ct
