// tc.cu -- tensor-core self-test: one kind::f16 MMA chain (M = 128, N = 32,
// K = 128; bf16 or fp16 operands) through shared-memory descriptors and tensor
// memory, the primitive of the precision-1 leaf filter.
#include "common.cuh"
#include "tc.cuh"

namespace ct {
namespace {

__global__ void __launch_bounds__(128) k_tc_selftest(const uint16_t *__restrict__ A, const uint16_t *__restrict__ B,
                                                     int fp16, float *__restrict__ D, int32_t *__restrict__ status,
                                                     int withhold) {
    __shared__ __align__(1024) unsigned char sA[128 * 256];
    __shared__ __align__(1024) unsigned char sB[32 * 256];
    __shared__ uint32_t tslot;
    __shared__ __align__(8) uint64_t mbar;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < 128 * 16; i += 128) {
        const int r = i >> 4, k8 = i & 15;
        *reinterpret_cast<uint4 *>(sA + tc::core_offset(r, k8)) =
            *reinterpret_cast<const uint4 *>(A + (size_t)r * 128 + k8 * 8);
    }
    for (int i = tid; i < 32 * 16; i += 128) {
        const int r = i >> 4, k8 = i & 15;
        *reinterpret_cast<uint4 *>(sB + tc::core_offset(r, k8)) =
            *reinterpret_cast<const uint4 *>(B + (size_t)r * 128 + k8 * 8);
    }
    if (warp == 0) tc::tmem_alloc(&tslot, 32);
    if (tid == 0) tc::mbar_init(&mbar, 1);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    if (tid == 0 && !withhold) {  // withheld (a test): no MMA and no commit, so the wait below runs out
        const uint32_t idesc = fp16 ? tc::idesc_f16_f32(128, 32) : tc::idesc_bf16_f32(128, 32);
        for (int s = 0; s < 8; ++s) {
            const uint64_t ad = tc::smem_desc(tc::smem_u32(sA) + s * 256, tc::kLBO, tc::kSBO);
            const uint64_t bd = tc::smem_desc(tc::smem_u32(sB) + s * 256, tc::kLBO, tc::kSBO);
            tc::mma_bf16(tmem, ad, bd, idesc, s > 0);
        }
        tc::mma_commit(&mbar);
    }
    const bool ok = tc::mbar_wait(&mbar, 0, 1u << 20);
    tc::fence_after_sync();
    if (__all_sync(0xffffffffu, ok)) {
        float v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16), v);
#pragma unroll
        for (int j = 0; j < 32; ++j) D[(size_t)(32 * warp + lane) * 32 + j] = v[j];
    } else if (lane == 0) {
        atomicOr(status, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 32);
}

}  // namespace

void tc_selftest(const void *A, const void *B, int fp16, float *D, cudaStream_t s, int withhold) {
    DBuf<int32_t> status(1, s);
    CT_CHECK_CUDA(cudaMemsetAsync(status.p, 0, sizeof(int32_t), s));
    k_tc_selftest<<<1, 128, 0, s>>>((const uint16_t *)A, (const uint16_t *)B, fp16, D, status.p, withhold);
    CT_COUNT_LAUNCH();
    CT_LAUNCH_CHECK();
    int32_t h = 0;
    to_host(&h, status.p, 1, s);
    if (h) CT_FAIL(CT_ETIMEOUT, "tensor-core completion wait gave up");
}

}  // namespace ct
