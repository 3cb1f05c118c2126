// Tensor-core (tcgen05) contractions of the seed network.
//
// osmodi_tc_gemm: a plain D = A B^T on the 5th-generation tensor cores --
// the building block of the network's convolutions, exposed as a step-level
// entry point so that the operand layout, the descriptors and the
// tensor-memory epilogue can be checked against a reference GEMM.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.cuh"
#include "tc.cuh"

namespace osm {
namespace {

typedef __nv_bfloat16 bf16;

constexpr long long kMbarPolls = 1LL << 22;  // bounded wait for the MMAs (~0.1 s)

// D[128][N] = A[128][K] B[N][K]^T; A, B BF16 with K contiguous, D FP32 row-major.
// One CTA of 128 threads: operands copied to shared memory in the K-major
// core-matrix layout, K / 16 MMAs issued by thread 0 into tensor memory,
// completion through an mbarrier, then every warp reads its 32 rows.
__global__ void __launch_bounds__(128) k_tc_gemm(const bf16* __restrict__ A, const bf16* __restrict__ B,
                                                float* __restrict__ D, int N, int K, int* err) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tbase;
    unsigned char* sA = smem;                         // 128 x K
    unsigned char* sB = smem + (size_t)128 * K * 2;   // N x K
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    uint32_t ncols = 32;
    while ((int)ncols < N) ncols <<= 1;
    if (warp == 0) {
        tc::tmem_alloc(&tbase, ncols);
        tc::tmem_relinquish();
    }
    if (t == 0) {
        tc::mbar_init(&mbar, 1);
        tc::mbar_fence_init();
    }
    // operands -> canonical layout (16-byte pieces: 8 values of K)
    const int kg = K / 8;
    for (int q = t; q < 128 * kg; q += 128) {
        const int m = q / kg, g = q % kg;
        const uint4 v = *reinterpret_cast<const uint4*>(A + (size_t)m * K + g * 8);
        *reinterpret_cast<uint4*>(sA + (size_t)g * 2048 + (m >> 3) * 128 + (m & 7) * 16) = v;
    }
    for (int q = t; q < N * kg; q += 128) {
        const int n = q / kg, g = q % kg;
        const uint4 v = *reinterpret_cast<const uint4*>(B + (size_t)n * K + g * 8);
        *reinterpret_cast<uint4*>(sB + (size_t)g * N * 16 + (n >> 3) * 128 + (n & 7) * 16) = v;
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tbase;
    if (t == 0) {
        const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
        const uint32_t id = tc::idesc_bf16_f32(128, N);
        for (int s = 0; s < K / 16; ++s) {
            const uint64_t ad = tc::sdesc(a0 + (uint32_t)s * 2 * 2048, 2048, 128);
            const uint64_t bd = tc::sdesc(b0 + (uint32_t)s * 2 * N * 16, (uint32_t)N * 16, 128);
            tc::mma_bf16(taddr, ad, bd, id, s > 0 ? 1u : 0u);
        }
        tc::mma_commit(&mbar);
    }
    const bool done = tc::mbar_wait(&mbar, 0, kMbarPolls);
    tc::fence_after_sync();
    if (!done) {
        if (lane == 0) atomicExch(err, 1);
    } else {
        const int row = warp * 32 + lane;
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) D[(size_t)row * N + c0 + i] = v[i];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, ncols);
}

}  // namespace
}  // namespace osm

extern "C" osmodi_status osmodi_tc_gemm(const void* A_dev, const void* B_dev, float* D_dev, int N, int K,
                                        int* err_dev, void* stream) {
    using namespace osm;
    if (!A_dev || !B_dev || !D_dev || !err_dev) return OSMODI_E_INVALID;
    if (N < 16 || N > 256 || N % 16 || K < 16 || K > 256 || K % 16) return OSMODI_E_INVALID;
    if (((uintptr_t)A_dev | (uintptr_t)B_dev) & 15u) return OSMODI_E_INVALID;
    const size_t smem = (size_t)(128 + N) * K * 2;
    OSM_CUDA(cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_tc_gemm<<<1, 128, smem, (cudaStream_t)stream>>>((const bf16*)A_dev, (const bf16*)B_dev, D_dev, N, K, err_dev);
    OSM_CUDA(cudaGetLastError());
    return OSMODI_OK;
}
