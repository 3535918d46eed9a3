// BF16 tensor-core (tcgen05) kernels of the learned relaxation surrogate.
//
// gemm_kernel: D (M x N, FP32) = A (M x K, BF16, row-major) * B (N x K, BF16, row-major)^T, one
// CTA (one warpgroup) per 128-row tile of A: the tile and B are staged in shared memory in the
// core-matrix layout, thread 0 issues the K / 16 MMAs into TMEM, the mbarrier of the commit
// releases the warpgroup, and each thread reads its row of D from its TMEM lane.
#include <cuda_runtime.h>

#include "lpdf_device.cuh"
#include "lpdf_tc.cuh"

namespace lpdf {

namespace {

constexpr int kTile = 128;              // rows per CTA (TMEM lanes)
constexpr int kMaxK = 128;
constexpr int kMaxN = 256;

struct GemmSmem {
    alignas(1024) unsigned char a[kTile * kMaxK * 2];
    alignas(1024) unsigned char b[kMaxN * kMaxK * 2];
    unsigned long long bar;
    uint32_t tmem;
};

__host__ __device__ inline uint32_t tmem_cols(int n)
{
    uint32_t c = 32;
    while ((int)c < n) c <<= 1;
    return c;
}

__global__ void __launch_bounds__(kTile, 1) gemm_kernel(const __nv_bfloat16* __restrict__ A,
                                                        const __nv_bfloat16* __restrict__ B, float* __restrict__ D,
                                                        int M, int N, int K, unsigned* __restrict__ error)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    GemmSmem& sm = *reinterpret_cast<GemmSmem*>(smem_raw);
    const int tid = threadIdx.x, wid = tid >> 5;
    const int r0 = blockIdx.x * kTile;
    // stage the operands (BF16, core-matrix layout)
    for (int i = tid; i < kTile * K; i += kTile) {
        const int r = i / K, k = i - (i / K) * K;
        const __nv_bfloat16 v = r0 + r < M ? A[(size_t)(r0 + r) * K + k] : __float2bfloat16(0.0f);
        *reinterpret_cast<__nv_bfloat16*>(sm.a + tc::core_offset(r, k, K)) = v;
    }
    for (int i = tid; i < N * K; i += kTile) {
        const int r = i / K, k = i - (i / K) * K;
        *reinterpret_cast<__nv_bfloat16*>(sm.b + tc::core_offset(r, k, K)) = B[(size_t)r * K + k];
    }
    const uint32_t ncols = tmem_cols(N);
    if (wid == 0) {
        tc::tmem_alloc(&sm.tmem, ncols);
        tc::tmem_relinquish();
    }
    if (tid == 0) tc::mbar_init1(&sm.bar);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = sm.tmem;
    if (tid == 0) tc::gemm_issue(tmem, sm.a, sm.b, N, K, &sm.bar);
    bool ok = tc::mbar_wait(&sm.bar, 0);
    if (!ok) {
        atomicOr(error, 1u);
        ok = tc::mbar_wait(&sm.bar, 0);   // the MMAs in flight once more, then stop
    }
    tc::fence_after_sync();
    if (ok) {
        const int row = r0 + tid;
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(32 * (wid & 3)) << 16) + (uint32_t)c0, v);
            tc::wait_ld();
            if (row < M)
#pragma unroll
                for (int j = 0; j < 16; ++j) D[(size_t)row * N + c0 + j] = v[j];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (wid == 0) tc::tmem_dealloc(tmem, ncols);
}

}  // namespace

cudaError_t launch_tc_gemm(const void* A, const void* B, float* D, int M, int N, int K, unsigned* error,
                           cudaStream_t st)
{
    if (M <= 0 || N < 16 || N > kMaxN || N % 16 || K < 16 || K > kMaxK || K % 16) return cudaErrorInvalidValue;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(GemmSmem));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    gemm_kernel<<<(unsigned)((M + kTile - 1) / kTile), kTile, sizeof(GemmSmem), st>>>(
        static_cast<const __nv_bfloat16*>(A), static_cast<const __nv_bfloat16*>(B), D, M, N, K, error);
    return cudaGetLastError();
}

}  // namespace lpdf
