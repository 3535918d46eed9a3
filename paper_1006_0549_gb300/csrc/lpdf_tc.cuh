// Fifth-generation tensor cores (tcgen05, sm_100a family) for the BF16 MLP of the learned
// relaxation surrogate: shared-memory matrix descriptors, the instruction descriptor, TMEM
// allocation and loads, MMA issue and completion through an mbarrier. Inline PTX only.
//
// Operand layout in shared memory: K-major, no swizzle. A matrix of R rows and K columns (BF16)
// is cut into core matrices of 8 rows x 8 columns (8 rows of 16 bytes, 128 bytes contiguous);
// core (r / 8, k / 8) starts at ((r / 8) * (K / 8) + k / 8) * 128 bytes. So the core next along
// K is 128 bytes away (leading-dimension byte offset) and the core next along the rows is
// (K / 8) * 128 bytes away (stride-dimension byte offset).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace lpdf {
namespace tc {

// byte offset of element (r, k) in the core-matrix layout of a matrix with K columns
__device__ __forceinline__ uint32_t core_offset(int r, int k, int K)
{
    return (uint32_t)((((r >> 3) * (K >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor (no swizzle): start address, leading and stride byte offsets
// (all in 16-byte units), descriptor version 1 at bits 46-47, layout type 0 (no swizzle)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9 and 10-12 = 1),
// both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// TMEM allocation by one warp: the base address is written to *slot (shared memory)
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A * B^T, A: M x 16 and B: N x 16 through their descriptors
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         bool accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}

// the MMAs issued so far by this thread arrive on the mbarrier when complete
__device__ __forceinline__ void mma_commit(unsigned long long* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane (32x32b shape: warp w of the warpgroup
// reads lanes 32 (w % 4) .. + 31, thread t lane 32 (w % 4) + t)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void mbar_init1(unsigned long long* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// bounded wait on phase `parity`: false when it gave up
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity)
{
#pragma unroll 1
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// One GEMM tile: D (128 x N, FP32 in TMEM at d_tmem) = A (128 x K) * B (N x K)^T, both in the
// core-matrix layout, issued by the calling (single) thread: K / 16 MMAs, then a commit.
__device__ __forceinline__ void gemm_issue(uint32_t d_tmem, const void* A, const void* B, int N, int K,
                                           unsigned long long* bar)
{
    const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
    const uint32_t sbo = (uint32_t)(K / 8) * 128u;
    const uint32_t idesc = idesc_bf16(128, N);
    for (int s = 0; s < K / 16; ++s) {
        // K-slice s: two cores along K, 256 bytes further
        const uint64_t ad = smem_desc(a0 + 256u * s, 128u, sbo);
        const uint64_t bd = smem_desc(b0 + 256u * s, 128u, sbo);
        mma_bf16(d_tmem, ad, bd, idesc, s > 0);
    }
    mma_commit(bar);
}

}  // namespace tc
}  // namespace lpdf
