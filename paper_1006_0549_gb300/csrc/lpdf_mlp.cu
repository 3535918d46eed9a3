// BF16 tensor-core (tcgen05) kernels of the learned relaxation surrogate.
//
// gemm_kernel: D (M x N, FP32) = A (M x K, BF16, row-major) * B (N x K, BF16, row-major)^T, one
// CTA (one warpgroup) per 128-row tile of A: the tile and B are staged in shared memory in the
// core-matrix layout, thread 0 issues the K / 16 MMAs into TMEM, the mbarrier of the commit
// releases the warpgroup, and each thread reads its row of D from its TMEM lane.
#include <cuda_runtime.h>

#include "lpdf_device.cuh"
#include "lpdf_internal.h"
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

// ==========================================================================================
// The surrogate network: 8 -> 128 -> 128 -> 128 -> 7, tanh, on 128-row tiles (layouts in
// lpdf_internal.h, namespace mlp).
// ==========================================================================================
namespace lpdf {

namespace {

using namespace mlp;

// element (r, k) of a row-major BF16 matrix (R x K) staged in the core layout, all threads
__device__ __forceinline__ void stage(unsigned char* dst, const __nv_bfloat16* __restrict__ src, int R, int K)
{
    for (int i = threadIdx.x; i < R * K; i += blockDim.x) {
        const int r = i / K, k = i - (i / K) * K;
        *reinterpret_cast<__nv_bfloat16*>(dst + tc::core_offset(r, k, K)) = src[i];
    }
}

__device__ __forceinline__ void put(unsigned char* dst, int r, int k, int K, float v)
{
    *reinterpret_cast<__nv_bfloat16*>(dst + tc::core_offset(r, k, K)) = __float2bfloat16(v);
}

// issue a GEMM from thread 0, wait (bounded) for it, order the TMEM reads after it
__device__ __forceinline__ bool gemm_sync(uint32_t tmem, const void* A, const void* B, int N, int K,
                                          unsigned long long* bar, uint32_t& phase, unsigned* error)
{
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x == 0) tc::gemm_issue(tmem, A, B, N, K, bar);
    bool ok = tc::mbar_wait(bar, phase);
    if (!ok) {
        atomicOr(error, 1u);
        ok = tc::mbar_wait(bar, phase);
    }
    phase ^= 1u;
    tc::fence_after_sync();
    return ok;
}

__device__ __forceinline__ uint32_t lane_addr(uint32_t tmem, int col)
{
    return tmem + ((uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16) + (uint32_t)col;
}

struct FwdSmem {
    alignas(1024) unsigned char x[kH * kInP * 2];
    alignas(1024) unsigned char h[kH * kH * 2];
    alignas(1024) unsigned char w1[kH * kInP * 2];
    alignas(1024) unsigned char w2[kH * kH * 2];
    alignas(1024) unsigned char w3[kH * kH * 2];
    alignas(1024) unsigned char w4[kOutP * kH * 2];
    float b[3 * kH + kOutP];
    unsigned long long bar;
    uint32_t tmem;
};

// Forward on rows [128 blockIdx, +128): feat (B x 8, FP32) standardised with the feature means and
// deviations of norm; out (may be NULL: B x 16, FP32, the 7 standardised outputs, then zeros);
// out_user (may be NULL: B x 7, the outputs in target units); with act != NULL also the three
// hidden activations (B x 128 BF16 each, for the backward pass).
__global__ void __launch_bounds__(kH, 1) mlp_fwd_kernel(const float* __restrict__ feat, int64_t B,
                                                        const float* __restrict__ P, const __nv_bfloat16* __restrict__ pack,
                                                        const float* __restrict__ norm, float* __restrict__ out,
                                                        float* __restrict__ out_user, __nv_bfloat16* __restrict__ act,
                                                        unsigned* __restrict__ error)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    FwdSmem& sm = *reinterpret_cast<FwdSmem*>(smem_raw);
    const int t = threadIdx.x, wid = t >> 5;
    const int64_t row = (int64_t)blockIdx.x * kH + t;
    stage(sm.w1, pack + pW1, kH, kInP);
    stage(sm.w2, pack + pW2, kH, kH);
    stage(sm.w3, pack + pW3, kH, kH);
    stage(sm.w4, pack + pW4, kOutP, kH);
    for (int i = t; i < 3 * kH; i += kH) sm.b[i] = P[(i < kH ? ob1 : (i < 2 * kH ? ob2 - kH : ob3 - 2 * kH)) + i];
    if (t < kOutP) sm.b[3 * kH + t] = P[ob4 + t];
    for (int k = 0; k < kInP; ++k) {
        float v = 0.0f;
        if (k < kIn && row < B) v = (feat[row * kIn + k] - norm[nFM + k]) / norm[nFS + k];
        put(sm.x, t, k, kInP, v);
    }
    if (wid == 0) {
        tc::tmem_alloc(&sm.tmem, kH);
        tc::tmem_relinquish();
    }
    if (t == 0) tc::mbar_init1(&sm.bar);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = sm.tmem;
    uint32_t phase = 0;
    bool ok = true;
    const unsigned char* a_op = sm.x;
    int K = kInP;
    const unsigned char* w_op[3] = {sm.w1, sm.w2, sm.w3};
    for (int l = 0; l < 3 && ok; ++l) {
        ok = gemm_sync(tmem, a_op, w_op[l], kH, K, &sm.bar, phase, error);
        if (!ok) break;
        for (int c0 = 0; c0 < kH; c0 += 16) {
            float v[16];
            tc::tmem_ld16(lane_addr(tmem, c0), v);
            tc::wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float a = tanhf(v[j] + sm.b[l * kH + c0 + j]);
                const __nv_bfloat16 ab = __float2bfloat16(a);
                *reinterpret_cast<__nv_bfloat16*>(sm.h + tc::core_offset(t, c0 + j, kH)) = ab;
                if (act && row < B) act[((size_t)l * B + row) * kH + c0 + j] = ab;
            }
        }
        a_op = sm.h;
        K = kH;
    }
    if (ok) ok = gemm_sync(tmem, sm.h, sm.w4, kOutP, kH, &sm.bar, phase, error);
    if (ok) {
        float v[16];
        tc::tmem_ld16(lane_addr(tmem, 0), v);
        tc::wait_ld();
        if (row < B && out)
#pragma unroll
            for (int j = 0; j < kOutP; ++j) out[row * kOutP + j] = j < kOut ? v[j] + sm.b[3 * kH + j] : 0.0f;
        if (row < B && out_user)
#pragma unroll
            for (int j = 0; j < kOut; ++j) out_user[row * kOut + j] = (v[j] + sm.b[3 * kH + j]) * norm[nTS + j] + norm[nTM + j];
    }
    tc::fence_before_sync();
    __syncthreads();
    if (wid == 0) tc::tmem_dealloc(tmem, kH);
}

struct BwdSmem {
    alignas(1024) unsigned char sat[kH * kH * 2];   // A operand, transposed activations [in][batch]
    alignas(1024) unsigned char sbt[kH * kH * 2];   // B operand, transposed dZ [out][batch]
    alignas(1024) unsigned char sar[kH * kH * 2];   // A operand, dZ rows [batch][out]
    alignas(1024) unsigned char t2[kH * kH * 2];    // W2^T [in][out]
    alignas(1024) unsigned char t3[kH * kH * 2];
    alignas(1024) unsigned char t4[kH * kOutP * 2];
    float wpart[4][kH];                             // per-warp column sums (bias gradients)
    unsigned long long bar;
    uint32_t tmem;
};

// column sums of v[0..15] (this thread's row, columns c0..c0+15) over the CTA, added to acc[c0..]
__device__ __forceinline__ void colsum16(float (*wpart)[kH], const float* v, int c0)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        float s = v[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) wpart[wid][c0 + j] = s;
    }
}

// Backward on rows [128 blockIdx, +128) of a batch of B rows: the gradient of the mean squared
// error over the 7 standardised outputs (weights w[7]) with respect to every parameter, as this
// CTA's partial sums (W^T layouts).
__global__ void __launch_bounds__(kH, 1) mlp_bwd_kernel(const float* __restrict__ feat, const float* __restrict__ tgt,
                                                        int64_t B, const __nv_bfloat16* __restrict__ pack,
                                                        const float* __restrict__ norm, const float* __restrict__ out,
                                                        const __nv_bfloat16* __restrict__ act,
                                                        float* __restrict__ part, unsigned* __restrict__ error)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    BwdSmem& sm = *reinterpret_cast<BwdSmem*>(smem_raw);
    const int t = threadIdx.x, wid = t >> 5;
    const int64_t row = (int64_t)blockIdx.x * kH + t;
    const bool live = row < B;
    float* const pp = part + (size_t)blockIdx.x * kPart;
    stage(sm.t2, pack + pT2, kH, kH);
    stage(sm.t3, pack + pT3, kH, kH);
    stage(sm.t4, pack + pT4, kH, kOutP);
    // dZ4 = d loss / d out: 2 (out - target) w_j / (7 B)
    float dz4[kOutP];
#pragma unroll
    for (int j = 0; j < kOutP; ++j) {
        float d = 0.0f;
        if (live && j < kOut) {
            const float y = (tgt[row * kOut + j] - norm[nTM + j]) / norm[nTS + j];
            d = 2.0f * (out[row * kOutP + j] - y) * norm[nW + j] / (float)(kOut * B);
        }
        dz4[j] = d;
    }
    colsum16(sm.wpart, dz4, 0);
    // dW4^T = A3^T dZ4: A = A3^T [in][batch], B = dZ4^T [out][batch]
    const __nv_bfloat16* a3 = act + (2 * (size_t)B + (live ? row : 0)) * kH;
    for (int i = 0; i < kH; ++i)
        *reinterpret_cast<__nv_bfloat16*>(sm.sat + tc::core_offset(i, t, kH)) = live ? a3[i] : __float2bfloat16(0.0f);
#pragma unroll
    for (int j = 0; j < kOutP; ++j) {
        put(sm.sbt, j, t, kH, dz4[j]);
        put(sm.sar, t, j, kOutP, dz4[j]);
    }
    if (wid == 0) {
        tc::tmem_alloc(&sm.tmem, kH);
        tc::tmem_relinquish();
    }
    if (t == 0) tc::mbar_init1(&sm.bar);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t < kOutP) pp[gb4 + t] = sm.wpart[0][t] + sm.wpart[1][t] + sm.wpart[2][t] + sm.wpart[3][t];
    const uint32_t tmem = sm.tmem;
    uint32_t phase = 0;
    bool ok = gemm_sync(tmem, sm.sat, sm.sbt, kOutP, kH, &sm.bar, phase, error);
    if (ok) {
        float v[16];
        tc::tmem_ld16(lane_addr(tmem, 0), v);
        tc::wait_ld();
#pragma unroll
        for (int j = 0; j < kOutP; ++j) pp[gW4 + t * kOutP + j] = v[j];
    }
    // hidden layers 3, 2, 1: dH = dZ W (A = dZ rows, B = W^T), dZ = dH (1 - a^2),
    // dW^T = A_prev^T dZ, bias gradient = column sums of dZ
    const unsigned char* tw[3] = {sm.t4, sm.t3, sm.t2};
    const int kw[3] = {kOutP, kH, kH};
    const int gw[3] = {gW3, gW2, gW1};
    const int gb[3] = {gb3, gb2, gb1};
    for (int s = 0; s < 3 && ok; ++s) {
        const int l = 2 - s;                       // hidden layer index (0-based) whose dZ is formed
        tc::fence_before_sync();
        ok = gemm_sync(tmem, sm.sar, tw[s], kH, kw[s], &sm.bar, phase, error);
        if (!ok) break;
        const __nv_bfloat16* al = act + ((size_t)l * B + (live ? row : 0)) * kH;
        for (int c0 = 0; c0 < kH; c0 += 16) {
            float v[16];
            tc::tmem_ld16(lane_addr(tmem, c0), v);
            tc::wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float a = live ? __bfloat162float(al[c0 + j]) : 0.0f;
                v[j] = live ? v[j] * (1.0f - a * a) : 0.0f;
                put(sm.sbt, c0 + j, t, kH, v[j]);
                put(sm.sar, t, c0 + j, kH, v[j]);
            }
            colsum16(sm.wpart, v, c0);
        }
        // A operand: the previous activations transposed (the standardised inputs for layer 1)
        if (l > 0) {
            const __nv_bfloat16* ap = act + ((size_t)(l - 1) * B + (live ? row : 0)) * kH;
            for (int i = 0; i < kH; ++i)
                *reinterpret_cast<__nv_bfloat16*>(sm.sat + tc::core_offset(i, t, kH)) =
                    live ? ap[i] : __float2bfloat16(0.0f);
        } else {
            for (int i = 0; i < kH; ++i) {
                float x = 0.0f;
                if (i < kIn && live) x = (feat[row * kIn + i] - norm[nFM + i]) / norm[nFS + i];
                put(sm.sat, i, t, kH, x);
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        pp[gb[s] + t] = sm.wpart[0][t] + sm.wpart[1][t] + sm.wpart[2][t] + sm.wpart[3][t];
        ok = gemm_sync(tmem, sm.sat, sm.sbt, kH, kH, &sm.bar, phase, error);
        if (!ok) break;
        // the loads are warp-collective: every thread loads, the rows that exist are stored
        const bool keep = t < (l > 0 ? kH : kInP);
        for (int c0 = 0; c0 < kH; c0 += 16) {
            float v[16];
            tc::tmem_ld16(lane_addr(tmem, c0), v);
            tc::wait_ld();
            if (keep)
#pragma unroll
                for (int j = 0; j < 16; ++j) pp[gw[s] + t * kH + c0 + j] = v[j];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (wid == 0) tc::tmem_dealloc(tmem, kH);
}

// grad (padded parameter layout) = the sum of the CTA partials in CTA order
__global__ void mlp_reduce_kernel(const float* __restrict__ part, int nparts, float* __restrict__ grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    int src;   // the partial that holds parameter i
    if (i < ob1) { const int o = i / kInP, k = i % kInP; src = gW1 + k * kH + o; }
    else if (i < oW2) src = gb1 + (i - ob1);
    else if (i < ob2) { const int j = i - oW2, o = j / kH, k = j % kH; src = gW2 + k * kH + o; }
    else if (i < oW3) src = gb2 + (i - ob2);
    else if (i < ob3) { const int j = i - oW3, o = j / kH, k = j % kH; src = gW3 + k * kH + o; }
    else if (i < oW4) src = gb3 + (i - ob3);
    else if (i < ob4) { const int j = i - oW4, o = j / kH, k = j % kH; src = gW4 + k * kOutP + o; }
    else src = gb4 + (i - ob4);
    double s = 0.0;
    for (int c = 0; c < nparts; ++c) s += part[(size_t)c * kPart + src];
    grad[i] = (float)s;
}

// parameters that exist (the padding stays zero)
__device__ __forceinline__ bool is_param(int i)
{
    if (i < ob1) return i % kInP < kIn;
    if (i >= oW4 && i < ob4) return (i - oW4) / kH < kOut;
    if (i >= ob4) return i - ob4 < kOut;
    return true;
}

// Adam step (t = step number from 1), then the BF16 packs
__global__ void mlp_adam_kernel(float* __restrict__ P, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, float lr, float b1, float b2, float eps, int step,
                                __nv_bfloat16* __restrict__ pack)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    float p = P[i];
    if (step > 0 && is_param(i)) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / (1.0f - powf(b1, (float)step)), vh = vi / (1.0f - powf(b2, (float)step));
        p -= lr * mh / (sqrtf(vh) + eps);
        P[i] = p;
    }
    if (!is_param(i)) {
        P[i] = 0.0f;
        p = 0.0f;
    }
    const __nv_bfloat16 pb = __float2bfloat16(p);
    if (i < ob1) {
        pack[pW1 + i] = pb;
    } else if (i >= oW2 && i < ob2) {
        const int j = i - oW2, o = j / kH, k = j % kH;
        pack[pW2 + j] = pb;
        pack[pT2 + k * kH + o] = pb;
    } else if (i >= oW3 && i < ob3) {
        const int j = i - oW3, o = j / kH, k = j % kH;
        pack[pW3 + j] = pb;
        pack[pT3 + k * kH + o] = pb;
    } else if (i >= oW4 && i < ob4) {
        const int j = i - oW4, o = j / kH, k = j % kH;
        pack[pW4 + j] = pb;
        pack[pT4 + k * kOutP + o] = pb;
    }
}

// loss[0] = the weighted mean squared error over the 7 standardised outputs (one block)
__global__ void mlp_loss_kernel(const float* __restrict__ out, const float* __restrict__ tgt, int64_t B,
                                const float* __restrict__ norm, double* __restrict__ loss)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < B; r += blockDim.x)
        for (int j = 0; j < kOut; ++j) {
            const double y = ((double)tgt[r * kOut + j] - norm[nTM + j]) / norm[nTS + j];
            const double d = (double)out[r * kOutP + j] - y;
            s += norm[nW + j] * d * d;
        }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss[0] = sh[0] / (double)(kOut * B);
}

// column c of the data set (features 0..7, then targets 8..14): mean and deviation (one block each;
// a deviation below 1e-6 max(1, |mean|) is taken as 1, so a constant column stays finite)
__global__ void mlp_fit_norm_kernel(const float* __restrict__ feat, const float* __restrict__ tgt, int64_t B,
                                    float* __restrict__ norm)
{
    __shared__ double sh[2][256];
    const int c = blockIdx.x;
    const float* src = c < kIn ? feat + c : tgt + (c - kIn);
    const int ld = c < kIn ? kIn : kOut;
    double s = 0.0, q = 0.0;
    for (int64_t r = threadIdx.x; r < B; r += blockDim.x) {
        const double v = src[r * ld];
        s += v;
        q += v * v;
    }
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = q;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mean = sh[0][0] / (double)B;
        const double var = fmax(sh[1][0] / (double)B - mean * mean, 0.0);
        double sd = sqrt(var);
        if (!(sd >= 1e-6 * fmax(1.0, fabs(mean)))) sd = 1.0;
        if (c < kIn) {
            norm[nFM + c] = (float)mean;
            norm[nFS + c] = (float)sd;
        } else {
            norm[nTM + c - kIn] = (float)mean;
            norm[nTS + c - kIn] = (float)sd;
        }
    }
}

}  // namespace

cudaError_t mlp_configure()
{
    cudaError_t e = cudaFuncSetAttribute(mlp_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FwdSmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BwdSmem));
    return e;
}

cudaError_t launch_mlp_forward(const float* feat, int64_t B, const float* P, const void* pack, const float* norm,
                               float* out, float* out_user, void* act, unsigned* error, cudaStream_t st)
{
    if (B <= 0) return cudaSuccess;
    mlp_fwd_kernel<<<(unsigned)((B + kH - 1) / kH), kH, sizeof(FwdSmem), st>>>(
        feat, B, P, static_cast<const __nv_bfloat16*>(pack), norm, out, out_user, static_cast<__nv_bfloat16*>(act),
        error);
    return cudaGetLastError();
}

cudaError_t launch_mlp_backward(const float* feat, const float* tgt, int64_t B, const void* pack, const float* norm,
                                const float* out, const void* act, float* part, float* grad, unsigned* error,
                                cudaStream_t st)
{
    if (B <= 0) return cudaSuccess;
    const unsigned nb = (unsigned)((B + kH - 1) / kH);
    mlp_bwd_kernel<<<nb, kH, sizeof(BwdSmem), st>>>(feat, tgt, B, static_cast<const __nv_bfloat16*>(pack), norm, out,
                                                    static_cast<const __nv_bfloat16*>(act), part, error);
    mlp_reduce_kernel<<<(kParams + 255) / 256, 256, 0, st>>>(part, (int)nb, grad);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* P, const float* grad, float* m, float* v, float lr, int step, void* pack,
                            cudaStream_t st)
{
    mlp_adam_kernel<<<(kParams + 255) / 256, 256, 0, st>>>(P, grad, m, v, lr, 0.9f, 0.999f, 1e-8f, step,
                                                           static_cast<__nv_bfloat16*>(pack));
    return cudaGetLastError();
}

cudaError_t launch_mlp_loss(const float* out, const float* tgt, int64_t B, const float* norm, double* loss,
                            cudaStream_t st)
{
    mlp_loss_kernel<<<1, 256, 0, st>>>(out, tgt, B, norm, loss);
    return cudaGetLastError();
}

cudaError_t launch_mlp_fit_norm(const float* feat, const float* tgt, int64_t B, float* norm, cudaStream_t st)
{
    if (B <= 0) return cudaSuccess;
    mlp_fit_norm_kernel<<<kIn + kOut, 256, 0, st>>>(feat, tgt, B, norm);
    return cudaGetLastError();
}

}  // namespace lpdf
