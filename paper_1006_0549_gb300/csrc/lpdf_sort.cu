// Element re-bucketing of the particle ensemble (keeps the particles of one element contiguous,
// so that a warp tile of the step kernel covers few elements).
//
// Deterministic counting sort by element: the result is ordered by (element, previous index),
// whatever the order in which the atomic scatter placed the indices:
//   1. count the particles of every element (warp-aggregated integer atomics); a particle with an
//      element id outside the mesh goes to an extra last bucket, so that every index is placed;
//   2. exclusive scan of the counts (one CTA);
//   3. scatter every particle's index into its element's bucket (atomic cursor);
//   4. sort each bucket ascending (bitonic sort in shared memory, one CTA per element);
//   5. gather every state row through the permutation into the second buffer.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lpdf_internal.h"

namespace lpdf {

namespace {

constexpr unsigned kFullMask = 0xffffffffu;

__global__ void count_kernel(const int* __restrict__ elem, int64_t n, int n_tri, int* __restrict__ cnt,
                             unsigned long long* __restrict__ status)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int e = -1;
    if (i < n) {
        e = elem[i];
        if ((unsigned)e >= (unsigned)n_tri) {
            atomicOr(&status[0], (unsigned long long)kErrLost);
            e = n_tri;
        }
    }
    const unsigned m = __match_any_sync(kFullMask, e);
    const int leader = __ffs(m) - 1;
    if (e >= 0 && (int)(threadIdx.x & 31) == leader) atomicAdd(&cnt[e], __popc(m));
}

// exclusive scan of cnt[0..n) into start[0..n], one CTA of 1024 threads
__global__ void scan_kernel(const int* __restrict__ cnt, int n, int* __restrict__ start)
{
    __shared__ int part[1024];
    const int t = threadIdx.x;
    const int chunk = (n + 1023) / 1024;
    const int b = t * chunk, e = min(n, b + chunk);
    int s = 0;
    for (int i = b; i < e; ++i) s += cnt[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - s;
    for (int i = b; i < e; ++i) {
        start[i] = run;
        run += cnt[i];
    }
    if (t == 1023) start[n] = part[1023];
}

__global__ void scatter_kernel(const int* __restrict__ elem, int64_t n, int n_tri, const int* __restrict__ start,
                               int* __restrict__ cursor, int* __restrict__ perm)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int e = -1;
    if (i < n) {
        e = elem[i];
        if ((unsigned)e >= (unsigned)n_tri) e = n_tri;
    }
    const unsigned m = __match_any_sync(kFullMask, e);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (e >= 0 && lane == leader) base = atomicAdd(&cursor[e], __popc(m));
    base = __shfl_sync(kFullMask, base, leader);
    if (e >= 0) perm[start[e] + base + __popc(m & ((1u << lane) - 1u))] = (int)i;
}

// one CTA per element: sort its bucket of previous indices ascending (bitonic, shared memory)
constexpr int kSegMax = 8192;

__global__ void segment_sort_kernel(const int* __restrict__ start, int* __restrict__ perm,
                                    unsigned long long* __restrict__ status)
{
    __shared__ int v[kSegMax];
    const int e = blockIdx.x;
    const int b = start[e], len = start[e + 1] - b;
    if (len <= 1) return;
    if (len > kSegMax) {
        if (threadIdx.x == 0) atomicOr(&status[0], (unsigned long long)kErrOverflow);
        return;
    }
    int p2 = 1;
    while (p2 < len) p2 <<= 1;
    for (int i = threadIdx.x; i < p2; i += blockDim.x) v[i] = i < len ? perm[b + i] : INT_MAX;
    __syncthreads();
    for (int k = 2; k <= p2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < p2; i += blockDim.x) {
                const int ij = i ^ j;
                if (ij > i) {
                    const int a = v[i], c = v[ij];
                    const bool up = (i & k) == 0;
                    if ((a > c) == up) { v[i] = c; v[ij] = a; }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < len; i += blockDim.x) perm[b + i] = v[i];
}

template <class T>
__global__ void gather_kernel(const T* __restrict__ src, T* __restrict__ dst, const int* __restrict__ perm, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[perm[i]];
}

}  // namespace

cudaError_t launch_sort(const DevMesh& m, const DevState& s, int ns, const DevState& dst, SortScratch& w,
                        unsigned long long* status, cudaStream_t st)
{
    if (s.n == 0) return cudaSuccess;
    const int E = m.n_tri;
    // buckets 0..E-1 are the elements, bucket E collects invalid element ids
    cudaError_t e = cudaMemsetAsync(w.cnt, 0, sizeof(int) * (size_t)(E + 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.cursor, 0, sizeof(int) * (size_t)(E + 1), st);
    if (e != cudaSuccess) return e;
    const unsigned g = (unsigned)((s.n + 255) / 256);
    count_kernel<<<g, 256, 0, st>>>(s.elem, s.n, E, w.cnt, status);
    scan_kernel<<<1, 1024, 0, st>>>(w.cnt, E + 1, w.start);
    scatter_kernel<<<g, 256, 0, st>>>(s.elem, s.n, E, w.start, w.cursor, w.perm);
    segment_sort_kernel<<<E + 1, 256, 0, st>>>(w.start, w.perm, status);
    const int64_t nblk = (s.n + 255) / 256;
    const unsigned gg = (unsigned)(nblk < 152 * 16 ? nblk : 152 * 16);
    gather_kernel<float><<<gg, 256, 0, st>>>(s.x, dst.x, w.perm, s.n);
    gather_kernel<float><<<gg, 256, 0, st>>>(s.y, dst.y, w.perm, s.n);
    gather_kernel<float><<<gg, 256, 0, st>>>(s.u, dst.u, w.perm, s.n);
    gather_kernel<float><<<gg, 256, 0, st>>>(s.v, dst.v, w.perm, s.n);
    gather_kernel<float><<<gg, 256, 0, st>>>(s.w, dst.w, w.perm, s.n);
    gather_kernel<float><<<gg, 256, 0, st>>>(s.om, dst.om, w.perm, s.n);
    for (int a = 0; a < ns; ++a)
        gather_kernel<float><<<gg, 256, 0, st>>>(s.psi + (size_t)a * s.cap, dst.psi + (size_t)a * dst.cap, w.perm, s.n);
    gather_kernel<int><<<gg, 256, 0, st>>>(s.elem, dst.elem, w.perm, s.n);
    gather_kernel<uint32_t><<<gg, 256, 0, st>>>(s.pid, dst.pid, w.perm, s.n);
    return cudaGetLastError();
}

}  // namespace lpdf
