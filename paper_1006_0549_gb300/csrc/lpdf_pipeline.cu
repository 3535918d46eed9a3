// The particle time step as a pipeline that keeps the ensemble in element order (sm_103a).
//
// Per step (Section "Governing equations": Eq. 2, 4, 5, 6, 9, forward Euler,
// statistics at the gridpoints, tracking through the unstructured grid):
//   T   element_fields_kernel: the node fields in element form (per element: the fields at vertex
//       0 and their x and y gradients), so a particle interpolates without the node indirection.
//   K1  advance_kernel: thread i takes the particle perm[i] of the current buffer (perm lists the
//       buffer in element order), advances it (Eq. 4, 5, 9 (IEM, or IECM with a reactive source),
//       2, wrap, reflection, sources), locates it with the barycentric neighbour walk and writes it
//       to position i of the next buffer. No barriers: a thread's walk never waits for another's.
//   H   histogram_kernel: each 256-particle block of the next buffer counts its particles per new
//       element (a sparse histogram: one record per distinct element) and gives every particle
//       its rank among the block's particles of the same element, in position order.
//   S1  exclusive scans: particles per element -> bucket starts; records per element -> list starts.
//   S2  record_scatter_kernel (a warp per record block): every record joins its element's record
//       list.
//   S3  key_offsets_kernel (a warp per element): the element's records in block order, and each
//       record's offset = bucket start + the counts of the element's records in earlier blocks.
//   S4  particle_scatter_kernel: perm_new[offset(record) + rank] = i. perm_new lists the next
//       buffer in (new element, position) order: a stable counting sort, fully deterministic.
//   K2  moments_kernel (a warp per element; with at most kHalfPpe particles per element on
//       average, FP32 sums, a half-warp per element): the element's particles, gathered through
//       perm_new in canonical order, a fixed reduce-scatter across the lanes (recursive halving),
//       one 64-bit fixed-point atomic add per node and quantity. Two precisions (lpdf_params
//       moment_sums): 0, lambda_a' q_k in FP32 summed in FP32 per lane over at most kLaneChunk
//       particles; 1, per lane the sums of q, dx q and dy q ((dx, dy) from vertex 0) in
//       compensated FP32 (double-floats), combined in FP64 with the element's FP64 affine
//       barycentric coefficients.
// Every step leaves perm_new as the next step's perm, so the ensemble is re-bucketed by element
// every step without a separate sort, and the reduction never needs a hash or a binning pass.
#include <algorithm>
#include <atomic>

#include "lpdf_device.cuh"

namespace lpdf {

namespace {

constexpr int kBlk = 256;          // H: positions per record block
constexpr int kLaneChunk = 8;      // K2: particles a lane sums before the warp reduction
constexpr int kLaneChunkDf = 16;   // the same with compensated sums (its warp reduction costs more)
constexpr int kHalfPpe = 384;      // K2: at most this many particles per element on average -> half-warps
constexpr int kScanItems = 4;      // scan: items per thread
constexpr int kScanThreads = 1024;
constexpr int kScanTile = kScanItems * kScanThreads;

__device__ __forceinline__ unsigned rec_hash(int key) { return ((unsigned)key * 2654435761u) >> 24; }   // 8 bits

// ------------------------------------------------------------------------------------------
// K1
// ------------------------------------------------------------------------------------------
// The state streams through once per step: its loads skip L1 (which keeps the element field
// rows and mesh records that the particles of an element share) and its stores are marked
// streaming.
__device__ __forceinline__ float ld_stream(const float* p)
{
    float v;
    asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int ld_stream(const int* p)
{
    int v;
    asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p)
{
    uint32_t v;
    asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// The rest of a walk that has met a wall edge (edge walls): mirror the position across the wall
// edge (U <- 2 U_w - U, U_w = (lid_u, 0, 0) on a moving wall), go on walking from the same
// element, at most kReflCap mirrorings and kHopCap hops in all. Returns the owner, or -1 (lost).
// Out of line: particles reach it only at walls.
static __device__ __noinline__ int walk_mirroring(const DevMesh& M, float lid_u, int e, int next, int& h, float& px,
                                                  float& py, float& u, float& v, float& w)
{
    for (int nref = 0;;) {
        if (next < 0) {
            if (nref >= kReflCap) return -1;
            const int k = -1 - next;
            mirror_across_edge(M, e, k, px, py);
            if (M.periodic) {
                // the image of a wall edge that is not parallel to the seam can leave the frame
                // in x: wrap it again (the frame of the element's component)
                float fx0 = M.x0, fx1 = M.x1;
                if (M.n_comp > 1) {
                    const float4 fr = __ldg(&M.cframe[__ldg(&M.ecomp[e])]);
                    fx0 = fr.x;
                    fx1 = fr.y;
                }
                if (px < fx0) px += M.period;
                else if (px >= fx1) px -= M.period;
                // the half-open frame: an image that rounds to x1 belongs to x0
                if (px >= fx1) px = fx0;
            }
            const bool moving = (__ldg(&M.en[e]).w >> (3 + k)) & 1;
            u = (moving ? 2.0f * lid_u : 0.0f) - u;
            v = -v;
            w = -w;
            ++nref;
        } else {
            if (h >= kHopCap) return -1;
            e = next;
            ++h;
        }
        int r = walk_test_fast<true>(M, e, px, py, next);
        if (r < 0) {
            const int c = walk_test_code(M, e, px, py);
            r = c == kWalkIn ? 1 : 0;
            if (!r) next = c;
        }
        if (r == 1) return e;
    }
}

// one particle, its state loaded: advanced, located and written to position i of the next buffer
template <int NS, int kKind>
__device__ __forceinline__ void advance_store(const DevMesh& M, const DevState& nxt, const float* __restrict__ EF,
                                              const StepParams& P, unsigned long long* __restrict__ status,
                                              int64_t i, ParticleState<NS>& p, unsigned& err, int& hops)
{
    bool bad;
    advance_particle<NS, true, kKind>(M, EF, P, p, err, bad);
    // barycentric neighbour walk from the old element; with edge walls, a position found beyond
    // a wall edge is mirrored across that edge (U <- 2 U_w - U) and the walk goes on
    const int e0 = p.elem;
    int e = e0, h = 0, ne = e0;
    bool lost = false;
#pragma unroll 1
    for (;;) {
        int next = -1;
        int r = walk_test_fast<kKind == 2>(M, e, p.x, p.y, next);
        if (r < 0) {
            const int c = walk_test_code(M, e, p.x, p.y);
            r = c == kWalkIn ? 1 : 0;
            if (!r) next = c;
        }
        if (r == 1) {
            ne = e;
            hops += h;
            break;
        }
        if (kKind == 2 && next < 0 && M.edge_walls) {
            // the mirroring walk writes through references: it gets copies, so that the state
            // itself never has its address taken and stays in registers on the common path
            float mx = p.x, my = p.y, mu = p.u, mv = p.v, mw = p.w;
            int mh = h;
            ne = walk_mirroring(M, P.lid_u, e, next, mh, mx, my, mu, mv, mw);
            p.x = mx;
            p.y = my;
            p.u = mu;
            p.v = mv;
            p.w = mw;
            h = mh;
            lost = ne < 0;
            hops += h;
            break;
        }
        if (next < 0 || h >= kHopCap) {
            lost = true;
            hops += next < 0 ? h : kHopCap + 1;
            break;
        }
        e = next;
        ++h;
    }
    if (lost) ne = e0;
    if (kKind == 2 && M.edge_walls) particle_sources<NS, kKind>(M, P, e0, p.x, p.y, p.psi);
    if (lost || bad) {
        err |= kErrLost;
        atomicAdd(&status[1], 1ull);
        atomicCAS(&status[2], ~0ull, (unsigned long long)p.pid);
    }
    __stcs(nxt.x + i, p.x);
    __stcs(nxt.y + i, p.y);
    __stcs(nxt.u + i, p.u);
    __stcs(nxt.v + i, p.v);
    __stcs(nxt.w + i, p.w);
    __stcs(nxt.om + i, p.om);
#pragma unroll
    for (int a = 0; a < NS; ++a) __stcs(nxt.psi + (size_t)a * nxt.cap + i, p.psi[a]);
    __stcs(nxt.elem + i, ne);
    __stcs(nxt.pid + i, p.pid);
}

// one particle: position i of the next buffer takes particle perm[i] of the current one
template <int NS, int kKind>
__device__ __forceinline__ void advance_one(const DevMesh& M, const DevState& cur, const DevState& nxt,
                                            const int* __restrict__ perm, const float* __restrict__ EF,
                                            const StepParams& P, unsigned long long* __restrict__ status, int64_t i,
                                            unsigned& err, int& hops)
{
    const int src = ld_stream(perm + i);
    ParticleState<NS> p;
    p.x = ld_stream(cur.x + src);
    p.y = ld_stream(cur.y + src);
    p.u = ld_stream(cur.u + src);
    p.v = ld_stream(cur.v + src);
    p.w = ld_stream(cur.w + src);
    p.om = ld_stream(cur.om + src);
#pragma unroll
    for (int a = 0; a < NS; ++a) p.psi[a] = ld_stream(cur.psi + (size_t)a * cur.cap + src);
    p.elem = ld_stream(cur.elem + src);
    p.pid = ld_stream(cur.pid + src);
    advance_store<NS, kKind>(M, nxt, EF, P, status, i, p, err, hops);
}

// K1 variants (the autotuner picks one per context; all give bit-identical results): ABLK
// threads per CTA, at least MINB CTAs per SM (the register cap), and the grid: kGrid 0, one
// particle per thread over the whole grid; 1, a persistent grid striding over ABLK-particle
// tiles; 2, a persistent grid whose warps take kQChunk-particle chunks in order from a counter
// (tiles, zero at launch). A warp then never waits for its CTA's other warps nor for a fixed
// share of tiles: the slow walks spread over all warps. 64 particles per chunk: 128 leave a
// tail of up to one chunk per warp at 5M particles, and 32 make the counter the bottleneck
// (781k claims per launch at 25M).
constexpr int kQChunk = 64;
template <int NS, int kKind, int ABLK, int MINB, int kGrid>
__global__ void __launch_bounds__(ABLK, MINB)
advance_kernel(const __grid_constant__ DevMesh M, const __grid_constant__ DevState cur,
               const __grid_constant__ DevState nxt, const int* __restrict__ perm, const float* __restrict__ EF,
               const __grid_constant__ StepParams P, unsigned long long* __restrict__ status,
               unsigned* __restrict__ tiles)
{
    const int lane = threadIdx.x & 31;
    unsigned err = 0;
    int hops = 0;
    if constexpr (kGrid == 2) {
        const int64_t nch = (cur.n + kQChunk - 1) / kQChunk;
        unsigned c = 0;
        if (lane == 0) c = atomicAdd(tiles, 1u);
        c = __shfl_sync(kFull, c, 0);
#pragma unroll 1
        while ((int64_t)c < nch) {
            // the next chunk is claimed before this one is worked on: its latency is hidden
            unsigned nx = 0;
            if (lane == 0) nx = atomicAdd(tiles, 1u);
#pragma unroll 1
            for (int k = 0; k < kQChunk / 32; ++k) {
                const int64_t i = (int64_t)c * kQChunk + 32 * k + lane;
                if (i < cur.n) advance_one<NS, kKind>(M, cur, nxt, perm, EF, P, status, i, err, hops);
            }
            c = __shfl_sync(kFull, nx, 0);
        }
    } else {
        const int64_t ntiles = (cur.n + ABLK - 1) / ABLK;
#pragma unroll 1
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += kGrid == 1 ? gridDim.x : ntiles) {
            const int64_t i = tile * ABLK + threadIdx.x;
            if (i < cur.n) advance_one<NS, kKind>(M, cur, nxt, perm, EF, P, status, i, err, hops);
        }
    }
    const unsigned e_or = __reduce_or_sync(kFull, err);
    const int h_sum = __reduce_add_sync(kFull, hops);
    if (lane == 0) {
        if (e_or) atomicOr(&status[0], (unsigned long long)e_or);
        if (h_sum) atomicAdd(&status[3], (unsigned long long)h_sum);
    }
}

// ------------------------------------------------------------------------------------------
// T: thread (e, q) writes float4 q of the three rows of element e
// ------------------------------------------------------------------------------------------
template <int NS>
__global__ void element_fields_kernel(const __grid_constant__ DevMesh M, const float* __restrict__ F,
                                      float* __restrict__ EF)
{
    constexpr int NFP = (22 + NS + 3) / 4 * 4, NQ4 = NFP / 4;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)M.n_tri * NQ4) return;
    const int e = (int)(t / NQ4), q = (int)(t - (int64_t)e * NQ4);
    const int4 V = __ldg(&M.ev[e]);
    const float4 A = __ldg(&M.ea[e]);   // b1 = A.z, g1 = A.w
    const float4 B = __ldg(&M.eb[e]);   // b2 = B.x, g2 = B.y
    const float4 fa = __ldg(reinterpret_cast<const float4*>(F) + (size_t)V.x * NQ4 + q);
    const float4 fb = __ldg(reinterpret_cast<const float4*>(F) + (size_t)V.y * NQ4 + q);
    const float4 fc = __ldg(reinterpret_cast<const float4*>(F) + (size_t)V.z * NQ4 + q);
    // F = fa + (fb - fa) lambda_1 + (fc - fa) lambda_2, lambda_1 = b1 dx + g1 dy, lambda_2 = b2 dx + g2 dy
    auto gx = [&](float a, float b, float c) { return fmaf(b - a, A.z, (c - a) * B.x); };
    auto gy = [&](float a, float b, float c) { return fmaf(b - a, A.w, (c - a) * B.y); };
    float4* R = reinterpret_cast<float4*>(EF) + (size_t)e * 3 * NQ4;
    R[q] = fa;
    R[NQ4 + q] = make_float4(gx(fa.x, fb.x, fc.x), gx(fa.y, fb.y, fc.y), gx(fa.z, fb.z, fc.z), gx(fa.w, fb.w, fc.w));
    R[2 * NQ4 + q] = make_float4(gy(fa.x, fb.x, fc.x), gy(fa.y, fb.y, fc.y), gy(fa.z, fb.z, fc.z), gy(fa.w, fb.w, fc.w));
}

// ------------------------------------------------------------------------------------------
// H: one warp per record block of kBlk positions, warp-synchronous (no block barriers)
// ------------------------------------------------------------------------------------------
constexpr int kHWarps = 8;             // warps (record blocks) per CTA
constexpr int kRows = kBlk / 32;       // rows of 32 positions in a record block
constexpr int kWHash = 256;            // per-warp hash slots (a block has at most kBlk elements)
static_assert(kWHash == 256 && kWHash >= kBlk, "rec_hash gives 8 bits; a block has at most kBlk elements");

__global__ void __launch_bounds__(32 * kHWarps) histogram_kernel(const int* __restrict__ elem, int64_t n,
                                                               uint16_t* __restrict__ rrank,
                                                               int* __restrict__ rec_key, int* __restrict__ rec_cnt,
                                                               int* __restrict__ nrec, int* __restrict__ kcnt,
                                                               int* __restrict__ krc, unsigned long long* __restrict__ status)
{
    __shared__ int hkey_s[kHWarps][kWHash];
    __shared__ unsigned short hcnt_s[kHWarps][kWHash];
    __shared__ unsigned char hrec_s[kHWarps][kWHash];
    __shared__ short used_s[kHWarps][kBlk];   // slot of each record, in insertion order
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t blk = (int64_t)blockIdx.x * kHWarps + wid;     // the record block of this warp
    const int64_t nblk = (n + kBlk - 1) / kBlk;
    if (blk >= nblk) return;
    int* const hkey = hkey_s[wid];
    unsigned short* const hcnt = hcnt_s[wid];
    unsigned char* const hrec = hrec_s[wid];
    short* const used = used_s[wid];
    for (int s = lane; s < kWHash; s += 32) hkey[s] = -1;
    const int64_t base = blk * kBlk;
    int key[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const int64_t i = base + r * 32 + lane;
        key[r] = i < n ? elem[i] : -1;
    }
    __syncwarp();
    unsigned err = 0;
    int nr = 0;                       // records so far (warp-uniform)
    int slot[kRows], rank[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const int k = key[r];
        const unsigned m = __match_any_sync(kFull, k);
        const int leader = __ffs(m) - 1;
        int s = -1, prefix = 0, fresh = 0;
        if (k >= 0 && lane == leader) {
            const unsigned h0 = rec_hash(k);
#pragma unroll 1
            for (int q = 0; q < kWHash; ++q) {
                const int t = (h0 + q) & (kWHash - 1);
                const int c = hkey[t];
                if (c == k) { s = t; break; }
                if (c == -1) {
                    // leaders of different elements of one row may probe the same empty slot
                    const int old = atomicCAS(&hkey[t], -1, k);
                    if (old == -1) { s = t; fresh = 1; break; }
                    if (old == k) { s = t; break; }
                }
            }
            if (fresh) hcnt[s] = 0;
        }
        // new records in lane order get consecutive record indices
        const unsigned nb = __ballot_sync(kFull, fresh);
        if (fresh) {
            const int r_new = nr + __popc(nb & lt);
            hrec[s] = (unsigned char)r_new;
            used[r_new] = (short)s;
        }
        nr += __popc(nb);
        __syncwarp();
        if (s >= 0) {
            prefix = hcnt[s];
            hcnt[s] = (unsigned short)(prefix + __popc(m));
        }
        s = __shfl_sync(kFull, s, leader);
        prefix = __shfl_sync(kFull, prefix, leader);
        slot[r] = s;
        rank[r] = prefix + __popc(m & lt);
        __syncwarp();
    }
    // records of this block
    for (int q = lane; q < nr; q += 32) {
        const int s = used[q];
        const int k = hkey[s], c = hcnt[s];
        const int64_t rid = blk * kBlk + q;
        rec_key[rid] = k;
        rec_cnt[rid] = c;
        atomicAdd(&kcnt[k], c);
        atomicAdd(&krc[k], 1);
    }
    if (lane == 0) nrec[blk] = nr;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const int64_t i = base + r * 32 + lane;
        if (key[r] >= 0 && consistent(slot[r] >= 0 && rank[r] < kBlk, err))
            rrank[i] = (uint16_t)(((unsigned)hrec[slot[r]] << 8) | (unsigned)rank[r]);
    }
    const unsigned e_or = __reduce_or_sync(kFull, err);
    if (lane == 0 && e_or) atomicOr(&status[0], (unsigned long long)e_or);
}

// ------------------------------------------------------------------------------------------
// S1: exclusive scan of two int arrays of length n (blockIdx.y picks the array)
// ------------------------------------------------------------------------------------------
struct ScanPair {
    const int* in[2];
    int* out[2];
    int* part[2];
    // select without dynamic indexing of the parameter arrays
    __device__ __forceinline__ const int* src(int a) const { return a ? in[1] : in[0]; }
    __device__ __forceinline__ int* dst(int a) const { return a ? out[1] : out[0]; }
    __device__ __forceinline__ int* tot(int a) const { return a ? part[1] : part[0]; }
};

__device__ __forceinline__ int block_scan_1024(int v, int* wsum, int& total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int s = wsum[lane];
        int x = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += t;
        }
        wsum[lane] = x - s;
        if (lane == 31) wsum[32] = x;
    }
    __syncthreads();
    total = wsum[32];
    const int r = wsum[wid] + incl - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(ScanPair sp, int n)
{
    __shared__ int wsum[33];
    const int a = blockIdx.y;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? sp.src(a)[base + k] : 0;
        sum += v[k];
    }
    int total;
    int run = block_scan_1024(sum, wsum, total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) sp.dst(a)[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) sp.tot(a)[blockIdx.x] = total;
}

// the tile totals (at most kScanTile of them) scanned in place
__global__ void __launch_bounds__(kScanThreads) scan_parts_kernel(ScanPair sp, int ntiles)
{
    __shared__ int wsum[33];
    const int a = blockIdx.y;
    const int base = threadIdx.x * kScanItems;
    int v[kScanItems];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < ntiles ? sp.tot(a)[base + k] : 0;
        sum += v[k];
    }
    int total;
    int run = block_scan_1024(sum, wsum, total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < ntiles) sp.tot(a)[base + k] = run;
        run += v[k];
    }
}

__global__ void scan_add_kernel(ScanPair sp, int n)
{
    const int a = blockIdx.y;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) sp.dst(a)[j] += sp.tot(a)[j / kScanTile];
}

// ------------------------------------------------------------------------------------------
// S2, S3, S4
// ------------------------------------------------------------------------------------------
// a warp per record block (a block holds a few records: one per distinct element)
__global__ void __launch_bounds__(256) record_scatter_kernel(const int* __restrict__ nrec, const int* __restrict__ rec_key,
                                                            const int* __restrict__ krstart, int* __restrict__ kcur,
                                                            int* __restrict__ klist, int64_t nblk)
{
    const int64_t blk = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (blk >= nblk) return;
    const int lane = threadIdx.x & 31;
    const int nr = nrec[blk];
    for (int t = lane; t < nr; t += 32) {
        const int rid = (int)blk * kBlk + t;
        const int key = rec_key[rid];
        klist[krstart[key] + atomicAdd(&kcur[key], 1)] = rid;
    }
}

// a warp per element: its records in block order (a record id is block * kBlk + slot, and an
// element has at most one record per block), then the running offsets
__global__ void __launch_bounds__(256) key_offsets_kernel(int n_keys, const int* __restrict__ kstart,
                                                          const int* __restrict__ krstart,
                                                          const int* __restrict__ klist, int* __restrict__ klist2,
                                                          const int* __restrict__ rec_cnt, int* __restrict__ rec_off)
{
    const int e = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= n_keys) return;
    const int r0 = krstart[e], r1 = krstart[e + 1], nr = r1 - r0;
    if (nr == 0) return;
    if (nr == 1) {
        if (lane == 0) rec_off[klist[r0]] = kstart[e];
        return;
    }
    // rank of every record id among the element's (ids are distinct)
    for (int j = lane; j < nr; j += 32) {
        const int id = klist[r0 + j];
        int rank = 0;
        for (int q = 0; q < nr; ++q) rank += klist[r0 + q] < id;
        klist2[r0 + rank] = id;
    }
    __syncwarp();
    int carry = kstart[e];
    for (int j0 = 0; j0 < nr; j0 += 32) {
        const int j = j0 + lane;
        const int id = j < nr ? klist2[r0 + j] : -1;
        const int c = id >= 0 ? rec_cnt[id] : 0;
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        if (id >= 0) rec_off[id] = carry + incl - c;
        carry += __shfl_sync(kFull, incl, 31);
    }
}

constexpr int kScatterPer = 4;   // particles per thread of the particle scatter

__global__ void particle_scatter_kernel(int64_t n, const uint16_t* __restrict__ rrank, const int* __restrict__ rec_off,
                                        int* __restrict__ perm_new)
{
    const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x) * kScatterPer + threadIdx.x;
    unsigned pk[kScatterPer];
    int off[kScatterPer];
#pragma unroll
    for (int k = 0; k < kScatterPer; ++k) {
        const int64_t i = i0 + (int64_t)k * blockDim.x;
        pk[k] = i < n ? rrank[i] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kScatterPer; ++k) {
        const int64_t i = i0 + (int64_t)k * blockDim.x;
        off[k] = i < n ? rec_off[(i / kBlk) * kBlk + (pk[k] >> 8)] : 0;
    }
#pragma unroll
    for (int k = 0; k < kScatterPer; ++k) {
        const int64_t i = i0 + (int64_t)k * blockDim.x;
        if (i < n) perm_new[off[k] + (pk[k] & 255u)] = (int)i;
    }
}

// ------------------------------------------------------------------------------------------
// K2
// ------------------------------------------------------------------------------------------
// Error-free transformations in FP32 (Knuth's two-sum; the two-product by FMA): a + b = s + e and
// a b = p + e exactly. A double-float is an unevaluated sum h + l of two FP32 values.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    const float t = __fadd_rn(a, b);
    const float bb = __fsub_rn(t, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(t, bb)), __fsub_rn(b, bb));
    s = t;
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e)
{
    const float t = __fmul_rn(a, b);
    e = fmaf(a, b, -t);
    p = t;
}
// (s + c) += (th + tl): the rounding error of s + th is kept exactly and added to c with tl
__device__ __forceinline__ void df_acc(float& s, float& c, float th, float tl)
{
    float e;
    two_sum(s, th, s, e);
    c = __fadd_rn(c, __fadd_rn(e, tl));
}
// the same on pairs of independent values (packed FP32x2 instructions of sm_100+)
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e)
{
    const float2 t = __fadd2_rn(a, b);
    const float2 bb = __fadd2_rn(t, neg2(a));
    e = __fadd2_rn(__fadd2_rn(a, neg2(__fadd2_rn(t, neg2(bb)))), __fadd2_rn(b, neg2(bb)));
    s = t;
}
__device__ __forceinline__ void df_acc2(float2& s, float2& c, float2 th, float2 tl)
{
    float2 e;
    two_sum2(s, th, s, e);
    c = __fadd2_rn(c, __fadd2_rn(e, tl));
}

// Quantity groups of the moment sums (columns of the node accumulators from COL0 on, NQTOT per node):
//   G = 0: 1, u, v, w, uu, uv, uw, vv, vw, ww, omega (the velocity and frequency statistics);
//   G = 1: psi_a, psi_a^2 (a < NS);  G = 2: u psi_a, v psi_a, w psi_a (the scalar fluxes of IECM).
// PROD(j): quantity j is a product of two state fields (a double-float); else it is exact in FP32.
template <int NS, int G>
struct QGroup {
    static constexpr int NQ = G == 0 ? 11 : (G == 1 ? 2 * NS : 3 * NS);
    static constexpr int COL0 = G == 1 ? 11 : 0;
    static constexpr int NQTOT = G == 2 ? 3 * NS : 11 + 2 * NS;
    static constexpr int NFLD = G == 0 ? 4 : (G == 1 ? NS : 3 + NS);   // gathered fields besides x, y
    __host__ __device__ static constexpr bool PROD(int j)
    {
        return G == 0 ? (j >= 4 && j <= 9) : (G == 1 ? j >= NS : true);
    }
};

template <int NS, int G>
__device__ __forceinline__ void gather_fields(const DevState& S, int j, float* f)
{
    if (G == 0) {
        f[0] = S.u[j];
        f[1] = S.v[j];
        f[2] = S.w[j];
        f[3] = S.om[j];
    } else if (G == 1) {
#pragma unroll
        for (int a = 0; a < NS; ++a) f[a] = S.psi[(size_t)a * S.cap + j];
    } else {
        f[0] = S.u[j];
        f[1] = S.v[j];
        f[2] = S.w[j];
#pragma unroll
        for (int a = 0; a < NS; ++a) f[3 + a] = S.psi[(size_t)a * S.cap + j];
    }
}

template <int NS, int G>
__device__ __forceinline__ void quantities_df(const float* f, float* qh, float* ql)
{
    if (G == 0) {
        const float u = f[0], v = f[1], w = f[2];
        qh[0] = 1.0f; qh[1] = u; qh[2] = v; qh[3] = w; qh[10] = f[3];
        ql[0] = ql[1] = ql[2] = ql[3] = ql[10] = 0.0f;
        two_prod(u, u, qh[4], ql[4]);
        two_prod(u, v, qh[5], ql[5]);
        two_prod(u, w, qh[6], ql[6]);
        two_prod(v, v, qh[7], ql[7]);
        two_prod(v, w, qh[8], ql[8]);
        two_prod(w, w, qh[9], ql[9]);
    } else if (G == 1) {
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            qh[a] = f[a];
            ql[a] = 0.0f;
            two_prod(f[a], f[a], qh[NS + a], ql[NS + a]);
        }
    } else {
#pragma unroll
        for (int a = 0; a < NS; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) two_prod(f[c], f[3 + a], qh[3 * a + c], ql[3 * a + c]);
    }
}

// One step of the warp reduce-scatter of double-float columns: with offset O, a lane keeps the half
// of its live columns that its lane bit O selects, in its low entries, and adds the partner's copy
// of them (a compensated addition). LA, LB: live entries of (ah, al) (columns i) and (bh, bl)
// (columns i + 32) before the step.
template <int O, int LA, int LB>
__device__ __forceinline__ void halve_df(float (&ah)[32], float (&al)[32], float (&bh)[32], float (&bl)[32], bool up)
{
#pragma unroll
    for (int i = 0; i < (LA < O ? LA : O); ++i) {
        const float loh = ah[i], lol = al[i];
        const float hih = O + i < LA ? ah[O + i] : 0.0f, hil = O + i < LA ? al[O + i] : 0.0f;
        const float rh = __shfl_xor_sync(kFull, up ? loh : hih, O), rl = __shfl_xor_sync(kFull, up ? lol : hil, O);
        float s, e;
        two_sum(up ? hih : loh, rh, s, e);
        ah[i] = s;
        al[i] = __fadd_rn(__fadd_rn(up ? hil : lol, rl), e);
    }
#pragma unroll
    for (int i = 0; i < (LB < O ? LB : O); ++i) {
        const float loh = bh[i], lol = bl[i];
        const float hih = O + i < LB ? bh[O + i] : 0.0f, hil = O + i < LB ? bl[O + i] : 0.0f;
        const float rh = __shfl_xor_sync(kFull, up ? loh : hih, O), rl = __shfl_xor_sync(kFull, up ? lol : hil, O);
        float s, e;
        two_sum(up ? hih : loh, rh, s, e);
        bh[i] = s;
        bl[i] = __fadd_rn(__fadd_rn(up ? hil : lol, rl), e);
    }
}

__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }

// Column sums of NK <= 64 per-lane double-floats over the warp, by recursive halving: after the
// steps with offsets 16, 8, 4, 2, 1 lane j holds the sums of columns j and j + 32 (zero when
// j + 32 >= NK). The order of the additions is fixed: every launch gives the same bits.
template <int NK>
__device__ __forceinline__ void warp_reduce_scatter_df(const float (&sh)[NK], const float (&sl)[NK], int lane,
                                                       float& h0, float& l0, float& h1, float& l1)
{
    static_assert(NK >= 1 && NK <= 64, "at most two columns per lane");
    constexpr int A0 = cmin(NK, 32), B0 = NK > 32 ? NK - 32 : 0;
    float ah[32], al[32], bh[32], bl[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        ah[i] = i < NK ? sh[i] : 0.0f;
        al[i] = i < NK ? sl[i] : 0.0f;
        bh[i] = 32 + i < NK ? sh[32 + i] : 0.0f;
        bl[i] = 32 + i < NK ? sl[32 + i] : 0.0f;
    }
    halve_df<16, A0, B0>(ah, al, bh, bl, (lane & 16) != 0);
    halve_df<8, cmin(A0, 16), cmin(B0, 16)>(ah, al, bh, bl, (lane & 8) != 0);
    halve_df<4, cmin(A0, 8), cmin(B0, 8)>(ah, al, bh, bl, (lane & 4) != 0);
    halve_df<2, cmin(A0, 4), cmin(B0, 4)>(ah, al, bh, bl, (lane & 2) != 0);
    halve_df<1, cmin(A0, 2), cmin(B0, 2)>(ah, al, bh, bl, (lane & 1) != 0);
    h0 = ah[0];
    l0 = al[0];
    h1 = B0 > 0 ? bh[0] : 0.0f;
    l1 = B0 > 0 ? bl[0] : 0.0f;
}

__device__ __forceinline__ long long to_fixed64(double v, unsigned& err)
{
    if (!(fabs(v) < (double)kFixLimit)) err |= kErrOverflow;
    return __double2ll_rn(v * 4294967296.0);
}

// One quantity group over the particles idx[0..LC) of a lane (a chunk of the element's particles).
// With (dx, dy) = p - vertex 0 formed exactly as double-floats, the barycentrics are affine,
// lambda_1 = b1 dx + g1 dy, lambda_2 = b2 dx + g2 dy, lambda_0 = 1 - lambda_1 - lambda_2, so the
// element's sums are
//   S_1 = b1 Tx + g1 Ty,  S_2 = b2 Tx + g2 Ty,  S_0 = T0 - S_1 - S_2,
//   T0 = sum q,  Tx = sum dx q,  Ty = sum dy q.
// T0, Tx, Ty are summed in double-float (exact products, compensated additions) per lane and over
// the warp; the FP64 coefficients of the element combine them in FP64 and each node sum gets one
// 64-bit fixed-point add per quantity.
template <int NS, int G>
__device__ __forceinline__ void moment_group(const DevState& S, const int* __restrict__ perm, int base, int end,
                                            float X0, float Y0, const double4& co, const int4& mv, int lane,
                                            unsigned long long* __restrict__ node_acc, unsigned& err)
{
    using Q = QGroup<NS, G>;
    constexpr int NQ = Q::NQ, NK = 3 * NQ, NF = Q::NFLD;
    constexpr int NP = (NQ + 1) / 2;
    float2 s0[NP], c0[NP], sxy[NQ], cxy[NQ];   // T0 of quantities (2i, 2i + 1); (Tx, Ty) of quantity j
#pragma unroll
    for (int k = 0; k < NP; ++k) s0[k] = c0[k] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < NQ; ++k) sxy[k] = cxy[k] = make_float2(0.0f, 0.0f);
    // the lane's particles base + lane + 32 k in canonical order, one per iteration (the loop is
    // not unrolled: its body is already several hundred instructions); the gather order two
    // particles ahead and the fields one particle ahead are loaded before a particle is summed
    int pos = base + lane;
    int j1 = pos < end ? perm[pos] : -1;
    int j2 = pos + 32 < end ? perm[pos + 32] : -1;
    float cx = 0.0f, cy = 0.0f, cf[NF];
    if (j1 >= 0) {
        cx = S.x[j1];
        cy = S.y[j1];
        gather_fields<NS, G>(S, j1, cf);
    }
#pragma unroll 1
    for (; j1 >= 0; pos += 32) {
        const int j3 = pos + 64 < end ? perm[pos + 64] : -1;
        float nx = 0.0f, ny = 0.0f, nf[NF];
        if (j2 >= 0) {
            nx = S.x[j2];
            ny = S.y[j2];
            gather_fields<NS, G>(S, j2, nf);
        }
        // (dx, dy) = p - vertex 0 as exact double-floats (dh + dl), x and y packed
        float2 dh, dl;
        two_sum2(make_float2(cx, cy), make_float2(-X0, -Y0), dh, dl);
        float qh[NQ], ql[NQ];
        quantities_df<NS, G>(cf, qh, ql);
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const int j = 2 * i;
            df_acc2(s0[i], c0[i], make_float2(qh[j], j + 1 < NQ ? qh[j + 1] : 0.0f),
                    make_float2(ql[j], j + 1 < NQ ? ql[j + 1] : 0.0f));
        }
#pragma unroll
        for (int j = 0; j < NQ; ++j) {
            // (dh + dl)(qh + ql): the exact product of the leading parts plus the cross terms
            const float2 q2 = make_float2(qh[j], qh[j]);
            const float2 ph = __fmul2_rn(dh, q2);
            float2 pl = __ffma2_rn(dh, q2, neg2(ph));
            pl = __ffma2_rn(dl, q2, pl);
            if (Q::PROD(j)) pl = __ffma2_rn(dh, make_float2(ql[j], ql[j]), pl);
            df_acc2(sxy[j], cxy[j], ph, pl);
        }
        j1 = j2;
        j2 = j3;
        cx = nx;
        cy = ny;
#pragma unroll
        for (int f = 0; f < NF; ++f) cf[f] = nf[f];
    }
    // columns T0 (0 .. NQ - 1), Tx (NQ ..), Ty (2 NQ ..); lane j ends with columns j and j + 32
    float sh[NK], sl[NK];
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
        sh[j] = j & 1 ? s0[j / 2].y : s0[j / 2].x;
        sl[j] = j & 1 ? c0[j / 2].y : c0[j / 2].x;
        sh[NQ + j] = sxy[j].x;
        sl[NQ + j] = cxy[j].x;
        sh[2 * NQ + j] = sxy[j].y;
        sl[2 * NQ + j] = cxy[j].y;
    }
    float h0, l0, h1, l1;
    warp_reduce_scatter_df<NK>(sh, sl, lane, h0, l0, h1, l1);
    // lane j < NQ: T0 (column j, its own), Tx (column NQ + j) and Ty (column 2 NQ + j)
    const int cxc = NQ + lane, cyc = 2 * NQ + lane;
    const float xh0 = __shfl_sync(kFull, h0, cxc & 31), xl0 = __shfl_sync(kFull, l0, cxc & 31);
    const float xh1 = __shfl_sync(kFull, h1, cxc & 31), xl1 = __shfl_sync(kFull, l1, cxc & 31);
    const float yh0 = __shfl_sync(kFull, h0, cyc & 31), yl0 = __shfl_sync(kFull, l0, cyc & 31);
    const float yh1 = __shfl_sync(kFull, h1, cyc & 31), yl1 = __shfl_sync(kFull, l1, cyc & 31);
    if (lane < NQ) {
        const double T0 = (double)h0 + (double)l0;
        const double Tx = cxc < 32 ? (double)xh0 + (double)xl0 : (double)xh1 + (double)xl1;
        const double Ty = cyc < 32 ? (double)yh0 + (double)yl0 : (double)yh1 + (double)yl1;
        const double S1 = co.x * Tx + co.y * Ty;
        const double S2 = co.z * Tx + co.w * Ty;
        const double S0 = (T0 - S1) - S2;
        const int col = Q::COL0 + lane;
        const long long v0 = to_fixed64(S0, err), v1 = to_fixed64(S1, err), v2 = to_fixed64(S2, err);
        if (v0 != 0) atomicAdd(&node_acc[(size_t)mv.x * Q::NQTOT + col], (unsigned long long)v0);
        if (v1 != 0) atomicAdd(&node_acc[(size_t)mv.y * Q::NQTOT + col], (unsigned long long)v1);
        if (v2 != 0) atomicAdd(&node_acc[(size_t)mv.z * Q::NQTOT + col], (unsigned long long)v2);
    }
}

// K2 with compensated sums (moment_sums = 1). kFlux: the sums of the scalar fluxes u_i psi_a
// (IECM) into their own accumulators instead
template <int NS, int MBLK, int MMINB, bool kFlux = false>
__global__ void __launch_bounds__(MBLK, MMINB) moments_kernel_df(const __grid_constant__ DevMesh M,
                                                      const __grid_constant__ DevState S,
                                                      const int* __restrict__ perm, const int* __restrict__ kstart,
                                                      unsigned long long* __restrict__ node_acc,
                                                      unsigned long long* __restrict__ status)
{
    const int e = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= M.n_tri) return;
    const int p0 = kstart[e], p1 = kstart[e + 1];
    if (p0 >= p1) return;
    const float4 A = __ldg(&M.ea[e]);
    const double2 c01 = __ldg(reinterpret_cast<const double2*>(M.ec + e)), c23 = __ldg(reinterpret_cast<const double2*>(M.ec + e) + 1);
    const double4 co = make_double4(c01.x, c01.y, c23.x, c23.y);
    const int4 mv = __ldg(&M.em[e]);
    unsigned err = 0;
    constexpr int LC = kLaneChunkDf;   // particles per lane and chunk
#pragma unroll 1
    for (int base = p0; base < p1; base += 32 * LC) {
        const int end = min(p1, base + 32 * LC);
        if (kFlux) {
            moment_group<NS, 2>(S, perm, base, end, A.x, A.y, co, mv, lane, node_acc, err);
        } else {
            moment_group<NS, 0>(S, perm, base, end, A.x, A.y, co, mv, lane, node_acc, err);
            moment_group<NS, 1>(S, perm, base, end, A.x, A.y, co, mv, lane, node_acc, err);
        }
    }
    const unsigned e_or = __reduce_or_sync(kFull, err);
    if (lane == 0 && e_or) atomicOr(&status[0], (unsigned long long)e_or);
}

// K2 with FP32 partial sums (moment_sums = 0, the throughput configuration): lambda_a' q_k formed
// in FP32 and accumulated in FP32 per lane over at most kLaneChunk particles, then a fixed
// reduce-scatter across the lanes, one 64-bit fixed-point atomic add per node and quantity. kFlux:
// the same reduction of the scalar fluxes u_i psi_a (IECM) into their own accumulators.
// One step of the warp reduce-scatter below: with offset O, a lane keeps the half of its live
// columns that its lane bit O selects, in its low entries, and adds the partner's copy of them.
// LA, LB: live entries of a (columns base + i) and b (columns base + i + 32) before the step.
template <int O, int LA, int LB>
__device__ __forceinline__ void halve(float (&a)[32], float (&b)[32], bool up)
{
#pragma unroll
    for (int i = 0; i < (LA < O ? LA : O); ++i) {
        const float lo = a[i], hi = O + i < LA ? a[O + i] : 0.0f;
        a[i] = (up ? hi : lo) + __shfl_xor_sync(kFull, up ? lo : hi, O);
    }
#pragma unroll
    for (int i = 0; i < (LB < O ? LB : O); ++i) {
        const float lo = b[i], hi = O + i < LB ? b[O + i] : 0.0f;
        b[i] = (up ? hi : lo) + __shfl_xor_sync(kFull, up ? lo : hi, O);
    }
}

// Column sums of NK <= 64 per-lane values over the warp, by recursive halving: after the steps
// with offsets 16, 8, 4, 2, 1 lane j holds the sums of columns j (lo) and j + 32 (hi, zero when
// j + 32 >= NK). About NK shuffles instead of a butterfly's 5 NK; the order of the additions is
// fixed, so every launch gives the same bits.
template <int NK>
__device__ __forceinline__ void warp_reduce_scatter(const float (&acc)[NK], int lane, float& lo, float& hi)
{
    static_assert(NK >= 1 && NK <= 64, "at most two columns per lane");
    constexpr int A0 = cmin(NK, 32), B0 = NK > 32 ? NK - 32 : 0;
    float a[32], b[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        a[i] = i < NK ? acc[i] : 0.0f;
        b[i] = 32 + i < NK ? acc[32 + i] : 0.0f;
    }
    halve<16, A0, B0>(a, b, (lane & 16) != 0);
    halve<8, cmin(A0, 16), cmin(B0, 16)>(a, b, (lane & 8) != 0);
    halve<4, cmin(A0, 8), cmin(B0, 8)>(a, b, (lane & 4) != 0);
    halve<2, cmin(A0, 4), cmin(B0, 4)>(a, b, (lane & 2) != 0);
    halve<1, cmin(A0, 2), cmin(B0, 2)>(a, b, (lane & 1) != 0);
    lo = a[0];
    hi = B0 > 0 ? b[0] : 0.0f;
}

template <int NS, int MBLK, int MMINB, bool kFlux = false>
__global__ void __launch_bounds__(MBLK, MMINB) moments_kernel_f32(const __grid_constant__ DevMesh M,
                                                      const __grid_constant__ DevState S,
                                                      const int* __restrict__ perm, const int* __restrict__ kstart,
                                                      unsigned long long* __restrict__ node_acc,
                                                      unsigned long long* __restrict__ status)
{
    constexpr int NQ = kFlux ? 3 * NS : 11 + 2 * NS, NK = 3 * NQ;
    const int e = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= M.n_tri) return;
    const int p0 = kstart[e], p1 = kstart[e + 1];
    if (p0 >= p1) return;
    const float4 X = __ldg(&M.ex[e]);
    const float4 Y = __ldg(&M.ey[e]);
    const int4 mv = __ldg(&M.em[e]);
    unsigned err = 0;
    constexpr int LC = kLaneChunk;   // particles per lane and chunk
#pragma unroll 1
    for (int base = p0; base < p1; base += 32 * LC) {
        float acc[NK];
#pragma unroll
        for (int k = 0; k < NK; ++k) acc[k] = 0.0f;
        const int end = min(p1, base + 32 * LC);
        // the lane's gather indices for the whole chunk first, then batches of MB particles per
        // lane; with one scalar the batches are double-buffered (the next batch's state loads
        // are issued before the current batch is accumulated), with more the registers go to one
        // batch at a time. The accumulation order per lane stays position order either way.
        constexpr int MB = NS <= 2 ? 4 : 2, NB = NS == 1 ? 2 : 1;
        static_assert(LC % MB == 0, "whole batches per chunk");
        int idx[LC];
#pragma unroll
        for (int k = 0; k < LC; ++k) {
            const int pos = base + lane + 32 * k;
            idx[k] = pos < end ? perm[pos] : -1;
        }
        float bx[NB][MB], by[NB][MB], bu[NB][MB], bv[NB][MB], bw[NB][MB], bo[NB][MB], bp[NB][MB][NS];
        auto gather = [&](int buf, int k0) {
#pragma unroll
            for (int k = 0; k < MB; ++k) {
                const int j = idx[k0 + k] >= 0 ? idx[k0 + k] : 0;
                bx[buf][k] = S.x[j];
                by[buf][k] = S.y[j];
                bu[buf][k] = S.u[j];
                bv[buf][k] = S.v[j];
                bw[buf][k] = S.w[j];
                if (!kFlux) bo[buf][k] = S.om[j];
#pragma unroll
                for (int a = 0; a < NS; ++a) bp[buf][k][a] = S.psi[(size_t)a * S.cap + j];
            }
        };
        if constexpr (NB == 2) gather(0, 0);
#pragma unroll
        for (int k0 = 0; k0 < LC; k0 += MB) {
            if (base + 32 * k0 >= end) break;
            const int cb = NB == 2 ? (k0 / MB) & 1 : 0;
            if constexpr (NB == 2) {
                if (k0 + MB < LC && base + 32 * (k0 + MB) < end) gather(cb ^ 1, k0 + MB);
            } else {
                gather(0, k0);
            }
            float* const sx = bx[cb];
            float* const sy = by[cb];
            float* const su = bu[cb];
            float* const sv = bv[cb];
            float* const sw = bw[cb];
            float* const so = bo[cb];
#pragma unroll
            for (int k = 0; k < MB; ++k) {
                if (idx[k0 + k] < 0) break;
                float q[NQ];
                float* const spk = bp[cb][k];
                const float u = su[k], v = sv[k], w = sw[k];
                if (kFlux) {
#pragma unroll
                    for (int a = 0; a < NS; ++a) {
                        q[3 * a] = u * spk[a];
                        q[3 * a + 1] = v * spk[a];
                        q[3 * a + 2] = w * spk[a];
                    }
                } else {
                    q[0] = 1.0f; q[1] = u; q[2] = v; q[3] = w;
                    q[4] = u * u; q[5] = u * v; q[6] = u * w; q[7] = v * v; q[8] = v * w; q[9] = w * w;
                    q[10] = so[k];
#pragma unroll
                    for (int a = 0; a < NS; ++a) {
                        q[11 + a] = spk[a];
                        q[11 + NS + a] = spk[a] * spk[a];
                    }
                }
                float l0, l1, l2;
                barycentric(X, Y, sx[k], sy[k], l0, l1, l2);
#pragma unroll
                for (int kq = 0; kq < NQ; ++kq) {
                    acc[kq] = fmaf(l0, q[kq], acc[kq]);
                    acc[NQ + kq] = fmaf(l1, q[kq], acc[NQ + kq]);
                    acc[2 * NQ + kq] = fmaf(l2, q[kq], acc[2 * NQ + kq]);
                }
            }
        }
        // the warp's column sums, scattered: lane j ends with columns j and j + 32
        float colsum[2];
        warp_reduce_scatter<NK>(acc, lane, colsum[0], colsum[1]);
        // lane j adds columns j and j + 32
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            const int col = lane + 32 * kk;
            const float mine = colsum[kk];
            if (col < NK) {
                const int c = col / NQ, qq = col - c * NQ;
                const int node = c == 0 ? mv.x : (c == 1 ? mv.y : mv.z);
                const long long v = to_fixed(mine, err);
                if (v != 0) atomicAdd(&node_acc[(size_t)node * NQ + qq], (unsigned long long)v);
            }
        }
    }
    const unsigned e_or = __reduce_or_sync(kFull, err);
    if (lane == 0 && e_or) atomicOr(&status[0], (unsigned long long)e_or);
}

// Half-warp column sums: lanes 0-15 and lanes 16-31 of a warp hold two different elements'
// columns (NK <= 64) and reduce them by recursive halving with offsets 8, 4, 2, 1, which never
// cross the halves; lane j of a half ends with columns j, j + 16, j + 32 and j + 48 (zero past NK).
// The order of the additions is fixed.
template <int NK>
__device__ __forceinline__ void half_reduce_scatter(const float (&acc)[NK], int lane, float (&col)[4])
{
    static_assert(NK >= 1 && NK <= 64, "at most four columns per lane");
    constexpr int A0 = cmin(NK, 16), B0 = NK > 16 ? cmin(NK - 16, 16) : 0;
    constexpr int C0 = NK > 32 ? cmin(NK - 32, 16) : 0, D0 = NK > 48 ? NK - 48 : 0;
    float a[32], b[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        a[i] = i < A0 ? acc[i] : 0.0f;
        b[i] = i < B0 ? acc[cmin(16 + i, NK - 1)] : 0.0f;
    }
    halve<8, A0, B0>(a, b, (lane & 8) != 0);
    halve<4, cmin(A0, 8), cmin(B0, 8)>(a, b, (lane & 4) != 0);
    halve<2, cmin(A0, 4), cmin(B0, 4)>(a, b, (lane & 2) != 0);
    halve<1, cmin(A0, 2), cmin(B0, 2)>(a, b, (lane & 1) != 0);
    col[0] = a[0];
    col[1] = B0 > 0 ? b[0] : 0.0f;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        a[i] = i < C0 ? acc[cmin(32 + i, NK - 1)] : 0.0f;
        b[i] = i < D0 ? acc[cmin(48 + i, NK - 1)] : 0.0f;
    }
    halve<8, C0, D0>(a, b, (lane & 8) != 0);
    halve<4, cmin(C0, 8), cmin(D0, 8)>(a, b, (lane & 4) != 0);
    halve<2, cmin(C0, 4), cmin(D0, 4)>(a, b, (lane & 2) != 0);
    halve<1, cmin(C0, 2), cmin(D0, 2)>(a, b, (lane & 1) != 0);
    col[2] = C0 > 0 ? a[0] : 0.0f;
    col[3] = D0 > 0 ? b[0] : 0.0f;
}

// K2 for sparsely populated elements (FP32 partial sums): a half-warp per element, so that a warp
// keeps two elements' chains of dependent loads (bucket bounds, gather indices, state) in flight
// instead of one. Otherwise as moments_kernel_f32: at most kLaneChunk particles per lane and chunk
// in position order, the fixed reduction, one fixed-point atomic per node and quantity. Both
// halves run the same number of chunks (an empty or missing element contributes nothing) because
// the reduction's shuffles span the warp.
template <int NS, int MBLK, int MMINB>
__global__ void __launch_bounds__(MBLK, MMINB) moments_kernel_f32h(const __grid_constant__ DevMesh M,
                                                       const __grid_constant__ DevState S,
                                                       const int* __restrict__ perm, const int* __restrict__ kstart,
                                                       unsigned long long* __restrict__ node_acc,
                                                       unsigned long long* __restrict__ status)
{
    constexpr int NQ = 11 + 2 * NS, NK = 3 * NQ;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (((t >> 5) << 1) >= M.n_tri) return;   // the warp's first element is past the end (warp-uniform)
    const int e = (int)(t >> 4);
    const int lane = threadIdx.x & 15;
    const bool valid = e < M.n_tri;
    int p0 = 0, p1 = 0;
    if (valid) {
        p0 = kstart[e];
        p1 = kstart[e + 1];
    }
    constexpr int LC = kLaneChunk;
    const int mine = (p1 - p0 + 16 * LC - 1) / (16 * LC);
    const int nchunk = max(mine, __shfl_xor_sync(kFull, mine, 16));
    if (nchunk == 0) return;                   // both elements empty (warp-uniform)
    float4 X = make_float4(0.f, 0.f, 0.f, 0.f), Y = X;
    int4 mv = make_int4(0, 0, 0, 0);
    if (valid && p1 > p0) {
        X = __ldg(&M.ex[e]);
        Y = __ldg(&M.ey[e]);
        mv = __ldg(&M.em[e]);
    }
    unsigned err = 0;
#pragma unroll 1
    for (int ci = 0; ci < nchunk; ++ci) {
        const int base = p0 + ci * 16 * LC;
        const int end = min(p1, base + 16 * LC);
        float acc[NK];
#pragma unroll
        for (int k = 0; k < NK; ++k) acc[k] = 0.0f;
        constexpr int MB = NS <= 2 ? 4 : 2, NB = NS == 1 ? 2 : 1;
        static_assert(LC % MB == 0, "whole batches per chunk");
        int idx[LC];
#pragma unroll
        for (int k = 0; k < LC; ++k) {
            const int pos = base + lane + 16 * k;
            idx[k] = pos < end ? perm[pos] : -1;
        }
        float bx[NB][MB], by[NB][MB], bu[NB][MB], bv[NB][MB], bw[NB][MB], bo[NB][MB], bp[NB][MB][NS];
        auto gather = [&](int buf, int k0) {
#pragma unroll
            for (int k = 0; k < MB; ++k) {
                const int j = idx[k0 + k] >= 0 ? idx[k0 + k] : 0;
                bx[buf][k] = S.x[j];
                by[buf][k] = S.y[j];
                bu[buf][k] = S.u[j];
                bv[buf][k] = S.v[j];
                bw[buf][k] = S.w[j];
                bo[buf][k] = S.om[j];
#pragma unroll
                for (int a = 0; a < NS; ++a) bp[buf][k][a] = S.psi[(size_t)a * S.cap + j];
            }
        };
        if (base < end) {
            if constexpr (NB == 2) gather(0, 0);
#pragma unroll
            for (int k0 = 0; k0 < LC; k0 += MB) {
                if (base + 16 * k0 >= end) break;
                const int cb = NB == 2 ? (k0 / MB) & 1 : 0;
                if constexpr (NB == 2) {
                    if (k0 + MB < LC && base + 16 * (k0 + MB) < end) gather(cb ^ 1, k0 + MB);
                } else {
                    gather(0, k0);
                }
#pragma unroll
                for (int k = 0; k < MB; ++k) {
                    if (idx[k0 + k] < 0) break;
                    float q[NQ];
                    const float u = bu[cb][k], v = bv[cb][k], w = bw[cb][k];
                    q[0] = 1.0f; q[1] = u; q[2] = v; q[3] = w;
                    q[4] = u * u; q[5] = u * v; q[6] = u * w; q[7] = v * v; q[8] = v * w; q[9] = w * w;
                    q[10] = bo[cb][k];
#pragma unroll
                    for (int a = 0; a < NS; ++a) {
                        q[11 + a] = bp[cb][k][a];
                        q[11 + NS + a] = bp[cb][k][a] * bp[cb][k][a];
                    }
                    float l0, l1, l2;
                    barycentric(X, Y, bx[cb][k], by[cb][k], l0, l1, l2);
#pragma unroll
                    for (int kq = 0; kq < NQ; ++kq) {
                        acc[kq] = fmaf(l0, q[kq], acc[kq]);
                        acc[NQ + kq] = fmaf(l1, q[kq], acc[NQ + kq]);
                        acc[2 * NQ + kq] = fmaf(l2, q[kq], acc[2 * NQ + kq]);
                    }
                }
            }
        }
        float col[4];
        half_reduce_scatter<NK>(acc, lane, col);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const int c_ = lane + 16 * kk;
            if (c_ < NK && base < end) {
                const int c = c_ / NQ, qq = c_ - c * NQ;
                const int node = c == 0 ? mv.x : (c == 1 ? mv.y : mv.z);
                const long long val = to_fixed(col[kk], err);
                if (val != 0) atomicAdd(&node_acc[(size_t)node * NQ + qq], (unsigned long long)val);
            }
        }
    }
    const unsigned e_or = __reduce_or_sync(kFull, err);
    if ((threadIdx.x & 31) == 0 && e_or) atomicOr(&status[0], (unsigned long long)e_or);
}

__global__ void iota_kernel(int* __restrict__ p, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = (int)i;
}

// the step counter of graph-replayed steps: set (add = 0) or advance (set = 0)
__global__ void step_counter_kernel(unsigned long long* __restrict__ c, unsigned long long set, unsigned long long add)
{
    *c = add ? *c + add : set;
}

inline unsigned nblocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t scan_pair(const int* in0, int* out0, const int* in1, int* out1, int n, int* part, cudaStream_t st)
{
    const int ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles > kScanTile) return cudaErrorInvalidValue;
    ScanPair sp{{in0, in1}, {out0, out1}, {part, part + kScanTile}};
    scan_tiles_kernel<<<dim3(ntiles, 2), kScanThreads, 0, st>>>(sp, n);
    scan_parts_kernel<<<dim3(1, 2), kScanThreads, 0, st>>>(sp, ntiles);
    scan_add_kernel<<<dim3(nblocks(n, 256), 2), 256, 0, st>>>(sp, n);
    return cudaGetLastError();
}

// SM count of the current device (kept per device: contexts may live on different GPUs)
int sm_count_cached()
{
    constexpr int kMaxDev = 64;
    static std::atomic<int> n_of_dev[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 1;
    int n = n_of_dev[dev].load(std::memory_order_relaxed);
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
        n_of_dev[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

template <int NS, int kKind, int ABLK, int MINB, int kGrid>
void launch_advance_v(const DevMesh& m, const DevState& cur, const DevState& nxt, const int* perm, const float* ef,
                      const StepParams& p, unsigned long long* status, unsigned* tiles, cudaStream_t st)
{
    const int64_t ntiles = (cur.n + ABLK - 1) / ABLK;
    const int64_t grid = kGrid ? std::min<int64_t>(ntiles, (int64_t)sm_count_cached() * MINB) : ntiles;
    advance_kernel<NS, kKind, ABLK, MINB, kGrid>
        <<<(unsigned)grid, ABLK, 0, st>>>(m, cur, nxt, perm, ef, p, status, tiles);
}

template <int NS, int kKind>
void launch_advance(int v, const DevMesh& m, const DevState& cur, const DevState& nxt, const int* perm,
                    const float* ef, const StepParams& p, unsigned long long* status, unsigned* tiles,
                    cudaStream_t st)
{
    switch (v) {
        case 1: launch_advance_v<NS, kKind, 128, 10, 1>(m, cur, nxt, perm, ef, p, status, tiles, st); break;
        case 2: launch_advance_v<NS, kKind, 128, 8, 0>(m, cur, nxt, perm, ef, p, status, tiles, st); break;
        case 3: launch_advance_v<NS, kKind, 256, 4, 1>(m, cur, nxt, perm, ef, p, status, tiles, st); break;
        case 4: launch_advance_v<NS, kKind, 64, 18, 1>(m, cur, nxt, perm, ef, p, status, tiles, st); break;
        case 5: launch_advance_v<NS, kKind, 128, 10, 2>(m, cur, nxt, perm, ef, p, status, tiles, st); break;
        default: launch_advance_v<NS, kKind, 256, 4, 0>(m, cur, nxt, perm, ef, p, status, tiles, st); break;
    }
}

template <int NS>
void launch_moments(int v, int mode, const DevMesh& m, const DevState& s, const int* perm, const int* kstart,
                    unsigned long long* node_acc, unsigned long long* status, cudaStream_t st)
{
    const int64_t threads = (int64_t)m.n_tri * 32;
    if (mode == 1) {
        switch (v) {
            case 1: moments_kernel_df<NS, 128, 4><<<nblocks(threads, 128), 128, 0, st>>>(m, s, perm, kstart, node_acc, status); break;
            case 2: moments_kernel_df<NS, 512, 1><<<nblocks(threads, 512), 512, 0, st>>>(m, s, perm, kstart, node_acc, status); break;
            case 3: moments_kernel_df<NS, 256, 1><<<nblocks(threads, 256), 256, 0, st>>>(m, s, perm, kstart, node_acc, status); break;
            default: moments_kernel_df<NS, 256, 2><<<nblocks(threads, 256), 256, 0, st>>>(m, s, perm, kstart, node_acc, status); break;
        }
        return;
    }
    // sparsely populated elements (at most kHalfPpe particles per element on average): a half-warp
    // per element. The rule depends on the ensemble only, so every launch variant gives the same bits.
    if (s.n <= (int64_t)kHalfPpe * m.n_tri) {
        const int64_t ht = ((int64_t)m.n_tri + 1) / 2 * 32;
        switch (v) {
            case 1: moments_kernel_f32h<NS, 128, 4><<<nblocks(ht, 128), 128, 0, st>>>(m, s, perm, kstart, node_acc, status); break;
            case 2: moments_kernel_f32h<NS, 512, 1><<<nblocks(ht, 512), 512, 0, st>>>(m, s, perm, kstart, node_acc, status); break;
            case 3: moments_kernel_f32h<NS, 256, 3><<<nblocks(ht, 256), 256, 0, st>>>(m, s, perm, kstart, node_acc, status); break;
            default: moments_kernel_f32h<NS, 256, 2><<<nblocks(ht, 256), 256, 0, st>>>(m, s, perm, kstart, node_acc, status); break;
        }
        return;
    }
    switch (v) {
        case 1: moments_kernel_f32<NS, 128, 4><<<nblocks(threads, 128), 128, 0, st>>>(m, s, perm, kstart, node_acc, status); break;
        case 2: moments_kernel_f32<NS, 512, 1><<<nblocks(threads, 512), 512, 0, st>>>(m, s, perm, kstart, node_acc, status); break;
        case 3: moments_kernel_f32<NS, 256, 3><<<nblocks(threads, 256), 256, 0, st>>>(m, s, perm, kstart, node_acc, status); break;
        default: moments_kernel_f32<NS, 256, 2><<<nblocks(threads, 256), 256, 0, st>>>(m, s, perm, kstart, node_acc, status); break;
    }
}

template <int NS>
cudaError_t run_pipeline(const DevMesh& m, const DevState& cur, const DevState& nxt, const float* fields,
                         const StepParams& p, PipeScratch& w, unsigned long long* node_acc, unsigned long long* status,
                         cudaStream_t st, const cudaEvent_t* ev, const StepTune& tune, unsigned long long* flux_acc)
{
    const int64_t n = cur.n;
    if (n == 0) return cudaSuccess;
    const int E = m.n_tri;
    const int64_t nblk = (n + kBlk - 1) / kBlk;
    cudaError_t e = cudaMemsetAsync(w.kwork, 0, sizeof(int) * (3 * (size_t)(E + 1) + 1), st);
    if (e != cudaSuccess) return e;
    int* kcnt = w.kwork;
    int* krc = w.kwork + (E + 1);
    int* kcur = w.kwork + 2 * (E + 1);
    unsigned* tiles = reinterpret_cast<unsigned*>(w.kwork + 3 * (E + 1));
    if (ev) cudaEventRecord(ev[0], st);
    constexpr int NQ4 = (22 + NS + 3) / 4;
    element_fields_kernel<NS><<<nblocks((int64_t)E * NQ4, 256), 256, 0, st>>>(m, fields, w.efields);
    // the kernel with the least code that covers the mesh and the model: walls off the frame,
    // IECM or reactions (kind 2); several components (kind 1); the plain step (kind 0)
    if (m.edge_walls || p.beta || p.react_k > 0.0f)
        launch_advance<NS, 2>(tune.adv, m, cur, nxt, w.perm, w.efields, p, status, tiles, st);
    else if (m.n_comp > 1) launch_advance<NS, 1>(tune.adv, m, cur, nxt, w.perm, w.efields, p, status, tiles, st);
    else launch_advance<NS, 0>(tune.adv, m, cur, nxt, w.perm, w.efields, p, status, tiles, st);
    if (ev) cudaEventRecord(ev[1], st);
    histogram_kernel<<<(unsigned)((nblk + kHWarps - 1) / kHWarps), 32 * kHWarps, 0, st>>>(
        nxt.elem, n, w.rrank, w.rec_key, w.rec_cnt, w.nrec, kcnt, krc, status);
    e = scan_pair(kcnt, w.kstart, krc, w.krstart, E + 1, w.scan_part, st);
    if (e != cudaSuccess) return e;
    record_scatter_kernel<<<nblocks(nblk * 32, 256), 256, 0, st>>>(w.nrec, w.rec_key, w.krstart, kcur, w.klist, nblk);
    key_offsets_kernel<<<nblocks((int64_t)E * 32, 256), 256, 0, st>>>(E, w.kstart, w.krstart, w.klist, w.klist2,
                                                                       w.rec_cnt, w.rec_off);
    particle_scatter_kernel<<<nblocks(n, 256 * kScatterPer), 256, 0, st>>>(n, w.rrank, w.rec_off, w.perm_new);
    if (ev) cudaEventRecord(ev[2], st);
    launch_moments<NS>(tune.mom, p.moment_sums, m, nxt, w.perm_new, w.kstart, node_acc, status, st);
    if (flux_acc) {
        if (p.moment_sums == 1)
            moments_kernel_df<NS, 256, 2, true><<<nblocks((int64_t)E * 32, 256), 256, 0, st>>>(m, nxt, w.perm_new,
                                                                                             w.kstart, flux_acc, status);
        else
            moments_kernel_f32<NS, 256, 2, true><<<nblocks((int64_t)E * 32, 256), 256, 0, st>>>(m, nxt, w.perm_new,
                                                                                              w.kstart, flux_acc, status);
    }
    if (ev) cudaEventRecord(ev[3], st);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pdf_step_pipeline(const DevMesh& m, const DevState& cur, const DevState& nxt, int ns,
                                     const float* fields, const StepParams& p, PipeScratch& w,
                                     unsigned long long* node_acc, unsigned long long* status, cudaStream_t st,
                                     const cudaEvent_t* ev, const StepTune& tune, unsigned long long* flux_acc)
{
    switch (ns) {
        case 1: return run_pipeline<1>(m, cur, nxt, fields, p, w, node_acc, status, st, ev, tune, flux_acc);
        case 2: return run_pipeline<2>(m, cur, nxt, fields, p, w, node_acc, status, st, ev, tune, flux_acc);
        case 3: return run_pipeline<3>(m, cur, nxt, fields, p, w, node_acc, status, st, ev, tune, flux_acc);
        case 4: return run_pipeline<4>(m, cur, nxt, fields, p, w, node_acc, status, st, ev, tune, flux_acc);
        default: return cudaErrorInvalidValue;
    }
}

int sm_count() { return sm_count_cached(); }

cudaError_t launch_step_counter(unsigned long long* c, unsigned long long set, unsigned long long add, cudaStream_t st)
{
    step_counter_kernel<<<1, 1, 0, st>>>(c, set, add);
    return cudaGetLastError();
}

cudaError_t launch_iota(int* p, int64_t n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    iota_kernel<<<nblocks(n, 256), 256, 0, st>>>(p, n);
    return cudaGetLastError();
}

}  // namespace lpdf
