// The particle time step (sm_103a): one forward-Euler step of every particle of the joint
// velocity-frequency-scalar PDF method (arXiv:1006.0549, Section "Governing equations": Eq. 2,
// 4, 5, 6, 9 in IEM form (the static entry point's kernel; IECM and reactive sources run in the
// pipeline); statistics at particle positions; tracking through the unstructured
// grid), fused with the reduction of the new state's moments to the gridpoints.
//
// A persistent CTA (128 threads, four per SM) walks a contiguous range of 512-particle
// sub-tiles. Per sub-tile:
//   1. bulk copy (TMA) of the state rows into shared memory;
//   2. every thread advances its 4 particles (Eq. 4, 5, 9, 2, wrap, reflection, sources) in
//      place, then locates them with a pooled neighbour walk (the thread's 4 walks share one
//      loop, so lanes stay busy while their particles need different hop counts); the rows
//      go back to global memory by bulk copy while the reduction proceeds;
//   3. binning by new element: a shared-memory hash collects the distinct new elements, which
//      are numbered in ascending order (bins); per (bin, warp) counts and ranks come from
//      match_any on each 32-particle row; one block scan gives every bin its range of sorted
//      positions and its accumulation units (runs of at most kUnit particles, aligned to the
//      bin start);
//   4. each thread accumulates one unit in FP32 registers (lambda_a' q_k for the 3 corners and
//      the 11 + 2 ns quantities); after a barrier the tile is dead and becomes a column-major
//      scratch of all units' partials; thread i then takes (bin, column) tasks: it sums the
//      column over the bin's units, converts the sum once to 64-bit fixed point and adds it to
//      the CTA node table (one add per bin and column, no two threads on the same word).
// The bins, units and lanes are a function of the sub-tile's contents only, and integer
// addition is associative: the gridpoint sums are bit-reproducible.
#include <algorithm>
#include <cstddef>
#include <mutex>

#include "lpdf_device.cuh"

namespace lpdf {

namespace {

constexpr int kThreads = 128;
constexpr int kWarps = kThreads / 32;
constexpr int kPPT = 4;                       // particles per thread per sub-tile
constexpr int kT = kThreads * kPPT;           // sub-tile: 512 particles
constexpr int kUnit = 6;                      // particles per accumulation unit
constexpr int kMaxBins = kThreads;            // distinct new elements per sub-tile (more: direct path)
constexpr int kHash = 2 * kThreads;           // bin hash slots
constexpr int kMaxUnits = kT / kUnit + kMaxBins;
constexpr unsigned short kNoBin = 0xFFFF;
constexpr int kScrPitch = kThreads + 1;       // hand-over scratch: [column][unit], padded

template <int NS>
struct Smem {
    static constexpr int NF = 8 + NS;         // x, y, u, v, w, omega, psi[NS], elem, pid
    static constexpr int NQ = 11 + 2 * NS;
    static constexpr int NT = 128;            // node-table slots
    static constexpr int F_X = 0, F_Y = 1, F_U = 2, F_V = 3, F_W = 4, F_OM = 5, F_PSI = 6, F_ELEM = 6 + NS,
                         F_PID = 7 + NS;
    alignas(128) float tile[NF][kT];          // bulk-copy rows (16-byte aligned)
    float lam[3][kT];                         // barycentrics of the new position in the new element
    unsigned short perm[kT];                  // sorted position -> tile index (first: bin key list)
    unsigned short ubin[kMaxUnits];           // unit -> bin
    int hkey[kHash];                          // bin hash: element id per slot, -1 empty
    unsigned short hbin[kHash];
    int binel[kMaxBins];                      // bin -> element
    unsigned short wcnt[kMaxBins][kWarps];    // counts per (bin, warp), then absolute offsets
    unsigned short bstart[kMaxBins + 1];
    unsigned short ustart[kMaxBins + 1];
    short cslot[kMaxBins][3];                 // node-table slot of each bin's corners (-1: global)
    int wsum[kWarps];
    int nbins, nunits, tfill, abort;
    NodeTable<NQ, NT> table;
    unsigned long long bar;
};

// the hand-over scratch (3 NQ columns x kScrPitch) lives in the tile and lam rows
template <int NS>
constexpr bool scratch_fits()
{
    return offsetof(Smem<NS>, lam) == sizeof(((Smem<NS>*)nullptr)->tile) &&
           (size_t)3 * Smem<NS>::NQ * kScrPitch * sizeof(float) <=
               sizeof(((Smem<NS>*)nullptr)->tile) + sizeof(((Smem<NS>*)nullptr)->lam);
}
static_assert(scratch_fits<1>() && scratch_fits<2>() && scratch_fits<3>() && scratch_fits<4>(), "scratch");
// four CTAs per SM: 228 KB of shared memory per SM, 1 KB of it reserved per CTA
static_assert(sizeof(Smem<1>) <= 56 * 1024 && sizeof(Smem<2>) <= 56 * 1024 && sizeof(Smem<3>) <= 56 * 1024 &&
                  sizeof(Smem<4>) <= 56 * 1024,
              "four CTAs per SM");

// exclusive block scan over kThreads threads; `total` gets the sum. Contains two barriers.
__device__ __forceinline__ int block_scan(int v, int* wsum, int& total)
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
    int off = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const int s = wsum[w];
        off += w < wid ? s : 0;
        tot += s;
    }
    __syncthreads();
    total = tot;
    return off + incl - v;
}

// The exact walk test with its weights returned by value (a small struct travels through the
// call's parameter space): the walk's own variables never have their address taken, so they are
// not given a home in local memory.
struct WalkLam {
    int code;   // kWalkIn, or the exit as walk_test's `next`
    float l0, l1, l2;
};
static __device__ __noinline__ WalkLam walk_test_lam(const DevMesh& M, int e, float px, float py)
{
    float lam[3] = {0.0f, 0.0f, 0.0f};
    WalkLam r;
    r.code = walk_decide(M, e, px, py, lam);
    r.l0 = lam[0];
    r.l1 = lam[1];
    r.l2 = lam[2];
    return r;
}

__device__ __forceinline__ unsigned hash_slot(int key) { return ((unsigned)key * 2654435761u) >> 24; }   // 8 bits
static_assert(kHash == 256, "hash_slot gives 8 bits");

// node-table slot of `node`, counting new insertions in `fill`
template <int NQ, int NT>
__device__ __forceinline__ int table_slot_counted(NodeTable<NQ, NT>& T, int node, int* fill)
{
    const unsigned h = ((unsigned)node * 2654435761u) >> 9;
#pragma unroll 1
    for (int p = 0; p < kProbe; ++p) {
        const int s = (h + p) & (NT - 1);
        const int k = T.key[s];
        if (k == node) return s;
        if (k == -1) {
            const int old = atomicCAS(&T.key[s], -1, node);
            if (old == -1) {
                atomicAdd(fill, 1);
                return s;
            }
            if (old == node) return s;
        }
    }
    return -1;
}

// ------------------------------------------------------------------------------------------
// The particle in tile column t: advanced in place (the element row keeps the walk's start).
// ------------------------------------------------------------------------------------------
template <int NS>
__device__ __forceinline__ void advance_state(const DevMesh& M, const float* __restrict__ F, const StepParams& P,
                                              Smem<NS>& sm, int t, unsigned& err, bool& bad)
{
    using SM = Smem<NS>;
    ParticleState<NS> q;
    q.x = sm.tile[SM::F_X][t];
    q.y = sm.tile[SM::F_Y][t];
    q.u = sm.tile[SM::F_U][t];
    q.v = sm.tile[SM::F_V][t];
    q.w = sm.tile[SM::F_W][t];
    q.om = sm.tile[SM::F_OM][t];
#pragma unroll
    for (int a = 0; a < NS; ++a) q.psi[a] = sm.tile[SM::F_PSI + a][t];
    q.elem = __float_as_int(sm.tile[SM::F_ELEM][t]);
    q.pid = __float_as_uint(sm.tile[SM::F_PID][t]);
    advance_particle<NS>(M, F, P, q, err, bad);
    sm.tile[SM::F_X][t] = q.x;
    sm.tile[SM::F_Y][t] = q.y;
    sm.tile[SM::F_U][t] = q.u;
    sm.tile[SM::F_V][t] = q.v;
    sm.tile[SM::F_W][t] = q.w;
    sm.tile[SM::F_OM][t] = q.om;
#pragma unroll
    for (int a = 0; a < NS; ++a) sm.tile[SM::F_PSI + a][t] = q.psi[a];
    sm.tile[SM::F_ELEM][t] = __int_as_float(q.elem);
}

// moment quantities of the particle in tile column t: 1, u, v, w, uu, uv, uw, vv, vw, ww, omega,
// psi_a, psi_a^2
template <int NS>
__device__ __forceinline__ void quantities(const Smem<NS>& sm, int t, float* q)
{
    using SM = Smem<NS>;
    const float u = sm.tile[SM::F_U][t], v = sm.tile[SM::F_V][t], w = sm.tile[SM::F_W][t];
    q[0] = 1.0f; q[1] = u; q[2] = v; q[3] = w;
    q[4] = u * u; q[5] = u * v; q[6] = u * w; q[7] = v * v; q[8] = v * w; q[9] = w * w;
    q[10] = sm.tile[SM::F_OM][t];
#pragma unroll
    for (int a = 0; a < NS; ++a) {
        const float ps = sm.tile[SM::F_PSI + a][t];
        q[11 + a] = ps;
        q[11 + NS + a] = ps * ps;
    }
}

// statistics node of corner c of bin b: the node-table key of its slot, else from the mesh
template <int NS>
__device__ __forceinline__ int bin_node(const Smem<NS>& sm, const DevMesh& M, int b, int c)
{
    const int slot = sm.cslot[b][c];
    if (slot >= 0) return sm.table.key[slot];
    const int4 mv = __ldg(&M.em[sm.binel[b]]);
    return c == 0 ? mv.x : (c == 1 ? mv.y : mv.z);
}

template <int NS>
__device__ __forceinline__ void flush_table(Smem<NS>& sm, unsigned long long* __restrict__ node_acc)
{
    using SM = Smem<NS>;
    constexpr int NQ = SM::NQ, NT = SM::NT;
    for (int i = threadIdx.x; i < NT * NQ; i += kThreads) {
        const int s = i / NQ, q = i - (i / NQ) * NQ;
        const int node = sm.table.key[s];
        const unsigned long long v = sm.table.acc[s][q];
        if (node >= 0 && v != 0ull) atomicAdd(&node_acc[(size_t)node * NQ + q], v);
        sm.table.acc[s][q] = 0ull;
    }
    __syncthreads();
    for (int s = threadIdx.x; s < NT; s += kThreads) sm.table.key[s] = -1;
    if (threadIdx.x == 0) sm.tfill = 0;
    __syncthreads();
}

template <int NS>
__global__ void __launch_bounds__(kThreads, 4)
pdf_step_kernel(const __grid_constant__ DevMesh M, const __grid_constant__ DevState S, const float* __restrict__ F,
                const __grid_constant__ StepParams P, unsigned long long* __restrict__ node_acc,
                unsigned long long* __restrict__ status, int64_t tiles_per_cta, int use_bulk)
{
    using SM = Smem<NS>;
    constexpr int NF = SM::NF, NQ = SM::NQ, NK = 3 * NQ, NT = SM::NT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SM& sm = *reinterpret_cast<SM*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int i = tid; i < NT; i += kThreads) sm.table.key[i] = -1;
    for (int i = tid; i < NT * NQ; i += kThreads) (&sm.table.acc[0][0])[i] = 0ull;
    if (tid == 0) {
        sm.tfill = 0;
        sm.abort = 0;
        mbar_init(&sm.bar, 1);
    }
    __syncthreads();

    unsigned err = 0;
    int hops = 0;
    uint32_t phase = 0;
    // global row of field f (psi rows are `cap` apart)
    auto grow = [&](int f) -> float* {
        if (f == SM::F_X) return S.x;
        if (f == SM::F_Y) return S.y;
        if (f == SM::F_U) return S.u;
        if (f == SM::F_V) return S.v;
        if (f == SM::F_W) return S.w;
        if (f == SM::F_OM) return S.om;
        if (f == SM::F_ELEM) return reinterpret_cast<float*>(S.elem);
        if (f == SM::F_PID) return reinterpret_cast<float*>(S.pid);
        return S.psi + (size_t)(f - SM::F_PSI) * S.cap;
    };

    const int64_t ntiles = (S.n + kT - 1) / kT;
    const int64_t tile0 = (int64_t)blockIdx.x * tiles_per_cta;
    const int64_t tile1 = min(ntiles, tile0 + tiles_per_cta);
    // the tile loop is uniform over the CTA (it contains CTA barriers)
    for (int64_t ti = tile0; ti < tile1; ++ti) {
        const int64_t base = ti * kT;
        const int nvalid = (int)min((int64_t)kT, S.n - base);
        const bool bulk = use_bulk && nvalid == kT;
        // ---- 1. stage the state rows -------------------------------------------------------
        if (bulk) {
            if (tid == 0) {
                bulk_wait_read_all();   // the previous sub-tile's bulk store has read the rows
                mbar_expect_tx(&sm.bar, (uint32_t)(NF * kT * sizeof(float)));
#pragma unroll
                for (int f = 0; f < NF; ++f) bulk_load(&sm.tile[f][0], grow(f) + base, kT * sizeof(float), &sm.bar);
            }
            bool ok = mbar_wait_bounded(&sm.bar, phase);
            if (__syncthreads_or(!ok)) {
                // give the copies in flight one more bounded wait, then stop this CTA's work
                if (tid == 0) {
                    mbar_wait_bounded(&sm.bar, phase);
                    atomicOr(&status[0], (unsigned long long)kErrTimeout);
                }
                break;
            }
            phase ^= 1u;
        } else {
            if (tid == 0) bulk_wait_read_all();
            __syncthreads();
            for (int f = 0; f < NF; ++f) {
                const float* g = grow(f) + base;
                for (int i = tid; i < nvalid; i += kThreads) sm.tile[f][i] = g[i];
            }
            __syncthreads();
        }
        // ---- 2a. advance the thread's particles (tile columns tid + 256 j) -------------------
        unsigned badmask = 0;
#pragma unroll 1
        for (int j = 0; j < kPPT; ++j) {
            const int t = j * kThreads + tid;
            if (t < nvalid) {
                bool bad;
                advance_state<NS>(M, F, P, sm, t, err, bad);
                badmask |= (unsigned)bad << j;
            }
        }
        // ---- 2b. pooled neighbour walk: two walks in flight per thread ---------------------------
        int mykey[kPPT];                       // new element per particle, -1 for none
#pragma unroll
        for (int j = 0; j < kPPT; ++j) mykey[j] = -1;
        {
            struct Walk {
                int j, e, e0, h;
                float px, py;
            };
            int jn = 0;                            // next particle of this thread to start
            auto start = [&](Walk& w) {
                const int t = jn * kThreads + tid;
                if (jn < kPPT && t < nvalid) {
                    w.j = jn++;
                    w.e = w.e0 = __float_as_int(sm.tile[SM::F_ELEM][t]);
                    w.px = sm.tile[SM::F_X][t];
                    w.py = sm.tile[SM::F_Y][t];
                    w.h = 0;
                } else {
                    w.j = -1;
                    w.e = 0;
                }
            };
            // one test of walk w; on a stop, record the particle and start the next one
            auto step = [&](Walk& w, bool found, int next, float* lam) {
                if (!(found || next < 0 || w.h >= kHopCap)) {
                    w.e = next;
                    ++w.h;
                    return;
                }
                const int t = w.j * kThreads + tid;
                int ne = w.e;
                bool lost = !found;
                hops += found ? w.h : (next < 0 ? w.h : kHopCap + 1);
                if (lost) {
                    ne = w.e0;
                    barycentric(__ldg(&M.ex[ne]), __ldg(&M.ey[ne]), w.px, w.py, lam[0], lam[1], lam[2]);
                }
                if ((badmask >> w.j) & 1u) lost = true;
                if (lost) {
                    err |= kErrLost;
                    atomicAdd(&status[1], 1ull);
                    atomicCAS(&status[2], ~0ull, (unsigned long long)__float_as_uint(sm.tile[SM::F_PID][t]));
                }
                sm.tile[SM::F_ELEM][t] = __int_as_float(ne);
                sm.lam[0][t] = lam[0];
                sm.lam[1][t] = lam[1];
                sm.lam[2][t] = lam[2];
                // w.j is thread-divergent: select the register without dynamic indexing
#pragma unroll
                for (int jj = 0; jj < kPPT; ++jj)
                    if (jj == w.j) mykey[jj] = ne;
                start(w);
            };
            Walk A, B;
            start(A);
            start(B);
#pragma unroll 1
            while (A.j >= 0 || B.j >= 0) {
                WalkLam ra = {kWalkIn, 0.0f, 0.0f, 0.0f}, rb = ra;
                if (A.j >= 0) ra = walk_test_lam(M, A.e, A.px, A.py);
                if (B.j >= 0) rb = walk_test_lam(M, B.e, B.px, B.py);
                if (A.j >= 0) {
                    float la[3] = {ra.l0, ra.l1, ra.l2};
                    step(A, ra.code == kWalkIn, ra.code == kWalkIn ? -1 : ra.code, la);
                }
                if (B.j >= 0) {
                    float lb[3] = {rb.l0, rb.l1, rb.l2};
                    step(B, rb.code == kWalkIn, rb.code == kWalkIn ? -1 : rb.code, lb);
                }
            }
        }
        // ---- 3a. insert the new elements into the bin hash (one insert per distinct key of a row)
        for (int i = tid; i < kHash; i += kThreads) sm.hkey[i] = -1;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kPPT; ++j) {
            const int k = mykey[j];
            const unsigned m = __match_any_sync(kFull, k);
            if (k >= 0 && lane == __ffs(m) - 1) {
                const unsigned h0 = hash_slot(k);
#pragma unroll 1
                for (int p = 0; p < kHash; ++p) {
                    const int s = (h0 + p) & (kHash - 1);
                    const int cur = sm.hkey[s];
                    if (cur == k) break;
                    if (cur == -1) {
                        const int old = atomicCAS(&sm.hkey[s], -1, k);
                        if (old == -1 || old == k) break;
                    }
                }
            }
        }
        // the state rows are final: write them back (every field but pid) while the reduction runs
        fence_async_shared();
        __syncthreads();
        if (bulk) {
            if (tid == 0) {
#pragma unroll
                for (int f = 0; f < NF - 1; ++f) bulk_store(grow(f) + base, &sm.tile[f][0], kT * sizeof(float));
                bulk_commit();
            }
        } else {
            for (int f = 0; f < NF - 1; ++f) {
                float* g = grow(f) + base;
                for (int i = tid; i < nvalid; i += kThreads) g[i] = sm.tile[f][i];
            }
        }
        // ---- 3b. bins: the distinct new elements in ascending order -------------------------------
        {
            int* const list = reinterpret_cast<int*>(sm.perm);   // kHash ints fit in perm
            const int s0 = 2 * tid, s1 = 2 * tid + 1;
            const int k0 = sm.hkey[s0], k1 = sm.hkey[s1];
            const int o0 = k0 >= 0, o1 = k1 >= 0;
            int total;
            const int c0 = block_scan(o0 + o1, sm.wsum, total);
            if (o0) list[c0] = k0;
            if (o1) list[c0 + o0] = k1;
            __syncthreads();
            // rank among the distinct keys (keys are distinct: a count of the smaller ones)
            int r0 = 0, r1 = 0;
            if (o0 | o1) {
#pragma unroll 4
                for (int i = 0; i < total; ++i) {
                    const int k = list[i];
                    r0 += k < k0;
                    r1 += k < k1;
                }
            }
            if (o0) {
                sm.hbin[s0] = r0 < kMaxBins ? (unsigned short)r0 : kNoBin;
                if (r0 < kMaxBins) sm.binel[r0] = k0;
            }
            if (o1) {
                sm.hbin[s1] = r1 < kMaxBins ? (unsigned short)r1 : kNoBin;
                if (r1 < kMaxBins) sm.binel[r1] = k1;
            }
            const int nb = min(total, kMaxBins);
            if (tid == 0) sm.nbins = nb;
            for (int i = tid; i < nb * kWarps; i += kThreads) (&sm.wcnt[0][0])[i] = 0;
        }
        __syncthreads();
        // ---- 3c. per (bin, warp) counts and ranks, row by row --------------------------------
        unsigned short mybin[kPPT];
        int myrank[kPPT];
#pragma unroll
        for (int j = 0; j < kPPT; ++j) {
            const int k = mykey[j];
            unsigned short b = kNoBin;
            if (k >= 0) {
                const unsigned h0 = hash_slot(k);
#pragma unroll 1
                for (int p = 0; p < kHash; ++p) {
                    const int s = (h0 + p) & (kHash - 1);
                    const int cur = sm.hkey[s];
                    if (cur == k) { b = sm.hbin[s]; break; }
                    if (cur == -1) break;
                }
            }
            mybin[j] = b;
            const unsigned m = __match_any_sync(kFull, (int)b);
            const int leader = __ffs(m) - 1;
            int prefix = 0;
            if (b != kNoBin && lane == leader) {
                prefix = sm.wcnt[b][wid];
                sm.wcnt[b][wid] = (unsigned short)(prefix + __popc(m));
            }
            prefix = __shfl_sync(kFull, prefix, leader);
            myrank[j] = prefix + __popc(m & lt);
        }
        __syncthreads();
        // ---- 4. bin ranges and accumulation units (one block scan of packed counts) -----------
        {
            const int nb = sm.nbins;
            int packed = 0, n_b = 0;
            if (tid < nb) {
#pragma unroll
                for (int w = 0; w < kWarps; ++w) {
                    const int c = sm.wcnt[tid][w];
                    sm.wcnt[tid][w] = (unsigned short)n_b;
                    n_b += c;
                }
                packed = n_b | (((n_b + kUnit - 1) / kUnit) << 16);
            }
            int total;
            const int excl = block_scan(packed, sm.wsum, total);
            if (tid < nb) {
                const int bs = excl & 0xFFFF;
                sm.bstart[tid] = (unsigned short)bs;
                sm.ustart[tid] = (unsigned short)(excl >> 16);
#pragma unroll
                for (int w = 0; w < kWarps; ++w) sm.wcnt[tid][w] = (unsigned short)(sm.wcnt[tid][w] + bs);
            }
            if (tid == 0) {
                sm.bstart[nb] = (unsigned short)(total & 0xFFFF);
                sm.ustart[nb] = (unsigned short)(total >> 16);
                sm.nunits = total >> 16;
            }
        }
        __syncthreads();
        // ---- 5. sorted positions, unit -> bin, node-table slots of the bins' corners ---------
        {
            const int nb = sm.nbins;
#pragma unroll
            for (int j = 0; j < kPPT; ++j) {
                const unsigned short b = mybin[j];
                if (b == kNoBin) continue;
                const int pos = sm.wcnt[b][wid] + myrank[j];
                if (consistent(pos < kT, err)) sm.perm[pos] = (unsigned short)(j * kThreads + tid);
            }
            if (tid < nb)
                for (int u = sm.ustart[tid]; u < sm.ustart[tid + 1]; ++u)
                    if (consistent(u < kMaxUnits, err)) sm.ubin[u] = (unsigned short)tid;
            for (int i = tid; i < 3 * nb; i += kThreads) {
                const int b = i / 3, c = i - 3 * (i / 3);
                const int ek = sm.binel[b];
                if (!consistent(ek >= 0 && ek < M.n_tri, err)) { sm.cslot[b][c] = -1; continue; }
                const int4 mv = __ldg(&M.em[ek]);
                const int node = c == 0 ? mv.x : (c == 1 ? mv.y : mv.z);
                sm.cslot[b][c] = (short)table_slot_counted(sm.table, node, &sm.tfill);
            }
        }
        __syncthreads();
        // ---- 6. accumulate units; hand the partials to column owners -------------------------
        {
            const int nu = min(sm.nunits, kMaxUnits);
            const int nb = sm.nbins;
            float acc[NK];
            // accumulate unit u into acc (sorted positions of its bin, two particles per pass)
            auto accumulate = [&](int u, int b) {
#pragma unroll
                for (int k = 0; k < NK; ++k) acc[k] = 0.0f;
                const int p0 = sm.bstart[b] + (u - sm.ustart[b]) * kUnit;
                const int p1 = min(p0 + kUnit, (int)sm.bstart[b + 1]);
                int p = p0;
#pragma unroll 1
                for (; p + 1 < p1; p += 2) {
                    const int t0 = sm.perm[p], t1 = sm.perm[p + 1];
                    if (!consistent(t0 < kT && t1 < kT, err)) return;
                    const float a0 = sm.lam[0][t0], a1 = sm.lam[1][t0], a2 = sm.lam[2][t0];
                    const float c0 = sm.lam[0][t1], c1 = sm.lam[1][t1], c2 = sm.lam[2][t1];
                    float q0[NQ], q1[NQ];
                    quantities<NS>(sm, t0, q0);
                    quantities<NS>(sm, t1, q1);
#pragma unroll
                    for (int k = 0; k < NQ; ++k) {
                        acc[k] = fmaf(c0, q1[k], fmaf(a0, q0[k], acc[k]));
                        acc[NQ + k] = fmaf(c1, q1[k], fmaf(a1, q0[k], acc[NQ + k]));
                        acc[2 * NQ + k] = fmaf(c2, q1[k], fmaf(a2, q0[k], acc[2 * NQ + k]));
                    }
                }
                if (p < p1) {
                    const int t0 = sm.perm[p];
                    if (!consistent(t0 < kT, err)) return;
                    const float a0 = sm.lam[0][t0], a1 = sm.lam[1][t0], a2 = sm.lam[2][t0];
                    float q0[NQ];
                    quantities<NS>(sm, t0, q0);
#pragma unroll
                    for (int k = 0; k < NQ; ++k) {
                        acc[k] = fmaf(a0, q0[k], acc[k]);
                        acc[NQ + k] = fmaf(a1, q0[k], acc[NQ + k]);
                        acc[2 * NQ + k] = fmaf(a2, q0[k], acc[2 * NQ + k]);
                    }
                }
            };
            // units beyond the first kThreads (sub-tiles spread over many elements): added
            // straight to the node table, one unit at a time
#pragma unroll 1
            for (int u = tid + kThreads; u < nu; u += kThreads) {
                const int b = sm.ubin[u];
                if (!consistent(b < nb, err)) continue;
                accumulate(u, b);
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int k = 0; k < NQ; ++k)
                        table_add(sm.table, (int)sm.cslot[b][c], bin_node(sm, M, b, c), k,
                                  to_fixed(acc[c * NQ + k], err), node_acc);
            }
            // particles without a bin (more than kMaxBins distinct elements in the sub-tile)
#pragma unroll 1
            for (int j = 0; j < kPPT; ++j) {
                const int t = j * kThreads + tid;
                if (mybin[j] != kNoBin || mykey[j] < 0) continue;
                const int4 mv = __ldg(&M.em[mykey[j]]);
                const int nd[3] = {mv.x, mv.y, mv.z};
                float q[NQ];
                quantities<NS>(sm, t, q);
                for (int c = 0; c < 3; ++c) {
                    const float l = sm.lam[c][t];
                    for (int k = 0; k < NQ; ++k) {
                        const long long v = to_fixed(l * q[k], err);
                        if (v != 0) atomicAdd(&node_acc[(size_t)nd[c] * NQ + k], (unsigned long long)v);
                    }
                }
            }
            // the first kThreads units: one per thread
            int b = -1;
            if (tid < nu) {
                b = sm.ubin[tid];
                if (consistent(b < nb, err)) accumulate(tid, b);
                else b = -1;
            }
            if (b < 0) {
#pragma unroll
                for (int k = 0; k < NK; ++k) acc[k] = 0.0f;
            }
            // every read of the tile (and the bulk store's) is over: the tile becomes the scratch
            if (tid == 0) bulk_wait_read_all();
            __syncthreads();
            float* const scr = &sm.tile[0][0];
#pragma unroll
            for (int k = 0; k < NK; ++k) scr[k * kScrPitch + tid] = acc[k];
            __syncthreads();
            // (bin, column) tasks: the column summed over the bin's units (those of the first kThreads)
            const int ntask = nb * NK;
#pragma unroll 1
            for (int i = tid; i < ntask; i += kThreads) {
                const int bb = i / NK, k = i - (i / NK) * NK;
                const int c = k / NQ, q = k - c * NQ;
                const int u0 = sm.ustart[bb], u1 = min((int)sm.ustart[bb + 1], kThreads);
                const float* col = scr + k * kScrPitch;
                float sum = 0.0f;
                for (int u = u0; u < u1; ++u) sum += col[u];
                if (u1 > u0)
                    table_add(sm.table, (int)sm.cslot[bb][c], bin_node(sm, M, bb, c), q, to_fixed(sum, err), node_acc);
            }
        }
        // generic reads of the tile are done before the next bulk load overwrites it
        fence_async_shared();
        __syncthreads();
        if (sm.tfill > NT / 2) flush_table<NS>(sm, node_acc);
    }
    // every bulk store must be complete before the CTA exits
    if (tid == 0) bulk_wait_all();
    __syncthreads();
    flush_table<NS>(sm, node_acc);
    // ---- status -------------------------------------------------------------------------------
    const unsigned e_or = __reduce_or_sync(kFull, err);
    const int h_sum = __reduce_add_sync(kFull, hops);
    if (lane == 0) {
        if (e_or) atomicOr(&status[0], (unsigned long long)e_or);
        if (h_sum) atomicAdd(&status[3], (unsigned long long)h_sum);
    }
}

template <int NS>
cudaError_t launch_step_ns(const DevMesh& m, const DevState& s, const float* fields, const StepParams& p,
                           unsigned long long* node_acc, unsigned long long* status, cudaStream_t st)
{
    const size_t smem = sizeof(Smem<NS>);
    // the shared-memory opt-in and the SM count belong to the device that is current: kept per
    // device, set once under a lock (host threads may call from several devices at once)
    constexpr int kMaxDev = 64;
    static std::mutex mu;
    static int sm_of_dev[kMaxDev] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    int n_sm = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (sm_of_dev[dev] == 0) {
            e = cudaFuncSetAttribute(pdf_step_kernel<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            int c = 0;
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
            sm_of_dev[dev] = c > 0 ? c : 1;
        }
        n_sm = sm_of_dev[dev];
    }
    const int64_t ntiles = (s.n + kT - 1) / kT;
    if (ntiles == 0) return cudaSuccess;
    // persistent CTAs, four per SM, each on a contiguous range of sub-tiles
    const int64_t grid = std::min<int64_t>(ntiles, 4 * (int64_t)n_sm);
    const int64_t per = (ntiles + grid - 1) / grid;
    const int64_t used = (ntiles + per - 1) / per;
    // bulk copies need 16-byte aligned rows: every base pointer and the psi row stride
    auto al = [](const void* q) { return ((uintptr_t)q & 15u) == 0; };
    const int use_bulk = al(s.x) && al(s.y) && al(s.u) && al(s.v) && al(s.w) && al(s.om) && al(s.psi) && al(s.elem) &&
                         al(s.pid) && (s.cap % 4 == 0);
    pdf_step_kernel<NS><<<(unsigned)used, kThreads, smem, st>>>(m, s, fields, p, node_acc, status, per, use_bulk);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pdf_step(const DevMesh& m, const DevState& s, int ns, const float* fields, const StepParams& p,
                            unsigned long long* node_acc, unsigned long long* status, cudaStream_t st)
{
    switch (ns) {
        case 1: return launch_step_ns<1>(m, s, fields, p, node_acc, status, st);
        case 2: return launch_step_ns<2>(m, s, fields, p, node_acc, status, st);
        case 3: return launch_step_ns<3>(m, s, fields, p, node_acc, status, st);
        case 4: return launch_step_ns<4>(m, s, fields, p, node_acc, status, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lpdf
