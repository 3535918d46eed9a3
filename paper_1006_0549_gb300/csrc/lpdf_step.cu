// The particle time step (sm_103a): one forward-Euler step of every particle of the joint
// velocity-frequency-scalar PDF method (arXiv:1006.0549, Section "Governing equations": Eq. 2,
// 4, 5, 6, 9 in IEM form; statistics at particle positions; tracking through the unstructured
// grid), fused with the reduction of the new state's moments to the gridpoints.
//
// A persistent CTA (256 threads, two per SM) walks a contiguous range of 1024-particle
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
//   4. each thread accumulates whole units in FP32 registers (lambda_a' q_k for the 3 corners
//      and the 11 + 2 ns quantities); the warp then hands its units' partials through a small
//      shared scratch, kGroup lanes at a time, to column owners: lane k sums column k over each
//      run of equal bins, converts the sum once to 64-bit fixed point and adds it to the CTA
//      node table (no two lanes of a warp add to the same word).
// The bins, units and lanes are a function of the sub-tile's contents only, and integer
// addition is associative: the gridpoint sums are bit-reproducible.
#include <algorithm>

#include "lpdf_device.cuh"

namespace lpdf {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kPPT = 4;                       // particles per thread per sub-tile
constexpr int kT = kThreads * kPPT;           // sub-tile: 1024 particles
constexpr int kUnit = 8;                      // particles per accumulation unit
constexpr int kMaxBins = 256;                 // distinct new elements per sub-tile (more: direct path)
constexpr int kHash = 512;                    // bin hash slots
constexpr int kMaxUnits = kT / kUnit + kMaxBins;
constexpr unsigned short kNoBin = 0xFFFF;
constexpr int kGroup = 8;                     // lanes per hand-over of unit partials

template <int NS>
struct Smem {
    static constexpr int NF = 8 + NS;         // x, y, u, v, w, omega, psi[NS], elem, pid
    static constexpr int NQ = 11 + 2 * NS;
    static constexpr int NT = NS <= 2 ? 256 : 128;   // node-table slots
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
    float scr[kWarps][kGroup][3 * NQ];        // unit partials on their way to the column owners
    int sbin[kWarps][kGroup];
    int wsum[kWarps];
    int nbins, nunits, tfill, abort;
    NodeTable<NQ, NT> table;
    unsigned long long bar;
};

static_assert(sizeof(Smem<1>) <= 112 * 1024 && sizeof(Smem<2>) <= 112 * 1024 && sizeof(Smem<3>) <= 112 * 1024 &&
                  sizeof(Smem<4>) <= 112 * 1024,
              "two CTAs per SM");

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

__device__ __forceinline__ unsigned hash_slot(int key) { return ((unsigned)key * 2654435761u) >> 23; }   // 9 bits

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
// Eq. 4, 5, 9 (IEM), 2; wrap and reflection; sources, for the particle in tile column t.
// The new state replaces the old one in the tile; the element row keeps the walk's start
// (the old element, or 0 when it is outside the mesh: `bad`).
// ------------------------------------------------------------------------------------------
template <int NS>
__device__ __forceinline__ void advance_state(const DevMesh& M, const float* __restrict__ F, const StepParams& P,
                                              Smem<NS>& sm, int t, unsigned& err, bool& bad)
{
    using SM = Smem<NS>;
    constexpr int NFP = (22 + NS + 3) / 4 * 4;
    const float x = sm.tile[SM::F_X][t], y = sm.tile[SM::F_Y][t];
    const float u = sm.tile[SM::F_U][t], v = sm.tile[SM::F_V][t], w = sm.tile[SM::F_W][t];
    const float om = sm.tile[SM::F_OM][t];
    const int elem = __float_as_int(sm.tile[SM::F_ELEM][t]);
    const uint32_t pid = __float_as_uint(sm.tile[SM::F_PID][t]);
    bad = (unsigned)elem >= (unsigned)M.n_tri;
    const int e = bad ? 0 : elem;
    const float4 X = __ldg(&M.ex[e]);
    const float4 Y = __ldg(&M.ey[e]);
    const int4 V = __ldg(&M.ev[e]);
    float l0, l1, l2;
    barycentric(X, Y, x, y, l0, l1, l2);
    // linear shape-function interpolation of the node fields
    float Fi[NFP];
    {
        const float4* R0 = reinterpret_cast<const float4*>(F) + (size_t)V.x * (NFP / 4);
        const float4* R1 = reinterpret_cast<const float4*>(F) + (size_t)V.y * (NFP / 4);
        const float4* R2 = reinterpret_cast<const float4*>(F) + (size_t)V.z * (NFP / 4);
#pragma unroll
        for (int q = 0; q < NFP / 4; ++q) {
            const float4 a = __ldg(R0 + q), b = __ldg(R1 + q), c = __ldg(R2 + q);
            Fi[4 * q + 0] = fmaf(l0, a.x, fmaf(l1, b.x, l2 * c.x));
            Fi[4 * q + 1] = fmaf(l0, a.y, fmaf(l1, b.y, l2 * c.y));
            Fi[4 * q + 2] = fmaf(l0, a.z, fmaf(l1, b.z, l2 * c.z));
            Fi[4 * q + 3] = fmaf(l0, a.w, fmaf(l1, b.w, l2 * c.w));
        }
    }
    // Wiener increments: Philox blocks 0 and 1 of counter (pid, step, 0<<16 | block)
    const uint4 r0 = philox4x32_10(make_uint4(pid, P.step_lo, P.step_hi, 0u), P.key0, P.key1);
    const uint4 r1 = philox4x32_10(make_uint4(pid, P.step_lo, P.step_hi, 1u), P.key0, P.key1);
    float z0, z1, z2, z3, z4, z5;
    box_muller(r0.x, r0.y, z0, z1);
    box_muller(r0.z, r0.w, z2, z3);
    box_muller(r1.x, r1.y, z4, z5);
    const float dW1 = P.sdt * z0, dW2 = P.sdt * z1;
    const float c0e = sqrtf(fmaxf(Fi[LPDF_F_C0EPS], 0.0f));
    const float Ur = u - Fi[LPDF_F_U + 0], Vr = v - Fi[LPDF_F_U + 1], Wr = w - Fi[LPDF_F_U + 2];
    // Eq. 4
    float un = u + (-Fi[LPDF_F_DPDX] + P.nu2 * Fi[LPDF_F_LAPU] + Fi[LPDF_F_G11] * Ur + Fi[LPDF_F_G11 + 1] * Vr) * P.dt
             + P.s2nu * (Fi[LPDF_F_DUDX] * dW1 + Fi[LPDF_F_DUDX + 1] * dW2) + c0e * (P.sdt * z2);
    float vn = v + (-Fi[LPDF_F_DPDX + 1] + P.nu2 * Fi[LPDF_F_LAPU + 1] + Fi[LPDF_F_G11 + 2] * Ur
                    + Fi[LPDF_F_G11 + 3] * Vr) * P.dt
             + P.s2nu * (Fi[LPDF_F_DUDX + 2] * dW1 + Fi[LPDF_F_DUDX + 3] * dW2) + c0e * (P.sdt * z3);
    float wn = w + (P.nu2 * Fi[LPDF_F_LAPU + 2] + Fi[LPDF_F_G11 + 4] * Wr) * P.dt
             + P.s2nu * (Fi[LPDF_F_DUDX + 4] * dW1 + Fi[LPDF_F_DUDX + 5] * dW2) + c0e * (P.sdt * z4);
    // Eq. 5 (S_omega of Eq. 6 is a node field)
    const float Om = Fi[LPDF_F_OMEGA];
    float omn = om - P.C3 * Om * (om - Om) * P.dt - Fi[LPDF_F_SOMEGA] * Om * om * P.dt
              + sqrtf(2.0f * P.C3 * P.C4 * Om * Om * fmaxf(om, 0.0f)) * (P.sdt * z5);
    omn = fabsf(omn);
    // Eq. 9, IEM form: 1/t_m = C_phi <omega> / 2
    const float mix = P.half_cphi * Om * P.dt;
    float psi[NS];
#pragma unroll
    for (int a = 0; a < NS; ++a) {
        const float ps = sm.tile[SM::F_PSI + a][t];
        psi[a] = ps - (ps - Fi[LPDF_F_PHI0 + a]) * mix;
    }
    // Eq. 2 with the velocity at t_n and the same dW_1, dW_2
    float qx = x + u * P.dt + P.s2nu * dW1;
    float qy = y + v * P.dt + P.s2nu * dW2;
    if (M.periodic) {
        if (qx < M.x0) qx += M.period;
        else if (qx >= M.x1) qx -= M.period;
        if (qx < M.x0 || qx >= M.x1) qx -= floorf((qx - M.x0) / M.period) * M.period;   // moves > one period
    }
#pragma unroll 1
    for (int it = 0; it < 8; ++it) {
        if (qy < M.y0) { qy = 2.0f * M.y0 - qy; un = -un; vn = -vn; wn = -wn; }
        else if (qy > M.y1) { qy = 2.0f * M.y1 - qy; un = 2.0f * P.lid_u - un; vn = -vn; wn = -wn; }
        else if (!M.periodic && qx < M.x0) { qx = 2.0f * M.x0 - qx; un = -un; vn = -vn; wn = -wn; }
        else if (!M.periodic && qx > M.x1) { qx = 2.0f * M.x1 - qx; un = -un; vn = -vn; wn = -wn; }
        else break;
    }
    // half-open domain [x0, x1) x [y0, y1)
    if (qx >= M.x1) qx = M.periodic ? M.x0 : nextafterf(M.x1, -CUDART_INF_F);
    if (qy >= M.y1) qy = nextafterf(M.y1, -CUDART_INF_F);
    // concentrated scalar sources
    for (int q = 0; q < P.n_src; ++q)
        if (in_source(qx, qy, P.src_x[q], P.src_y[q], P.src_r[q])) {
#pragma unroll
            for (int a = 0; a < NS; ++a)
                if (a == P.src_alpha[q]) psi[a] = 1.0f;
        }
    if (!(isfinite(un) && isfinite(vn) && isfinite(wn) && isfinite(omn) && isfinite(qx) && isfinite(qy)))
        err |= kErrNonFinite;
    sm.tile[SM::F_X][t] = qx;
    sm.tile[SM::F_Y][t] = qy;
    sm.tile[SM::F_U][t] = un;
    sm.tile[SM::F_V][t] = vn;
    sm.tile[SM::F_W][t] = wn;
    sm.tile[SM::F_OM][t] = omn;
#pragma unroll
    for (int a = 0; a < NS; ++a) sm.tile[SM::F_PSI + a][t] = psi[a];
    sm.tile[SM::F_ELEM][t] = __int_as_float(e);
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
__global__ void __launch_bounds__(kThreads, 2)
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
        // ---- 2b. pooled neighbour walk over the thread's particles ----------------------------
        int mykey[kPPT];                       // new element per particle, -1 for none
#pragma unroll
        for (int j = 0; j < kPPT; ++j) mykey[j] = -1;
        {
            int j = 0, h = 0, e = -1, e0 = -1;
            float px = 0.0f, py = 0.0f;
            if (tid < nvalid) {
                e = e0 = __float_as_int(sm.tile[SM::F_ELEM][tid]);
                px = sm.tile[SM::F_X][tid];
                py = sm.tile[SM::F_Y][tid];
            } else {
                j = kPPT;
            }
#pragma unroll 1
            while (j < kPPT) {
                float lam[3];
                int next = -1;
                const bool found = walk_test(M, e, px, py, lam, next);
                const bool stop = found || next < 0 || h >= kHopCap;
                if (!stop) {
                    e = next;
                    ++h;
                    continue;
                }
                const int t = j * kThreads + tid;
                int ne = e;
                bool lost = !found;
                hops += found ? h : (next < 0 ? h : kHopCap + 1);
                if (lost) {
                    ne = e0;
                    barycentric(__ldg(&M.ex[ne]), __ldg(&M.ey[ne]), px, py, lam[0], lam[1], lam[2]);
                }
                if ((badmask >> j) & 1u) lost = true;
                if (lost) {
                    err |= kErrLost;
                    atomicAdd(&status[1], 1ull);
                    atomicCAS(&status[2], ~0ull, (unsigned long long)__float_as_uint(sm.tile[SM::F_PID][t]));
                }
                sm.tile[SM::F_ELEM][t] = __int_as_float(ne);
                sm.lam[0][t] = lam[0];
                sm.lam[1][t] = lam[1];
                sm.lam[2][t] = lam[2];
                // j is thread-divergent: select the register without dynamic indexing
#pragma unroll
                for (int jj = 0; jj < kPPT; ++jj)
                    if (jj == j) mykey[jj] = ne;
                ++j;
                const int t2 = j * kThreads + tid;
                if (j < kPPT && t2 < nvalid) {
                    e = e0 = __float_as_int(sm.tile[SM::F_ELEM][t2]);
                    px = sm.tile[SM::F_X][t2];
                    py = sm.tile[SM::F_Y][t2];
                    h = 0;
                } else {
                    j = kPPT;
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
                sm.cslot[b][c] = (short)table_slot_counted(sm.table, c == 0 ? mv.x : (c == 1 ? mv.y : mv.z), &sm.tfill);
            }
        }
        __syncthreads();
        // ---- 6. accumulate units; hand the partials to column owners -------------------------
        {
            const int nu = min(sm.nunits, kMaxUnits);
            const int nb = sm.nbins;
            // warp-uniform rounds: lane `lane` of warp `wid` takes unit r * kThreads + wid * 32 + lane
#pragma unroll 1
            for (int ub = wid * 32; ub < nu; ub += kThreads) {
                const int u = ub + lane;
                int b = -1;
                float acc[NK];
#pragma unroll
                for (int k = 0; k < NK; ++k) acc[k] = 0.0f;
                if (u < nu) {
                    b = sm.ubin[u];
                    if (!consistent(b < nb, err)) b = -1;
                }
                if (b >= 0) {
                    const int p0 = sm.bstart[b] + (u - sm.ustart[b]) * kUnit;
                    const int p1 = min(p0 + kUnit, (int)sm.bstart[b + 1]);
#pragma unroll 1
                    for (int p = p0; p < p1; ++p) {
                        const int t = sm.perm[p];
                        if (!consistent(t < kT, err)) break;
                        const float l0 = sm.lam[0][t], l1 = sm.lam[1][t], l2 = sm.lam[2][t];
                        float q[NQ];
                        quantities<NS>(sm, t, q);
#pragma unroll
                        for (int k = 0; k < NQ; ++k) {
                            acc[k] = fmaf(l0, q[k], acc[k]);
                            acc[NQ + k] = fmaf(l1, q[k], acc[NQ + k]);
                            acc[2 * NQ + k] = fmaf(l2, q[k], acc[2 * NQ + k]);
                        }
                    }
                }
                // hand-over, kGroup lanes at a time: lane k owns columns k and k + 32
#pragma unroll 1
                for (int g = 0; g < 32; g += kGroup) {
                    if (lane >= g && lane < g + kGroup) {
#pragma unroll
                        for (int k = 0; k < NK; ++k) sm.scr[wid][lane - g][k] = acc[k];
                        sm.sbin[wid][lane - g] = b;
                    }
                    __syncwarp();
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const int k = lane + 32 * kk;
                        if (k >= NK) break;
                        const int c = k / NQ, q = k - c * NQ;
                        int cur = -1;
                        float sum = 0.0f;
#pragma unroll
                        for (int l = 0; l <= kGroup; ++l) {
                            const int bl = l < kGroup ? sm.sbin[wid][l] : -2;
                            if (bl != cur) {
                                if (cur >= 0) {
                                    const int4 mv = __ldg(&M.em[sm.binel[cur]]);
                                    table_add(sm.table, (int)sm.cslot[cur][c], c == 0 ? mv.x : (c == 1 ? mv.y : mv.z),
                                              q, to_fixed(sum, err), node_acc);
                                }
                                cur = bl;
                                sum = 0.0f;
                            }
                            if (l < kGroup) sum += sm.scr[wid][l][k];
                        }
                    }
                    __syncwarp();
                }
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
    static int n_sm = 0;
    if (n_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(pdf_step_kernel<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    const int64_t ntiles = (s.n + kT - 1) / kT;
    if (ntiles == 0) return cudaSuccess;
    // persistent CTAs, two per SM, each on a contiguous range of sub-tiles
    const int64_t grid = std::min<int64_t>(ntiles, 2 * (int64_t)n_sm);
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
