// Kernels of the particle time step (sm_103a).
//
// pdf_step_kernel: one forward-Euler step of every particle of the joint velocity-frequency-
// scalar PDF method (arXiv:1006.0549, Section "Governing equations": Eq. 2, 4, 5, 6, 9 in IEM
// form, forward Euler, statistics at particle positions, tracking through the unstructured
// grid) fused with the reduction of the new state's moments to gridpoints.
//
// Work decomposition: a CTA (8 warps) owns a contiguous range of particles (particles are kept
// sorted by element, so a range covers few elements); each warp takes 128-particle tiles of it.
// Per tile:
//   1. every lane advances 4 particles (lane l: tile particles l, l+32, l+64, l+96) and stores
//      the new state (coalesced);
//   2. the warp sorts its 128 (new element, particle) pairs by element, stably, with warp
//      minimum reductions and a prefix scan per distinct element, and scatters the reduction
//      inputs (lambda', u, v, w, omega, psi) into shared memory in that order;
//   3. lane l accumulates sorted positions 4l..4l+3 serially in FP32 registers; segments that
//      end inside the lane's chunk go straight to the CTA node table; the lane's last segment
//      is combined across lanes column by column (a warp segmented reduction through shared
//      memory) before it goes to the table;
//   4. the CTA node table holds 64-bit fixed-point sums keyed by gridpoint; at the end of the
//      CTA's range it is added to the global gridpoint accumulators (one atomic add per
//      touched node and quantity). Integer addition is associative, so the result does not
//      depend on CTA or warp scheduling: the sums are bit-reproducible.
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "lpdf_internal.h"

namespace lpdf {

constexpr int kTPB = 256;
constexpr int kWarps = kTPB / 32;
constexpr int kPPL = 4;                    // particles per lane per tile
constexpr int kTile = 32 * kPPL;           // 128 particles per warp tile
constexpr int kSubTile = kWarps * kTile;   // 1024 particles per CTA sub-tile
constexpr int kSubTilesPerCTA = 4;         // CTA range = 4096 particles
constexpr int kRange = kSubTile * kSubTilesPerCTA;
constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): 10 rounds of two 32x32->64 products
// with the round multipliers, the high words xored with the other counter words and the round
// key, the key advanced by the Weyl increments between rounds.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// (w + 1/2) 2^-32, rounded to FP32
__device__ __forceinline__ float u01(uint32_t w) { return fmaf((float)w, 0x1p-32f, 0x1p-33f); }

// Box-Muller (1958): r = sqrt(-2 ln u0), angle 2 pi u1
__device__ __forceinline__ void box_muller(uint32_t w0, uint32_t w1, float& z0, float& z1)
{
    const float r = sqrtf(-2.0f * logf(u01(w0)));
    float s, c;
    sincospif(2.0f * u01(w1), &s, &c);
    z0 = r * c;
    z1 = r * s;
}

// ------------------------------------------------------------------------------------------
// Exact orientation (rare fallback): sign of (ax-cx)(by-cy) - (ay-cy)(bx-cx) by exact FP64
// expansion arithmetic (Shewchuk 1997: two-sum, FMA two-product, grow-expansion).
// ------------------------------------------------------------------------------------------
__device__ __noinline__ int orient_exact(double ax, double ay, double bx, double by, double cx, double cy)
{
    double t[16];
    int nt = 0;
    auto tsum = [](double a, double b, double& s, double& e) {
        s = a + b;
        const double bv = s - a, av = s - bv;
        e = (a - av) + (b - bv);
    };
    double d[8];
    tsum(ax, -cx, d[0], d[1]);
    tsum(by, -cy, d[2], d[3]);
    tsum(ay, -cy, d[4], d[5]);
    tsum(bx, -cx, d[6], d[7]);
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double p = d[i] * d[2 + j];
            t[nt++] = p;
            t[nt++] = fma(d[i], d[2 + j], -p);
            double q = d[4 + i] * d[6 + j];
            t[nt++] = -q;
            t[nt++] = -fma(d[4 + i], d[6 + j], -q);
        }
    double h[17];
    int nh = 0;
    for (int i = 0; i < nt; ++i) {
        double q = t[i];
        int m = 0;
        for (int k = 0; k < nh; ++k) {
            double s, e;
            tsum(q, h[k], s, e);
            if (e != 0.0) h[m++] = e;
            q = s;
        }
        if (q != 0.0) h[m++] = q;
        nh = m;
    }
    if (nh == 0) return 0;
    return h[nh - 1] > 0.0 ? 1 : -1;
}

// orientation of p relative to directed edge a->b, (bx-ax)(py-ay) - (by-ay)(px-ax): FP32
// value for navigation and its exact sign (error-bounded FP32 filter, exact FP64 fallback).
__device__ __forceinline__ float orient_sign(float ax, float ay, float bx, float by, float px, float py, int& sgn)
{
    const float dx1 = __fsub_rn(bx, ax), dy1 = __fsub_rn(by, ay);
    const float dx2 = __fsub_rn(px, ax), dy2 = __fsub_rn(py, ay);
    const float t1 = __fmul_rn(dx1, dy2), t2 = __fmul_rn(dy1, dx2);
    const float val = __fsub_rn(t1, t2);
    const float detsum = __fadd_rn(fabsf(t1), fabsf(t2));
    // (3 + 16 eps) eps with eps = 2^-24 is 1.79e-7; 2e-7 leaves room for the rounding of the bound
    const float bound = 2.0e-7f * detsum;
    if (detsum > 1e-25f && val > bound) { sgn = 1; return val; }
    if (detsum > 1e-25f && -val > bound) { sgn = -1; return val; }
    sgn = orient_exact((double)bx, (double)by, (double)px, (double)py, (double)ax, (double)ay);
    return val;
}

// an edge a->b of a CCW triangle owns the points on it iff it is a "top-left" edge
__device__ __forceinline__ bool edge_owns(float ax, float ay, float bx, float by)
{
    return (by < ay) || (by == ay && bx > ax);
}

// Barycentric neighbour walk from element e to the unique owner of (px, py). Exact inside
// tests in the element's own frame; in a periodic image frame only navigation. Returns the
// owner, -1 on a wall exit, -2 at the hop cap.
__device__ int locate_walk(const DevMesh& M, int e, float px, float py, int& hops)
{
    for (int h = 0; h <= kHopCap; ++h) {
        const float4 X = __ldg(&M.ex[e]);
        const float4 Y = __ldg(&M.ey[e]);
        const int4 N = __ldg(&M.en[e]);
        const float xs[3] = {X.x, X.y, X.z}, ys[3] = {Y.x, Y.y, Y.z};
        const int nb[3] = {N.x, N.y, N.z};
        float sh = 0.0f;
        if (M.periodic) sh = rintf((X.w - px) / M.period) * M.period;
        int best = -1;
        float bestv = 0.0f;
        bool all_in = true;
        if (sh == 0.0f) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int a = k, b = (k + 1) % 3;
                int s;
                const float val = orient_sign(xs[a], ys[a], xs[b], ys[b], px, py, s);
                const bool in = s > 0 || (s == 0 && edge_owns(xs[a], ys[a], xs[b], ys[b]));
                if (!in) {
                    all_in = false;
                    if (best < 0 || val < bestv) { best = k; bestv = val; }
                }
            }
            if (all_in) { hops = h; return e; }
        } else {
            const float qx = px + sh;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int a = k, b = (k + 1) % 3;
                const float val = (xs[b] - xs[a]) * (py - ys[a]) - (ys[b] - ys[a]) * (qx - xs[a]);
                const bool in = (val > 0.0f) || nb[k] < 0;
                if (!in && (best < 0 || val < bestv)) { best = k; bestv = val; }
            }
            if (best < 0) best = (N.w & 1) ? 0 : (N.w & 2) ? 1 : (N.w & 4) ? 2 : 0;
        }
        const int n = best == 0 ? N.x : (best == 1 ? N.y : N.z);
        if (n < 0) { hops = h; return -1; }
        e = n;
    }
    hops = kHopCap + 1;
    return -2;
}

// a*d - b*c with one rounding error bound of 1.5 ulp (Kahan's FMA determinant)
__device__ __forceinline__ float det2(float a, float b, float c, float d)
{
    const float w = b * c;
    const float e = fmaf(-b, c, w);
    const float f = fmaf(a, d, -w);
    return f + e;
}

__device__ __forceinline__ void barycentric(const float4& X, const float4& Y, float px, float py, float& l0,
                                            float& l1, float& l2)
{
    l0 = det2(X.y - px, Y.y - py, X.z - px, Y.z - py) * Y.w;
    l1 = det2(X.z - px, Y.z - py, X.x - px, Y.x - py) * Y.w;
    l2 = det2(X.x - px, Y.x - py, X.y - px, Y.y - py) * Y.w;
}

__device__ __forceinline__ bool in_source(float px, float py, float sx, float sy, float r)
{
    const float dx = __fsub_rn(px, sx), dy = __fsub_rn(py, sy);
    return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)) < __fmul_rn(r, r);
}

// ------------------------------------------------------------------------------------------
// One particle: Eq. 4, 5, 9 (IEM), 2; wrap and reflection; exact location; sources.
// ------------------------------------------------------------------------------------------
template <int NS>
struct Particle {
    float x, y, u, v, w, om, psi[NS];
    int elem;
};

template <int NS>
__device__ __forceinline__ bool advance(const DevMesh& M, const float* __restrict__ F, const StepParams& P,
                                        uint32_t pid, Particle<NS>& s, float lam[3], unsigned& err, int& hops)
{
    constexpr int NFP = (22 + NS + 3) / 4 * 4;
    // an element id outside the mesh (corrupt input) is reported as a lost particle
    const bool bad_elem = (unsigned)s.elem >= (unsigned)M.n_tri;
    const int e = bad_elem ? 0 : s.elem;
    const float4 X = __ldg(&M.ex[e]);
    const float4 Y = __ldg(&M.ey[e]);
    const int4 V = __ldg(&M.ev[e]);
    float l0, l1, l2;
    barycentric(X, Y, s.x, s.y, l0, l1, l2);
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
    const float Ur = s.u - Fi[LPDF_F_U + 0], Vr = s.v - Fi[LPDF_F_U + 1], Wr = s.w - Fi[LPDF_F_U + 2];
    // Eq. 4
    float un = s.u + (-Fi[LPDF_F_DPDX] + P.nu2 * Fi[LPDF_F_LAPU] + Fi[LPDF_F_G11] * Ur + Fi[LPDF_F_G11 + 1] * Vr) * P.dt
             + P.s2nu * (Fi[LPDF_F_DUDX] * dW1 + Fi[LPDF_F_DUDX + 1] * dW2) + c0e * (P.sdt * z2);
    float vn = s.v + (-Fi[LPDF_F_DPDX + 1] + P.nu2 * Fi[LPDF_F_LAPU + 1] + Fi[LPDF_F_G11 + 2] * Ur + Fi[LPDF_F_G11 + 3] * Vr) * P.dt
             + P.s2nu * (Fi[LPDF_F_DUDX + 2] * dW1 + Fi[LPDF_F_DUDX + 3] * dW2) + c0e * (P.sdt * z3);
    float wn = s.w + (P.nu2 * Fi[LPDF_F_LAPU + 2] + Fi[LPDF_F_G11 + 4] * Wr) * P.dt
             + P.s2nu * (Fi[LPDF_F_DUDX + 4] * dW1 + Fi[LPDF_F_DUDX + 5] * dW2) + c0e * (P.sdt * z4);
    // Eq. 5 (S_omega of Eq. 6 is a node field)
    const float Om = Fi[LPDF_F_OMEGA];
    float omn = s.om - P.C3 * Om * (s.om - Om) * P.dt - Fi[LPDF_F_SOMEGA] * Om * s.om * P.dt
              + sqrtf(2.0f * P.C3 * P.C4 * Om * Om * fmaxf(s.om, 0.0f)) * (P.sdt * z5);
    omn = fabsf(omn);
    // Eq. 9, IEM form: 1/t_m = C_phi <omega> / 2
    const float mix = P.half_cphi * Om * P.dt;
#pragma unroll
    for (int a = 0; a < NS; ++a) s.psi[a] = s.psi[a] - (s.psi[a] - Fi[LPDF_F_PHI0 + a]) * mix;
    // Eq. 2 with the velocity at t_n and the same dW_1, dW_2
    float qx = s.x + s.u * P.dt + P.s2nu * dW1;
    float qy = s.y + s.v * P.dt + P.s2nu * dW2;
    if (M.periodic) qx -= floorf((qx - M.x0) / M.period) * M.period;
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
    int h = 0;
    int ne = locate_walk(M, e, qx, qy, h);
    hops += h;
    const bool lost = ne < 0 || bad_elem;
    if (lost) { err |= kErrLost; if (ne < 0) ne = e; }
    // concentrated scalar sources
    for (int q = 0; q < P.n_src; ++q)
        if (in_source(qx, qy, P.src_x[q], P.src_y[q], P.src_r[q])) {
#pragma unroll
            for (int a = 0; a < NS; ++a)
                if (a == P.src_alpha[q]) s.psi[a] = 1.0f;
        }
    if (!(isfinite(un) && isfinite(vn) && isfinite(wn) && isfinite(omn) && isfinite(qx) && isfinite(qy)))
        err |= kErrNonFinite;
    // shape functions at the new position for the moments
    const float4 X2 = __ldg(&M.ex[ne]);
    const float4 Y2 = __ldg(&M.ey[ne]);
    barycentric(X2, Y2, qx, qy, lam[0], lam[1], lam[2]);
    s.x = qx; s.y = qy; s.u = un; s.v = vn; s.w = wn; s.om = omn; s.elem = ne;
    return lost;
}

// ------------------------------------------------------------------------------------------
// CTA node table: 64-bit fixed-point moment sums keyed by statistics node. A lookup probes at
// most kProbe slots; a node that finds no slot goes straight to the global accumulators.
// ------------------------------------------------------------------------------------------
constexpr int kProbe = 16;

template <int NQ, int NT>
struct NodeTable {
    int key[NT];
    unsigned long long acc[NT][NQ];
};

template <int NQ, int NT>
__device__ __forceinline__ int table_slot(NodeTable<NQ, NT>& T, int node)
{
    const unsigned h = ((unsigned)node * 2654435761u) >> 9;
#pragma unroll 1
    for (int p = 0; p < kProbe; ++p) {
        const int s = (h + p) & (NT - 1);
        const int k = T.key[s];
        if (k == node) return s;
        if (k == -1) {
            const int old = atomicCAS(&T.key[s], -1, node);
            if (old == -1 || old == node) return s;
        }
    }
    return -1;
}

__device__ __forceinline__ long long to_fixed(float v, unsigned& err)
{
    if (!(fabsf(v) < kFixLimit)) err |= kErrOverflow;
    return __float2ll_rn(v * 4294967296.0f);
}

template <int NQ, int NT>
__device__ __forceinline__ void table_add(NodeTable<NQ, NT>& T, int slot, int node, int q, long long v,
                                          unsigned long long* __restrict__ node_acc)
{
    if (v == 0) return;
    if (slot >= 0) atomicAdd(&T.acc[slot][q], (unsigned long long)v);
    else atomicAdd(&node_acc[(size_t)node * NQ + q], (unsigned long long)v);
}

// ------------------------------------------------------------------------------------------
// The fused step kernel.
// ------------------------------------------------------------------------------------------
template <int NS>
struct StepSmem {
    static constexpr int NV = 7 + NS;          // lambda0..2, u, v, w, omega, psi
    static constexpr int NQ = 11 + 2 * NS;
    static constexpr int NK = 3 * NQ;          // columns: corner-major, quantity-minor
    static constexpr int WB = (NV * kTile > 32 * NK) ? NV * kTile : 32 * NK;
    static constexpr int NT = 256;
    float wbuf[kWarps][WB];                    // reduction inputs (tile order), later lane partials
    int wkey[kWarps][kTile];                   // new element of every tile particle (tile order)
    unsigned char perm[kWarps][kTile];         // sorted position -> tile index
    unsigned char wbin[kWarps][kTile];         // sorted position -> bin
    int bkey[kWarps][kTile];                   // bin -> element
    int blast[kWarps][32];
    NodeTable<NQ, NT> table;
};

template <int NS>
__global__ void __launch_bounds__(kTPB, 2)
pdf_step_kernel(const __grid_constant__ DevMesh M, const __grid_constant__ DevState S, const float* __restrict__ F,
                const __grid_constant__ StepParams P,
                unsigned long long* __restrict__ node_acc, unsigned long long* __restrict__ status)
{
    using SM = StepSmem<NS>;
    constexpr int NV = SM::NV, NQ = SM::NQ, NK = SM::NK, NT = SM::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SM& sm = *reinterpret_cast<SM*>(smem_raw);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < NT; i += kTPB) sm.table.key[i] = -1;
    for (int i = threadIdx.x; i < NT * NQ; i += kTPB) (&sm.table.acc[0][0])[i] = 0ull;
    __syncthreads();

    unsigned err = 0;
    int hops = 0;
    const int64_t range0 = (int64_t)blockIdx.x * kRange;
    float* wb = sm.wbuf[wid];
    int* wkey = sm.wkey[wid];
    unsigned char* perm = sm.perm[wid];
    unsigned char* wbin = sm.wbin[wid];
    int* bkey = sm.bkey[wid];

    for (int sub = 0; sub < kSubTilesPerCTA; ++sub) {
        const int64_t tb = range0 + (int64_t)sub * kSubTile + (int64_t)wid * kTile;
        if (tb >= S.n) break;
        // ---- 1. advance 4 particles per lane (tile index j*32 + lane), store, stage inputs
#pragma unroll 1
        for (int j = 0; j < kPPL; ++j) {
            const int t = j * 32 + lane;
            const int64_t i = tb + t;
            int key = INT_MAX;
            if (i < S.n) {
                Particle<NS> p;
                p.x = S.x[i]; p.y = S.y[i]; p.u = S.u[i]; p.v = S.v[i]; p.w = S.w[i]; p.om = S.om[i];
#pragma unroll
                for (int a = 0; a < NS; ++a) p.psi[a] = S.psi[(size_t)a * S.cap + i];
                p.elem = S.elem[i];
                const uint32_t pid = S.pid[i];
                float lam[3];
                if (advance<NS>(M, F, P, pid, p, lam, err, hops)) {
                    atomicAdd(&status[1], 1ull);
                    atomicCAS(&status[2], ~0ull, (unsigned long long)pid);
                }
                S.x[i] = p.x; S.y[i] = p.y; S.u[i] = p.u; S.v[i] = p.v; S.w[i] = p.w; S.om[i] = p.om;
#pragma unroll
                for (int a = 0; a < NS; ++a) S.psi[(size_t)a * S.cap + i] = p.psi[a];
                S.elem[i] = p.elem;
                key = p.elem;
                wb[0 * kTile + t] = lam[0]; wb[1 * kTile + t] = lam[1]; wb[2 * kTile + t] = lam[2];
                wb[3 * kTile + t] = p.u; wb[4 * kTile + t] = p.v; wb[5 * kTile + t] = p.w; wb[6 * kTile + t] = p.om;
#pragma unroll
                for (int a = 0; a < NS; ++a) wb[(7 + a) * kTile + t] = p.psi[a];
            }
            wkey[t] = key;
        }
        __syncwarp();
        // ---- 2. stable warp sort of the tile by new element: perm[sorted pos] = tile index
        int n = 0, nb = 0;
        {
            int key[kPPL];
#pragma unroll
            for (int j = 0; j < kPPL; ++j) key[j] = wkey[j * 32 + lane];
            int mn = min(min(key[0], key[1]), min(key[2], key[3]));
            int cur = __reduce_min_sync(kFull, mn);
            while (cur != INT_MAX) {
                int c = 0;
#pragma unroll
                for (int j = 0; j < kPPL; ++j) c += (key[j] == cur);
                int incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int tt = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += tt;
                }
                const int total = __shfl_sync(kFull, incl, 31);
                int p0 = n + incl - c;
#pragma unroll
                for (int j = 0; j < kPPL; ++j)
                    if (key[j] == cur) { perm[p0] = (unsigned char)(j * 32 + lane); wbin[p0] = (unsigned char)nb; ++p0; }
                if (lane == 0) bkey[nb] = cur;
                n += total;
                ++nb;
                int nx = INT_MAX;
#pragma unroll
                for (int j = 0; j < kPPL; ++j)
                    if (key[j] > cur) nx = min(nx, key[j]);
                cur = __reduce_min_sync(kFull, nx);
            }
        }
        __syncwarp();
        // ---- 3. per-lane serial accumulation over sorted positions 4l..4l+3 ------------
        float acc[NK];
#pragma unroll
        for (int k = 0; k < NK; ++k) acc[k] = 0.0f;
        int curb = -1;
        const int pbeg = kPPL * lane;
#pragma unroll 1
        for (int p = pbeg; p < pbeg + kPPL && p < n; ++p) {
            const int b = wbin[p];
            if (b != curb) {
                if (curb >= 0) {
                    // a segment that ends inside this lane's chunk: straight to the node table
                    const int4 mv = __ldg(&M.em[bkey[curb]]);
                    const int s0 = table_slot(sm.table, mv.x), s1 = table_slot(sm.table, mv.y),
                              s2 = table_slot(sm.table, mv.z);
#pragma unroll
                    for (int k = 0; k < NQ; ++k) {
                        table_add(sm.table, s0, mv.x, k, to_fixed(acc[k], err), node_acc);
                        table_add(sm.table, s1, mv.y, k, to_fixed(acc[NQ + k], err), node_acc);
                        table_add(sm.table, s2, mv.z, k, to_fixed(acc[2 * NQ + k], err), node_acc);
                        acc[k] = 0.0f; acc[NQ + k] = 0.0f; acc[2 * NQ + k] = 0.0f;
                    }
                }
                curb = b;
            }
            const int t = perm[p];
            const float l0 = wb[0 * kTile + t], l1 = wb[1 * kTile + t], l2 = wb[2 * kTile + t];
            float q[NQ];
            const float u = wb[3 * kTile + t], v = wb[4 * kTile + t], w = wb[5 * kTile + t];
            q[0] = 1.0f; q[1] = u; q[2] = v; q[3] = w;
            q[4] = u * u; q[5] = u * v; q[6] = u * w; q[7] = v * v; q[8] = v * w; q[9] = w * w;
            q[10] = wb[6 * kTile + t];
#pragma unroll
            for (int a = 0; a < NS; ++a) {
                const float ps = wb[(7 + a) * kTile + t];
                q[11 + a] = ps;
                q[11 + NS + a] = ps * ps;
            }
#pragma unroll
            for (int k = 0; k < NQ; ++k) {
                acc[k] = fmaf(l0, q[k], acc[k]);
                acc[NQ + k] = fmaf(l1, q[k], acc[NQ + k]);
                acc[2 * NQ + k] = fmaf(l2, q[k], acc[2 * NQ + k]);
            }
        }
        __syncwarp();
        // ---- 4. combine the lanes' last segments column by column ---------------------
        float* part = wb;   // reuses the staged inputs: 32 x NK
#pragma unroll
        for (int k = 0; k < NK; ++k) part[lane * NK + k] = acc[k];
        sm.blast[wid][lane] = curb;
        __syncwarp();
#pragma unroll 1
        for (int k = lane; k < NK; k += 32) {
            const int c = k / NQ, qq = k - c * NQ;
            float s = 0.0f;
            int b = -1;
#pragma unroll 1
            for (int l = 0; l < 32; ++l) {
                const int bl = sm.blast[wid][l];
                if (bl != b) {
                    if (b >= 0) {
                        const int4 mv = __ldg(&M.em[bkey[b]]);
                        const int node = c == 0 ? mv.x : (c == 1 ? mv.y : mv.z);
                        table_add(sm.table, table_slot(sm.table, node), node, qq, to_fixed(s, err), node_acc);
                    }
                    b = bl;
                    s = 0.0f;
                }
                s += part[l * NK + k];
            }
            if (b >= 0) {
                const int4 mv = __ldg(&M.em[bkey[b]]);
                const int node = c == 0 ? mv.x : (c == 1 ? mv.y : mv.z);
                table_add(sm.table, table_slot(sm.table, node), node, qq, to_fixed(s, err), node_acc);
            }
        }
        __syncwarp();
    }
    // ---- 5. flush the CTA node table --------------------------------------------------
    __syncthreads();
    for (int i = threadIdx.x; i < NT * NQ; i += kTPB) {
        const int s = i / NQ, q = i - (i / NQ) * NQ;
        const int node = sm.table.key[s];
        const unsigned long long v = sm.table.acc[s][q];
        if (node >= 0 && v != 0ull) atomicAdd(&node_acc[(size_t)node * NQ + q], v);
    }
    // ---- status -----------------------------------------------------------------------
    const unsigned e_or = __reduce_or_sync(kFull, err);
    const int h_sum = __reduce_add_sync(kFull, hops);
    if (lane == 0) {
        if (e_or) atomicOr(&status[0], (unsigned long long)e_or);
        if (h_sum) atomicAdd(&status[3], (unsigned long long)h_sum);
    }
}

template <int NS>
static cudaError_t launch_step_ns(const DevMesh& m, const DevState& s, const float* fields, const StepParams& p,
                                  unsigned long long* node_acc, unsigned long long* status, cudaStream_t st)
{
    const size_t smem = sizeof(StepSmem<NS>);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(pdf_step_kernel<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int64_t grid = (s.n + kRange - 1) / kRange;
    if (grid == 0) return cudaSuccess;
    pdf_step_kernel<NS><<<(unsigned)grid, kTPB, smem, st>>>(m, s, fields, p, node_acc, status);
    return cudaGetLastError();
}

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

// ------------------------------------------------------------------------------------------
// Particle initialisation: uniform position in the generating element (s = sqrt(r1):
// lambda = (1-s, s(1-r2), s r2)), exact location, Gaussian velocity about the interpolated
// mean, Erlang(m) frequency with the interpolated mean, psi = 0. Philox tag 1, blocks 0..2.
// ------------------------------------------------------------------------------------------
template <int NS>
__global__ void particles_init_kernel(const __grid_constant__ DevMesh M, const __grid_constant__ DevState S, int n_per_elem, const float* __restrict__ init,
                                      int m_erlang, uint32_t k0, uint32_t k1, unsigned long long* status)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t P = (int64_t)M.n_tri * n_per_elem;
    unsigned err = 0;
    if (i < P) {
        const int e = (int)(i / n_per_elem);
        const uint32_t pid = (uint32_t)i;
        const uint4 a = philox4x32_10(make_uint4(pid, 0u, 0u, (1u << 16) | 0u), k0, k1);
        const uint4 b = philox4x32_10(make_uint4(pid, 0u, 0u, (1u << 16) | 1u), k0, k1);
        const uint4 c = philox4x32_10(make_uint4(pid, 0u, 0u, (1u << 16) | 2u), k0, k1);
        const float4 X = __ldg(&M.ex[e]), Y = __ldg(&M.ey[e]);
        const float sq = sqrtf(u01(a.x)), r2 = u01(a.y);
        const float l0 = 1.0f - sq, l1 = sq * (1.0f - r2), l2 = sq * r2;
        float px = fmaf(l0, X.x, fmaf(l1, X.y, l2 * X.z));
        float py = fmaf(l0, Y.x, fmaf(l1, Y.y, l2 * Y.z));
        if (px >= M.x1) px = M.periodic ? M.x0 : nextafterf(M.x1, -CUDART_INF_F);
        if (py >= M.y1) py = nextafterf(M.y1, -CUDART_INF_F);
        int hops = 0;
        int ne = locate_walk(M, e, px, py, hops);
        if (ne < 0) { err |= kErrLost; ne = e; }
        const float4 X2 = __ldg(&M.ex[ne]), Y2 = __ldg(&M.ey[ne]);
        const int4 V = __ldg(&M.ev[ne]);
        float m0, m1, m2;
        barycentric(X2, Y2, px, py, m0, m1, m2);
        float Fi[5];
#pragma unroll
        for (int f = 0; f < 5; ++f)
            Fi[f] = fmaf(m0, __ldg(&init[(size_t)V.x * 8 + f]), fmaf(m1, __ldg(&init[(size_t)V.y * 8 + f]), m2 * __ldg(&init[(size_t)V.z * 8 + f])));
        float z0, z1, z2, z3;
        box_muller(a.z, a.w, z0, z1);
        box_muller(b.x, b.y, z2, z3);
        const uint32_t ew[6] = {b.z, b.w, c.x, c.y, c.z, c.w};
        float sum = 0.0f;
        for (int k = 0; k < m_erlang; ++k) sum += -logf(u01(ew[k]));
        S.x[i] = px; S.y[i] = py;
        S.u[i] = Fi[0] + Fi[3] * z0;
        S.v[i] = Fi[1] + Fi[3] * z1;
        S.w[i] = Fi[2] + Fi[3] * z2;
        S.om[i] = Fi[4] * sum / (float)m_erlang;
#pragma unroll
        for (int q = 0; q < NS; ++q) S.psi[(size_t)q * S.cap + i] = 0.0f;
        S.elem[i] = ne;
        S.pid[i] = pid;
    }
    if (err) atomicOr(&status[0], (unsigned long long)err);
}

cudaError_t launch_particles_init(const DevMesh& m, const DevState& s, int ns, int n_per_elem, const float* node_init,
                                  int m_erlang, uint64_t seed, unsigned long long* status, cudaStream_t st)
{
    const int64_t P = (int64_t)m.n_tri * n_per_elem;
    const unsigned grid = (unsigned)((P + 255) / 256);
    if (grid == 0) return cudaSuccess;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    switch (ns) {
        case 1: particles_init_kernel<1><<<grid, 256, 0, st>>>(m, s, n_per_elem, node_init, m_erlang, k0, k1, status); break;
        case 2: particles_init_kernel<2><<<grid, 256, 0, st>>>(m, s, n_per_elem, node_init, m_erlang, k0, k1, status); break;
        case 3: particles_init_kernel<3><<<grid, 256, 0, st>>>(m, s, n_per_elem, node_init, m_erlang, k0, k1, status); break;
        case 4: particles_init_kernel<4><<<grid, 256, 0, st>>>(m, s, n_per_elem, node_init, m_erlang, k0, k1, status); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Gridpoint statistics from the fixed-point sums: raw sums, or means and central moments
// (mean = S_q/S_0, central = S_qq/S_0 - mean^2). Periodic partners read their master's sums.
// ------------------------------------------------------------------------------------------
__global__ void grid_statistics_kernel(const int* __restrict__ master, int n_nodes, int ns,
                                       const unsigned long long* __restrict__ acc, double* __restrict__ out, int raw)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_nodes) return;
    const int nq = 11 + 2 * ns;
    const int m = master[n];
    double S[11 + 2 * kMaxNS];
    for (int k = 0; k < nq; ++k) S[k] = (double)(long long)acc[(size_t)m * nq + k] * (1.0 / kFixScale);
    double* o = out + (size_t)n * nq;
    if (raw) {
        for (int k = 0; k < nq; ++k) o[k] = S[k];
        return;
    }
    const double s0 = S[0];
    o[0] = s0;
    if (s0 == 0.0) {
        for (int k = 1; k < nq; ++k) o[k] = 0.0;
        return;
    }
    const double inv = 1.0 / s0;
    const double mu = S[1] * inv, mv = S[2] * inv, mw = S[3] * inv;
    o[1] = mu; o[2] = mv; o[3] = mw;
    o[4] = S[4] * inv - mu * mu; o[5] = S[5] * inv - mu * mv; o[6] = S[6] * inv - mu * mw;
    o[7] = S[7] * inv - mv * mv; o[8] = S[8] * inv - mv * mw; o[9] = S[9] * inv - mw * mw;
    o[10] = S[10] * inv;
    for (int a = 0; a < ns; ++a) {
        const double mp = S[11 + a] * inv;
        o[11 + a] = mp;
        o[11 + ns + a] = S[11 + ns + a] * inv - mp * mp;
    }
}

cudaError_t launch_grid_statistics(const DevMesh& m, int ns, const unsigned long long* node_acc, double* out, int raw,
                                   cudaStream_t st)
{
    const unsigned grid = (unsigned)((m.n_nodes + 255) / 256);
    grid_statistics_kernel<<<grid, 256, 0, st>>>(m.master, m.n_nodes, ns, node_acc, out, raw);
    return cudaGetLastError();
}

}  // namespace lpdf
