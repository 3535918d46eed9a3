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

// Box-Muller (1958) on the special-function unit: r^2 = -2 ln u0 (lg2.approx: absolute error
// ~2^-22 in log2), r = r^2 * rsqrt(r^2), angle theta = 2 pi u1 - pi in [-pi, pi), where the SFU
// sine and cosine are accurate to ~2^-21.4 absolute; cos(theta + pi) = -cos(theta) and
// sin(theta + pi) = -sin(theta), so z0 = r cos(2 pi u1), z1 = r sin(2 pi u1) as in the oracle.
__device__ __forceinline__ void box_muller(uint32_t w0, uint32_t w1, float& z0, float& z1)
{
    const float r2 = -2.0f * __logf(u01(w0));
    const float r = r2 > 0.0f ? r2 * rsqrtf(r2) : 0.0f;
    const float th = fmaf(6.28318530717958648f, u01(w1), -3.14159265358979324f);
    float sn, cs;
    __sincosf(th, &sn, &cs);
    z0 = -r * cs;
    z1 = -r * sn;
}

// accurate variant for the initialisation kernel (not on the hot path)
__device__ __forceinline__ void box_muller_accurate(uint32_t w0, uint32_t w1, float& z0, float& z1)
{
    const float r = sqrtf(-2.0f * logf(u01(w0)));
    float sn, cs;
    sincospif(2.0f * u01(w1), &sn, &cs);
    z0 = r * cs;
    z1 = r * sn;
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

// orientation of p relative to directed edge a->b, (bx-ax)(py-ay) - (by-ay)(px-ax): the FP32
// value (Kahan's FMA determinant: at most 1.5 ulp of the result beyond the rounding of the four
// differences) and its exact sign. Filter: every rounding above is bounded by 3.5 eps32 (|t1| +
// |t2|) (eps32 = 2^-24); 4e-7 (~6.7 eps32) also covers the rounding of the bound. Undecided
// cases go to the exact FP64 expansion.
__device__ __forceinline__ float orient_sign(float ax, float ay, float bx, float by, float px, float py, int& sgn)
{
    const float dx1 = __fsub_rn(bx, ax), dy1 = __fsub_rn(by, ay);
    const float dx2 = __fsub_rn(px, ax), dy2 = __fsub_rn(py, ay);
    const float w = dy1 * dx2;
    const float e = fmaf(-dy1, dx2, w);
    const float f = fmaf(dx1, dy2, -w);
    const float val = f + e;
    const float detsum = fmaf(fabsf(dx1), fabsf(dy2), fabsf(w));
    const float bound = 4.0e-7f * detsum;
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
// owner (and its barycentrics, from the orientation values of the last test), -1 on a wall
// exit, -2 at the hop cap.
__device__ int locate_walk(const DevMesh& M, int e, float px, float py, int& hops, float lam[3])
{
    for (int h = 0; h <= kHopCap; ++h) {
        const float4 X = __ldg(&M.ex[e]);
        const float4 Y = __ldg(&M.ey[e]);
        const int4 N = __ldg(&M.en[e]);
        const float xs[3] = {X.x, X.y, X.z}, ys[3] = {Y.x, Y.y, Y.z};
        const int nb[3] = {N.x, N.y, N.z};
        // nearest periodic image of the point relative to this element (elements are much
        // smaller than the period, so |centroid - x| > period/2 means the other image)
        float sh = 0.0f;
        if (M.periodic) {
            const float d = X.w - px;
            if (fabsf(d) > 0.5f * M.period) sh = copysignf(M.period, d);
        }
        int best = -1;
        float bestv = 0.0f;
        if (sh == 0.0f) {
            bool all_in = true;
            float vv[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int a = k, b = (k + 1) % 3;
                int s;
                vv[k] = orient_sign(xs[a], ys[a], xs[b], ys[b], px, py, s);
                const bool in = s > 0 || (s == 0 && edge_owns(xs[a], ys[a], xs[b], ys[b]));
                if (!in) {
                    all_in = false;
                    if (best < 0 || vv[k] < bestv) { best = k; bestv = vv[k]; }
                }
            }
            if (all_in) {
                // edge k = (v_k, v_k+1) is opposite vertex k+2: lambda_{k+2} = orient_k / (2 area)
                lam[2] = vv[0] * Y.w;
                lam[0] = vv[1] * Y.w;
                lam[1] = vv[2] * Y.w;
                hops = h;
                return e;
            }
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
    int h = 0;
    int ne = locate_walk(M, e, qx, qy, h, lam);
    hops += h;
    const bool lost = ne < 0 || bad_elem;
    if (lost) {
        err |= kErrLost;
        if (ne < 0) ne = e;
        barycentric(__ldg(&M.ex[ne]), __ldg(&M.ey[ne]), qx, qy, lam[0], lam[1], lam[2]);
    }
    // concentrated scalar sources
    for (int q = 0; q < P.n_src; ++q)
        if (in_source(qx, qy, P.src_x[q], P.src_y[q], P.src_r[q])) {
#pragma unroll
            for (int a = 0; a < NS; ++a)
                if (a == P.src_alpha[q]) s.psi[a] = 1.0f;
        }
    if (!(isfinite(un) && isfinite(vn) && isfinite(wn) && isfinite(omn) && isfinite(qx) && isfinite(qy)))
        err |= kErrNonFinite;
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
// Bulk-copy (TMA) and mbarrier helpers (inline PTX, sm_90+ forms valid on sm_103a).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: gives up after ~2^22 polls (each poll may suspend the thread briefly)
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, uint32_t parity)
{
#pragma unroll 1
    for (int it = 0; it < (1 << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, unsigned long long* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Adds a whole 3 x NQ partial (corner-major) to the table: rare path, kept out of line so that
// the hot loop stays small in the instruction cache.
template <int NQ, int NT>
__device__ __noinline__ void flush_partial(NodeTable<NQ, NT>& T, const float* acc, int4 nodes, const short* slots,
                                           unsigned long long* __restrict__ node_acc, unsigned* err)
{
    const int nd[3] = {nodes.x, nodes.y, nodes.z};
    for (int c = 0; c < 3; ++c)
        for (int k = 0; k < NQ; ++k) table_add(T, (int)slots[c], nd[c], k, to_fixed(acc[c * NQ + k], *err), node_acc);
}

// ------------------------------------------------------------------------------------------
// The fused step kernel.
// ------------------------------------------------------------------------------------------
template <int NS>
struct alignas(16) WarpTile {
    static constexpr int NF = 8 + NS;          // x, y, u, v, w, omega, psi[NS], elem, pid
    static constexpr int NQ = 11 + 2 * NS;
    static constexpr int NK = 3 * NQ;          // columns: corner-major, quantity-minor
    static constexpr int F_X = 0, F_Y = 1, F_U = 2, F_V = 3, F_W = 4, F_OM = 5, F_PSI = 6, F_ELEM = 6 + NS,
                         F_PID = 7 + NS;
    static constexpr int LAM = NF * kTile;     // 3 rows of lambda' after the state rows
    static constexpr int KEY = LAM + 3 * kTile;
    static constexpr int RAW = KEY + kTile;
    static constexpr int WB = RAW > 32 * NK ? RAW : 32 * NK;   // the lane partials reuse it all
    static constexpr int NL = NS == 1 ? 8 : (NS == 2 ? 4 : 2);   // parked partials of segments that end mid-chunk
    alignas(16) float buf[WB];                 // bulk-copy rows start on 16-byte boundaries
    int dkey[kTile];                           // this tile's distinct new elements, ascending
    int blast[32];
    float lpart[NL][NK];                       // parked partials
    int lbin[NL];
    int nlist;
    int ndist;
    unsigned long long bar;
};

// Internal consistency check of the binning: a failed check records kErrCheck in the status
// word and the caller skips the access, so a logic error can never become a wild address.
__device__ __forceinline__ bool consistent(bool ok, unsigned& err)
{
    if (!ok) err |= kErrCheck;
    return ok;
}

// CTA-level binning of one 1024-particle sub-tile by new element
constexpr int kMaxBins = 64;
constexpr int kRows = kWarps * kPPL;            // (warp, j) rows of 32 particles

template <int NS>
struct StepSmem {
    static constexpr int NQ = 11 + 2 * NS;
    static constexpr int NT = 128;
    WarpTile<NS> w[kWarps];
    int binkey[kSubTile];                      // bin -> element (ascending)
    short cslot[kMaxBins][3];                  // bin of the current pass -> node-table slot of each corner
    int cnt[kMaxBins][kRows];                  // particles of bin b in row r, then exclusive offsets
    unsigned short cperm[kSubTile];            // sorted position -> (warp << 7) | tile index
    unsigned char cbin[kSubTile];              // sorted position -> bin
    int nbins;
    int ntot;
    int wsum[kWarps];
    NodeTable<NQ, NT> table;
};

// Parked partials of the warp (segments that ended inside a lane's chunk): lane k adds column
// k (and k + 32) of every entry to the node table. Each value is converted on its own, so the
// order of the entries does not matter.
template <int NS>
__device__ __forceinline__ void flush_parked(const DevMesh& M, StepSmem<NS>& sm, WarpTile<NS>& W, int b0, int lane,
                                             unsigned long long* __restrict__ node_acc, unsigned& err)
{
    constexpr int NQ = WarpTile<NS>::NQ, NK = WarpTile<NS>::NK;
    const int nl = min(W.nlist, WarpTile<NS>::NL);
    for (int k = lane; k < NK; k += 32) {
        const int c = k / NQ, q = k - c * NQ;
        for (int e = 0; e < nl; ++e) {
            const int b = W.lbin[e];
            if (!consistent(b >= 0 && b < kMaxBins && b0 + b < sm.nbins, err)) continue;
            const int ek = sm.binkey[b0 + b];
            if (!consistent(ek >= 0 && ek < M.n_tri, err)) continue;
            const int4 mv = __ldg(&M.em[ek]);
            table_add(sm.table, (int)sm.cslot[b][c], c == 0 ? mv.x : (c == 1 ? mv.y : mv.z), q,
                      to_fixed(W.lpart[e][k], err), node_acc);
        }
    }
}

// Column combine of the lanes' last segments: lanes holding the same bin are contiguous; lane k
// sums column k (and k + 32) over each run of lanes and adds it to the node table. The partials
// go through `part` (32 x NK floats).
template <int NS>
__device__ __forceinline__ void combine_lanes(const DevMesh& M, StepSmem<NS>& sm, WarpTile<NS>& W, float* part,
                                              const float* acc, int curb, int b0, int lane,
                                              unsigned long long* __restrict__ node_acc, unsigned& err)
{
    constexpr int NQ = WarpTile<NS>::NQ, NK = WarpTile<NS>::NK;
#pragma unroll
    for (int k = 0; k < NK; ++k) part[lane * NK + k] = acc[k];
    W.blast[lane] = curb;
    __syncwarp();
    const int k0 = lane, k1 = lane + 32;
    const bool has1 = k1 < NK;
    const int c0 = k0 / NQ, q0 = k0 - c0 * NQ;
    const int c1 = k1 / NQ, q1 = k1 - c1 * NQ;
    auto put = [&](int b, int c, int q, float v) {
        if (!consistent(b >= 0 && b < kMaxBins && b0 + b < sm.nbins, err)) return;
        const int ek = sm.binkey[b0 + b];
        if (!consistent(ek >= 0 && ek < M.n_tri, err)) return;
        const int4 mv = __ldg(&M.em[ek]);
        table_add(sm.table, (int)sm.cslot[b][c], c == 0 ? mv.x : (c == 1 ? mv.y : mv.z), q, to_fixed(v, err), node_acc);
    };
    float s0 = 0.0f, s1 = 0.0f;
    int b = W.blast[0];
#pragma unroll 4
    for (int l = 0; l < 32; ++l) {
        const int bl = W.blast[l];
        if (bl != b) {
            if (b >= 0) {
                put(b, c0, q0, s0);
                if (has1) put(b, c1, q1, s1);
            }
            b = bl;
            s0 = 0.0f;
            s1 = 0.0f;
        }
        s0 += part[l * NK + k0];
        if (has1) s1 += part[l * NK + k1];
    }
    if (b >= 0) {
        put(b, c0, q0, s0);
        if (has1) put(b, c1, q1, s1);
    }
}

template <int NS>
__global__ void __launch_bounds__(kTPB, 2)
pdf_step_kernel(const __grid_constant__ DevMesh M, const __grid_constant__ DevState S, const float* __restrict__ F,
                const __grid_constant__ StepParams P, unsigned long long* __restrict__ node_acc,
                unsigned long long* __restrict__ status, int use_bulk)
{
    using SM = StepSmem<NS>;
    using WT = WarpTile<NS>;
    constexpr int NF = WT::NF, NQ = WT::NQ, NK = WT::NK, NT = SM::NT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SM& sm = *reinterpret_cast<SM*>(smem_raw);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    WT& W = sm.w[wid];
    for (int i = threadIdx.x; i < NT; i += kTPB) sm.table.key[i] = -1;
    for (int i = threadIdx.x; i < NT * NQ; i += kTPB) (&sm.table.acc[0][0])[i] = 0ull;
    if (lane == 0) mbar_init(&W.bar, 1);
    __syncthreads();

    unsigned err = 0;
    int hops = 0;
    uint32_t phase = 0;
    bool abort = false;
    const int64_t range0 = (int64_t)blockIdx.x * kRange;
    float* const tile = W.buf;
    float* const lamr = W.buf + WT::LAM;
    float* const keyr = W.buf + WT::KEY;          // new element ids, as float bit patterns
    // global row of field f (psi rows are `cap` apart)
    auto grow = [&](int f) -> float* {
        if (f == WT::F_X) return S.x;
        if (f == WT::F_Y) return S.y;
        if (f == WT::F_U) return S.u;
        if (f == WT::F_V) return S.v;
        if (f == WT::F_W) return S.w;
        if (f == WT::F_OM) return S.om;
        if (f == WT::F_ELEM) return reinterpret_cast<float*>(S.elem);
        if (f == WT::F_PID) return reinterpret_cast<float*>(S.pid);
        return S.psi + (size_t)(f - WT::F_PSI) * S.cap;
    };

    // the sub-tile loop is uniform over the CTA (it contains CTA barriers)
    for (int sub = 0; sub < kSubTilesPerCTA; ++sub) {
        const int64_t sb = range0 + (int64_t)sub * kSubTile;
        if (sb >= S.n) break;
        const int64_t tb = sb + (int64_t)wid * kTile;
        const int64_t rem = S.n - tb;
        int nvalid = rem <= 0 ? 0 : (rem < (int64_t)kTile ? (int)rem : kTile);
        if (abort) nvalid = 0;
        const bool bulk = use_bulk && nvalid == kTile;
        // the previous tile's bulk store must have finished reading the buffer, and the generic
        // reads and writes of the previous tile must be ordered before the next bulk load
        if (lane == 0) bulk_wait_read_all();
        fence_async_shared();
        __syncwarp();
        // ---- 1. stage the tile's state in shared memory ---------------------------------
        if (bulk) {
            if (lane == 0) {
                mbar_expect_tx(&W.bar, (uint32_t)(NF * kTile * sizeof(float)));
#pragma unroll
                for (int f = 0; f < NF; ++f) bulk_load(tile + f * kTile, grow(f) + tb, kTile * sizeof(float), &W.bar);
            }
            if (mbar_wait_bounded(&W.bar, phase)) {
                phase ^= 1u;
            } else {
                // give the copies in flight one more bounded wait, then stop this warp's work
                err |= kErrTimeout;
                mbar_wait_bounded(&W.bar, phase);
                abort = true;
                nvalid = 0;
            }
        } else if (nvalid > 0) {
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const float* g = grow(f) + tb;
                for (int t = lane; t < nvalid; t += 32) tile[f * kTile + t] = g[t];
            }
            __syncwarp();
        }
        // ---- 2. advance; lane l takes tile particles l, l+32, l+64, l+96 -----------------
#pragma unroll 1
        for (int j = 0; j < kPPL; ++j) {
            const int t = j * 32 + lane;
            int key = INT_MAX;
            if (t < nvalid) {
                Particle<NS> p;
                p.x = tile[WT::F_X * kTile + t]; p.y = tile[WT::F_Y * kTile + t];
                p.u = tile[WT::F_U * kTile + t]; p.v = tile[WT::F_V * kTile + t];
                p.w = tile[WT::F_W * kTile + t]; p.om = tile[WT::F_OM * kTile + t];
#pragma unroll
                for (int a = 0; a < NS; ++a) p.psi[a] = tile[(WT::F_PSI + a) * kTile + t];
                p.elem = __float_as_int(tile[WT::F_ELEM * kTile + t]);
                const uint32_t pid = __float_as_uint(tile[WT::F_PID * kTile + t]);
                float lam[3];
                if (advance<NS>(M, F, P, pid, p, lam, err, hops)) {
                    atomicAdd(&status[1], 1ull);
                    atomicCAS(&status[2], ~0ull, (unsigned long long)pid);
                }
                tile[WT::F_X * kTile + t] = p.x; tile[WT::F_Y * kTile + t] = p.y;
                tile[WT::F_U * kTile + t] = p.u; tile[WT::F_V * kTile + t] = p.v;
                tile[WT::F_W * kTile + t] = p.w; tile[WT::F_OM * kTile + t] = p.om;
#pragma unroll
                for (int a = 0; a < NS; ++a) tile[(WT::F_PSI + a) * kTile + t] = p.psi[a];
                tile[WT::F_ELEM * kTile + t] = __int_as_float(p.elem);
                lamr[t] = lam[0]; lamr[kTile + t] = lam[1]; lamr[2 * kTile + t] = lam[2];
                key = p.elem;
            }
            keyr[t] = __int_as_float(key);
        }
        // ---- 3. write the tile back (bulk store of every field but pid) -----------------
        if (bulk && !abort) {
            fence_async_shared();
            __syncwarp();
            if (lane == 0) {
#pragma unroll
                for (int f = 0; f < NF - 1; ++f) bulk_store(grow(f) + tb, tile + f * kTile, kTile * sizeof(float));
                bulk_commit();
            }
        } else if (nvalid > 0) {
            __syncwarp();
#pragma unroll
            for (int f = 0; f < NF - 1; ++f) {
                float* g = grow(f) + tb;
                for (int t = lane; t < nvalid; t += 32) g[t] = tile[f * kTile + t];
            }
        }
        // ---- 4. the tile's distinct new elements, ascending (warp minimum loop) ------------
        int key[kPPL];
#pragma unroll
        for (int j = 0; j < kPPL; ++j) key[j] = __float_as_int(keyr[j * 32 + lane]);
        {
            int nd = 0;
            int cur = __reduce_min_sync(kFull, min(min(key[0], key[1]), min(key[2], key[3])));
            while (cur != INT_MAX) {
                if (lane == 0 && consistent(nd < kTile, err)) W.dkey[nd] = cur;
                ++nd;
                int nx = INT_MAX;
#pragma unroll
                for (int j = 0; j < kPPL; ++j)
                    if (key[j] > cur) nx = min(nx, key[j]);
                cur = __reduce_min_sync(kFull, nx);
            }
            if (lane == 0) W.ndist = nd;
        }
        __syncthreads();
        // ---- 5. merge the warps' sorted lists into the CTA bins (warp 0) ------------------
        if (wid == 0) {
            // lane l looks after list entries l and l+32 of every warp's list: a k-way merge by
            // repeated minimum over the heads
            int head[kWarps];
#pragma unroll
            for (int w = 0; w < kWarps; ++w) head[w] = 0;
            int nbins = 0;
            for (;;) {
                int mn = INT_MAX;
#pragma unroll
                for (int w = 0; w < kWarps; ++w)
                    if (head[w] < sm.w[w].ndist) mn = min(mn, sm.w[w].dkey[head[w]]);
                if (mn == INT_MAX) break;
#pragma unroll
                for (int w = 0; w < kWarps; ++w)
                    if (head[w] < sm.w[w].ndist && sm.w[w].dkey[head[w]] == mn) ++head[w];
                if (lane == 0 && consistent(nbins < kSubTile, err)) sm.binkey[nbins] = mn;
                ++nbins;
            }
            if (lane == 0) sm.nbins = nbins;
        }
        __syncthreads();
        const int nbins = sm.nbins;
        int gbin[kPPL];
#pragma unroll
        for (int j = 0; j < kPPL; ++j) {
            int b = -1;
            if (key[j] != INT_MAX) {
                int lo = 0, hi = nbins - 1;           // binary search: binkey is ascending
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (sm.binkey[mid] < key[j]) lo = mid + 1; else hi = mid;
                }
                b = lo;
            }
            gbin[j] = b;
        }
        // passes over ranges of at most kMaxBins bins (one pass unless the sub-tile is scattered)
        for (int b0 = 0; b0 < nbins; b0 += kMaxBins) {
            const int nbp = min(kMaxBins, nbins - b0);
            const bool last = b0 + kMaxBins >= nbins;
            // ---- 6. stable counting sort of this pass's particles by bin -----------------
            for (int i = threadIdx.x; i < nbp * kRows; i += kTPB) (&sm.cnt[0][0])[i] = 0;
            __syncthreads();
            int bin[kPPL], rank[kPPL];
#pragma unroll
            for (int j = 0; j < kPPL; ++j) {
                const int b = (gbin[j] >= b0 && gbin[j] < b0 + nbp) ? gbin[j] - b0 : -1;
                const unsigned m = __match_any_sync(kFull, b);
                rank[j] = __popc(m & lt);
                bin[j] = b;
                if (b >= 0 && rank[j] == 0) sm.cnt[b][wid * kPPL + j] = __popc(m);
            }
            __syncthreads();
            // exclusive scan over (bin, row), bin-major: each thread owns a run of entries
            {
                constexpr int PER = (kMaxBins * kRows) / kTPB;
                const int n = nbp * kRows;
                const int e0 = threadIdx.x * PER;
                int v[PER];
                int sum = 0;
#pragma unroll
                for (int i = 0; i < PER; ++i) {
                    v[i] = (e0 + i < n) ? (&sm.cnt[0][0])[e0 + i] : 0;
                    sum += v[i];
                }
                int incl = sum;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int tt = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += tt;
                }
                if (lane == 31) sm.wsum[wid] = incl;
                __syncthreads();
                int woff = 0;
#pragma unroll
                for (int w = 0; w < kWarps; ++w) woff += (w < wid) ? sm.wsum[w] : 0;
                if (threadIdx.x == kTPB - 1) sm.ntot = woff + incl;
                int run = woff + incl - sum;
#pragma unroll
                for (int i = 0; i < PER; ++i) {
                    if (e0 + i < n) (&sm.cnt[0][0])[e0 + i] = run;
                    run += v[i];
                }
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < kPPL; ++j)
                if (bin[j] >= 0) {
                    const int pos = sm.cnt[bin[j]][wid * kPPL + j] + rank[j];
                    if (!consistent(pos >= 0 && pos < kSubTile, err)) continue;
                    sm.cperm[pos] = (unsigned short)((wid << 7) | (j * 32 + lane));
                    sm.cbin[pos] = (unsigned char)bin[j];
                }
            // node-table slots of every bin's three corners
            for (int i = threadIdx.x; i < 3 * nbp; i += kTPB) {
                const int b = i / 3, c = i - 3 * (i / 3);
                const int ek = sm.binkey[b0 + b];
                if (!consistent(ek >= 0 && ek < M.n_tri, err)) { sm.cslot[b][c] = -1; continue; }
                const int4 mv = __ldg(&M.em[ek]);
                sm.cslot[b][c] = (short)table_slot(sm.table, c == 0 ? mv.x : (c == 1 ? mv.y : mv.z));
            }
            if (lane == 0) W.nlist = 0;
            __syncthreads();
            // ---- 7. warp w reduces sorted positions 128w .. 128w+127; lane l takes 4 --------
            const int ntot = consistent(sm.ntot >= 0 && sm.ntot <= kSubTile, err) ? sm.ntot : 0;
            float acc[NK];
#pragma unroll
            for (int k = 0; k < NK; ++k) acc[k] = 0.0f;
            int curb = -1;
            const int pbeg = wid * kTile + kPPL * lane;
#pragma unroll 1
            for (int p = pbeg; p < pbeg + kPPL && p < ntot; ++p) {
                const int b = sm.cbin[p];
                if (!consistent(b < nbp && sm.cperm[p] < kSubTile, err)) break;
                if (b != curb) {
                    if (curb >= 0) {
                        // a segment that ends inside this lane's chunk: park its FP32 partial
                        const int slot = atomicAdd(&W.nlist, 1);
                        if (slot < WT::NL) {
#pragma unroll
                            for (int k = 0; k < NK; ++k) { W.lpart[slot][k] = acc[k]; acc[k] = 0.0f; }
                            W.lbin[slot] = curb;
                        } else {
                            float spill[NK];
#pragma unroll
                            for (int k = 0; k < NK; ++k) { spill[k] = acc[k]; acc[k] = 0.0f; }
                            flush_partial(sm.table, spill, __ldg(&M.em[sm.binkey[b0 + curb]]), sm.cslot[curb], node_acc,
                                          &err);
                        }
                    }
                    curb = b;
                }
                const int cp = sm.cperm[p];
                const WT& Src = sm.w[cp >> 7];
                const int t = cp & 127;
                const float* sl = Src.buf + WT::LAM;
                const float l0 = sl[t], l1 = sl[kTile + t], l2 = sl[2 * kTile + t];
                float q[NQ];
                const float u = Src.buf[WT::F_U * kTile + t], v = Src.buf[WT::F_V * kTile + t],
                            w = Src.buf[WT::F_W * kTile + t];
                q[0] = 1.0f; q[1] = u; q[2] = v; q[3] = w;
                q[4] = u * u; q[5] = u * v; q[6] = u * w; q[7] = v * v; q[8] = v * w; q[9] = w * w;
                q[10] = Src.buf[WT::F_OM * kTile + t];
#pragma unroll
                for (int a = 0; a < NS; ++a) {
                    const float ps = Src.buf[(WT::F_PSI + a) * kTile + t];
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
            flush_parked<NS>(M, sm, W, b0, lane, node_acc, err);
            if (last) {
                // every warp has read the tiles it needs; the bulk stores must have read them too:
                // then the lane partials may reuse this warp's tile buffer
                if (lane == 0) bulk_wait_read_all();
                __syncthreads();
                combine_lanes<NS>(M, sm, W, W.buf, acc, curb, b0, lane, node_acc, err);
            } else {
                // more passes follow and still need the tiles: flush this lane's last segment
                if (curb >= 0) {
                    float spill[NK];
#pragma unroll
                    for (int k = 0; k < NK; ++k) spill[k] = acc[k];
                    flush_partial(sm.table, spill, __ldg(&M.em[sm.binkey[b0 + curb]]), sm.cslot[curb], node_acc, &err);
                }
                __syncthreads();
            }
        }
        __syncwarp();
    }
    // every bulk store of this warp must be complete before the CTA exits
    if (lane == 0) bulk_wait_all();
    // ---- 9. flush the CTA node table ----------------------------------------------------
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
    // bulk copies need 16-byte aligned rows: every base pointer and the psi row stride
    auto al = [](const void* q) { return ((uintptr_t)q & 15u) == 0; };
    const int use_bulk = al(s.x) && al(s.y) && al(s.u) && al(s.v) && al(s.w) && al(s.om) && al(s.psi) && al(s.elem) &&
                         al(s.pid) && (s.cap % 4 == 0);
    pdf_step_kernel<NS><<<(unsigned)grid, kTPB, smem, st>>>(m, s, fields, p, node_acc, status, use_bulk);
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
        float lw[3];
        int ne = locate_walk(M, e, px, py, hops, lw);
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
        box_muller_accurate(a.z, a.w, z0, z1);
        box_muller_accurate(b.x, b.y, z2, z3);
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
