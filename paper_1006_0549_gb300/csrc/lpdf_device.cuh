// Device helpers shared by the kernels of liblpdf (sm_103a): counter-based normals, exact
// orientation and point location on the triangle mesh, interpolation, the CTA node table of
// 64-bit fixed-point moment sums, and bulk-copy (TMA) / mbarrier wrappers.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "lpdf_internal.h"

namespace lpdf {

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

// -2 ln u for u = (w + 1/2) 2^-32. Near u = 1 both the FP32 rounding of u and a logarithm with a
// bounded absolute error would leave a large relative error in the (small) result; there
// v = 1 - u = (~w + 1/2) 2^-32 is formed exactly from the integer and -ln(1 - v) summed as its
// series v + v^2/2 + ... + v^6/6 (v < 1/16: the remainder is below 1e-8 relative).
__device__ __forceinline__ float neg2log_tail(uint32_t w)
{
    const float v = fmaf((float)(~w), 0x1p-32f, 0x1p-33f);
    const float s = fmaf(v, fmaf(v, fmaf(v, fmaf(v, fmaf(v, 1.0f / 6.0f, 0.2f), 0.25f), 1.0f / 3.0f), 0.5f), 1.0f);
    return 2.0f * v * s;
}

// Box-Muller (1958) on the special-function unit: r^2 = -2 ln u0 (lg2.approx: absolute error
// ~2^-22 in log2, used for u0 <= 15/16 where -ln u0 >= 0.064), r = r^2 * rsqrt(r^2), angle
// theta = 2 pi u1 - pi in [-pi, pi), where the SFU sine and cosine are accurate to ~2^-21.4
// absolute; cos(theta + pi) = -cos(theta) and sin(theta + pi) = -sin(theta), so
// z0 = r cos(2 pi u1), z1 = r sin(2 pi u1) as in the oracle.
__device__ __forceinline__ void box_muller(uint32_t w0, uint32_t w1, float& z0, float& z1)
{
    const float r2 = w0 >= 0xF0000000u ? neg2log_tail(w0) : -2.0f * __logf(u01(w0));
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
    const float r = sqrtf(w0 >= 0xF0000000u ? neg2log_tail(w0) : -2.0f * logf(u01(w0)));
    float sn, cs;
    sincospif(2.0f * u01(w1), &sn, &cs);
    z0 = r * cs;
    z1 = r * sn;
}

// ------------------------------------------------------------------------------------------
// Exact orientation (rare fallback): sign of (ax-cx)(by-cy) - (ay-cy)(bx-cx) by exact FP64
// expansion arithmetic (Shewchuk 1997: two-sum, FMA two-product, grow-expansion).
// ------------------------------------------------------------------------------------------
static __device__ __noinline__ int orient_exact(double ax, double ay, double bx, double by, double cx, double cy)
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

// The same orientation for the periodic image (px + sh, py) of a point (sh = +-period): the
// difference px + sh - ax is formed with one rounding, as in the own frame, because one of
// ax - sh (sh > 0: an element near the seam at x1) or px + sh (sh < 0: a point near x1) is exact
// by Sterbenz's lemma when the two lie within a factor of two of each other; otherwise (an
// element far from the seam) the sign comes from the exact FP64 expansion of the image, whose x
// coordinate px + sh is exact in FP64. Returns the FP32 value (for choosing among exits) and the
// exact sign.
__device__ __forceinline__ float orient_sign_image(float ax, float ay, float bx, float by, float px, float py, float sh,
                                                   int& sgn)
{
    const bool shift_element = sh > 0.0f;
    const bool exact = shift_element ? (ax >= 0.5f * sh && ax <= 2.0f * sh) : (px >= -0.5f * sh && px <= -2.0f * sh);
    const float dx1 = __fsub_rn(bx, ax), dy1 = __fsub_rn(by, ay);
    const float dx2 = shift_element ? __fsub_rn(px, __fsub_rn(ax, sh)) : __fsub_rn(__fadd_rn(px, sh), ax);
    const float dy2 = __fsub_rn(py, ay);
    const float w = dy1 * dx2;
    const float e = fmaf(-dy1, dx2, w);
    const float f = fmaf(dx1, dy2, -w);
    const float val = f + e;
    const float detsum = fmaf(fabsf(dx1), fabsf(dy2), fabsf(w));
    const float bound = 4.0e-7f * detsum;
    if (exact && detsum > 1e-25f && val > bound) { sgn = 1; return val; }
    if (exact && detsum > 1e-25f && -val > bound) { sgn = -1; return val; }
    sgn = orient_exact((double)bx, (double)by, (double)px + (double)sh, (double)py, (double)ax, (double)ay);
    return val;
}

// an edge a->b of a CCW triangle owns the points on it iff it is a "top-left" edge
__device__ __forceinline__ bool edge_owns(float ax, float ay, float bx, float by)
{
    return (by < ay) || (by == ay && bx > ax);
}

// The exit of a walk test in a periodic image frame (sh = +-period). The image (px + sh, py) is
// tested as a point of the own frame (exact orientation, top-left rule), so an edge the walk
// crosses is inside for the next element and the walk never steps back, even from a vertex on
// the seam. The image of a point of the frame lies inside no element of the image frame: the test
// only picks the exit, never a wall. A periodic edge the image is not inside of first (it leads
// toward the point's own frame), the most negative one; else the most negative other edge; when
// the image lies beyond walls only (where the seam meets a wall), the element's periodic edge;
// else the interior neighbour nearest the seam. Out of line: few particles cross the seam.
static __device__ __noinline__ int image_exit(const DevMesh& M, int e, float px, float py, float sh)
{
    const float4 X = __ldg(&M.ex[e]);
    const float4 Y = __ldg(&M.ey[e]);
    const int4 N = __ldg(&M.en[e]);
    const float xs[3] = {X.x, X.y, X.z}, ys[3] = {Y.x, Y.y, Y.z};
    const int nb[3] = {N.x, N.y, N.z};
    int best = -1, per = -1;
    float bestv = 0.0f, perv = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int a = k, b = (k + 1) % 3;
        if (nb[k] < 0) continue;
        int s;
        const float val = orient_sign_image(xs[a], ys[a], xs[b], ys[b], px, py, sh, s);
        if (s > 0 || (s == 0 && edge_owns(xs[a], ys[a], xs[b], ys[b]))) continue;
        if ((N.w >> k) & 1) {
            if (per < 0 || val < perv) { per = k; perv = val; }
        } else if (best < 0 || val < bestv) {
            best = k;
            bestv = val;
        }
    }
    if (per >= 0) return per;
    if (best >= 0) return best;
    best = (N.w & 1) ? 0 : (N.w & 2) ? 1 : (N.w & 4) ? 2 : -1;
    if (best >= 0) return best;
    // sh < 0: the image lies left of this element, toward x0; sh > 0: right, toward x1
    float bc = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (nb[k] < 0) continue;
        const float c = __ldg(&M.ex[nb[k]]).w;
        if (best < 0 || (sh < 0.0f ? c < bc : c > bc)) { best = k; bc = c; }
    }
    return best >= 0 ? best : 0;
}

// One test of the barycentric neighbour walk at element e: true if e is the unique owner of
// (px, py) (exact inside tests in the element's own frame; lam = its barycentrics, from the
// orientation values); otherwise `next` = the neighbour across the exit edge (the edge with the
// most negative orientation value, the lowest local index on ties), -1 - k for a wall edge k
// (with edge walls a point on a wall edge is inside: those walls are closed). In a
// periodic image frame the test only navigates. Out of line: the step calls it only when the
// certified fast test is undecided, and its registers stay out of the step's hot loop.
// the decision of walk_test: kWalkIn when (px, py) is in e (then lam, when given, receives the
// barycentric weights), else the exit as walk_test's `next`
constexpr int kWalkIn = 0x7fffffff;
__device__ __forceinline__ int walk_decide(const DevMesh& M, int e, float px, float py, float* lam)
{
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
            // with edge walls a point on a wall edge belongs to the element (walls are closed);
            // otherwise the domain is the half-open frame and the top-left rule decides
            const bool in = s > 0 || (s == 0 && ((M.edge_walls && nb[k] < 0) || edge_owns(xs[a], ys[a], xs[b], ys[b])));
            if (!in) {
                all_in = false;
                // the exit: the most negative across an interior edge, else across a wall
                const bool better = best < 0 || (nb[k] >= 0 && nb[best] < 0) ||
                                    ((nb[k] >= 0) == (nb[best] >= 0) && vv[k] < bestv);
                if (better) { best = k; bestv = vv[k]; }
            }
        }
        if (all_in) {
            // edge k = (v_k, v_k+1) is opposite vertex k+2: lambda_{k+2} = orient_k / (2 area)
            if (lam) {
                lam[2] = vv[0] * Y.w;
                lam[0] = vv[1] * Y.w;
                lam[1] = vv[2] * Y.w;
            }
            return kWalkIn;
        }
    } else {
        best = image_exit(M, e, px, py, sh);
    }
    const int next = best == 0 ? N.x : (best == 1 ? N.y : N.z);
    return next < 0 ? -1 - best : next;   // a wall: -1 - (the exit edge)
}

static __device__ __noinline__ bool walk_test(const DevMesh& M, int e, float px, float py, float lam[3], int& next)
{
    const int c = walk_decide(M, e, px, py, lam);
    if (c == kWalkIn) return true;
    next = c;
    return false;
}

// walk_test without the weights, returning its decision (kWalkIn or the exit): the caller's
// variables never have their address taken, so they stay in registers
static __device__ __noinline__ int walk_test_code(const DevMesh& M, int e, float px, float py)
{
    return walk_decide(M, e, px, py, nullptr);
}

// The most negative lambda (vertex a) of the fast walk test lies across a wall: leave through the
// most negative interior edge that is certainly crossed instead; the wall (-1 - its edge) only
// when no interior edge can be crossed; kWalkUndecided when an interior edge is within its
// rounding bound. Returns the exit (the walk's `next`) or kWalkUndecided. Out of line: the step
// reaches it only at walls.
constexpr int kWalkUndecided = -0x7fffffff - 1;
static __device__ __noinline__ int fast_wall_exit(float l0, float l1, float l2, float E0, float E1, float E2, int4 N,
                                                  int a)
{
    const float lv[3] = {l0, l1, l2}, ev[3] = {E0, E1, E2};
    const int nv[3] = {N.y, N.z, N.x};
    int b = -1;
    for (int q = 0; q < 3; ++q) {
        if (nv[q] < 0) continue;
        if (lv[q] < -ev[q]) {
            if (b < 0 || lv[q] < lv[b]) b = q;
        } else if (!(lv[q] > ev[q])) {
            return kWalkUndecided;
        }
    }
    if (b >= 0) return nv[b];
    return -1 - (a == 2 ? 0 : a + 1);
}

// The walk test in the affine barycentric form relative to vertex 0, with a certified error
// bound: 1 = (px, py) is strictly inside e; 0 = it is certainly outside, leave through `next`
// (the edge opposite the most negative certainly negative lambda across an interior edge; if
// only walls are crossed, -1 - k for the wall edge k of the most negative one); -1 = undecided
// (within the rounding bound of an edge, or in a periodic image frame): the caller runs
// walk_test. Preferring interior exits keeps the walk inside a non-convex domain: a point of the
// domain can lie beyond the line of some wall edge, never beyond every negative edge's line.
// Bound: with u = 2^-24, dx = fl(px - x_v0) (x_v0 exact in FP32) and the coefficients rounded
// from FP64, |lambda_a' - lambda_a| <= 4.01 u (|b_a dx| + |g_a dy|) for a = 1, 2, and for
// lambda_0 = 1 - lambda_1 - lambda_2 that sum plus 2 u (1 + |lambda_1| + |lambda_2|); the
// constants below carry a margin for the rounding of the bounds themselves.
template <bool kWalls = false>
__device__ __forceinline__ int walk_test_fast(const DevMesh& M, int e, float px, float py, int& next)
{
    const float4* W = M.ew + 4 * (size_t)e;
    const float4 A = __ldg(W);
    const float4 B = __ldg(W + 1);
    const int4 N = __ldg(reinterpret_cast<const int4*>(W + 2));
    if (M.periodic && fabsf(B.z - px) > 0.5f * M.period) return -1;
    const float dx = __fsub_rn(px, A.x), dy = __fsub_rn(py, A.y);
    const float t1 = A.z * dx, s1 = A.w * dy, t2 = B.x * dx, s2 = B.y * dy;
    const float l1 = t1 + s1, l2 = t2 + s2;
    const float l0 = (1.0f - l1) - l2;
    const float E1 = 3.0e-7f * (fabsf(t1) + fabsf(s1)) + 1e-30f;
    const float E2 = 3.0e-7f * (fabsf(t2) + fabsf(s2)) + 1e-30f;
    const float E0 = E1 + E2 + 1.5e-7f * (1.0f + fabsf(l1) + fabsf(l2));
    if (l0 > E0 && l1 > E1 && l2 > E2) return 1;
    // the most negative lambda, lowest index on ties; vertex a is opposite edge (a + 1) % 3
    // (edge k runs from vertex k to vertex k + 1)
    int a = 0;
    float lm = l0;
    if (l1 < lm) { a = 1; lm = l1; }
    if (l2 < lm) { a = 2; lm = l2; }
    const float Ea = a == 0 ? E0 : (a == 1 ? E1 : E2);
    if (!(lm < -Ea)) return -1;
    next = a == 0 ? N.y : (a == 1 ? N.z : N.x);
    if (next >= 0) return 0;
    if (kWalls) {
        const int c = fast_wall_exit(l0, l1, l2, E0, E1, E2, N, a);
        if (c == kWalkUndecided) return -1;
        next = c;
        return 0;
    }
    next = -1 - (a == 2 ? 0 : a + 1);   // a wall: -1 - (the exit edge)
    return 0;
}

// Mirror image of (px, py) across the line of edge k of element e, in FP64 with every operation
// rounded once in this order, then rounded to FP32: d = b - a, t = ((p - a).d) / (d.d), foot
// f = a + t d, p' = 2 f - p. A point within about an ulp beyond the wall can have an image that
// rounds back onto itself; it then moves one FP32 step along the edge's inward normal (-d_y, d_x),
// so that the walk makes progress.
static __device__ __noinline__ void mirror_across_edge(const DevMesh& M, int e, int k, float& px, float& py)
{
    const float4 X = __ldg(&M.ex[e]);
    const float4 Y = __ldg(&M.ey[e]);
    const float xs[3] = {X.x, X.y, X.z}, ys[3] = {Y.x, Y.y, Y.z};
    const int b = k == 2 ? 0 : k + 1;
    const double ax = xs[k], ay = ys[k];
    const double dx = __dsub_rn(xs[b], ax), dy = __dsub_rn(ys[b], ay);
    const double qx = __dsub_rn(px, ax), qy = __dsub_rn(py, ay);
    const double t = __ddiv_rn(__dadd_rn(__dmul_rn(qx, dx), __dmul_rn(qy, dy)),
                               __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
    const double fx = __dadd_rn(ax, __dmul_rn(t, dx)), fy = __dadd_rn(ay, __dmul_rn(t, dy));
    const float nx = __double2float_rn(__dsub_rn(__dmul_rn(2.0, fx), (double)px));
    const float ny = __double2float_rn(__dsub_rn(__dmul_rn(2.0, fy), (double)py));
    if (nx == px && ny == py) {
        if (dy != 0.0) px = nextafterf(px, dy < 0.0 ? CUDART_INF_F : -CUDART_INF_F);
        if (dx != 0.0) py = nextafterf(py, dx > 0.0 ? CUDART_INF_F : -CUDART_INF_F);
        return;
    }
    px = nx;
    py = ny;
}

// The whole walk from element e: the owner of (px, py) (and its barycentrics), -1 on a wall
// exit, -2 at the hop cap.
__device__ __forceinline__ int locate_walk(const DevMesh& M, int e, float px, float py, int& hops, float lam[3])
{
#pragma unroll 1
    for (int h = 0; h <= kHopCap; ++h) {
        int next;
        if (walk_test(M, e, px, py, lam, next)) { hops = h; return e; }
        if (next < 0) { hops = h; return -1; }   // (the caller starts inside the domain)
        e = next;
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

// ------------------------------------------------------------------------------------------
// One particle's state in registers, and its forward-Euler step (Section "Governing
// equations"): Eq. 4 for U, Eq. 5 for omega, Eq. 9 for psi (IEM, or IECM with a reactive
// source), Eq. 2 for X with the same dW_1, dW_2; periodic wrap, wall reflection, the half-open
// domain and the scalar sources.
// ------------------------------------------------------------------------------------------
template <int NS>
struct ParticleState {
    float x, y, u, v, w, om, psi[NS];
    int elem;
    uint32_t pid;
};

__device__ __forceinline__ bool in_source(float px, float py, float sx, float sy, float r)
{
    const float dx = __fsub_rn(px, sx), dy = __fsub_rn(py, sy);
    return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)) < __fmul_rn(r, r);
}

// psi_alpha <- 1 inside the concentrated sources (discs) of `sp` (the step's parameters, or a
// component's: both carry n_src, src_x, src_y, src_r, src_alpha), on the final FP32 position
template <int NS, class SP>
__device__ __forceinline__ void apply_sources(const SP& sp, float px, float py, float* psi)
{
    // outside the discs' box: px < x - r (or another side) for every disc, so the rounded
    // difference is at least r in magnitude and the rounded squared distance is not below r^2
    if (!(px >= sp.src_box[0] && px <= sp.src_box[1] && py >= sp.src_box[2] && py <= sp.src_box[3])) return;
    for (int q = 0; q < sp.n_src; ++q)
        if (in_source(px, py, sp.src_x[q], sp.src_y[q], sp.src_r[q])) {
#pragma unroll
            for (int a = 0; a < NS; ++a)
                if (a == sp.src_alpha[q]) psi[a] = 1.0f;
        }
}

// the sources of the particle's component (a multi-component mesh), or the step's
template <int NS, int kKind>
__device__ __forceinline__ void particle_sources(const DevMesh& M, const StepParams& P, int e, float px, float py,
                                                 float* psi)
{
    if (kKind >= 1 && M.n_comp > 1) apply_sources<NS>(P.comp[__ldg(&M.ecomp[e])], px, py, psi);
    else apply_sources<NS>(P, px, py, psi);
}

// Interpolated node fields at the particle, two sources:
//   kElementTable = false: F is the node table (n_nodes x nfp); the P1 shape functions of the
//                          element weight its three node rows;
//   kElementTable = true:  F is the element table (n_tri x 3 x nfp: the fields at vertex 0 and
//                          their x and y gradients on the element), so F(p) = F0 + Gx dx + Gy dy
//                          with (dx, dy) = p - vertex 0; the same P1 interpolant.
template <int NS, bool kElementTable>
__device__ __forceinline__ void interpolate_fields(const DevMesh& M, const float* __restrict__ F, int e, float x,
                                                   float y, float* Fi)
{
    constexpr int NFP = (22 + NS + 3) / 4 * 4;
    if (kElementTable) {
        const float4 A = __ldg(&M.ea[e]);
        const float dx = __fsub_rn(x, A.x), dy = __fsub_rn(y, A.y);
        const float4* R = reinterpret_cast<const float4*>(F) + (size_t)e * (3 * NFP / 4);
#pragma unroll
        for (int q = 0; q < NFP / 4; ++q) {
            const float4 a = __ldg(R + q), gx = __ldg(R + NFP / 4 + q), gy = __ldg(R + 2 * (NFP / 4) + q);
            Fi[4 * q + 0] = fmaf(gx.x, dx, fmaf(gy.x, dy, a.x));
            Fi[4 * q + 1] = fmaf(gx.y, dx, fmaf(gy.y, dy, a.y));
            Fi[4 * q + 2] = fmaf(gx.z, dx, fmaf(gy.z, dy, a.z));
            Fi[4 * q + 3] = fmaf(gx.w, dx, fmaf(gy.w, dy, a.w));
        }
    } else {
        const float4 X = __ldg(&M.ex[e]);
        const float4 Y = __ldg(&M.ey[e]);
        const int4 V = __ldg(&M.ev[e]);
        float l0, l1, l2;
        barycentric(X, Y, x, y, l0, l1, l2);
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
}

// On return p holds the new state except the element, which is the walk's start: the old
// element, or 0 when the old one is outside the mesh (`bad`). kKind selects the code compiled in:
// 0 one component, walls on the frame's sides, IEM; 1 also several independent components (the
// particle's component, that of its element, gives the frame, the Philox key and the sources);
// 2 also walls off the frame (mirrored in the walk, not here), IECM and reactive sources.
template <int NS, bool kElementTable = false, int kKind = 0>
__device__ __forceinline__ void advance_particle(const DevMesh& M, const float* __restrict__ F, const StepParams& P,
                                                 ParticleState<NS>& p, unsigned& err, bool& bad)
{
    constexpr int NFP = (22 + NS + 3) / 4 * 4;
    const float x = p.x, y = p.y, u = p.u, v = p.v, w = p.w, om = p.om;
    bad = (unsigned)p.elem >= (unsigned)M.n_tri;
    const int e = bad ? 0 : p.elem;
    float fx0 = M.x0, fx1 = M.x1, fy0 = M.y0, fy1 = M.y1;
    uint32_t key0 = P.key0, key1 = P.key1;
    if (kKind >= 1 && M.n_comp > 1) {
        const int c = __ldg(&M.ecomp[e]);
        const float4 fr = __ldg(&M.cframe[c]);
        fx0 = fr.x;
        fx1 = fr.y;
        fy0 = fr.z;
        fy1 = fr.w;
        key0 = P.comp[c].key0;
        key1 = P.comp[c].key1;
    }
    // Wiener increments: Philox blocks 0 and 1 of counter (pid, step, 0<<16 | block)
    uint32_t step_lo = P.step_lo, step_hi = P.step_hi;
    if (P.step_dev) {
        const unsigned long long sn = *P.step_dev + P.step_add;
        step_lo = (uint32_t)sn;
        step_hi = (uint32_t)(sn >> 32);
    }
    const uint4 r0 = philox4x32_10(make_uint4(p.pid, step_lo, step_hi, 0u), key0, key1);
    const uint4 r1 = philox4x32_10(make_uint4(p.pid, step_lo, step_hi, 1u), key0, key1);
    float z0, z1, z2, z3, z4, z5;
    box_muller(r0.x, r0.y, z0, z1);
    box_muller(r0.z, r0.w, z2, z3);
    box_muller(r1.x, r1.y, z4, z5);
    // linear shape-function interpolation of the node fields (after the random numbers: fewer
    // registers live across the loads)
    float Fi[NFP];
    interpolate_fields<NS, kElementTable>(M, F, e, x, y, Fi);
    const float dW1 = P.sdt * z0, dW2 = P.sdt * z1;
    // square roots by the special-function unit's reciprocal square root (about 2 ulp; the step's
    // tolerance is 1e-5): sqrt(a) = a rsqrt(a) for a > 0
    const float c0a = fmaxf(Fi[LPDF_F_C0EPS], 0.0f);
    const float c0e = c0a > 0.0f ? c0a * rsqrtf(c0a) : 0.0f;
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
    const float oma = 2.0f * P.C3 * P.C4 * Om * Om * fmaxf(om, 0.0f);
    float omn = om - P.C3 * Om * (om - Om) * P.dt - Fi[LPDF_F_SOMEGA] * Om * om * P.dt
              + (oma > 0.0f ? oma * rsqrtf(oma) : 0.0f) * (P.sdt * z5);
    omn = fabsf(omn);
    // Eq. 9: relaxation to the conditional mean, 1/t_m = C_phi <omega> / 2
    const float mix = P.half_cphi * Om * P.dt;
    if (kKind == 2 && (P.beta || P.react_k > 0.0f)) {
        // IECM: <phi_a|V> = <phi_a> + beta_a . (U - <U>), beta interpolated by the shape functions of
        // the element's nodes; the reactive source psi_ra + psi_rb -> psi_rp; all from the state at t_n
        float cond[NS], src[NS];
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            cond[a] = Fi[LPDF_F_PHI0 + a];
            src[a] = 0.0f;
        }
        if (P.beta) {
            const float4 X = __ldg(&M.ex[e]), Y = __ldg(&M.ey[e]);
            const int4 V = __ldg(&M.ev[e]);
            float l0, l1, l2;
            barycentric(X, Y, x, y, l0, l1, l2);
            const float* b0 = P.beta + (size_t)V.x * 3 * NS;
            const float* b1 = P.beta + (size_t)V.y * 3 * NS;
            const float* b2 = P.beta + (size_t)V.z * 3 * NS;
#pragma unroll
            for (int a = 0; a < NS; ++a) {
                float bc[3];
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    bc[c] = fmaf(l0, __ldg(b0 + 3 * a + c), fmaf(l1, __ldg(b1 + 3 * a + c), l2 * __ldg(b2 + 3 * a + c)));
                cond[a] += bc[0] * Ur + bc[1] * Vr + bc[2] * Wr;
            }
        }
        if (P.react_k > 0.0f) {
            float pa = 0.0f, pb = 0.0f;
#pragma unroll
            for (int a = 0; a < NS; ++a) {
                if (a == P.react_a) pa = p.psi[a];
                if (a == P.react_b) pb = p.psi[a];
            }
            const float r = P.react_k * pa * pb;
#pragma unroll
            for (int a = 0; a < NS; ++a) {
                if (a == P.react_a) src[a] -= r;
                if (a == P.react_b) src[a] -= r;
                if (a == P.react_p) src[a] += r;
            }
        }
#pragma unroll
        for (int a = 0; a < NS; ++a) p.psi[a] = p.psi[a] - (p.psi[a] - cond[a]) * mix + src[a] * P.dt;
    } else {
        // IEM: <phi|V> = <phi>
#pragma unroll
        for (int a = 0; a < NS; ++a) p.psi[a] = p.psi[a] - (p.psi[a] - Fi[LPDF_F_PHI0 + a]) * mix;
    }
    // Eq. 2 with the velocity at t_n and the same dW_1, dW_2
    float qx = x + u * P.dt + P.s2nu * dW1;
    float qy = y + v * P.dt + P.s2nu * dW2;
    if (M.periodic) {
        if (qx < fx0) qx += M.period;
        else if (qx >= fx1) qx -= M.period;
        if (qx < fx0 || qx >= fx1) qx -= floorf((qx - fx0) / M.period) * M.period;   // moves > one period
    }
    if (!(kKind == 2 && M.edge_walls) && !(qy >= fy0 && qy < fy1 && qx >= fx0 && qx < fx1)) {
        // walls on the frame's sides: mirror at the frame (edge walls are mirrored in the walk);
        // a position inside the half-open frame needs neither this nor the clamp below
#pragma unroll 1
        for (int it = 0; it < 8; ++it) {
            if (qy < fy0) { qy = 2.0f * fy0 - qy; un = -un; vn = -vn; wn = -wn; }
            else if (qy > fy1) { qy = 2.0f * fy1 - qy; un = 2.0f * P.lid_u - un; vn = -vn; wn = -wn; }
            else if (!M.periodic && qx < fx0) { qx = 2.0f * fx0 - qx; un = -un; vn = -vn; wn = -wn; }
            else if (!M.periodic && qx > fx1) { qx = 2.0f * fx1 - qx; un = -un; vn = -vn; wn = -wn; }
            else break;
        }
        // half-open domain [x0, x1) x [y0, y1)
        if (qx >= fx1) qx = M.periodic ? fx0 : nextafterf(fx1, -CUDART_INF_F);
        if (qy >= fy1) qy = nextafterf(fy1, -CUDART_INF_F);
    } else if (M.periodic && qx >= fx1) {
        qx = fx0;
    }
    // concentrated scalar sources (with edge walls: after the walk, on the mirrored position)
    if (!(kKind == 2 && M.edge_walls)) particle_sources<NS, kKind>(M, P, e, qx, qy, p.psi);
    if (!(isfinite(un) && isfinite(vn) && isfinite(wn) && isfinite(omn) && isfinite(qx) && isfinite(qy)))
        err |= kErrNonFinite;
    p.x = qx;
    p.y = qy;
    p.u = un;
    p.v = vn;
    p.w = wn;
    p.om = omn;
    p.elem = e;
}

// Internal consistency check: a failed check records kErrCheck in the status word and the
// caller skips the access, so a logic error can never become a wild address.
__device__ __forceinline__ bool consistent(bool ok, unsigned& err)
{
    if (!ok) err |= kErrCheck;
    return ok;
}

}  // namespace lpdf
