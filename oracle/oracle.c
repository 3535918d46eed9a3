/*
 * FP64 CPU oracle for the per-particle time step of the fully Lagrangian joint
 * velocity-frequency-scalar PDF method (Bakosi, Franzese & Boybeyi, arXiv:1006.0549).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously-correct statement of
 * what the particle step computes. Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load it. The product path never calls it, and it shares
 * no code, header, table or constant generator with the CUDA library.
 *
 * What it follows:
 *   position            Eq. 2   dX_i = U_i dt + (2 nu)^(1/2) dW_i, same dW_i as in Eq. 4
 *   velocity (GLM)      Eq. 4   dU_i = -d<P>/dx_i dt + 2 nu lap<U_i> dt + (2 nu)^(1/2) d<U_i>/dx_j dW_j
 *                                      + G_ij (U_j - <U_j>) dt + (C_0 eps)^(1/2) dW'_i
 *   frequency           Eq. 5   d omega = -C_3 <w>(w - <w>) dt - S_w <w> w dt + (2 C_3 C_4 <w>^2 w)^(1/2) dW
 *   frequency source    Eq. 6   S_w enters as a node field
 *   mixing              Eq. 9   d psi = -(psi - <phi|V>)/t_m dt + S(psi) dt,  t_m = 2/(C_phi <omega>):
 *                               IEM (<phi|V> -> <phi>), or IECM with <phi|V> linear in V, and an
 *                               optional second-order reaction psi_a + psi_b -> psi_p
 *   time integration    forward Euler (Section "Governing equations", summary paragraph);
 *                       every right-hand side uses the state at t_n
 *   statistics          extracted at gridpoints of the unstructured mesh, evaluated at particle
 *                       positions with linear shape functions (same paragraph)
 *   tracking            particles are tracked through the grid (Introduction, item iii)
 *   walls               only the no-slip condition on particles (Introduction): reflection
 *
 * Readings where the paper is silent (each is stated once here and in the design notes):
 *   - Wiener increments are sqrt(dt) * N(0,1); normals come from Philox4x32-10 (Salmon et al.,
 *     SC'11) keyed (seed) and countered (pid, step, tag<<16 | block), Box-Muller (1958) pairs.
 *   - sqrt(max(omega, 0)) inside Eq. 5, then omega <- |omega|.
 *   - reflection mirrors the position across the wall and sets U <- 2 U_w - U; on a mesh with
 *     walls of any shape (wall edges off the bounding box) the walk mirrors across the wall edge
 *     it meets (FP64, rounded to FP32; an image that rounds back onto the point steps one FP32
 *     value along the inward normal; the image is wrapped into the periodic frame again).
 *   - the walk leaves through the edge of the most negative barycentric, interior edges before
 *     walls; in a periodic image frame it only navigates toward the seam (seam_exit).
 *   - a point exactly on an edge belongs to the element for which that edge is "top-left"
 *     (edge a->b of a CCW triangle includes its points iff b.y < a.y or (b.y == a.y and b.x > a.x));
 *     the domain is half-open ([x0,x1) x [y0,y1)), so positions equal to x1 or y1 are moved to the
 *     next FP32 value inside (periodic x: to x0).
 *   - statistics estimator: S_k(n) = sum_p lambda_n(X_p) q_k(p); mean = S_q/S_0;
 *     central moment = S_qq/S_0 - mean^2.
 *
 * Exact geometric predicate: orient2d by exact floating-point expansion arithmetic
 * (Shewchuk, "Adaptive Precision Floating-Point Arithmetic and Fast Robust Geometric
 * Predicates", 1997): error-bounded FP64 filter, then an exact expansion sum.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_HOP_CAP 64
#define ORACLE_REFL_CAP 8
#define ORACLE_MAX_SOURCES 8
#define ORACLE_MAX_NS 8

/* ------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11). Round: two 32x32->64 multiplications by the round multipliers, the high halves
 * xored with the other counter words and the round key; key bumped by the Weyl constants
 * between rounds.                                                                         */
/* ------------------------------------------------------------------------------------ */
static const uint32_t PHILOX_M0 = 0xD2511F53u, PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u, PHILOX_W1 = 0xBB67AE85u;

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* the 8 words of blocks 0 and 1 for (seed, pid, step, tag) */
static void philox_words(uint64_t seed, uint32_t pid, uint64_t step, uint32_t tag, uint32_t blk0,
                         int nblk, uint32_t* w)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int b = 0; b < nblk; ++b) {
        uint32_t ctr[4] = {pid, (uint32_t)step, (uint32_t)(step >> 32), (tag << 16) | (blk0 + (uint32_t)b)};
        oracle_philox4x32_10(ctr, key, w + 4 * b);
    }
}

static double word_to_uniform(uint32_t w) { return ((double)w + 0.5) * 0x1p-32; }

/* Box-Muller: (u0, u1) -> r cos(2 pi u1), r sin(2 pi u1), r = sqrt(-2 ln u0) */
static void box_muller(double u0, double u1, double* z0, double* z1)
{
    const double r = sqrt(-2.0 * log(u0));
    const double t = 2.0 * M_PI * u1;
    *z0 = r * cos(t);
    *z1 = r * sin(t);
}

/* Six standard normals of one particle update: z0,z1 = dW_1,dW_2 (Eq. 2 and Eq. 4),
 * z2..z4 = dW'_1..3 (Eq. 4), z5 = dW (Eq. 5); all before the sqrt(dt) scaling. */
void oracle_normals6(uint64_t seed, uint32_t pid, uint64_t step, uint32_t tag, double z[6])
{
    uint32_t w[8];
    philox_words(seed, pid, step, tag, 0, 2, w);
    box_muller(word_to_uniform(w[0]), word_to_uniform(w[1]), &z[0], &z[1]);
    box_muller(word_to_uniform(w[2]), word_to_uniform(w[3]), &z[2], &z[3]);
    box_muller(word_to_uniform(w[4]), word_to_uniform(w[5]), &z[4], &z[5]);
}

/* ------------------------------------------------------------------------------------ */
/* Exact orient2d (Shewchuk 1997): sign of det[[ax-cx, ay-cy],[bx-cx, by-cy]].             */
/* ------------------------------------------------------------------------------------ */
static void two_sum(double a, double b, double* s, double* e)
{
    double x = a + b, bv = x - a, av = x - bv;
    *s = x;
    *e = (a - av) + (b - bv);
}

static void two_prod(double a, double b, double* p, double* e)
{
    double x = a * b;
    *p = x;
    *e = fma(a, b, -x);
}

/* h <- h + b exactly (Grow-Expansion); h is nonoverlapping, increasing magnitude */
static int grow_expansion(int n, double* h, double b)
{
    double q = b;
    int m = 0;
    double tmp[40];
    for (int i = 0; i < n; ++i) {
        double s, e;
        two_sum(q, h[i], &s, &e);
        if (e != 0.0) tmp[m++] = e;
        q = s;
    }
    if (q != 0.0) tmp[m++] = q;
    memcpy(h, tmp, sizeof(double) * (size_t)m);
    return m;
}

int oracle_orient2d_sign(double ax, double ay, double bx, double by, double cx, double cy)
{
    const double detleft = (ax - cx) * (by - cy);
    const double detright = (ay - cy) * (bx - cx);
    const double det = detleft - detright;
    const double eps = 0x1p-53;
    const double errbound = (3.0 + 16.0 * eps) * eps * (fabs(detleft) + fabs(detright));
    if (det > errbound) return 1;
    if (-det > errbound) return -1;
    /* exact: every difference as a two-term expansion, every product of terms exact */
    double acx, acxt, acy, acyt, bcx, bcxt, bcy, bcyt;
    two_sum(ax, -cx, &acx, &acxt);
    two_sum(ay, -cy, &acy, &acyt);
    two_sum(bx, -cx, &bcx, &bcxt);
    two_sum(by, -cy, &bcy, &bcyt);
    const double A[2] = {acx, acxt}, B[2] = {bcy, bcyt};
    const double C[2] = {acy, acyt}, D[2] = {bcx, bcxt};
    double h[40];
    int n = 0;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double p, e;
            two_prod(A[i], B[j], &p, &e);
            n = grow_expansion(n, h, p);
            n = grow_expansion(n, h, e);
            two_prod(C[i], D[j], &p, &e);
            n = grow_expansion(n, h, -p);
            n = grow_expansion(n, h, -e);
        }
    if (n == 0) return 0;
    return h[n - 1] > 0.0 ? 1 : (h[n - 1] < 0.0 ? -1 : 0);
}

/* ------------------------------------------------------------------------------------ */
/* Mesh                                                                                  */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    int n_nodes, n_tri;
    double *x, *y;
    int *tri, *tag, *nbr, *master;
    double* cx;
    double period;
    double x0, x1, y0, y1;
    int edge_walls;   /* 1: some wall edge is off the sides of the bounding box */
} OMesh;

void oracle_mesh_free(OMesh* m)
{
    if (!m) return;
    free(m->x); free(m->y); free(m->tri); free(m->tag); free(m->nbr); free(m->master); free(m->cx);
    free(m);
}

/* Builds the oracle's own adjacency: interior edges by shared node pairs, periodic edges by
 * matching the y values of their end points on x = x0 and x = x1. */
OMesh* oracle_mesh_new(const double* node_xy, int n_nodes, const int* tri, int n_tri, const int* tag,
                       double period, double x0, double x1, double y0, double y1)
{
    OMesh* m = (OMesh*)calloc(1, sizeof(OMesh));
    m->n_nodes = n_nodes; m->n_tri = n_tri; m->period = period;
    m->x0 = x0; m->x1 = x1; m->y0 = y0; m->y1 = y1;
    m->x = (double*)malloc(sizeof(double) * (size_t)n_nodes);
    m->y = (double*)malloc(sizeof(double) * (size_t)n_nodes);
    m->master = (int*)malloc(sizeof(int) * (size_t)n_nodes);
    m->tri = (int*)malloc(sizeof(int) * 3 * (size_t)n_tri);
    m->tag = (int*)malloc(sizeof(int) * 3 * (size_t)n_tri);
    m->nbr = (int*)malloc(sizeof(int) * 3 * (size_t)n_tri);
    m->cx = (double*)malloc(sizeof(double) * (size_t)n_tri);
    for (int i = 0; i < n_nodes; ++i) { m->x[i] = node_xy[2 * i]; m->y[i] = node_xy[2 * i + 1]; m->master[i] = i; }
    memcpy(m->tri, tri, sizeof(int) * 3 * (size_t)n_tri);
    memcpy(m->tag, tag, sizeof(int) * 3 * (size_t)n_tri);
    for (int e = 0; e < n_tri; ++e) {
        m->cx[e] = (m->x[tri[3 * e]] + m->x[tri[3 * e + 1]] + m->x[tri[3 * e + 2]]) / 3.0;
        for (int k = 0; k < 3; ++k) m->nbr[3 * e + k] = -1;
    }
    /* node -> element lists */
    int* cnt = (int*)calloc((size_t)n_nodes + 1, sizeof(int));
    for (int i = 0; i < 3 * n_tri; ++i) cnt[tri[i] + 1]++;
    for (int i = 0; i < n_nodes; ++i) cnt[i + 1] += cnt[i];
    int* fill = (int*)calloc((size_t)n_nodes, sizeof(int));
    int* lst = (int*)malloc(sizeof(int) * 3 * (size_t)n_tri);
    for (int e = 0; e < n_tri; ++e)
        for (int k = 0; k < 3; ++k) { int n = tri[3 * e + k]; lst[cnt[n] + fill[n]++] = e; }
    for (int e = 0; e < n_tri; ++e)
        for (int k = 0; k < 3; ++k) {
            int a = tri[3 * e + k], b = tri[3 * e + (k + 1) % 3];
            for (int t = cnt[a]; t < cnt[a + 1]; ++t) {
                int f = lst[t];
                if (f == e) continue;
                for (int kk = 0; kk < 3; ++kk) {
                    int fa = tri[3 * f + kk], fb = tri[3 * f + (kk + 1) % 3];
                    if (fa == b && fb == a) m->nbr[3 * e + k] = f;
                }
            }
        }
    if (period > 0.0) {
        /* periodic edges: left (x == x0) against right (x == x1) with equal y end points */
        for (int e = 0; e < n_tri; ++e)
            for (int k = 0; k < 3; ++k) {
                if (tag[3 * e + k] != 3) continue;
                int a = tri[3 * e + k], b = tri[3 * e + (k + 1) % 3];
                double ya = m->y[a], yb = m->y[b];
                int on_left = (m->x[a] == x0);
                for (int f = 0; f < n_tri && m->nbr[3 * e + k] < 0; ++f)
                    for (int kk = 0; kk < 3; ++kk) {
                        if (tag[3 * f + kk] != 3) continue;
                        int fa = tri[3 * f + kk], fb = tri[3 * f + (kk + 1) % 3];
                        int f_left = (m->x[fa] == x0);
                        if (f_left == on_left) continue;
                        if (m->y[fa] == yb && m->y[fb] == ya) { m->nbr[3 * e + k] = f; break; }
                    }
            }
        for (int i = 0; i < n_nodes; ++i) {
            if (m->x[i] != x1) continue;
            for (int j = 0; j < n_nodes; ++j)
                if (m->x[j] == x0 && m->y[j] == m->y[i]) { m->master[i] = j; break; }
        }
    }
    /* walls off the sides of the bounding box: mirror across wall edges during location */
    m->edge_walls = 0;
    for (int e = 0; e < n_tri; ++e)
        for (int k = 0; k < 3; ++k) {
            if (tag[3 * e + k] != 1 && tag[3 * e + k] != 2) continue;
            int a = tri[3 * e + k], b = tri[3 * e + (k + 1) % 3];
            double ax = m->x[a], ay = m->y[a], bx = m->x[b], by = m->y[b];
            int on_side = (ax == bx && (ax == x0 || ax == x1)) || (ay == by && (ay == y0 || ay == y1));
            if (!on_side) m->edge_walls = 1;
        }
    free(cnt); free(fill); free(lst);
    return m;
}

int oracle_mesh_edge_walls(const OMesh* m) { return m->edge_walls; }

int oracle_mesh_neighbors(const OMesh* m, int* out)
{
    memcpy(out, m->nbr, sizeof(int) * 3 * (size_t)m->n_tri);
    return 0;
}

int oracle_mesh_masters(const OMesh* m, int* out)
{
    memcpy(out, m->master, sizeof(int) * (size_t)m->n_nodes);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Point location                                                                        */
/* ------------------------------------------------------------------------------------ */
static int edge_included(double ax, double ay, double bx, double by)
{
    return (by < ay) || (by == ay && bx > ax);
}

/* 1 if p is inside-or-owned-on edge a->b, else 0 */
static int edge_in(double ax, double ay, double bx, double by, double px, double py)
{
    int s = oracle_orient2d_sign(ax, ay, bx, by, px, py);
    if (s > 0) return 1;
    if (s < 0) return 0;
    return edge_included(ax, ay, bx, by);
}

/* inside-or-owned test of element e: a point on an edge belongs to the element for which the
 * edge is "top-left", except that with walls off the frame (edge_walls) a point on a wall edge
 * belongs to its element (those walls are closed) */
int oracle_inside(const OMesh* m, int e, double px, double py)
{
    for (int k = 0; k < 3; ++k) {
        int a = m->tri[3 * e + k], b = m->tri[3 * e + (k + 1) % 3];
        if (m->edge_walls && m->nbr[3 * e + k] < 0) {
            if (oracle_orient2d_sign(m->x[a], m->y[a], m->x[b], m->y[b], px, py) < 0) return 0;
        } else if (!edge_in(m->x[a], m->y[a], m->x[b], m->y[b], px, py)) {
            return 0;
        }
    }
    return 1;
}

/* owner of p by testing every element; -1 if none, -2 - count if several */
int oracle_locate_brute(const OMesh* m, double px, double py)
{
    int owner = -1, count = 0;
    for (int e = 0; e < m->n_tri; ++e)
        if (oracle_inside(m, e, px, py)) { owner = e; ++count; }
    if (count > 1) return -2 - count;
    return owner;
}

/* nearest periodic image offset of p relative to element e (0 when not periodic) */
static double image_shift(const OMesh* m, int e, double px)
{
    if (m->period <= 0.0) return 0.0;
    double k = floor((m->cx[e] - px) / m->period + 0.5);
    return k * m->period;
}

/* The exit of a walk step in a periodic image frame (sh != 0), where the image of the point lies
 * inside no element and the step only moves toward the seam. An edge counts as crossed by the
 * image when the image is not inside it by the exact test of the own frame (top-left rule), so an
 * edge the walk crosses is inside for the next element and the walk never steps back, even from
 * a vertex on the seam; walls are never crossed here. A periodic edge crossed by the image
 * (`per`, the most negative) is taken first, since the point's own frame is on the other side;
 * else the most negative other crossed edge (`best`); else the element's periodic edge; else,
 * when the image lies beyond walls only (at a corner of the seam), the interior neighbour nearest
 * the seam: the least centroid x for sh < 0 (the image lies toward x0), the greatest for sh > 0. */
static int seam_exit(const OMesh* m, int e, double sh, int per, int best)
{
    if (per >= 0) return per;
    if (best >= 0) return best;
    for (int k = 0; k < 3; ++k)
        if (m->tag[3 * e + k] == 3) return k;
    double bc = 0.0;
    for (int k = 0; k < 3; ++k) {
        int n = m->nbr[3 * e + k];
        if (n < 0) continue;
        float c = (float)m->cx[n];
        if (best < 0 || (sh < 0.0 ? c < bc : c > bc)) { best = k; bc = c; }
    }
    return best >= 0 ? best : 0;
}

/* Barycentric neighbour walk: start at `start`; while p is not inside, leave through the edge
 * whose barycentric is most negative among the interior edges it lies beyond, else through the
 * most negative wall edge (ties: lowest local index). Inside tests are exact and
 * only made in the element's own frame (image shift 0); in a shifted frame the walk only
 * navigates. Returns the owner, -1 on a wall exit (cannot happen in a convex domain), -2 when
 * the hop cap is reached. */
int oracle_locate_walk(const OMesh* m, int start, double px, double py, int* hops_out)
{
    int e = start;
    for (int h = 0; h <= ORACLE_HOP_CAP; ++h) {
        double sh = image_shift(m, e, px);
        double qx = px + sh;
        int best = -1, per = -1;
        double bestv = 0.0, perv = 0.0;
        int all_in = 1;
        for (int k = 0; k < 3; ++k) {
            int a = m->tri[3 * e + k], b = m->tri[3 * e + (k + 1) % 3];
            double ax = m->x[a], ay = m->y[a], bx = m->x[b], by = m->y[b];
            double val = (bx - ax) * (py - ay) - (by - ay) * (qx - ax);
            int in;
            if (sh == 0.0) {
                in = (m->edge_walls && m->nbr[3 * e + k] < 0) ? oracle_orient2d_sign(ax, ay, bx, by, qx, py) >= 0
                                                               : edge_in(ax, ay, bx, by, qx, py);
            } else {
                /* shifted frame: the image is tested as a point of the own frame (exact orientation,
                 * top-left rule), walls excepted (never crossed here); it lies inside no element */
                all_in = 0;
                in = (m->nbr[3 * e + k] < 0) || edge_in(ax, ay, bx, by, qx, py);
                if (!in && m->tag[3 * e + k] == 3 && (per < 0 || val < perv)) { per = k; perv = val; }
            }
            if (!in) {
                all_in = 0;
                /* the exit: the most negative across an interior edge, else across a wall */
                int nk = m->nbr[3 * e + k] >= 0, nb = best >= 0 && m->nbr[3 * e + best] >= 0;
                if (best < 0 || (nk && !nb) || (nk == nb && val < bestv)) { best = k; bestv = val; }
            }
        }
        if (sh == 0.0 && all_in) { if (hops_out) *hops_out = h; return e; }
        if (sh != 0.0) best = seam_exit(m, e, sh, per, best);
        int n = m->nbr[3 * e + best];
        if (n < 0) { if (hops_out) *hops_out = h; return -1; }
        e = n;
    }
    if (hops_out) *hops_out = ORACLE_HOP_CAP + 1;
    return -2;
}

/* The walk of oracle_locate_walk for walls of any shape: when it would leave through a wall edge
 * (edge k of element e, from node a to node b), the FP32 position is mirrored across the edge's
 * line -- t = ((p - a).d)/(d.d), foot f = a + t d, p' = 2 f - p with d = b - a, in FP64, then
 * rounded to FP32; an image that rounds back onto the point moves one FP32 step along the inward
 * normal (-d_y, d_x) -- the velocity becomes 2 U_w - U (U_w = (lid_u, 0, 0) on a moving-wall edge,
 * else 0), and the walk goes on from e; at most ORACLE_REFL_CAP mirrorings. Returns the owner or
 * a negative value as oracle_locate_walk. */
int oracle_locate_walk_reflect(const OMesh* m, int start, float* px, float* py, double* U, double* V, double* W,
                               double lid_u, int* hops_out, int* nref_out)
{
    int e = start, nref = 0, h = 0;
    for (;;) {
        double sh = image_shift(m, e, *px);
        double qx = *px + sh;
        int best = -1, per = -1;
        double bestv = 0.0, perv = 0.0;
        int all_in = 1;
        for (int k = 0; k < 3; ++k) {
            int a = m->tri[3 * e + k], b = m->tri[3 * e + (k + 1) % 3];
            double ax = m->x[a], ay = m->y[a], bx = m->x[b], by = m->y[b];
            double val = (bx - ax) * ((double)*py - ay) - (by - ay) * (qx - ax);
            int in;
            if (sh == 0.0) {
                in = (m->edge_walls && m->nbr[3 * e + k] < 0) ? oracle_orient2d_sign(ax, ay, bx, by, qx, *py) >= 0
                                                               : edge_in(ax, ay, bx, by, qx, *py);
            } else {
                all_in = 0;
                in = (m->nbr[3 * e + k] < 0) || edge_in(ax, ay, bx, by, qx, *py);
                if (!in && m->tag[3 * e + k] == 3 && (per < 0 || val < perv)) { per = k; perv = val; }
            }
            if (!in) {
                all_in = 0;
                /* the exit: the most negative across an interior edge, else across a wall */
                int nk = m->nbr[3 * e + k] >= 0, nb = best >= 0 && m->nbr[3 * e + best] >= 0;
                if (best < 0 || (nk && !nb) || (nk == nb && val < bestv)) { best = k; bestv = val; }
            }
        }
        if (sh == 0.0 && all_in) { *hops_out = h; *nref_out = nref; return e; }
        if (sh != 0.0) best = seam_exit(m, e, sh, per, best);
        int n = m->nbr[3 * e + best];
        if (n < 0) {
            if (nref >= ORACLE_REFL_CAP) { *hops_out = h; *nref_out = nref; return -1; }
            int a = m->tri[3 * e + best], b = m->tri[3 * e + (best + 1) % 3];
            double dx = m->x[b] - m->x[a], dy = m->y[b] - m->y[a];
            double t = (((double)*px - m->x[a]) * dx + ((double)*py - m->y[a]) * dy) / (dx * dx + dy * dy);
            double fx = m->x[a] + t * dx, fy = m->y[a] + t * dy;
            float nx = (float)(2.0 * fx - (double)*px), ny = (float)(2.0 * fy - (double)*py);
            if (nx == *px && ny == *py) {
                /* an image that rounds back onto the point (within about an ulp beyond the wall):
                 * one FP32 step along the inward normal (-dy, dx) of the edge */
                if (dy != 0.0) *px = nextafterf(*px, dy < 0.0 ? INFINITY : -INFINITY);
                if (dx != 0.0) *py = nextafterf(*py, dx > 0.0 ? INFINITY : -INFINITY);
            } else {
                *px = nx;
                *py = ny;
            }
            /* the image across a wall edge not parallel to the seam can leave the frame in x */
            if (m->period > 0.0) {
                if (*px < (float)m->x0) *px = (float)((double)*px + m->period);
                else if (*px >= (float)m->x1) *px = (float)((double)*px - m->period);
                /* the half-open frame: an image that rounds to x1 belongs to x0 */
                if (*px >= (float)m->x1) *px = (float)m->x0;
            }
            *U = (m->tag[3 * e + best] == 2 ? 2.0 * lid_u : 0.0) - *U;
            *V = -*V;
            *W = -*W;
            ++nref;
            continue;
        }
        if (h >= ORACLE_HOP_CAP) { *hops_out = ORACLE_HOP_CAP + 1; *nref_out = nref; return -2; }
        e = n;
        ++h;
    }
}

/* barycentric coordinates of p in element e (element's own frame), FP64 */
static void barycentric(const OMesh* m, int e, double px, double py, double lam[3])
{
    const int* t = m->tri + 3 * e;
    double x0 = m->x[t[0]], y0 = m->y[t[0]], x1 = m->x[t[1]], y1 = m->y[t[1]], x2 = m->x[t[2]], y2 = m->y[t[2]];
    double A = (x1 - x0) * (y2 - y0) - (y1 - y0) * (x2 - x0);
    lam[0] = ((x1 - px) * (y2 - py) - (y1 - py) * (x2 - px)) / A;
    lam[1] = ((x2 - px) * (y0 - py) - (y2 - py) * (x0 - px)) / A;
    lam[2] = ((x0 - px) * (y1 - py) - (y0 - py) * (x1 - px)) / A;
}

void oracle_barycentric(const OMesh* m, int e, double px, double py, double* lam)
{
    barycentric(m, e, px, py, lam);
}

/* ------------------------------------------------------------------------------------ */
/* Parameters                                                                            */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    double nu, dt, C3, C4, Cphi, lid_u;
    uint64_t seed;
    int32_t ns;
    int32_t n_sources;
    double src_x[ORACLE_MAX_SOURCES], src_y[ORACLE_MAX_SOURCES], src_r[ORACLE_MAX_SOURCES];
    int32_t src_alpha[ORACLE_MAX_SOURCES];
    /* reactive source of Eq. 9: psi_a + psi_b -> psi_p at rate react_k (none when react_k <= 0) */
    double react_k;
    int32_t react_a, react_b, react_p;
} OParams;

/* node-field columns */
enum { F_U = 0, F_V, F_W, F_DUDX, F_DUDY, F_DVDX, F_DVDY, F_DWDX, F_DWDY, F_LAPU, F_LAPV, F_LAPW,
       F_DPDX, F_DPDY, F_G11, F_G12, F_G21, F_G22, F_G33, F_C0EPS, F_OMEGA, F_SOMEGA, F_PHI0 };

static void interpolate(const OMesh* m, const float* fields, int nfp, int nf, int e, const double lam[3], double* out)
{
    const int* t = m->tri + 3 * e;
    for (int f = 0; f < nf; ++f) {
        double s = 0.0;
        for (int a = 0; a < 3; ++a) s += lam[a] * (double)fields[(size_t)t[a] * (size_t)nfp + (size_t)f];
        out[f] = s;
    }
}

/* scalar source test, taken in FP32 like the kernel: (x-xs)^2 + (y-ys)^2 < r^2, each op rounded */
static int in_source_f32(float px, float py, float sx, float sy, float r)
{
    volatile float dx = px - sx;
    volatile float dy = py - sy;
    volatile float dxx = dx * dx;
    volatile float dyy = dy * dy;
    volatile float d2 = dxx + dyy;
    volatile float r2 = r * r;
    return d2 < r2;
}

/* ------------------------------------------------------------------------------------ */
/* One forward-Euler step of every particle.                                              */
/* State arrays: FP32 input; FP64 output (positions are FP32 values).                     */
/* aux (4 per particle): position before the boundary treatment (x, y), number of         */
/* reflections, walk hops.                                                                */
/* locate_mode: 0 walk, 1 brute force, 2 both (a disagreement counts as lost).            */
/* Returns the number of particles that could not be located.                            */
/* ------------------------------------------------------------------------------------ */
long oracle_pdf_step(const OMesh* m, const OParams* p, const float* fields, int nfp, const float* beta, long P,
                     const float* x, const float* y, const float* u, const float* v, const float* w,
                     const float* om, const float* psi, const int* elem, const uint32_t* pid,
                     uint64_t step, int locate_mode,
                     double* ox, double* oy, double* ou, double* ov, double* ow, double* oom, double* opsi,
                     int* oelem, double* aux)
{
    const int ns = p->ns;
    const int nf = 22 + ns;
    const double dt = p->dt, sdt = sqrt(dt), s2nu = sqrt(2.0 * p->nu);
    const int periodic = m->period > 0.0;
    long lost = 0;
    for (long i = 0; i < P; ++i) {
        const int e = elem[i];
        double X = x[i], Y = y[i], U = u[i], V = v[i], W = w[i], OM = om[i];
        double lam[3];
        barycentric(m, e, X, Y, lam);
        double F[22 + ORACLE_MAX_NS];
        interpolate(m, fields, nfp, nf, e, lam, F);
        double z[6];
        oracle_normals6(p->seed, pid[i], step, 0u, z);
        const double dW1 = sdt * z[0], dW2 = sdt * z[1];
        const double dWp1 = sdt * z[2], dWp2 = sdt * z[3], dWp3 = sdt * z[4], dWw = sdt * z[5];
        const double c0e = sqrt(fmax(F[F_C0EPS], 0.0));
        const double Ur = U - F[F_U], Vr = V - F[F_V], Wr = W - F[F_W];
        /* Eq. 4 */
        double Un = U + (-F[F_DPDX] + 2.0 * p->nu * F[F_LAPU] + F[F_G11] * Ur + F[F_G12] * Vr) * dt
                      + s2nu * (F[F_DUDX] * dW1 + F[F_DUDY] * dW2) + c0e * dWp1;
        double Vn = V + (-F[F_DPDY] + 2.0 * p->nu * F[F_LAPV] + F[F_G21] * Ur + F[F_G22] * Vr) * dt
                      + s2nu * (F[F_DVDX] * dW1 + F[F_DVDY] * dW2) + c0e * dWp2;
        double Wn = W + (2.0 * p->nu * F[F_LAPW] + F[F_G33] * Wr) * dt
                      + s2nu * (F[F_DWDX] * dW1 + F[F_DWDY] * dW2) + c0e * dWp3;
        /* Eq. 5 with S_w from Eq. 6 as a node field */
        const double Om = F[F_OMEGA];
        double OMn = OM - p->C3 * Om * (OM - Om) * dt - F[F_SOMEGA] * Om * OM * dt
                        + sqrt(2.0 * p->C3 * p->C4 * Om * Om * fmax(OM, 0.0)) * dWw;
        OMn = fabs(OMn);
        /* Eq. 9: relaxation to the conditional mean with 1/t_m = C_phi <omega> / 2; IEM takes
         * <phi|V> = <phi>, IECM (beta given) <phi_a|V> = <phi_a> + beta_a . (U - <U>) with beta
         * interpolated like the other node fields; plus the reactive source, from the state at t_n */
        double PSIn[ORACLE_MAX_NS], PS[ORACLE_MAX_NS], S[ORACLE_MAX_NS];
        for (int a = 0; a < ns; ++a) {
            PS[a] = psi[(size_t)a * (size_t)P + (size_t)i];
            S[a] = 0.0;
        }
        if (p->react_k > 0.0) {
            const double r = p->react_k * PS[p->react_a] * PS[p->react_b];
            S[p->react_a] -= r;
            S[p->react_b] -= r;
            S[p->react_p] += r;
        }
        double B[3 * ORACLE_MAX_NS];
        if (beta) interpolate(m, beta, 3 * ns, 3 * ns, e, lam, B);
        for (int a = 0; a < ns; ++a) {
            double cond = F[F_PHI0 + a];
            if (beta) cond += B[3 * a] * Ur + B[3 * a + 1] * Vr + B[3 * a + 2] * Wr;
            PSIn[a] = PS[a] - (PS[a] - cond) * (0.5 * p->Cphi * Om) * dt + S[a] * dt;
        }
        /* Eq. 2, with the state at t_n */
        double qx = X + U * dt + s2nu * dW1;
        double qy = Y + V * dt + s2nu * dW2;
        if (aux) { aux[4 * i + 0] = qx; aux[4 * i + 1] = qy; }
        /* periodic wrap, then wall reflections (U <- 2 U_w - U; lid at y1 moves with (lid_u,0,0)) */
        if (periodic) {
            double k = floor((qx - m->x0) / m->period);
            qx -= k * m->period;
        }
        int nref = 0;
        for (int it = 0; it < 8 && !m->edge_walls; ++it) {
            if (qy < m->y0) { qy = 2.0 * m->y0 - qy; Un = -Un; Vn = -Vn; Wn = -Wn; ++nref; }
            else if (qy > m->y1) { qy = 2.0 * m->y1 - qy; Un = 2.0 * p->lid_u - Un; Vn = -Vn; Wn = -Wn; ++nref; }
            else if (!periodic && qx < m->x0) { qx = 2.0 * m->x0 - qx; Un = -Un; Vn = -Vn; Wn = -Wn; ++nref; }
            else if (!periodic && qx > m->x1) { qx = 2.0 * m->x1 - qx; Un = -Un; Vn = -Vn; Wn = -Wn; ++nref; }
            else break;
        }
        float pxf = (float)qx, pyf = (float)qy;
        const float x0f = (float)m->x0, x1f = (float)m->x1, y1f = (float)m->y1;
        if (!m->edge_walls) {
            if (pxf >= x1f) pxf = periodic ? x0f : nextafterf(x1f, -INFINITY);
            if (pyf >= y1f) pyf = nextafterf(y1f, -INFINITY);
        } else if (periodic && pxf >= x1f) {
            pxf = x0f;
        }
        /* point location */
        int hops = 0, ne;
        if (m->edge_walls) {
            /* walls of any shape: mirrored across the wall edge through which the walk leaves */
            ne = oracle_locate_walk_reflect(m, e, &pxf, &pyf, &Un, &Vn, &Wn, p->lid_u, &hops, &nref);
            if (locate_mode == 2 && ne >= 0 && oracle_locate_brute(m, pxf, pyf) != ne) ne = -3;
        } else if (locate_mode == 1) {
            ne = oracle_locate_brute(m, pxf, pyf);
        } else {
            ne = oracle_locate_walk(m, e, pxf, pyf, &hops);
            if (locate_mode == 2) {
                int nb = oracle_locate_brute(m, pxf, pyf);
                if (nb != ne) ne = -3;
            }
        }
        if (ne < 0) { ++lost; ne = e; }
        /* scalar sources (Section "Two testcases"): psi_alpha = 1 inside the source disc */
        for (int s = 0; s < p->n_sources; ++s)
            if (in_source_f32(pxf, pyf, (float)p->src_x[s], (float)p->src_y[s], (float)p->src_r[s]))
                PSIn[p->src_alpha[s]] = 1.0;
        ox[i] = pxf; oy[i] = pyf; ou[i] = Un; ov[i] = Vn; ow[i] = Wn; oom[i] = OMn;
        for (int a = 0; a < ns; ++a) opsi[(size_t)a * (size_t)P + (size_t)i] = PSIn[a];
        oelem[i] = ne;
        if (aux) { aux[4 * i + 2] = nref; aux[4 * i + 3] = hops; }
    }
    return lost;
}

/* ------------------------------------------------------------------------------------ */
/* Gridpoint statistics: raw sums S_k(n) = sum_p lambda_n(X_p) q_k(p), q = 1, u, v, w, uu, uv,
 * uw, vv, vw, ww, omega, psi_a (ns), psi_a^2 (ns). Sabs holds sum_p |lambda_n| |q_k| (the
 * scale of the rounding error of any evaluation of S). Periodic duplicates are folded:
 * both copies hold the total.                                                           */
/* ------------------------------------------------------------------------------------ */
void oracle_moments(const OMesh* m, int ns, long P, const double* x, const double* y, const double* u,
                    const double* v, const double* w, const double* om, const double* psi, const int* elem,
                    double* S, double* Sabs)
{
    const int nq = 11 + 2 * ns;
    memset(S, 0, sizeof(double) * (size_t)m->n_nodes * (size_t)nq);
    if (Sabs) memset(Sabs, 0, sizeof(double) * (size_t)m->n_nodes * (size_t)nq);
    double q[11 + 2 * ORACLE_MAX_NS];
    for (long i = 0; i < P; ++i) {
        const int e = elem[i];
        double lam[3];
        barycentric(m, e, x[i], y[i], lam);
        q[0] = 1.0; q[1] = u[i]; q[2] = v[i]; q[3] = w[i];
        q[4] = u[i] * u[i]; q[5] = u[i] * v[i]; q[6] = u[i] * w[i];
        q[7] = v[i] * v[i]; q[8] = v[i] * w[i]; q[9] = w[i] * w[i];
        q[10] = om[i];
        for (int a = 0; a < ns; ++a) {
            double ps = psi[(size_t)a * (size_t)P + (size_t)i];
            q[11 + a] = ps;
            q[11 + ns + a] = ps * ps;
        }
        for (int c = 0; c < 3; ++c) {
            const size_t n = (size_t)m->tri[3 * e + c];
            for (int k = 0; k < nq; ++k) {
                S[n * nq + k] += lam[c] * q[k];
                if (Sabs) Sabs[n * nq + k] += fabs(lam[c]) * fabs(q[k]);
            }
        }
    }
    for (int n = 0; n < m->n_nodes; ++n) {
        int mn = m->master[n];
        if (mn == n) continue;
        for (int k = 0; k < nq; ++k) {
            S[(size_t)mn * nq + k] += S[(size_t)n * nq + k];
            if (Sabs) Sabs[(size_t)mn * nq + k] += Sabs[(size_t)n * nq + k];
        }
    }
    for (int n = 0; n < m->n_nodes; ++n) {
        int mn = m->master[n];
        if (mn == n) continue;
        for (int k = 0; k < nq; ++k) {
            S[(size_t)n * nq + k] = S[(size_t)mn * nq + k];
            if (Sabs) Sabs[(size_t)n * nq + k] = Sabs[(size_t)mn * nq + k];
        }
    }
}

/* means and central moments: [S0, <u>, <v>, <w>, <u'u'>, <u'v'>, <u'w'>, <v'v'>, <v'w'>, <w'w'>,
 * <omega>, <psi_a>, <psi_a'^2>]; a node with S0 == 0 gets zeros. */
/* Scalar-flux sums for IECM: F(n) = sum_p lambda_n(X_p) (u psi_a, v psi_a, w psi_a), a = 0..ns-1,
 * per node (3 ns columns); periodic duplicates folded as in oracle_moments. */
void oracle_flux_moments(const OMesh* m, int ns, long P, const double* x, const double* y, const double* u,
                         const double* v, const double* w, const double* psi, const int* elem, double* F)
{
    const int nq = 3 * ns;
    memset(F, 0, sizeof(double) * (size_t)m->n_nodes * (size_t)nq);
    for (long i = 0; i < P; ++i) {
        const int e = elem[i];
        double lam[3];
        barycentric(m, e, x[i], y[i], lam);
        for (int k = 0; k < 3; ++k) {
            const int n = m->master[m->tri[3 * e + k]];
            for (int a = 0; a < ns; ++a) {
                const double ps = psi[(size_t)a * (size_t)P + (size_t)i];
                F[(size_t)n * nq + 3 * a + 0] += lam[k] * u[i] * ps;
                F[(size_t)n * nq + 3 * a + 1] += lam[k] * v[i] * ps;
                F[(size_t)n * nq + 3 * a + 2] += lam[k] * w[i] * ps;
            }
        }
    }
    for (int n = 0; n < m->n_nodes; ++n)
        if (m->master[n] != n)
            memcpy(F + (size_t)n * nq, F + (size_t)m->master[n] * nq, sizeof(double) * (size_t)nq);
}

void oracle_grid_statistics(int n_nodes, int ns, const double* S, double* out)
{
    const int nq = 11 + 2 * ns;
    for (int n = 0; n < n_nodes; ++n) {
        const double* s = S + (size_t)n * nq;
        double* o = out + (size_t)n * nq;
        const double s0 = s[0];
        o[0] = s0;
        if (s0 == 0.0) { for (int k = 1; k < nq; ++k) o[k] = 0.0; continue; }
        const double mu = s[1] / s0, mv = s[2] / s0, mw = s[3] / s0;
        o[1] = mu; o[2] = mv; o[3] = mw;
        o[4] = s[4] / s0 - mu * mu; o[5] = s[5] / s0 - mu * mv; o[6] = s[6] / s0 - mu * mw;
        o[7] = s[7] / s0 - mv * mv; o[8] = s[8] / s0 - mv * mw; o[9] = s[9] / s0 - mw * mw;
        o[10] = s[10] / s0;
        for (int a = 0; a < ns; ++a) {
            const double mp = s[11 + a] / s0;
            o[11 + a] = mp;
            o[11 + ns + a] = s[11 + ns + a] / s0 - mp * mp;
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* Particle initialisation: n_per_elem particles per element, pid = e*n_per_elem + j,
 * position uniform in the element (s = sqrt(r1): lambda = (1-s, s(1-r2), s r2)), located
 * exactly, U = <U>(X) + sigma(X) z, omega = <omega>(X)/m * sum_{i<m} -ln(e_i) (Erlang(m) with
 * mean <omega>, m = 1/C_4), psi = 0. Random words: Philox tag 1, blocks 0..2, step 0.
 * node_init per node: <U>, <V>, <W>, sigma, <omega>, pad x3.                               */
/* ------------------------------------------------------------------------------------ */
long oracle_particles_init(const OMesh* m, const OParams* p, int n_per_elem, const float* node_init,
                           int m_erlang, double* ox, double* oy, double* ou, double* ov, double* ow,
                           double* oom, double* opsi, int* oelem, uint32_t* opid)
{
    const long P = (long)m->n_tri * n_per_elem;
    long lost = 0;
    for (int e = 0; e < m->n_tri; ++e)
        for (int j = 0; j < n_per_elem; ++j) {
            const long i = (long)e * n_per_elem + j;
            const uint32_t id = (uint32_t)i;
            uint32_t wd[12];
            philox_words(p->seed, id, 0, 1u, 0, 3, wd);
            const double r1 = word_to_uniform(wd[0]), r2 = word_to_uniform(wd[1]);
            const double s = sqrt(r1);
            const double l0 = 1.0 - s, l1 = s * (1.0 - r2), l2 = s * r2;
            const int* t = m->tri + 3 * e;
            double X = l0 * m->x[t[0]] + l1 * m->x[t[1]] + l2 * m->x[t[2]];
            double Y = l0 * m->y[t[0]] + l1 * m->y[t[1]] + l2 * m->y[t[2]];
            float pxf = (float)X, pyf = (float)Y;
            const float x1f = (float)m->x1, y1f = (float)m->y1;
            if (pxf >= x1f) pxf = (m->period > 0.0) ? (float)m->x0 : nextafterf(x1f, -INFINITY);
            if (pyf >= y1f) pyf = nextafterf(y1f, -INFINITY);
            int hops;
            int ne = oracle_locate_walk(m, e, pxf, pyf, &hops);
            if (ne < 0) { ++lost; ne = e; }
            double lam[3];
            barycentric(m, ne, pxf, pyf, lam);
            double Fi[5];
            const int* tn = m->tri + 3 * ne;
            for (int f = 0; f < 5; ++f) {
                double acc = 0.0;
                for (int a = 0; a < 3; ++a) acc += lam[a] * (double)node_init[(size_t)tn[a] * 8 + (size_t)f];
                Fi[f] = acc;
            }
            double z0, z1, z2, z3;
            box_muller(word_to_uniform(wd[2]), word_to_uniform(wd[3]), &z0, &z1);
            box_muller(word_to_uniform(wd[4]), word_to_uniform(wd[5]), &z2, &z3);
            double sum = 0.0;
            for (int k = 0; k < m_erlang; ++k) sum += -log(word_to_uniform(wd[6 + k]));
            ox[i] = pxf; oy[i] = pyf;
            ou[i] = Fi[0] + Fi[3] * z0;
            ov[i] = Fi[1] + Fi[3] * z1;
            ow[i] = Fi[2] + Fi[3] * z2;
            oom[i] = Fi[4] * sum / (double)m_erlang;
            for (int a = 0; a < p->ns; ++a) opsi[(size_t)a * (size_t)P + (size_t)i] = 0.0;
            oelem[i] = ne;
            opid[i] = id;
        }
    return lost;
}
