// Host side of liblpdf: the C ABI declared in include/lpdf.h (mesh building, context and
// device memory management, argument checking, launches).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include "lpdf_internal.h"

using namespace lpdf;


namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(expr)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess) return fail(LPDF_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t n)
{
    return cudaMalloc((void**)p, sizeof(T) * (n ? n : 1));
}

bool is_f32(double v) { return (double)(float)v == v; }

// the box x0, x1, y0, y1 around the discs (x - r .. x + r, y - r .. y + r), each bound rounded
// outward to FP32; empty (+inf, -inf, +inf, -inf) without discs
void source_box(int n, const float* sx, const float* sy, const float* sr, float box[4])
{
    double lo[2] = {HUGE_VAL, HUGE_VAL}, hi[2] = {-HUGE_VAL, -HUGE_VAL};
    for (int i = 0; i < n; ++i) {
        const double c[2] = {sx[i], sy[i]};
        for (int d = 0; d < 2; ++d) {
            lo[d] = std::min(lo[d], c[d] - (double)sr[i]);
            hi[d] = std::max(hi[d], c[d] + (double)sr[i]);
        }
    }
    for (int d = 0; d < 2; ++d) {
        float l = (float)lo[d], h = (float)hi[d];
        if ((double)l > lo[d]) l = std::nextafter(l, -HUGE_VALF);
        if ((double)h < hi[d]) h = std::nextafter(h, HUGE_VALF);
        box[2 * d] = l;
        box[2 * d + 1] = h;
    }
}

CompParams comp_params(uint64_t seed, int n_src, const float* sx, const float* sy, const float* sr, const int32_t* sa)
{
    CompParams c{};
    c.key0 = (uint32_t)seed;
    c.key1 = (uint32_t)(seed >> 32);
    c.n_src = n_src;
    for (int i = 0; i < n_src; ++i) {
        c.src_x[i] = sx[i];
        c.src_y[i] = sy[i];
        c.src_r[i] = sr[i];
        c.src_alpha[i] = sa[i];
    }
    source_box(n_src, sx, sy, sr, c.src_box);
    return c;
}

// drops the captured step graphs (the state, its order or the configuration changed)
void drop_graphs(lpdf_ctx* c)
{
    for (int k = 0; k < 2; ++k) {
        if (c->graph[k]) cudaGraphExecDestroy(c->graph[k]);
        c->graph[k] = nullptr;
        c->graph_fields[k] = nullptr;
        c->graph_state[k] = nullptr;
        c->graph_perm[k] = nullptr;
    }
}

cudaError_t alloc_pipe(PipeScratch& w, int64_t cap, size_t E, int ns)
{
    const size_t nrec = (size_t)((cap + 255) / 256) * 256;
    cudaError_t e = cudaSuccess;
    if ((e = dalloc(&w.perm, cap)) || (e = dalloc(&w.perm_new, cap)) || (e = dalloc(&w.rrank, cap)) ||
        (e = dalloc(&w.rec_key, nrec)) || (e = dalloc(&w.rec_cnt, nrec)) || (e = dalloc(&w.rec_off, nrec)) ||
        (e = dalloc(&w.nrec, nrec / 256)) || (e = dalloc(&w.kwork, 3 * (E + 1) + 1)) || (e = dalloc(&w.kstart, E + 1)) ||
        (e = dalloc(&w.krstart, E + 1)) || (e = dalloc(&w.klist, nrec)) || (e = dalloc(&w.klist2, nrec)) ||
        (e = dalloc(&w.scan_part, 2 * 4096)) || (e = dalloc(&w.efields, E * 3 * (size_t)nfields_padded(ns))))
        return e;
    return cudaSuccess;
}

void free_mesh_device(DevMesh& d)
{
    cudaFree(d.ex); cudaFree(d.ey); cudaFree(d.en); cudaFree(d.ev); cudaFree(d.em); cudaFree(d.master);
    cudaFree(d.ea); cudaFree(d.eb); cudaFree(d.ec); cudaFree(d.ew); cudaFree(d.ecomp); cudaFree(d.cframe);
    d = DevMesh();
}

}  // namespace

int lpdf::lpdf_set_error(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

StepParams lpdf::make_step_params(const lpdf_params& p, const lpdf_mesh* m, uint64_t step)
{
    StepParams s{};
    s.dt = (float)p.dt;
    s.sdt = (float)std::sqrt(p.dt);
    s.s2nu = (float)std::sqrt(2.0 * p.nu);
    s.nu2 = (float)(2.0 * p.nu);
    s.C3 = (float)p.C3;
    s.C4 = (float)p.C4;
    s.half_cphi = (float)(0.5 * p.Cphi);
    s.lid_u = (float)p.lid_u;
    s.key0 = (uint32_t)p.seed;
    s.key1 = (uint32_t)(p.seed >> 32);
    s.step_lo = (uint32_t)step;
    s.step_hi = (uint32_t)(step >> 32);
    s.react_k = p.react_k > 0.0 ? (float)p.react_k : 0.0f;
    s.react_a = p.react_a;
    s.react_b = p.react_b;
    s.react_p = p.react_p;
    s.n_src = p.n_sources;
    for (int i = 0; i < p.n_sources; ++i) {
        s.src_x[i] = p.src_x[i];
        s.src_y[i] = p.src_y[i];
        s.src_r[i] = p.src_r[i];
        s.src_alpha[i] = p.src_alpha[i];
    }
    source_box(p.n_sources, p.src_x, p.src_y, p.src_r, s.src_box);
    (void)m;
    s.moment_sums = p.moment_sums;
    return s;
}

namespace {

int check_params(const lpdf_params* p)
{
    if (!p) return fail(LPDF_ERR_ARG, "params is NULL");
    if (p->ns < 1 || p->ns > LPDF_MAX_SCALARS)
        return fail(LPDF_ERR_UNSUPPORTED, "ns = %d outside 1..%d", p->ns, LPDF_MAX_SCALARS);
    if (p->n_sources < 0 || p->n_sources > LPDF_MAX_SOURCES)
        return fail(LPDF_ERR_ARG, "n_sources = %d outside 0..%d", p->n_sources, LPDF_MAX_SOURCES);
    for (int i = 0; i < p->n_sources; ++i)
        if (p->src_alpha[i] < 0 || p->src_alpha[i] >= p->ns)
            return fail(LPDF_ERR_ARG, "source %d sets scalar %d, but ns = %d", i, p->src_alpha[i], p->ns);
    if (!(p->dt > 0.0) || !(p->nu >= 0.0)) return fail(LPDF_ERR_ARG, "need dt > 0 and nu >= 0");
    if (p->mixing < 0 || p->mixing > 1) return fail(LPDF_ERR_ARG, "mixing = %d (0 IEM, 1 IECM)", p->mixing);
    if (p->moment_sums < 0 || p->moment_sums > 1)
        return fail(LPDF_ERR_ARG, "moment_sums = %d (0 FP32 partial sums, 1 compensated)", p->moment_sums);
    if (p->react_k > 0.0 && (p->react_a < 0 || p->react_a >= p->ns || p->react_b < 0 || p->react_b >= p->ns ||
                             p->react_p < 0 || p->react_p >= p->ns))
        return fail(LPDF_ERR_ARG, "reaction scalars %d + %d -> %d outside 0..%d", p->react_a, p->react_b, p->react_p,
                    p->ns - 1);
    return LPDF_OK;
}

}  // namespace

int lpdf::mesh_fem(const lpdf_mesh* mesh, Fem** out)
{
    std::lock_guard<std::mutex> lock(mesh->fem_mutex);
    if (!mesh->fem) {
        Fem* F = nullptr;
        cudaError_t e = fem_build(mesh->node_xy.data(), mesh->d.n_nodes, mesh->tri.data(), mesh->d.n_tri,
                                  mesh->tag.data(), mesh->master, mesh->node_comp, mesh->period, &F);
        if (e != cudaSuccess) return fail(LPDF_ERR_CUDA, "gridpoint tables: %s", cudaGetErrorString(e));
        mesh->fem = F;
    }
    *out = mesh->fem;
    return LPDF_OK;
}

extern "C" {

void lpdf_params_default(lpdf_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->nu = 1.0 / 180.0;
    p->dt = 1e-3;
    p->C3 = 5.0;
    p->C4 = 0.25;
    p->Cphi = 2.0;
    p->C0 = 2.1;
    p->Comega1 = 0.5;
    p->Comega2 = 0.73;
    p->CL = 0.134;
    p->Ceta = 72.0;
    p->lid_u = 0.0;
    p->seed = 1;
    p->ns = 1;
    p->n_sources = 0;
}

const char* lpdf_last_error(void) { return g_err.c_str(); }
const char* lpdf_version(void) { return "lpdf 0.1 (sm_103a)"; }

}  // extern "C"

namespace {

// The mesh tables of n_comp independent components (n_comp = 1: an ordinary mesh). Component c
// owns nodes [node_off[c], node_off[c + 1]) and elements [tri_off[c], tri_off[c + 1]); its
// frame is its own bounding box and its periodic edges and nodes pair within it.
int build_mesh(const double* node_xy, int32_t n_nodes, const int32_t* tri, int32_t n_tri, const int32_t* edge_tag,
               int32_t n_comp, const int32_t* node_off, const int32_t* tri_off, double period_x, lpdf_mesh** out)
{
    if (!node_xy || !tri || !edge_tag || !out) return fail(LPDF_ERR_ARG, "mesh_load: NULL argument");
    if (n_nodes < 3 || n_tri < 1) return fail(LPDF_ERR_ARG, "mesh_load: n_nodes = %d, n_tri = %d", n_nodes, n_tri);
    if (n_comp < 1 || node_off[0] != 0 || tri_off[0] != 0 || node_off[n_comp] != n_nodes || tri_off[n_comp] != n_tri)
        return fail(LPDF_ERR_ARG, "mesh_load: component offsets do not cover the nodes and elements");
    for (int c = 0; c < n_comp; ++c)
        if (node_off[c + 1] - node_off[c] < 3 || tri_off[c + 1] <= tri_off[c])
            return fail(LPDF_ERR_ARG, "mesh_load: component %d is empty", c);
    *out = nullptr;
    const bool periodic = period_x > 0.0;
    std::vector<double> fr(4 * (size_t)n_comp);   // per component x0, x1, y0, y1
    std::vector<int32_t> ncomp(n_nodes), ecomp(n_tri);
    for (int c = 0; c < n_comp; ++c) {
        double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
        for (int i = node_off[c]; i < node_off[c + 1]; ++i) {
            const double x = node_xy[2 * i], y = node_xy[2 * i + 1];
            if (!is_f32(x) || !is_f32(y)) return fail(LPDF_ERR_ARG, "node %d coordinates are not FP32 values", i);
            x0 = std::min(x0, x); x1 = std::max(x1, x); y0 = std::min(y0, y); y1 = std::max(y1, y);
            ncomp[i] = c;
        }
        if (periodic && (float)(x1 - x0) != (float)period_x)
            return fail(LPDF_ERR_MESH, "component %d: period %.9g differs from the x extent %.9g", c, period_x, x1 - x0);
        fr[4 * c] = x0; fr[4 * c + 1] = x1; fr[4 * c + 2] = y0; fr[4 * c + 3] = y1;
        for (int e = tri_off[c]; e < tri_off[c + 1]; ++e) ecomp[e] = c;
    }
    double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
    for (int c = 0; c < n_comp; ++c) {
        x0 = std::min(x0, fr[4 * c]); x1 = std::max(x1, fr[4 * c + 1]);
        y0 = std::min(y0, fr[4 * c + 2]); y1 = std::max(y1, fr[4 * c + 3]);
    }
    std::vector<float> ex(4 * (size_t)n_tri), ey(4 * (size_t)n_tri), ea(4 * (size_t)n_tri), eb(4 * (size_t)n_tri);
    std::vector<double> ec(4 * (size_t)n_tri);
    std::vector<int32_t> en(4 * (size_t)n_tri, -1), ev(4 * (size_t)n_tri, 0), em(4 * (size_t)n_tri, 0);
    for (int e = 0; e < n_tri; ++e) {
        const int* t = tri + 3 * e;
        for (int k = 0; k < 3; ++k) {
            if (t[k] < 0 || t[k] >= n_nodes) return fail(LPDF_ERR_MESH, "element %d has node id %d", e, t[k]);
            if (ncomp[t[k]] != ecomp[e])
                return fail(LPDF_ERR_MESH, "element %d of component %d uses node %d of component %d", e, ecomp[e], t[k],
                            ncomp[t[k]]);
        }
        const double ax = node_xy[2 * t[0]], ay = node_xy[2 * t[0] + 1];
        const double bx = node_xy[2 * t[1]], by = node_xy[2 * t[1] + 1];
        const double cx = node_xy[2 * t[2]], cy = node_xy[2 * t[2] + 1];
        const double A = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
        if (!(A > 0.0)) return fail(LPDF_ERR_MESH, "element %d is not counter-clockwise (2A = %g)", e, A);
        ex[4 * e + 0] = (float)ax; ex[4 * e + 1] = (float)bx; ex[4 * e + 2] = (float)cx;
        ex[4 * e + 3] = (float)((ax + bx + cx) / 3.0);
        ey[4 * e + 0] = (float)ay; ey[4 * e + 1] = (float)by; ey[4 * e + 2] = (float)cy;
        ey[4 * e + 3] = (float)(1.0 / A);
        ea[4 * e + 0] = (float)ax;
        ea[4 * e + 1] = (float)ay;
        ea[4 * e + 2] = (float)((cy - ay) / A);
        ea[4 * e + 3] = (float)(-(cx - ax) / A);
        eb[4 * e + 0] = (float)(-(by - ay) / A);
        eb[4 * e + 1] = (float)((bx - ax) / A);
        eb[4 * e + 2] = ex[4 * e + 3];
        eb[4 * e + 3] = 0.0f;
        ec[4 * e + 0] = (cy - ay) / A;
        ec[4 * e + 1] = -(cx - ax) / A;
        ec[4 * e + 2] = -(by - ay) / A;
        ec[4 * e + 3] = (bx - ax) / A;
        for (int k = 0; k < 3; ++k) ev[4 * e + k] = t[k];
        ev[4 * e + 3] = 0;
        en[4 * e + 3] = 0;   // bit k: edge k is periodic
    }
    // interior adjacency by shared (ordered) node pairs
    std::unordered_map<uint64_t, int64_t> half;   // (a,b) -> e*3+k
    half.reserve(3 * (size_t)n_tri);
    for (int e = 0; e < n_tri; ++e)
        for (int k = 0; k < 3; ++k) {
            const uint32_t a = (uint32_t)tri[3 * e + k], b = (uint32_t)tri[3 * e + (k + 1) % 3];
            const uint64_t key = ((uint64_t)a << 32) | b;
            if (!half.emplace(key, (int64_t)e * 3 + k).second)
                return fail(LPDF_ERR_MESH, "directed edge %u->%u appears twice", a, b);
        }
    std::vector<std::pair<double, int64_t>> left_edges, right_edges;   // keyed by min y
    bool edge_walls = false;
    for (int e = 0; e < n_tri; ++e)
        for (int k = 0; k < 3; ++k) {
            const uint32_t a = (uint32_t)tri[3 * e + k], b = (uint32_t)tri[3 * e + (k + 1) % 3];
            const int tag = edge_tag[3 * e + k];
            if (tag < 0 || tag > 3) return fail(LPDF_ERR_MESH, "element %d edge %d: bad tag %d", e, k, tag);
            auto it = half.find(((uint64_t)b << 32) | a);
            if (it != half.end()) {
                if (tag != LPDF_EDGE_INTERIOR)
                    return fail(LPDF_ERR_MESH, "element %d edge %d is shared but tagged %d", e, k, tag);
                en[4 * e + k] = (int32_t)(it->second / 3);
                continue;
            }
            if (tag == LPDF_EDGE_INTERIOR)
                return fail(LPDF_ERR_MESH, "element %d edge %d is a boundary edge tagged interior", e, k);
            if (tag == LPDF_EDGE_WALL || tag == LPDF_EDGE_MOVING_WALL) {
                if (tag == LPDF_EDGE_MOVING_WALL) en[4 * e + 3] |= (8 << k);   // bit 3 + k: moving wall
                // a wall edge off the sides of its component's frame makes the mesh "edge walls"
                const int c = ecomp[e];
                const double ax = node_xy[2 * a], ay = node_xy[2 * a + 1], bx = node_xy[2 * b], by = node_xy[2 * b + 1];
                const bool on_side = (ax == bx && (ax == fr[4 * c] || ax == fr[4 * c + 1])) ||
                                     (ay == by && (ay == fr[4 * c + 2] || ay == fr[4 * c + 3]));
                if (!on_side) edge_walls = true;
            }
            if (tag == LPDF_EDGE_PERIODIC) {
                if (!periodic) return fail(LPDF_ERR_MESH, "periodic edge without period_x");
                const double ax = node_xy[2 * a], bx = node_xy[2 * b];
                const double ymin = std::min(node_xy[2 * a + 1], node_xy[2 * b + 1]);
                const double cx0 = fr[4 * ecomp[e]], cx1 = fr[4 * ecomp[e] + 1];
                if (ax == cx0 && bx == cx0) left_edges.push_back({ymin, (int64_t)e * 3 + k});
                else if (ax == cx1 && bx == cx1) right_edges.push_back({ymin, (int64_t)e * 3 + k});
                else return fail(LPDF_ERR_MESH, "periodic edge of element %d is not on x0 or x1", e);
            }
        }
    if (periodic) {
        if (left_edges.size() != right_edges.size())
            return fail(LPDF_ERR_MESH, "%zu left vs %zu right periodic edges", left_edges.size(), right_edges.size());
        // partners are found within the component, by the y values of their ends
        std::map<std::tuple<int, double, double>, int64_t> rmap;
        for (auto& r : right_edges) {
            const int e = (int)(r.second / 3), k = (int)(r.second % 3);
            const int a = tri[3 * e + k], b = tri[3 * e + (k + 1) % 3];
            rmap[{ecomp[e], node_xy[2 * a + 1], node_xy[2 * b + 1]}] = r.second;
        }
        for (auto& l : left_edges) {
            const int e = (int)(l.second / 3), k = (int)(l.second % 3);
            const int a = tri[3 * e + k], b = tri[3 * e + (k + 1) % 3];
            // the partner runs the other way: its (a, b) y values are this edge's (b, a)
            auto it = rmap.find({ecomp[e], node_xy[2 * b + 1], node_xy[2 * a + 1]});
            if (it == rmap.end()) return fail(LPDF_ERR_MESH, "left periodic edge of element %d has no partner", e);
            const int f = (int)(it->second / 3), kk = (int)(it->second % 3);
            en[4 * e + k] = f;
            en[4 * f + kk] = e;
            en[4 * e + 3] |= (1 << k);
            en[4 * f + 3] |= (1 << kk);
        }
    }
    // periodic node pairing: node on x1 -> node on x0 of its component with the same y
    std::vector<int32_t> master(n_nodes);
    for (int i = 0; i < n_nodes; ++i) master[i] = i;
    if (periodic) {
        std::map<std::pair<int, double>, int> left_nodes;
        for (int i = 0; i < n_nodes; ++i)
            if (node_xy[2 * i] == fr[4 * ncomp[i]]) left_nodes[{ncomp[i], node_xy[2 * i + 1]}] = i;
        for (int i = 0; i < n_nodes; ++i)
            if (node_xy[2 * i] == fr[4 * ncomp[i] + 1]) {
                auto it = left_nodes.find({ncomp[i], node_xy[2 * i + 1]});
                if (it == left_nodes.end()) return fail(LPDF_ERR_MESH, "node %d on x1 has no partner on x0", i);
                master[i] = it->second;
            }
    }
    for (int e = 0; e < n_tri; ++e)
        for (int k = 0; k < 3; ++k) em[4 * e + k] = master[tri[3 * e + k]];

    lpdf_mesh* m = new lpdf_mesh();
    cudaGetDevice(&m->device);
    DevMesh& d = m->d;
    d.n_nodes = n_nodes;
    d.n_tri = n_tri;
    d.x0 = (float)x0; d.x1 = (float)x1; d.y0 = (float)y0; d.y1 = (float)y1;
    d.periodic = periodic ? 1 : 0;
    d.n_comp = n_comp;
    d.edge_walls = edge_walls ? 1 : 0;
    std::vector<float> cf(4 * (size_t)n_comp);
    for (size_t q = 0; q < cf.size(); ++q) cf[q] = (float)fr[q];
    d.period = periodic ? (float)period_x : 0.0f;
    m->box[0] = x0; m->box[1] = x1; m->box[2] = y0; m->box[3] = y1;
    std::vector<float> ew(16 * (size_t)n_tri, 0.0f);
    for (int e = 0; e < n_tri; ++e) {
        for (int q = 0; q < 4; ++q) {
            ew[16 * (size_t)e + q] = ea[4 * (size_t)e + q];
            ew[16 * (size_t)e + 4 + q] = eb[4 * (size_t)e + q];
            std::memcpy(&ew[16 * (size_t)e + 8 + q], &en[4 * (size_t)e + q], sizeof(float));
        }
    }
    cudaError_t ce = cudaSuccess;
    if ((ce = dalloc(&d.ex, n_tri)) != cudaSuccess || (ce = dalloc(&d.ey, n_tri)) != cudaSuccess ||
        (ce = dalloc(&d.en, n_tri)) != cudaSuccess || (ce = dalloc(&d.ev, n_tri)) != cudaSuccess ||
        (ce = dalloc(&d.em, n_tri)) != cudaSuccess || (ce = dalloc(&d.master, n_nodes)) != cudaSuccess ||
        (ce = dalloc(&d.ea, n_tri)) != cudaSuccess || (ce = dalloc(&d.eb, n_tri)) != cudaSuccess ||
        (ce = dalloc(&d.ec, n_tri)) != cudaSuccess || (ce = dalloc(&d.ew, 4 * (size_t)n_tri)) != cudaSuccess ||
        (ce = cudaMemcpy(d.ec, ec.data(), sizeof(double) * ec.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (ce = cudaMemcpy(d.ew, ew.data(), sizeof(float) * ew.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (ce = cudaMemcpy(d.ea, ea.data(), sizeof(float) * ea.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (ce = cudaMemcpy(d.eb, eb.data(), sizeof(float) * eb.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (ce = cudaMemcpy(d.ex, ex.data(), sizeof(float) * ex.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (ce = cudaMemcpy(d.ey, ey.data(), sizeof(float) * ey.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (ce = cudaMemcpy(d.en, en.data(), sizeof(int32_t) * en.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (ce = cudaMemcpy(d.ev, ev.data(), sizeof(int32_t) * ev.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (ce = cudaMemcpy(d.em, em.data(), sizeof(int32_t) * em.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (ce = cudaMemcpy(d.master, master.data(), sizeof(int32_t) * master.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (n_comp > 1 && ((ce = dalloc(&d.ecomp, n_tri)) != cudaSuccess || (ce = dalloc(&d.cframe, n_comp)) != cudaSuccess ||
                        (ce = cudaMemcpy(d.ecomp, ecomp.data(), sizeof(int32_t) * n_tri, cudaMemcpyHostToDevice)) != cudaSuccess ||
                        (ce = cudaMemcpy(d.cframe, cf.data(), sizeof(float) * cf.size(), cudaMemcpyHostToDevice)) != cudaSuccess))) {
        free_mesh_device(d);
        delete m;
        return fail(LPDF_ERR_CUDA, "mesh upload: %s", cudaGetErrorString(ce));
    }
    m->nbr.resize(3 * (size_t)n_tri);
    for (int e = 0; e < n_tri; ++e)
        for (int k = 0; k < 3; ++k) m->nbr[3 * e + k] = en[4 * e + k];
    m->master = std::move(master);
    m->node_xy.assign(node_xy, node_xy + 2 * (size_t)n_nodes);
    m->tri.assign(tri, tri + 3 * (size_t)n_tri);
    m->tag.assign(edge_tag, edge_tag + 3 * (size_t)n_tri);
    m->node_comp = std::move(ncomp);
    m->elem_comp = std::move(ecomp);
    m->period = periodic ? period_x : 0.0;
    *out = m;
    return LPDF_OK;
}

}  // namespace

extern "C" {

int lpdf_mesh_load(const double* node_xy, int32_t n_nodes, const int32_t* tri, int32_t n_tri,
                   const int32_t* edge_tag, double period_x, lpdf_mesh** out)
{
    const int32_t node_off[2] = {0, n_nodes}, tri_off[2] = {0, n_tri};
    return build_mesh(node_xy, n_nodes, tri, n_tri, edge_tag, 1, node_off, tri_off, period_x, out);
}

int lpdf_mesh_load_multi(const double* node_xy, int32_t n_nodes, const int32_t* tri, int32_t n_tri,
                         const int32_t* edge_tag, int32_t n_comp, const int32_t* node_off, const int32_t* tri_off,
                         double period_x, lpdf_mesh** out)
{
    if (n_comp < 1 || !node_off || !tri_off) return fail(LPDF_ERR_ARG, "mesh_load_multi: n_comp = %d", n_comp);
    return build_mesh(node_xy, n_nodes, tri, n_tri, edge_tag, n_comp, node_off, tri_off, period_x, out);
}

void lpdf_mesh_free(lpdf_mesh* mesh)
{
    if (!mesh) return;
    free_mesh_device(mesh->d);
    fem_free(mesh->fem);
    delete mesh;
}

int lpdf_mesh_info(const lpdf_mesh* m, int32_t* n_nodes, int32_t* n_tri, double* box)
{
    if (!m) return fail(LPDF_ERR_ARG, "mesh is NULL");
    if (n_nodes) *n_nodes = m->d.n_nodes;
    if (n_tri) *n_tri = m->d.n_tri;
    if (box) std::memcpy(box, m->box, sizeof m->box);
    return LPDF_OK;
}

int lpdf_mesh_neighbors(const lpdf_mesh* m, int32_t* out)
{
    if (!m || !out) return fail(LPDF_ERR_ARG, "mesh_neighbors: NULL argument");
    std::memcpy(out, m->nbr.data(), sizeof(int32_t) * m->nbr.size());
    return LPDF_OK;
}

int lpdf_mesh_masters(const lpdf_mesh* m, int32_t* out)
{
    if (!m || !out) return fail(LPDF_ERR_ARG, "mesh_masters: NULL argument");
    std::memcpy(out, m->master.data(), sizeof(int32_t) * m->master.size());
    return LPDF_OK;
}

int lpdf_ctx_create(const lpdf_mesh* mesh, const lpdf_params* params, int64_t capacity, lpdf_ctx** out)
{
    if (!mesh || !out) return fail(LPDF_ERR_ARG, "ctx_create: NULL argument");
    *out = nullptr;
    int rc = check_params(params);
    if (rc) return rc;
    if (capacity < 1) return fail(LPDF_ERR_ARG, "capacity = %lld", (long long)capacity);
    const int64_t cap = (capacity + 127) / 128 * 128;
    lpdf_ctx* c = new lpdf_ctx();
    c->mesh = mesh;
    c->params = *params;
    c->ns = params->ns;
    DevState& s = c->s;
    s.n = 0;
    s.cap = cap;
    const int nq = nquant(c->ns);
    cudaError_t ce = cudaSuccess;
    DevState& s2 = c->s2;
    s2.n = 0;
    s2.cap = cap;
    const size_t E = (size_t)mesh->d.n_tri;
    if ((ce = dalloc(&s.x, cap)) || (ce = dalloc(&s.y, cap)) || (ce = dalloc(&s.u, cap)) || (ce = dalloc(&s.v, cap)) ||
        (ce = dalloc(&s.w, cap)) || (ce = dalloc(&s.om, cap)) || (ce = dalloc(&s.psi, cap * c->ns)) ||
        (ce = dalloc(&s.elem, cap)) || (ce = dalloc(&s.pid, cap)) ||
        (ce = dalloc(&s2.x, cap)) || (ce = dalloc(&s2.y, cap)) || (ce = dalloc(&s2.u, cap)) || (ce = dalloc(&s2.v, cap)) ||
        (ce = dalloc(&s2.w, cap)) || (ce = dalloc(&s2.om, cap)) || (ce = dalloc(&s2.psi, cap * c->ns)) ||
        (ce = dalloc(&s2.elem, cap)) || (ce = dalloc(&s2.pid, cap)) ||
        (ce = dalloc(&c->sort.cnt, E + 1)) || (ce = dalloc(&c->sort.cursor, E + 1)) ||
        (ce = dalloc(&c->sort.start, E + 2)) || (ce = dalloc(&c->sort.perm, cap)) ||
        (ce = dalloc(&c->node_acc, (size_t)mesh->d.n_nodes * nq)) || (ce = dalloc(&c->status, 4)) ||
        (ce = alloc_pipe(c->pipe, cap, E, c->ns)) || (ce = dalloc(&c->comp, mesh->d.n_comp)) ||
        (ce = dalloc(&c->init_pbase, mesh->d.n_comp + 1)) || (ce = dalloc(&c->init_ppe, mesh->d.n_comp)) ||
        (ce = dalloc(&c->init_toff, mesh->d.n_comp + 1)) || (ce = dalloc(&c->init_key, 2 * mesh->d.n_comp)) ||
        (ce = dalloc(&c->step_dev, 1)) ||
        (params->mixing == 1 && (ce = dalloc(&c->flux_acc, (size_t)mesh->d.n_nodes * 3 * c->ns)))) {
        lpdf_ctx_free(c);
        return fail(LPDF_ERR_CUDA, "ctx_create: %s", cudaGetErrorString(ce));
    }
    cudaMemset(c->node_acc, 0, sizeof(unsigned long long) * (size_t)mesh->d.n_nodes * nq);
    c->comp_host.assign(mesh->d.n_comp, comp_params(params->seed, params->n_sources, params->src_x, params->src_y,
                                                    params->src_r, params->src_alpha));
    if ((ce = cudaMemcpy(c->comp, c->comp_host.data(), sizeof(CompParams) * c->comp_host.size(),
                         cudaMemcpyHostToDevice)) != cudaSuccess) {
        lpdf_ctx_free(c);
        return fail(LPDF_ERR_CUDA, "ctx_create: %s", cudaGetErrorString(ce));
    }
    const unsigned long long st0[4] = {0ull, 0ull, ~0ull, 0ull};
    if ((ce = cudaMemcpy(c->status, st0, sizeof st0, cudaMemcpyHostToDevice)) != cudaSuccess) {
        lpdf_ctx_free(c);
        return fail(LPDF_ERR_CUDA, "ctx_create: %s", cudaGetErrorString(ce));
    }
    *out = c;
    return LPDF_OK;
}

void lpdf_ctx_free(lpdf_ctx* c)
{
    if (!c) return;
    for (DevState* s : {&c->s, &c->s2}) {
        cudaFree(s->x); cudaFree(s->y); cudaFree(s->u); cudaFree(s->v); cudaFree(s->w); cudaFree(s->om);
        cudaFree(s->psi); cudaFree(s->elem); cudaFree(s->pid);
    }
    cudaFree(c->sort.cnt); cudaFree(c->sort.cursor); cudaFree(c->sort.start); cudaFree(c->sort.perm);
    for (auto& q : c->ev_pending)
        for (cudaEvent_t e : q) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
    PipeScratch& w = c->pipe;
    void* pp[] = {w.perm, w.perm_new, w.rrank, w.rec_key, w.rec_cnt, w.rec_off, w.nrec, w.kwork, w.kstart,
                  w.krstart, w.klist, w.klist2, w.scan_part, w.efields};
    for (void* q : pp) cudaFree(q);
    cudaFree(c->node_acc); cudaFree(c->status);
    cudaFree(c->comp); cudaFree(c->init_pbase); cudaFree(c->init_ppe); cudaFree(c->init_toff); cudaFree(c->init_key);
    cudaFree(c->step_dev);
    cudaFree(c->flux_acc);
    drop_graphs(c);
    if (c->graph_stream) cudaStreamDestroy(c->graph_stream);
    delete c;
}

int lpdf_ctx_set_params(lpdf_ctx* c, const lpdf_params* p)
{
    if (!c) return fail(LPDF_ERR_ARG, "ctx is NULL");
    int rc = check_params(p);
    if (rc) return rc;
    if (p->ns != c->ns) return fail(LPDF_ERR_ARG, "ns cannot change (%d -> %d)", c->ns, p->ns);
    if (p->mixing == 1 && !c->flux_acc)
        return fail(LPDF_ERR_ARG, "IECM needs a context created with mixing = 1 (its flux sums)");
    c->params = *p;
    drop_graphs(c);
    if (!c->comp_set) {
        c->comp_host.assign(c->mesh->d.n_comp, comp_params(p->seed, p->n_sources, p->src_x, p->src_y, p->src_r,
                                                           p->src_alpha));
        CUDA_TRY(cudaMemcpy(c->comp, c->comp_host.data(), sizeof(CompParams) * c->comp_host.size(),
                            cudaMemcpyHostToDevice));
    }
    return LPDF_OK;
}

int lpdf_ctx_set_components(lpdf_ctx* c, const lpdf_component* comps, int32_t n)
{
    if (!c || !comps) return fail(LPDF_ERR_ARG, "ctx_set_components: NULL argument");
    if (n != c->mesh->d.n_comp)
        return fail(LPDF_ERR_ARG, "ctx_set_components: %d components for a mesh of %d", n, c->mesh->d.n_comp);
    for (int k = 0; k < n; ++k) {
        const lpdf_component& q = comps[k];
        if (q.n_sources < 0 || q.n_sources > LPDF_MAX_SOURCES)
            return fail(LPDF_ERR_ARG, "component %d: n_sources = %d", k, q.n_sources);
        for (int i = 0; i < q.n_sources; ++i)
            if (q.src_alpha[i] < 0 || q.src_alpha[i] >= c->ns)
                return fail(LPDF_ERR_ARG, "component %d: source %d sets scalar %d, but ns = %d", k, i, q.src_alpha[i],
                            c->ns);
    }
    for (int k = 0; k < n; ++k) {
        const lpdf_component& q = comps[k];
        c->comp_host[k] = comp_params(q.seed, q.n_sources, q.src_x, q.src_y, q.src_r, q.src_alpha);
    }
    CUDA_TRY(cudaMemcpy(c->comp, c->comp_host.data(), sizeof(CompParams) * n, cudaMemcpyHostToDevice));
    c->comp_set = true;
    drop_graphs(c);
    return LPDF_OK;
}

int64_t lpdf_ctx_size(const lpdf_ctx* c) { return c ? c->s.n : -1; }

static int init_with(lpdf_ctx* c, const std::vector<int>& ppe, const float* node_init, int32_t m_erlang,
                     cudaStream_t st)
{
    if (m_erlang < 1 || m_erlang > 6) return fail(LPDF_ERR_ARG, "m_erlang = %d outside 1..6", m_erlang);
    const DevMesh& d = c->mesh->d;
    const int nc = d.n_comp;
    std::vector<long long> pbase(nc + 1, 0);
    std::vector<int> toff(nc + 1, 0);
    std::vector<uint32_t> key(2 * nc);
    // element ranges of the components, from the element -> component map the mesh keeps on the host
    int e = 0;
    for (int k = 0; k < nc; ++k) {
        toff[k] = e;
        while (e < d.n_tri && (nc == 1 || c->mesh->elem_comp[e] == k)) ++e;
        if (ppe[k] < 1) return fail(LPDF_ERR_ARG, "particles per element of component %d = %d", k, ppe[k]);
        pbase[k + 1] = pbase[k] + (long long)(e - toff[k]) * ppe[k];
        key[2 * k] = c->comp_host[k].key0;
        key[2 * k + 1] = c->comp_host[k].key1;
    }
    toff[nc] = e;
    const int64_t P = pbase[nc];
    if (P > c->s.cap) return fail(LPDF_ERR_ARG, "%lld particles exceed capacity %lld", (long long)P, (long long)c->s.cap);
    for (int k = 0; k < nc; ++k)
        if (pbase[k + 1] - pbase[k] > (long long)UINT32_MAX) return fail(LPDF_ERR_ARG, "particle ids are 32-bit");
    CUDA_TRY(cudaMemcpy(c->init_pbase, pbase.data(), sizeof(long long) * pbase.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c->init_ppe, ppe.data(), sizeof(int) * nc, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c->init_toff, toff.data(), sizeof(int) * toff.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c->init_key, key.data(), sizeof(uint32_t) * key.size(), cudaMemcpyHostToDevice));
    c->s.n = P;
    drop_graphs(c);
    const InitLayout L{c->init_pbase, c->init_ppe, c->init_toff, c->init_key, nc};
    CUDA_TRY(launch_particles_init(d, c->s, c->ns, L, P, node_init, m_erlang, c->status, st));
    // generated element by element: the buffer is already in element order
    CUDA_TRY(launch_iota(c->pipe.perm, P, st));
    return LPDF_OK;
}

int lpdf_particles_init(lpdf_ctx* c, int32_t n_per_elem, const float* node_init, int32_t m_erlang, void* stream)
{
    if (!c || !node_init) return fail(LPDF_ERR_ARG, "particles_init: NULL argument");
    if (n_per_elem < 1) return fail(LPDF_ERR_ARG, "n_per_elem = %d", n_per_elem);
    return init_with(c, std::vector<int>(c->mesh->d.n_comp, n_per_elem), node_init, m_erlang, (cudaStream_t)stream);
}

int lpdf_particles_init_multi(lpdf_ctx* c, const int32_t* n_per_elem, const float* node_init, int32_t m_erlang,
                              void* stream)
{
    if (!c || !n_per_elem || !node_init) return fail(LPDF_ERR_ARG, "particles_init_multi: NULL argument");
    return init_with(c, std::vector<int>(n_per_elem, n_per_elem + c->mesh->d.n_comp), node_init, m_erlang,
                     (cudaStream_t)stream);
}

static int copy_state(lpdf_ctx* c, int64_t n, bool in, float* x, float* y, float* u, float* v, float* w, float* om,
                      float* psi, int32_t* elem, uint32_t* pid, int on_device, cudaStream_t st)
{
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : (in ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
    DevState& s = c->s;
    struct Item { void* dev; void* usr; size_t bytes; };
    const size_t fb = sizeof(float) * (size_t)n;
    Item items[] = {{s.x, x, fb}, {s.y, y, fb}, {s.u, u, fb}, {s.v, v, fb}, {s.w, w, fb}, {s.om, om, fb},
                    {s.elem, elem, sizeof(int32_t) * (size_t)n}, {s.pid, pid, sizeof(uint32_t) * (size_t)n}};
    if (n == 0) return LPDF_OK;
    for (auto& it : items) {
        if (!it.usr) continue;
        CUDA_TRY(in ? cudaMemcpyAsync(it.dev, it.usr, it.bytes, k, st) : cudaMemcpyAsync(it.usr, it.dev, it.bytes, k, st));
    }
    if (psi)
        for (int a = 0; a < c->ns; ++a) {
            float* dev = s.psi + (size_t)a * s.cap;
            float* usr = psi + (size_t)a * n;
            CUDA_TRY(in ? cudaMemcpyAsync(dev, usr, fb, k, st) : cudaMemcpyAsync(usr, dev, fb, k, st));
        }
    return LPDF_OK;
}

int lpdf_set_state(lpdf_ctx* c, int64_t n, const float* x, const float* y, const float* u, const float* v,
                   const float* w, const float* om, const float* psi, const int32_t* elem, const uint32_t* pid,
                   int on_device, void* stream)
{
    if (c) drop_graphs(c);
    if (!c) return fail(LPDF_ERR_ARG, "ctx is NULL");
    if (n < 0 || n > c->s.cap) return fail(LPDF_ERR_ARG, "n = %lld outside 0..%lld", (long long)n, (long long)c->s.cap);
    if (n > 0 && (!x || !y || !u || !v || !w || !om || !psi || !elem || !pid))
        return fail(LPDF_ERR_ARG, "set_state needs every array");
    c->s.n = n;
    const int rc = copy_state(c, n, true, (float*)x, (float*)y, (float*)u, (float*)v, (float*)w, (float*)om,
                              (float*)psi, (int32_t*)elem, (uint32_t*)pid, on_device, (cudaStream_t)stream);
    if (rc) return rc;
    // any order is valid input; the first step brings the ensemble into element order
    CUDA_TRY(launch_iota(c->pipe.perm, n, (cudaStream_t)stream));
    return LPDF_OK;
}

int lpdf_get_state(const lpdf_ctx* c, float* x, float* y, float* u, float* v, float* w, float* om, float* psi,
                   int32_t* elem, uint32_t* pid, int on_device, void* stream)
{
    if (!c) return fail(LPDF_ERR_ARG, "ctx is NULL");
    return copy_state(const_cast<lpdf_ctx*>(c), c->s.n, false, x, y, u, v, w, om, psi, elem, pid, on_device,
                      (cudaStream_t)stream);
}

int lpdf_sort(lpdf_ctx* c, void* stream)
{
    if (c) drop_graphs(c);
    if (!c) return fail(LPDF_ERR_ARG, "sort: NULL argument");
    c->s2.n = c->s.n;
    CUDA_TRY(launch_sort(c->mesh->d, c->s, c->ns, c->s2, c->sort, c->status, (cudaStream_t)stream));
    std::swap(c->s, c->s2);
    CUDA_TRY(launch_iota(c->pipe.perm, c->s.n, (cudaStream_t)stream));
    return LPDF_OK;
}

int lpdf_pdf_step(lpdf_ctx* c, const float* node_fields, uint64_t step, void* stream)
{
    if (!c || !node_fields) return fail(LPDF_ERR_ARG, "pdf_step: NULL argument");
    const cudaStream_t st = (cudaStream_t)stream;
    ++c->nsteps;
    const int nq = nquant(c->ns);
    CUDA_TRY(cudaMemsetAsync(c->node_acc, 0, sizeof(unsigned long long) * (size_t)c->mesh->d.n_nodes * nq, st));
    StepParams p = make_step_params(c->params, c->mesh, step);
    p.comp = c->mesh->d.n_comp > 1 ? c->comp : nullptr;
    p.beta = c->params.mixing == 1 ? c->iecm_beta : nullptr;
    if (c->flux_acc)
        CUDA_TRY(cudaMemsetAsync(c->flux_acc, 0, sizeof(unsigned long long) * (size_t)c->mesh->d.n_nodes * 3 * c->ns, st));
    c->s2.n = c->s.n;
    std::array<cudaEvent_t, 4> ev{};
    if (c->timing) {
        for (auto& e : ev) {
            if (!c->ev_free.empty()) {
                e = c->ev_free.back();
                c->ev_free.pop_back();
            } else {
                CUDA_TRY(cudaEventCreate(&e));
            }
        }
        c->ev_pending.push_back(ev);
    }
    CUDA_TRY(launch_pdf_step_pipeline(c->mesh->d, c->s, c->s2, c->ns, node_fields, p, c->pipe, c->node_acc,
                                      c->status, st, c->timing ? ev.data() : nullptr, c->tune, c->flux_acc));
    // the new state is in the second buffer, listed in element order by perm_new
    std::swap(c->s, c->s2);
    std::swap(c->pipe.perm, c->pipe.perm_new);
    return LPDF_OK;
}

static int capture_steps(lpdf_ctx* c, const float* fields, int slot)
{
    if (c->graph[slot]) cudaGraphExecDestroy(c->graph[slot]);
    c->graph[slot] = nullptr;
    if (!c->graph_stream) CUDA_TRY(cudaStreamCreateWithFlags(&c->graph_stream, cudaStreamNonBlocking));
    const cudaStream_t cs = c->graph_stream;
    (void)sm_count();   // device queries stay outside the capture
    CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const int nq = nquant(c->ns);
    DevState a = c->s, b = c->s2;
    PipeScratch w = c->pipe;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMemsetAsync(c->node_acc, 0, sizeof(unsigned long long) * (size_t)c->mesh->d.n_nodes * nq, cs);
        if (e == cudaSuccess && c->flux_acc)
            e = cudaMemsetAsync(c->flux_acc, 0, sizeof(unsigned long long) * (size_t)c->mesh->d.n_nodes * 3 * c->ns, cs);
        StepParams p = make_step_params(c->params, c->mesh, 0);
        p.comp = c->mesh->d.n_comp > 1 ? c->comp : nullptr;
        p.beta = c->params.mixing == 1 ? c->iecm_beta : nullptr;
        p.step_dev = c->step_dev;
        p.step_add = (unsigned)k;
        b.n = a.n;
        if (e == cudaSuccess)
            e = launch_pdf_step_pipeline(c->mesh->d, a, b, c->ns, fields, p, w, c->node_acc, c->status, cs, nullptr,
                                         c->tune, c->flux_acc);
        std::swap(a, b);
        std::swap(w.perm, w.perm_new);
    }
    if (e == cudaSuccess) e = launch_step_counter(c->step_dev, 0ull, 2ull, cs);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph[slot], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->graph[slot] = nullptr;
        return fail(LPDF_ERR_CUDA, "pdf_steps: graph capture: %s", cudaGetErrorString(e));
    }
    c->graph_fields[slot] = fields;
    c->graph_state[slot] = c->s.x;
    c->graph_perm[slot] = c->pipe.perm;
    return LPDF_OK;
}

int lpdf_pdf_steps(lpdf_ctx* c, const float* node_fields, uint64_t step0, int32_t nsteps, void* stream)
{
    if (!c || !node_fields) return fail(LPDF_ERR_ARG, "pdf_steps: NULL argument");
    if (nsteps < 0) return fail(LPDF_ERR_ARG, "pdf_steps: nsteps = %d", nsteps);
    const cudaStream_t st = (cudaStream_t)stream;
    const int pairs = nsteps / 2;
    if (pairs > 0 && c->s.n > 0) {
        int slot = -1;
        for (int k = 0; k < 2; ++k)
            if (c->graph[k] && c->graph_fields[k] == node_fields && c->graph_state[k] == c->s.x &&
                c->graph_perm[k] == c->pipe.perm)
                slot = k;
        if (slot < 0) {
            slot = c->graph_next;
            c->graph_next ^= 1;
            if (const int rc = capture_steps(c, node_fields, slot)) return rc;
        }
        CUDA_TRY(launch_step_counter(c->step_dev, step0, 0ull, st));
        for (int k = 0; k < pairs; ++k) CUDA_TRY(cudaGraphLaunch(c->graph[slot], st));
        c->nsteps += 2 * pairs;
    } else if (pairs > 0) {
        for (int k = 0; k < 2 * pairs; ++k)
            if (const int rc = lpdf_pdf_step(c, node_fields, step0 + k, stream)) return rc;
    }
    if (nsteps % 2) return lpdf_pdf_step(c, node_fields, step0 + 2 * (uint64_t)pairs, stream);
    return LPDF_OK;
}

int lpdf_ctx_set_tune(lpdf_ctx* c, int32_t adv, int32_t mom)
{
    if (!c) return fail(LPDF_ERR_ARG, "ctx is NULL");
    if (adv < 0 || adv >= kAdvVariants || mom < 0 || mom >= kMomVariants)
        return fail(LPDF_ERR_ARG, "set_tune: adv = %d (0..%d), mom = %d (0..%d)", adv, kAdvVariants - 1, mom,
                    kMomVariants - 1);
    c->tune.adv = adv;
    c->tune.mom = mom;
    drop_graphs(c);
    return LPDF_OK;
}

int lpdf_ctx_autotune(lpdf_ctx* c, const float* node_fields, uint64_t step0, int32_t steps_per_trial, int32_t rounds,
                      int32_t* choice, double* trial_ms, int32_t* steps_used, void* stream)
{
    if (!c || !node_fields) return fail(LPDF_ERR_ARG, "autotune: NULL argument");
    if (steps_per_trial < 1 || rounds < 1)
        return fail(LPDF_ERR_ARG, "autotune: steps_per_trial = %d, rounds = %d", steps_per_trial, rounds);
    const cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    uint64_t step = step0;
    int rc = LPDF_OK;
    auto trial = [&](int adv, int mom, double& ms) -> int {
        c->tune.adv = adv;
        c->tune.mom = mom;
        if (int r = lpdf_pdf_step(c, node_fields, step++, stream)) return r;   // warm-up of this variant
        if (cudaEventRecord(e0, st) != cudaSuccess) return fail(LPDF_ERR_CUDA, "autotune: event record");
        for (int k = 0; k < steps_per_trial; ++k)
            if (int r = lpdf_pdf_step(c, node_fields, step++, stream)) return r;
        float t = 0.0f;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
            return fail(LPDF_ERR_CUDA, "autotune: event timing");
        ms = t / steps_per_trial;
        return LPDF_OK;
    };
    const bool timing = c->timing;
    c->timing = false;
    StepTune best = c->tune;
    // every variant once per round, the rounds interleaved and run in alternating order (a variant
    // is not always timed right after the same one); a variant's time is its fastest trial
    double t_adv[kAdvVariants], t_mom[kMomVariants];
    for (double& t : t_adv) t = 1e300;
    for (double& t : t_mom) t = 1e300;
    for (int r = 0; r < rounds && rc == LPDF_OK; ++r)
        for (int j = 0; j < kAdvVariants && rc == LPDF_OK; ++j) {
            const int v = r % 2 ? kAdvVariants - 1 - j : j;
            double ms = 0.0;
            rc = trial(v, best.mom, ms);
            t_adv[v] = std::min(t_adv[v], ms);
        }
    for (int v = 0; v < kAdvVariants; ++v)
        if (t_adv[v] < t_adv[best.adv]) best.adv = v;
    for (int r = 0; r < rounds && rc == LPDF_OK; ++r)
        for (int j = 0; j < kMomVariants && rc == LPDF_OK; ++j) {
            const int v = r % 2 ? kMomVariants - 1 - j : j;
            double ms = 0.0;
            rc = trial(best.adv, v, ms);
            t_mom[v] = std::min(t_mom[v], ms);
        }
    for (int v = 0; v < kMomVariants; ++v)
        if (t_mom[v] < t_mom[best.mom]) best.mom = v;
    if (trial_ms) {
        for (int v = 0; v < kAdvVariants; ++v) trial_ms[v] = t_adv[v];
        for (int v = 0; v < kMomVariants; ++v) trial_ms[kAdvVariants + v] = t_mom[v];
    }
    c->timing = timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->tune = best;
    drop_graphs(c);
    if (choice) {
        choice[0] = best.adv;
        choice[1] = best.mom;
    }
    if (steps_used) *steps_used = (int32_t)(step - step0);
    return rc;
}

int lpdf_ctx_set_iecm(lpdf_ctx* c, const float* beta)
{
    if (!c) return fail(LPDF_ERR_ARG, "ctx is NULL");
    c->iecm_beta = beta;
    drop_graphs(c);
    return LPDF_OK;
}

int lpdf_grid_flux_statistics(lpdf_ctx* c, double* out, int raw, void* stream)
{
    if (!c || !out) return fail(LPDF_ERR_ARG, "grid_flux_statistics: NULL argument");
    if (!c->flux_acc) return fail(LPDF_ERR_ARG, "grid_flux_statistics: the context was created with mixing = 0");
    CUDA_TRY(launch_flux_statistics(c->mesh->d.master, c->mesh->d.n_nodes, c->ns, c->node_acc, c->flux_acc, out, raw,
                                    (cudaStream_t)stream));
    return LPDF_OK;
}

int lpdf_iecm_coefficients(const lpdf_mesh* mesh, int32_t ns, const double* stats, const double* flux, float* beta,
                           void* stream)
{
    if (!mesh || !stats || !flux || !beta) return fail(LPDF_ERR_ARG, "iecm_coefficients: NULL argument");
    if (ns < 1 || ns > LPDF_MAX_SCALARS) return fail(LPDF_ERR_UNSUPPORTED, "iecm_coefficients: ns = %d", ns);
    CUDA_TRY(launch_iecm_coefficients(mesh->d.n_nodes, ns, stats, flux, beta, (cudaStream_t)stream));
    return LPDF_OK;
}

int lpdf_ctx_set_timing(lpdf_ctx* c, int enable)
{
    if (!c) return fail(LPDF_ERR_ARG, "ctx is NULL");
    c->timing = enable != 0;
    return LPDF_OK;
}

int lpdf_ctx_timings(lpdf_ctx* c, double* out_ms, int64_t* steps)
{
    if (!c || !out_ms) return fail(LPDF_ERR_ARG, "ctx_timings: NULL argument");
    out_ms[0] = out_ms[1] = out_ms[2] = 0.0;
    for (auto& q : c->ev_pending) {
        CUDA_TRY(cudaEventSynchronize(q[3]));
        for (int k = 0; k < 3; ++k) {
            float ms = 0.0f;
            CUDA_TRY(cudaEventElapsedTime(&ms, q[k], q[k + 1]));
            out_ms[k] += ms;
        }
        for (cudaEvent_t e : q) c->ev_free.push_back(e);
    }
    if (steps) *steps = (int64_t)c->ev_pending.size();
    c->ev_pending.clear();
    return LPDF_OK;
}

int lpdf_status(lpdf_ctx* c, int64_t* out, void* stream)
{
    if (!c) return fail(LPDF_ERR_ARG, "ctx is NULL");
    const cudaStream_t st = (cudaStream_t)stream;
    unsigned long long h[4];
    CUDA_TRY(cudaMemcpyAsync(h, c->status, sizeof h, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    const unsigned long long st0[4] = {0ull, 0ull, ~0ull, 0ull};
    CUDA_TRY(cudaMemcpyAsync(c->status, st0, sizeof st0, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (out) {
        out[0] = (int64_t)h[0];
        out[1] = (int64_t)h[1];
        out[2] = h[2] == ~0ull ? -1 : (int64_t)h[2];
        out[3] = (int64_t)h[3];
    }
    if (h[0] & kErrLost) return fail(LPDF_ERR_LOST_PARTICLE, "%llu particle(s) lost, e.g. pid %llu", h[1], h[2]);
    if (h[0] & kErrNonFinite) return fail(LPDF_ERR_NONFINITE, "non-finite particle state");
    if (h[0] & kErrOverflow) return fail(LPDF_ERR_OVERFLOW, "fixed-point moment range exceeded");
    if (h[0] & kErrTimeout) return fail(LPDF_ERR_CUDA, "a bulk-copy wait in the step kernel timed out");
    if (h[0] & kErrCheck) return fail(LPDF_ERR_CUDA, "an internal consistency check of the step kernel failed");
    return LPDF_OK;
}

int lpdf_grid_statistics(lpdf_ctx* c, double* out, int raw, void* stream)
{
    if (!c || !out) return fail(LPDF_ERR_ARG, "grid_statistics: NULL argument");
    CUDA_TRY(launch_grid_statistics(c->mesh->d, c->ns, c->node_acc, out, raw ? 1 : 0, (cudaStream_t)stream));
    return LPDF_OK;
}


int lpdf_elliptic_relax_solve(const lpdf_mesh* mesh, const lpdf_params* params, const double* stats,
                              float* fields, double tol, int32_t maxit, int32_t* iters, void* stream)
{
    if (!mesh || !params || !stats || !fields) return fail(LPDF_ERR_ARG, "elliptic_relax_solve: NULL argument");
    if (params->ns < 1 || params->ns > LPDF_MAX_SCALARS)
        return fail(LPDF_ERR_UNSUPPORTED, "elliptic_relax_solve: ns = %d outside 1..%d", params->ns,
                    LPDF_MAX_SCALARS);
    if (params->gmodel < 0 || params->gmodel > 1 || params->pressure_solve < 0 || params->pressure_solve > 1)
        return fail(LPDF_ERR_ARG, "elliptic_relax_solve: gmodel = %d, pressure_solve = %d", params->gmodel,
                    params->pressure_solve);
    if (!(tol > 0.0) || maxit < 1)
        return fail(LPDF_ERR_ARG, "elliptic_relax_solve: tol = %g, maxit = %d", tol, maxit);
    Fem* F = nullptr;
    if (const int rc = mesh_fem(mesh, &F)) return rc;
    int it[2] = {0, 0};
    const cudaError_t e = node_fields_solve(*F, stats, *params, fields, tol, maxit, it, (cudaStream_t)stream);
    if (iters) {
        iters[0] = it[0];
        iters[1] = it[1];
    }
    if (e == cudaErrorNotReady)
        return fail(LPDF_ERR_CG_NOCONV, "elliptic_relax_solve: no convergence to %g in %d iterations (%d, %d)", tol,
                    maxit, it[0], it[1]);
    if (e != cudaSuccess) return fail(LPDF_ERR_CUDA, "elliptic_relax_solve: %s", cudaGetErrorString(e));
    return LPDF_OK;
}

int lpdf_tc_gemm_bf16(const void* A, const void* B, float* D, int32_t M, int32_t N, int32_t K, void* stream)
{
    if (!A || !B || !D) return fail(LPDF_ERR_ARG, "tc_gemm_bf16: NULL argument");
    if (M < 1 || N < 16 || N > 256 || N % 16 || K < 16 || K > 128 || K % 16)
        return fail(LPDF_ERR_ARG, "tc_gemm_bf16: shape M = %d, N = %d, K = %d", M, N, K);
    static unsigned* err_dev = nullptr;
    if (!err_dev) CUDA_TRY(cudaMalloc(&err_dev, sizeof(unsigned)));
    const cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaMemsetAsync(err_dev, 0, sizeof(unsigned), st));
    CUDA_TRY(launch_tc_gemm(A, B, D, M, N, K, err_dev, st));
    unsigned err = 0;
    CUDA_TRY(cudaMemcpyAsync(&err, err_dev, sizeof err, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (err) return fail(LPDF_ERR_CUDA, "tc_gemm_bf16: a bounded wait for the tensor-core MMAs gave up");
    return LPDF_OK;
}

}  // extern "C"
