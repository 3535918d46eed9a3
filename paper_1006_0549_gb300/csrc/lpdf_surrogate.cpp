// The learned surrogate of the elliptic-relaxation solve: the lpdf_mlp object (FP32 master
// parameters, BF16 packs for the tensor-core kernels, Adam moments, scratch), its training and
// gradient calls, and the surrogate solve with its fallback to the plain solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "lpdf_internal.h"

using namespace lpdf;

struct lpdf_mlp {
    float* P = nullptr;         // mlp::kParams, padded layout
    void* pack = nullptr;       // mlp::kPack BF16
    float* norm = nullptr;      // mlp::kNorm
    float* m = nullptr;         // Adam moments
    float* v = nullptr;
    float* grad = nullptr;      // mlp::kParams
    float* part = nullptr;      // per-tile partial gradients
    void* act = nullptr;        // 3 x max_batch x 128 BF16
    float* out = nullptr;       // max_batch x 16
    double* losses = nullptr;   // per training step
    int losses_cap = 0;
    unsigned* error = nullptr;
    int64_t max_batch = 0;
    int step = 0;
    // surrogate solve scratch, grown on demand
    float* s_feat = nullptr;
    float* s_out = nullptr;
    float* s_fields = nullptr;
    double* s_cmp = nullptr;
    int64_t s_feat_cap = 0, s_out_cap = 0, s_fields_cap = 0;
    // fallback policy
    int check_every = 50;
    double threshold = 0.02;
    int64_t calls = 0;
    bool net_ok = false;
    bool check_next = false;   // lpdf_mlp_request_check
};

namespace {

#define TRY(expr)                                                                               \
    do {                                                                                        \
        cudaError_t e_ = (expr);                                                                \
        if (e_ != cudaSuccess) return lpdf_set_error(LPDF_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

using namespace lpdf::mlp;

// compact ABI order -> padded device layout (and back)
void to_padded(const float* c, std::vector<float>& p)
{
    p.assign(kParams, 0.0f);
    size_t at = 0;
    for (int o = 0; o < kH; ++o)
        for (int k = 0; k < kIn; ++k) p[oW1 + o * kInP + k] = c[at++];
    for (int o = 0; o < kH; ++o) p[ob1 + o] = c[at++];
    for (int i = 0; i < kH * kH; ++i) p[oW2 + i] = c[at++];
    for (int o = 0; o < kH; ++o) p[ob2 + o] = c[at++];
    for (int i = 0; i < kH * kH; ++i) p[oW3 + i] = c[at++];
    for (int o = 0; o < kH; ++o) p[ob3 + o] = c[at++];
    for (int o = 0; o < kOut; ++o)
        for (int k = 0; k < kH; ++k) p[oW4 + o * kH + k] = c[at++];
    for (int o = 0; o < kOut; ++o) p[ob4 + o] = c[at++];
}

void to_compact(const std::vector<float>& p, float* c)
{
    size_t at = 0;
    for (int o = 0; o < kH; ++o)
        for (int k = 0; k < kIn; ++k) c[at++] = p[oW1 + o * kInP + k];
    for (int o = 0; o < kH; ++o) c[at++] = p[ob1 + o];
    for (int i = 0; i < kH * kH; ++i) c[at++] = p[oW2 + i];
    for (int o = 0; o < kH; ++o) c[at++] = p[ob2 + o];
    for (int i = 0; i < kH * kH; ++i) c[at++] = p[oW3 + i];
    for (int o = 0; o < kH; ++o) c[at++] = p[ob3 + o];
    for (int o = 0; o < kOut; ++o)
        for (int k = 0; k < kH; ++k) c[at++] = p[oW4 + o * kH + k];
    for (int o = 0; o < kOut; ++o) c[at++] = p[ob4 + o];
}

static_assert(kH * kIn + kH + 2 * (kH * kH + kH) + kOut * kH + kOut == LPDF_MLP_NPARAMS, "parameter count");
static_assert(kNorm == LPDF_MLP_NNORM, "standardisation block");

int check_error_flag(lpdf_mlp* m, cudaStream_t st, const char* what)
{
    unsigned h = 0;
    TRY(cudaMemcpyAsync(&h, m->error, sizeof h, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    if (h) {
        cudaMemsetAsync(m->error, 0, sizeof(unsigned), st);
        return lpdf_set_error(LPDF_ERR_CUDA, "%s: a bounded wait for the tensor-core MMAs gave up", what);
    }
    return LPDF_OK;
}

int grow(float** p, int64_t& cap, int64_t need)
{
    if (need <= cap) return LPDF_OK;
    cudaFree(*p);
    *p = nullptr;
    cap = 0;
    TRY(cudaMalloc((void**)p, sizeof(float) * (size_t)need));
    cap = need;
    return LPDF_OK;
}

}  // namespace

int lpdf_mlp_create(int64_t max_batch, lpdf_mlp** out)
{
    if (!out || max_batch < 1) return lpdf_set_error(LPDF_ERR_ARG, "mlp_create: max_batch = %lld", (long long)max_batch);
    *out = nullptr;
    TRY(mlp_configure());
    lpdf_mlp* m = new lpdf_mlp();
    m->max_batch = max_batch;
    const int64_t tiles = (max_batch + kH - 1) / kH;
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc((void**)&m->P, sizeof(float) * kParams)) ||
        (e = cudaMalloc(&m->pack, 2 * (size_t)kPack)) || (e = cudaMalloc((void**)&m->norm, sizeof(float) * kNorm)) ||
        (e = cudaMalloc((void**)&m->m, sizeof(float) * kParams)) ||
        (e = cudaMalloc((void**)&m->v, sizeof(float) * kParams)) ||
        (e = cudaMalloc((void**)&m->grad, sizeof(float) * kParams)) ||
        (e = cudaMalloc((void**)&m->part, sizeof(float) * kPart * (size_t)tiles)) ||
        (e = cudaMalloc(&m->act, 2 * 3 * (size_t)kH * (size_t)(tiles * kH))) ||
        (e = cudaMalloc((void**)&m->out, sizeof(float) * kOutP * (size_t)(tiles * kH))) ||
        (e = cudaMalloc((void**)&m->s_cmp, sizeof(double) * 2)) ||
        (e = cudaMalloc((void**)&m->error, sizeof(unsigned))) || (e = cudaMemset(m->error, 0, sizeof(unsigned)))) {
        lpdf_mlp_free(m);
        return lpdf_set_error(LPDF_ERR_CUDA, "mlp_create: %s", cudaGetErrorString(e));
    }
    std::vector<float> zero(LPDF_MLP_NPARAMS, 0.0f), norm(kNorm, 0.0f);
    for (int j = 0; j < kIn; ++j) norm[nFS + j] = 1.0f;
    for (int j = 0; j < kOut; ++j) norm[nW + j] = norm[nTS + j] = 1.0f;
    if (const int rc = lpdf_mlp_set_params(m, zero.data(), norm.data())) {
        lpdf_mlp_free(m);
        return rc;
    }
    *out = m;
    return LPDF_OK;
}

void lpdf_mlp_free(lpdf_mlp* m)
{
    if (!m) return;
    void* ps[] = {m->P, m->pack, m->norm, m->m, m->v, m->grad, m->part, m->act, m->out, m->losses, m->error,
                  m->s_feat, m->s_out, m->s_fields, m->s_cmp};
    for (void* p : ps) cudaFree(p);
    delete m;
}

int lpdf_mlp_set_params(lpdf_mlp* m, const float* params, const float* norm)
{
    if (!m || !params) return lpdf_set_error(LPDF_ERR_ARG, "mlp_set_params: NULL argument");
    std::vector<float> p;
    to_padded(params, p);
    TRY(cudaMemcpy(m->P, p.data(), sizeof(float) * kParams, cudaMemcpyHostToDevice));
    if (norm) TRY(cudaMemcpy(m->norm, norm, sizeof(float) * kNorm, cudaMemcpyHostToDevice));
    TRY(cudaMemset(m->m, 0, sizeof(float) * kParams));
    TRY(cudaMemset(m->v, 0, sizeof(float) * kParams));
    m->step = 0;
    TRY(launch_mlp_adam(m->P, m->grad, m->m, m->v, 0.0f, 0, m->pack, nullptr));   // step 0: packs only
    TRY(cudaDeviceSynchronize());
    return LPDF_OK;
}

int lpdf_mlp_get_params(lpdf_mlp* m, float* params, float* norm)
{
    if (!m) return lpdf_set_error(LPDF_ERR_ARG, "mlp_get_params: NULL argument");
    TRY(cudaDeviceSynchronize());
    if (params) {
        std::vector<float> p(kParams);
        TRY(cudaMemcpy(p.data(), m->P, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
        to_compact(p, params);
    }
    if (norm) TRY(cudaMemcpy(norm, m->norm, sizeof(float) * kNorm, cudaMemcpyDeviceToHost));
    return LPDF_OK;
}

int lpdf_mlp_fit_norm(lpdf_mlp* m, const float* feat, const float* tgt, int64_t B, void* stream)
{
    if (!m || !feat || !tgt || B < 1) return lpdf_set_error(LPDF_ERR_ARG, "mlp_fit_norm: bad argument");
    TRY(launch_mlp_fit_norm(feat, tgt, B, m->norm, (cudaStream_t)stream));
    return LPDF_OK;
}

int lpdf_mlp_forward(lpdf_mlp* m, const float* feat, int64_t B, float* out, void* stream)
{
    if (!m || B < 0 || (B > 0 && (!feat || !out))) return lpdf_set_error(LPDF_ERR_ARG, "mlp_forward: bad argument");
    TRY(launch_mlp_forward(feat, B, m->P, m->pack, m->norm, nullptr, out, nullptr, m->error, (cudaStream_t)stream));
    return LPDF_OK;
}

int lpdf_mlp_gradient(lpdf_mlp* m, const float* feat, const float* tgt, int64_t B, float* grad, double* loss,
                      void* stream)
{
    if (!m || !feat || !tgt || !grad || B < 1 || B > m->max_batch)
        return lpdf_set_error(LPDF_ERR_ARG, "mlp_gradient: bad argument (B = %lld)", (long long)B);
    const cudaStream_t st = (cudaStream_t)stream;
    if (m->losses_cap < 1) {
        TRY(cudaMalloc((void**)&m->losses, sizeof(double) * 1));
        m->losses_cap = 1;
    }
    TRY(launch_mlp_forward(feat, B, m->P, m->pack, m->norm, m->out, nullptr, m->act, m->error, st));
    TRY(launch_mlp_backward(feat, tgt, B, m->pack, m->norm, m->out, m->act, m->part, m->grad, m->error, st));
    TRY(launch_mlp_loss(m->out, tgt, B, m->norm, m->losses, st));
    std::vector<float> g(kParams);
    double l = 0.0;
    TRY(cudaMemcpyAsync(g.data(), m->grad, sizeof(float) * kParams, cudaMemcpyDeviceToHost, st));
    TRY(cudaMemcpyAsync(&l, m->losses, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (const int rc = check_error_flag(m, st, "mlp_gradient")) return rc;
    to_compact(g, grad);
    if (loss) *loss = l;
    return LPDF_OK;
}

int lpdf_mlp_train(lpdf_mlp* m, const float* feat, const float* tgt, int64_t B, int64_t batch, int32_t steps,
                   float lr, double* losses, void* stream)
{
    if (!m || !feat || !tgt || B < 1 || batch < 1 || batch > B || batch > m->max_batch || steps < 0 || !(lr > 0.0f))
        return lpdf_set_error(LPDF_ERR_ARG, "mlp_train: bad argument (B = %lld, batch = %lld, steps = %d)",
                              (long long)B, (long long)batch, steps);
    const cudaStream_t st = (cudaStream_t)stream;
    if (m->losses_cap < steps) {
        cudaFree(m->losses);
        m->losses = nullptr;
        m->losses_cap = 0;
        TRY(cudaMalloc((void**)&m->losses, sizeof(double) * steps));
        m->losses_cap = steps;
    }
    const int64_t nchunk = B / batch;
    for (int s = 0; s < steps; ++s) {
        const int64_t off = (s % nchunk) * batch;
        const float* f = feat + off * kIn;
        const float* t = tgt + off * kOut;
        TRY(launch_mlp_forward(f, batch, m->P, m->pack, m->norm, m->out, nullptr, m->act, m->error, st));
        TRY(launch_mlp_backward(f, t, batch, m->pack, m->norm, m->out, m->act, m->part, m->grad, m->error, st));
        TRY(launch_mlp_loss(m->out, t, batch, m->norm, m->losses + s, st));
        TRY(launch_mlp_adam(m->P, m->grad, m->m, m->v, lr, ++m->step, m->pack, st));
    }
    if (losses && steps > 0)
        TRY(cudaMemcpyAsync(losses, m->losses, sizeof(double) * steps, cudaMemcpyDeviceToHost, st));
    return check_error_flag(m, st, "mlp_train");
}

int lpdf_surrogate_features(const lpdf_mesh* mesh, const lpdf_params* params, const double* stats,
                            const float* fields, float* feat, float* tgt, void* stream)
{
    if (!mesh || !params || !stats || !feat || (fields && !tgt))
        return lpdf_set_error(LPDF_ERR_ARG, "surrogate_features: NULL argument");
    if (params->ns < 1 || params->ns > LPDF_MAX_SCALARS)
        return lpdf_set_error(LPDF_ERR_UNSUPPORTED, "surrogate_features: ns = %d", params->ns);
    Fem* F = nullptr;
    if (const int rc = mesh_fem(mesh, &F)) return rc;
    TRY(surrogate_features(*F, stats, params->ns, fields, params->C0, feat, tgt, (cudaStream_t)stream));
    return LPDF_OK;
}

int lpdf_mlp_set_policy(lpdf_mlp* m, int32_t check_every, double threshold)
{
    if (!m || check_every < 0 || !(threshold >= 0.0)) return lpdf_set_error(LPDF_ERR_ARG, "mlp_set_policy: bad argument");
    m->check_every = check_every;
    m->threshold = threshold;
    return LPDF_OK;
}

int lpdf_mlp_request_check(lpdf_mlp* m)
{
    if (!m) return lpdf_set_error(LPDF_ERR_ARG, "mlp_request_check: NULL argument");
    m->check_next = true;
    return LPDF_OK;
}

int lpdf_surrogate_relax_solve(const lpdf_mesh* mesh, lpdf_mlp* m, const lpdf_params* params, const double* stats,
                               float* fields, double tol, int32_t maxit, double* info, void* stream)
{
    if (!mesh || !m || !params || !stats || !fields)
        return lpdf_set_error(LPDF_ERR_ARG, "surrogate_relax_solve: NULL argument");
    if (params->gmodel != 0) return lpdf_set_error(LPDF_ERR_ARG, "surrogate_relax_solve: gmodel = %d", params->gmodel);
    if (params->ns < 1 || params->ns > LPDF_MAX_SCALARS)
        return lpdf_set_error(LPDF_ERR_UNSUPPORTED, "surrogate_relax_solve: ns = %d", params->ns);
    const cudaStream_t st = (cudaStream_t)stream;
    Fem* F = nullptr;
    if (const int rc = mesh_fem(mesh, &F)) return rc;
    const int64_t N = mesh->d.n_nodes;
    const int nfp = nfields_padded(params->ns);
    if (const int rc = grow(&m->s_feat, m->s_feat_cap, N * kIn)) return rc;
    if (const int rc = grow(&m->s_out, m->s_out_cap, N * kOutP)) return rc;
    const bool check = m->check_next || (m->check_every > 0 && m->calls % m->check_every == 0);
    m->check_next = false;
    ++m->calls;
    const bool use_net = check || m->net_ok;
    const bool use_plain = check || !m->net_ok;
    double err = -1.0;
    float* net_fields = fields;
    if (check) {
        if (const int rc = grow(&m->s_fields, m->s_fields_cap, N * nfp)) return rc;
        net_fields = m->s_fields;
    }
    int it[2] = {0, 0};
    if (use_net) {
        TRY(surrogate_features(*F, stats, params->ns, nullptr, params->C0, m->s_feat, nullptr, st));
        TRY(launch_mlp_forward(m->s_feat, N, m->P, m->pack, m->norm, m->s_out, nullptr, nullptr, m->error, st));
        const cudaError_t e = node_fields_solve(*F, stats, *params, net_fields, tol, maxit, it, st, m->s_out, m->norm);
        if (e == cudaErrorNotReady)
            return lpdf_set_error(LPDF_ERR_CG_NOCONV, "surrogate_relax_solve: pressure CG did not converge");
        TRY(e);
    }
    if (use_plain) {
        const cudaError_t e = node_fields_solve(*F, stats, *params, fields, tol, maxit, it, st);
        if (e == cudaErrorNotReady)
            return lpdf_set_error(LPDF_ERR_CG_NOCONV, "surrogate_relax_solve: no convergence to %g in %d iterations",
                                  tol, maxit);
        TRY(e);
    }
    if (check) {
        double h[2] = {0.0, 0.0};
        TRY(fields_compare(net_fields, fields, (int)N, nfp, m->s_cmp, st));
        TRY(cudaMemcpyAsync(h, m->s_cmp, sizeof h, cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        err = h[1] > 0.0 ? std::sqrt(h[0] / h[1]) : (h[0] > 0.0 ? INFINITY : 0.0);
        m->net_ok = err <= m->threshold;
    }
    if (const int rc = check_error_flag(m, st, "surrogate_relax_solve")) return rc;
    if (info) {
        info[0] = check ? 1.0 : 0.0;
        info[1] = err;
        info[2] = use_plain ? 1.0 : 0.0;
        info[3] = (double)m->calls;
    }
    return LPDF_OK;
}
