// Particle initialisation and gridpoint statistics (sm_103a). The particle step itself is in
// lpdf_pipeline.cu (and lpdf_step.cu for the no-allocation entry point).
#include "lpdf_device.cuh"

namespace lpdf {

// ------------------------------------------------------------------------------------------
// Particle initialisation: uniform position in the generating element (s = sqrt(r1):
// lambda = (1-s, s(1-r2), s r2)), exact location, Gaussian velocity about the interpolated
// mean, Erlang(m) frequency with the interpolated mean, psi = 0. Philox tag 1, blocks 0..2.
// Component c (one for an ordinary mesh) holds particles [pbase[c], pbase[c + 1]), ppe[c] per
// element of its element range, with ids counted from 0 and its own Philox key.
// ------------------------------------------------------------------------------------------
template <int NS>
__global__ void particles_init_kernel(const __grid_constant__ DevMesh M, const __grid_constant__ DevState S,
                                      const __grid_constant__ InitLayout L, const float* __restrict__ init,
                                      int m_erlang, unsigned long long* status)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned err = 0;
    if (i < L.pbase[L.n_comp]) {
        int lo = 0, hi = L.n_comp - 1;   // the component: pbase[lo] <= i < pbase[lo + 1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (L.pbase[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        const int64_t local = i - L.pbase[lo];
        const int e = L.tri_off[lo] + (int)(local / L.ppe[lo]);
        const uint32_t pid = (uint32_t)local;
        const uint32_t k0 = L.key[2 * lo], k1 = L.key[2 * lo + 1];
        const uint4 a = philox4x32_10(make_uint4(pid, 0u, 0u, (1u << 16) | 0u), k0, k1);
        const uint4 b = philox4x32_10(make_uint4(pid, 0u, 0u, (1u << 16) | 1u), k0, k1);
        const uint4 c = philox4x32_10(make_uint4(pid, 0u, 0u, (1u << 16) | 2u), k0, k1);
        const float4 X = __ldg(&M.ex[e]), Y = __ldg(&M.ey[e]);
        const float sq = sqrtf(u01(a.x)), r2 = u01(a.y);
        const float l0 = 1.0f - sq, l1 = sq * (1.0f - r2), l2 = sq * r2;
        float px = fmaf(l0, X.x, fmaf(l1, X.y, l2 * X.z));
        float py = fmaf(l0, Y.x, fmaf(l1, Y.y, l2 * Y.z));
        float fx0 = M.x0, fx1 = M.x1, fy1 = M.y1;
        if (M.n_comp > 1) {
            const float4 fr = __ldg(&M.cframe[lo]);
            fx0 = fr.x;
            fx1 = fr.y;
            fy1 = fr.w;
        }
        if (!M.edge_walls) {
            if (px >= fx1) px = M.periodic ? fx0 : nextafterf(fx1, -CUDART_INF_F);
            if (py >= fy1) py = nextafterf(fy1, -CUDART_INF_F);
        } else if (M.periodic && px >= fx1) {
            px = fx0;
        }
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

cudaError_t launch_particles_init(const DevMesh& m, const DevState& s, int ns, const InitLayout& L, int64_t P,
                                  const float* node_init, int m_erlang, unsigned long long* status, cudaStream_t st)
{
    const unsigned grid = (unsigned)((P + 255) / 256);
    if (grid == 0) return cudaSuccess;
    switch (ns) {
        case 1: particles_init_kernel<1><<<grid, 256, 0, st>>>(m, s, L, node_init, m_erlang, status); break;
        case 2: particles_init_kernel<2><<<grid, 256, 0, st>>>(m, s, L, node_init, m_erlang, status); break;
        case 3: particles_init_kernel<3><<<grid, 256, 0, st>>>(m, s, L, node_init, m_erlang, status); break;
        case 4: particles_init_kernel<4><<<grid, 256, 0, st>>>(m, s, L, node_init, m_erlang, status); break;
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

// ------------------------------------------------------------------------------------------
// IECM (Eq. 9): scalar fluxes at the gridpoints, and the slopes of the conditional mean
// ------------------------------------------------------------------------------------------
__global__ void flux_statistics_kernel(const int* __restrict__ master, int n_nodes, int ns,
                                       const unsigned long long* __restrict__ acc,
                                       const unsigned long long* __restrict__ facc, double* __restrict__ out, int raw)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_nodes) return;
    const int m = master[n];
    const int nq = 11 + 2 * ns, nf = 3 * ns;
    double* o = out + (size_t)n * nf;
    const double s0 = (double)(long long)acc[(size_t)m * nq] * (1.0 / kFixScale);
    for (int a = 0; a < ns; ++a)
        for (int c = 0; c < 3; ++c) {
            const double f = (double)(long long)facc[(size_t)m * nf + 3 * a + c] * (1.0 / kFixScale);
            if (raw) {
                o[3 * a + c] = f;
            } else if (s0 == 0.0) {
                o[3 * a + c] = 0.0;
            } else {
                const double su = (double)(long long)acc[(size_t)m * nq + 1 + c] * (1.0 / kFixScale);
                const double sp = (double)(long long)acc[(size_t)m * nq + 11 + a] * (1.0 / kFixScale);
                o[3 * a + c] = f / s0 - (su / s0) * (sp / s0);
            }
        }
}

// beta_a = R^-1 c_a by Cramer's rule (R symmetric, from the statistics columns uu, uv, uw, vv, vw,
// ww); beta_a = 0 where det R <= 1e-12 (trace R / 3)^3
__global__ void iecm_coefficients_kernel(int n_nodes, int ns, const double* __restrict__ stats,
                                         const double* __restrict__ flux, float* __restrict__ beta)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_nodes) return;
    const double* st = stats + (size_t)n * (11 + 2 * ns);
    const double a11 = st[4], a12 = st[5], a13 = st[6], a22 = st[7], a23 = st[8], a33 = st[9];
    // cofactors of the symmetric matrix
    const double c11 = a22 * a33 - a23 * a23, c12 = a13 * a23 - a12 * a33, c13 = a12 * a23 - a13 * a22;
    const double c22 = a11 * a33 - a13 * a13, c23 = a12 * a13 - a11 * a23, c33 = a11 * a22 - a12 * a12;
    const double det = a11 * c11 + a12 * c12 + a13 * c13;
    const double tr = fmax((a11 + a22 + a33) / 3.0, 0.0);
    const bool ok = det > 1e-12 * tr * tr * tr;
    for (int a = 0; a < ns; ++a) {
        const double* f = flux + (size_t)n * 3 * ns + 3 * a;
        float* b = beta + (size_t)n * 3 * ns + 3 * a;
        if (!ok) {
            b[0] = b[1] = b[2] = 0.0f;
            continue;
        }
        b[0] = (float)((c11 * f[0] + c12 * f[1] + c13 * f[2]) / det);
        b[1] = (float)((c12 * f[0] + c22 * f[1] + c23 * f[2]) / det);
        b[2] = (float)((c13 * f[0] + c23 * f[1] + c33 * f[2]) / det);
    }
}

cudaError_t launch_flux_statistics(const int* master, int n_nodes, int ns, const unsigned long long* node_acc,
                                   const unsigned long long* flux_acc, double* out, int raw, cudaStream_t st)
{
    if (n_nodes <= 0) return cudaSuccess;
    flux_statistics_kernel<<<(n_nodes + 255) / 256, 256, 0, st>>>(master, n_nodes, ns, node_acc, flux_acc, out, raw);
    return cudaGetLastError();
}

cudaError_t launch_iecm_coefficients(int n_nodes, int ns, const double* stats, const double* flux, float* beta,
                                     cudaStream_t st)
{
    if (n_nodes <= 0) return cudaSuccess;
    iecm_coefficients_kernel<<<(n_nodes + 255) / 256, 256, 0, st>>>(n_nodes, ns, stats, flux, beta);
    return cudaGetLastError();
}

}  // namespace lpdf
