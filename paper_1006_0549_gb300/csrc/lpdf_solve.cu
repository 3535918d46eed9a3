// The gridpoint side of the method (Introduction, item ii: the grid is used to solve for the
// Eulerian quantities): node fields for the particle step from gridpoint statistics.
//
//   * recovery: element gradients of the P1 mean fields, area-weighted to the nodes; the
//     Laplacian is the recovered divergence of the recovered gradient;
//   * k = <u_i u_i>/2, eps = k <omega> (the paragraph before Eq. 5), production
//     P = -<u_i u_j> d<U_i>/dx_j and S_omega = C_omega2 - C_omega1 P/eps (Eq. 6);
//   * G_ij from elliptic relaxation (the paragraph after Eq. 4): P1 finite elements for
//     wp_ij - L^2 lap wp_ij = -3/4 C0 eps delta_ij with wall values wp_ij = -4.5 eps n_i n_j,
//     L = CL max(k^1.5/eps, Ceta nu^0.75/eps^0.25) (L^2 averaged over each element's nodes),
//     solved by a Jacobi-preconditioned conjugate gradient in FP64 on the four components at
//     once; G_ij = (wp_ij - eps delta_ij/2)/k and C0 eps = -2/3 (eps + <u_i u_j> G_ij) (the
//     k-consistency condition), or the simplified Langevin model;
//   * mean pressure (optional; Section "Governing equations", the projection on the grid): weak
//     form of lap p = -d_i d_j (<U_i><U_j> + <u_i u_j>) with its natural boundary condition and
//     zero mean, by the same CG; a fixed mean gradient is added.
// Every reduction (gradient averaging, matrix assembly, dot products) is a gather in a fixed
// order, so the results are bit-reproducible run to run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

#include "lpdf_internal.h"

namespace lpdf {

namespace {

constexpr int kDotThreads = 256;
constexpr int kCheckEvery = 8;   // CG iterations between host-side convergence tests

template <class T>
cudaError_t upload(T** d, const std::vector<T>& h)
{
    cudaError_t e = cudaMalloc((void**)d, sizeof(T) * std::max<size_t>(1, h.size()));
    if (e != cudaSuccess || h.empty()) return e;
    return cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
}

inline unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------- recovery
// element gradient of m DOF fields (row stride ld): out[(e m + i) 2 + j] = d_j f_i
__global__ void elem_grad_kernel(const Fem F, const double* __restrict__ f, int m, int ld, double* __restrict__ out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= F.E) return;
    const int d0 = F.edof[3 * e], d1 = F.edof[3 * e + 1], d2 = F.edof[3 * e + 2];
    const double* g = F.grad + 6 * e;
    for (int i = 0; i < m; ++i) {
        const double a = f[(size_t)d0 * ld + i], b = f[(size_t)d1 * ld + i], c = f[(size_t)d2 * ld + i];
        out[((size_t)e * m + i) * 2 + 0] = a * g[0] + b * g[2] + c * g[4];
        out[((size_t)e * m + i) * 2 + 1] = a * g[1] + b * g[3] + c * g[5];
    }
}

// area-weighted average of m element values to the DOFs: out[d ld + i]
__global__ void recover_kernel(const Fem F, const double* __restrict__ ev, int m, double* __restrict__ out, int ld)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= F.ndof) return;
    const double inv = 1.0 / F.darea[d];
    for (int i = 0; i < m; ++i) {
        double s = 0.0;
        for (int t = F.de_ptr[d]; t < F.de_ptr[d + 1]; ++t) {
            const int e = F.de_el[t] / 3;
            s += F.area[e] * ev[(size_t)e * m + i];
        }
        out[(size_t)d * ld + i] = s * inv;
    }
}

// element divergence of a recovered gradient field g (d/dx at g[d ld], d/dy at g[d ld + 1])
__global__ void elem_div_kernel(const Fem F, const double* __restrict__ g, int ld, double* __restrict__ out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= F.E) return;
    const double* gr = F.grad + 6 * e;
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        const size_t d = F.edof[3 * e + a];
        s += g[d * ld] * gr[2 * a] + g[d * ld + 1] * gr[2 * a + 1];
    }
    out[e] = s;
}

// ---------------------------------------------------------------- per-DOF statistics
// statistics rows (S0, means, central moments, <omega>, <phi>, ...) of the DOF's master node
__global__ void dof_stats_kernel(const Fem F, const double* __restrict__ st, int nq, int ns, double* __restrict__ U,
                                 double* __restrict__ R, double* __restrict__ om, double* __restrict__ phi,
                                 double* __restrict__ k, double* __restrict__ eps)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= F.ndof) return;
    const double* s = st + (size_t)F.dof_node[d] * nq;
    for (int i = 0; i < 3; ++i) U[3 * d + i] = s[1 + i];
    for (int i = 0; i < 6; ++i) R[6 * d + i] = s[4 + i];
    om[d] = s[10];
    for (int a = 0; a < ns; ++a) phi[(size_t)d * ns + a] = s[11 + a];
    const double kk = 0.5 * (s[4] + s[7] + s[9]);
    k[d] = kk;
    eps[d] = kk * s[10];
}

// ---------------------------------------------------------------- assembly
__global__ void elem_L2_kernel(const Fem F, const double* __restrict__ k, const double* __restrict__ eps, double CL,
                               double Ceta, double nu, double* __restrict__ L2e)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= F.E) return;
    const double kol = Ceta * pow(nu, 0.75);
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        const int d = F.edof[3 * e + a];
        const double ep = fmax(eps[d], 1e-12);
        const double L = CL * fmax(pow(fmax(k[d], 0.0), 1.5) / ep, kol / pow(ep, 0.25));
        s += L * L;
    }
    L2e[e] = s / 3.0;
}

// A = M + sum_e L2_e K_e (fixed contribution order per CSR entry); diag = its diagonal
__global__ void assemble_kernel(const Fem F, const double* __restrict__ L2e, double* __restrict__ A,
                                double* __restrict__ diag)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= F.ndof) return;
    for (int j = F.row[i]; j < F.row[i + 1]; ++j) {
        double s = 0.0;
        for (int t = F.cptr[j]; t < F.cptr[j + 1]; ++t) {
            const int c = F.cel[t];
            const int e = c / 9, a = (c / 3) % 3, b = c % 3;
            const double* g = F.grad + 6 * e;
            s += L2e[e] * (F.area[e] * (g[2 * a] * g[2 * b] + g[2 * a + 1] * g[2 * b + 1]));
        }
        A[j] = F.Mval[j] + s;
        if (F.col[j] == i) diag[i] = A[j];
    }
}

__global__ void diag_kernel(const Fem F, const double* __restrict__ A, double* __restrict__ diag)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= F.ndof) return;
    for (int j = F.row[i]; j < F.row[i + 1]; ++j)
        if (F.col[j] == i) diag[i] = A[j];
}

// ---------------------------------------------------------------- batched PCG (nv <= 4 vectors)
// vectors are stored component-major: v[c n + i]

// y_c = A x_c; rows of fixed (wall) DOFs give 0 when `mask` is set
__global__ void spmv_kernel(const Fem F, const double* __restrict__ A, const double* __restrict__ x,
                            double* __restrict__ y, int mask, int nv)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= F.ndof) return;
    const size_t n = F.ndof;
    double s[4] = {0, 0, 0, 0};
    if (!(mask && F.wall[i]))
        for (int t = F.row[i]; t < F.row[i + 1]; ++t) {
            const int j = F.col[t];
            const double a = A[t];
            for (int c = 0; c < nv; ++c) s[c] += a * x[c * n + j];
        }
    for (int c = 0; c < nv; ++c) y[c * n + i] = s[c];
}

// r = b - y (0 on fixed rows); z = r / diag; p = z
__global__ void cg_start_kernel(const Fem F, const double* __restrict__ b, const double* __restrict__ y,
                                const double* __restrict__ diag, double* __restrict__ r, double* __restrict__ z,
                                double* __restrict__ p, int mask, int nv)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= F.ndof) return;
    const size_t n = F.ndof;
    const bool fixed = mask && F.wall[i];
    for (int c = 0; c < nv; ++c) {
        const double rr = fixed ? 0.0 : b[c * n + i] - y[c * n + i];
        r[c * n + i] = rr;
        z[c * n + i] = rr / diag[i];
        p[c * n + i] = rr / diag[i];
    }
}

// per-block partial sums of x_c . y_c, fixed order
__global__ void dot_kernel(const double* __restrict__ x, const double* __restrict__ y, int n, int nv,
                           double* __restrict__ part)
{
    __shared__ double sh[4][kDotThreads];
    double s[4] = {0, 0, 0, 0};
    for (int i = blockIdx.x * kDotThreads + threadIdx.x; i < n; i += gridDim.x * kDotThreads)
        for (int c = 0; c < nv; ++c) s[c] += x[(size_t)c * n + i] * y[(size_t)c * n + i];
    for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] = s[c];
    __syncthreads();
    for (int o = kDotThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 4; ++c) part[(size_t)c * gridDim.x + blockIdx.x] = sh[c][0];
}

// CG scalars, kept on the device (4 slots each): rz, the last plain dot, alpha, beta,
// |r_0|^2, |r|^2
enum { kRZ = 0, kDot = 4, kAlpha = 8, kBeta = 12, kR0 = 16, kRR = 20, kNScal = 24 };

// sum the block partials of one dot product, then per mode
// 0: sc[slot + c] = sum; 1: alpha = rz / sum; 2: beta = sum / rz, rz = sum
__global__ void scalar_kernel(const double* __restrict__ part, int nb, int nv, int slot, int mode,
                              double* __restrict__ sc)
{
    const int c = threadIdx.x;
    if (c >= nv) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(size_t)c * nb + b];
    if (mode == 0) {
        sc[slot + c] = s;
    } else if (mode == 1) {
        sc[kAlpha + c] = s != 0.0 ? sc[kRZ + c] / s : 0.0;
    } else {
        sc[kBeta + c] = sc[kRZ + c] != 0.0 ? s / sc[kRZ + c] : 0.0;
        sc[kRZ + c] = s;
    }
}

// x_c += alpha_c p_c ; r_c -= alpha_c q_c ; z_c = r_c / diag
__global__ void cg_update_kernel(int n, int nv, const double* __restrict__ sc, const double* __restrict__ diag,
                                 const double* __restrict__ p, const double* __restrict__ q, double* __restrict__ x,
                                 double* __restrict__ r, double* __restrict__ z)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int c = 0; c < nv; ++c) {
        const size_t o = (size_t)c * n + i;
        const double a = sc[kAlpha + c];
        x[o] += a * p[o];
        const double rr = r[o] - a * q[o];
        r[o] = rr;
        z[o] = rr / diag[i];
    }
}

// p_c = z_c + beta_c p_c
__global__ void cg_direction_kernel(int n, int nv, const double* __restrict__ sc, const double* __restrict__ z,
                                    double* __restrict__ p)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int c = 0; c < nv; ++c) {
        const size_t o = (size_t)c * n + i;
        p[o] = z[o] + sc[kBeta + c] * p[o];
    }
}

// q_c = A p_c (0 on fixed rows) and block partials of p_c . q_c (fixed order)
__global__ void spmv_dot_kernel(const Fem F, const double* __restrict__ A, const double* __restrict__ p,
                                double* __restrict__ q, int mask, int nv, double* __restrict__ part)
{
    __shared__ double sh[4][kDotThreads];
    const size_t n = F.ndof;
    double acc[4] = {0, 0, 0, 0};
    for (int i = blockIdx.x * kDotThreads + threadIdx.x; i < F.ndof; i += gridDim.x * kDotThreads) {
        double s[4] = {0, 0, 0, 0};
        if (!(mask && F.wall[i]))
            for (int t = F.row[i]; t < F.row[i + 1]; ++t) {
                const int j = F.col[t];
                const double a = A[t];
                for (int c = 0; c < nv; ++c) s[c] += a * p[c * n + j];
            }
        for (int c = 0; c < nv; ++c) {
            q[c * n + i] = s[c];
            acc[c] += p[c * n + i] * s[c];
        }
    }
    for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int o = kDotThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 4; ++c) part[(size_t)c * gridDim.x + blockIdx.x] = sh[c][0];
}

// x += alpha p; r -= alpha q; z = r / diag; block partials of r . z and r . r
__global__ void update_dot_kernel(int n, int nv, const double* __restrict__ sc, const double* __restrict__ diag,
                                  const double* __restrict__ p, const double* __restrict__ q, double* __restrict__ x,
                                  double* __restrict__ r, double* __restrict__ z, double* __restrict__ part_rz,
                                  double* __restrict__ part_rr)
{
    __shared__ double sh[8][kDotThreads];
    double a_rz[4] = {0, 0, 0, 0}, a_rr[4] = {0, 0, 0, 0};
    for (int i = blockIdx.x * kDotThreads + threadIdx.x; i < n; i += gridDim.x * kDotThreads)
        for (int c = 0; c < nv; ++c) {
            const size_t o = (size_t)c * n + i;
            const double al = sc[kAlpha + c];
            x[o] += al * p[o];
            const double rr = r[o] - al * q[o];
            r[o] = rr;
            const double zz = rr / diag[i];
            z[o] = zz;
            a_rz[c] += rr * zz;
            a_rr[c] += rr * rr;
        }
    for (int c = 0; c < 4; ++c) {
        sh[c][threadIdx.x] = a_rz[c];
        sh[4 + c][threadIdx.x] = a_rr[c];
    }
    __syncthreads();
    for (int o = kDotThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int c = 0; c < 8; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 4; ++c) {
            part_rz[(size_t)c * gridDim.x + blockIdx.x] = sh[c][0];
            part_rr[(size_t)c * gridDim.x + blockIdx.x] = sh[4 + c][0];
        }
}

// beta = rz_new / rz, rz = rz_new, rr (for the convergence test)
__global__ void scalar_beta_kernel(const double* __restrict__ part_rz, const double* __restrict__ part_rr, int nb,
                                   int nv, double* __restrict__ sc)
{
    const int c = threadIdx.x;
    if (c >= nv) return;
    double rz = 0.0, rr = 0.0;
    for (int b = 0; b < nb; ++b) {
        rz += part_rz[(size_t)c * nb + b];
        rr += part_rr[(size_t)c * nb + b];
    }
    sc[kBeta + c] = sc[kRZ + c] != 0.0 ? rz / sc[kRZ + c] : 0.0;
    sc[kRZ + c] = rz;
    sc[kRR + c] = rr;
}

// ---------------------------------------------------------------- right-hand sides
// elliptic relaxation: sources wp^h (11, 12, 22, 33); wall values in x (the CG's start, whose
// interior is `prev`, or 0) and in xref (interior 0: the reference of the convergence test)
__global__ void er_setup_kernel(const Fem F, const double* __restrict__ eps, double C0, double* __restrict__ src,
                                double* __restrict__ x, const double* __restrict__ prev, double* __restrict__ xref)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= F.ndof) return;
    const size_t n = F.ndof;
    const double e = eps[d];
    const double n1 = F.normal[2 * d], n2 = F.normal[2 * d + 1];
    const double s = -0.75 * C0 * e;
    const bool w = F.wall[d];
    src[0 * n + d] = s;
    src[1 * n + d] = 0.0;
    src[2 * n + d] = s;
    src[3 * n + d] = s;
    const double wv[4] = {-4.5 * e * n1 * n1, -4.5 * e * n1 * n2, -4.5 * e * n2 * n2, 0.0};
    for (int c = 0; c < 4; ++c) {
        xref[c * n + d] = w ? wv[c] : 0.0;
        x[c * n + d] = w ? wv[c] : (prev ? prev[c * n + d] : 0.0);
    }
}

// T = <U><U> + <uu> in the plane: (T00, T01, T10, T11) per DOF
__global__ void pressure_T_kernel(const Fem F, const double* __restrict__ U, const double* __restrict__ R,
                                  double* __restrict__ T)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= F.ndof) return;
    const double u = U[3 * d], v = U[3 * d + 1];
    T[4 * d + 0] = u * u + R[6 * d + 0];
    T[4 * d + 1] = u * v + R[6 * d + 1];
    T[4 * d + 2] = u * v + R[6 * d + 1];
    T[4 * d + 3] = v * v + R[6 * d + 3];
}

// b_d = -sum_(e, a: edof(e, a) = d) area_e grad(l_a) . (div T)_e, gT = element gradients of T
__global__ void pressure_rhs_kernel(const Fem F, const double* __restrict__ gT, double* __restrict__ b)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= F.ndof) return;
    double s = 0.0;
    for (int t = F.de_ptr[d]; t < F.de_ptr[d + 1]; ++t) {
        const int e = F.de_el[t] / 3, a = F.de_el[t] % 3;
        const double* g = gT + (size_t)e * 8;
        const double div0 = g[0] + g[3];    // d_x T00 + d_y T01
        const double div1 = g[4] + g[7];    // d_x T10 + d_y T11
        const double* gr = F.grad + 6 * e;
        s += -F.area[e] * (gr[2 * a] * div0 + gr[2 * a + 1] * div1);
    }
    b[d] = s;
}

__global__ void fill_kernel(int n, double v, double* __restrict__ x)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

__global__ void subtract_mean_kernel(int n, const double* __restrict__ sum, double* __restrict__ x)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] -= sum[0] / n;
}

// ---------------------------------------------------------------- the output fields
__global__ void fields_kernel(const Fem F, int ns, int nfp, const double* __restrict__ U, const double* __restrict__ R,
                              const double* __restrict__ om, const double* __restrict__ phi,
                              const double* __restrict__ k, const double* __restrict__ eps,
                              const double* __restrict__ gU, const double* __restrict__ lapU,
                              const double* __restrict__ gp, const double* __restrict__ wp, int gmodel, double C0,
                              double Comega1, double Comega2, double dpdx0, double dpdy0,
                              const float* __restrict__ surr, const float* __restrict__ snorm, float* __restrict__ out)
{
    const int nd = blockIdx.x * blockDim.x + threadIdx.x;
    if (nd >= F.N) return;
    const int d = F.dof[nd];
    const size_t n = F.ndof;
    const double* r = R + 6 * (size_t)d;       // uu, uv, uw, vv, vw, ww
    const double* g = gU + 6 * (size_t)d;      // dU/dx, dU/dy, dV/dx, dV/dy, dW/dx, dW/dy
    const double kk = k[d], e = eps[d], Om = om[d];
    const double prod = -(r[0] * g[0] + r[1] * g[1] + r[1] * g[2] + r[3] * g[3] + r[2] * g[4] + r[4] * g[5]);
    const double Som = e > 1e-12 ? Comega2 - Comega1 * prod / e : Comega2;
    double G11, G12, G21, G22, G33, c0e;
    if (surr) {
        // the surrogate's targets: G_ij / <omega> and C_0 epsilon / (k <omega>), standardised
        double y[6];
        for (int j = 0; j < 6; ++j)
            y[j] = (double)surr[(size_t)nd * mlp::kOutP + j] * snorm[mlp::nTS + j] + snorm[mlp::nTM + j];
        G11 = Om * y[0];
        G12 = Om * y[1];
        G21 = Om * y[2];
        G22 = Om * y[3];
        G33 = Om * y[4];
        c0e = fmax(0.0, kk * Om * y[5]);
    } else if (gmodel == 1) {
        G11 = G22 = G33 = -(0.5 + 0.75 * C0) * Om;
        G12 = G21 = 0.0;
        c0e = C0 * e;
    } else {
        const double kc = fmax(kk, 1e-12);
        G11 = (wp[0 * n + d] - 0.5 * e) / kc;
        G12 = wp[1 * n + d] / kc;
        G22 = (wp[2 * n + d] - 0.5 * e) / kc;
        G33 = (wp[3 * n + d] - 0.5 * e) / kc;
        c0e = fmax(0.0, -2.0 / 3.0 * (e + r[0] * G11 + 2.0 * r[1] * G12 + r[3] * G22 + r[5] * G33));
        G21 = G12;
    }
    float* o = out + (size_t)nd * nfp;
    o[LPDF_F_U + 0] = (float)U[3 * d];
    o[LPDF_F_U + 1] = (float)U[3 * d + 1];
    o[LPDF_F_U + 2] = (float)U[3 * d + 2];
    for (int i = 0; i < 6; ++i) o[LPDF_F_DUDX + i] = (float)g[i];
    for (int i = 0; i < 3; ++i) o[LPDF_F_LAPU + i] = (float)lapU[3 * (size_t)d + i];
    o[LPDF_F_DPDX] = (float)(gp[2 * d] + dpdx0);
    o[LPDF_F_DPDX + 1] = (float)(gp[2 * d + 1] + dpdy0);
    o[LPDF_F_G11] = (float)G11;
    o[LPDF_F_G11 + 1] = (float)G12;
    o[LPDF_F_G11 + 2] = (float)G21;
    o[LPDF_F_G11 + 3] = (float)G22;
    o[LPDF_F_G11 + 4] = (float)G33;
    o[LPDF_F_C0EPS] = (float)c0e;
    o[LPDF_F_OMEGA] = (float)Om;
    o[LPDF_F_SOMEGA] = (float)Som;
    for (int a = 0; a < ns; ++a) o[LPDF_F_PHI0 + a] = (float)phi[(size_t)d * ns + a];
    for (int i = LPDF_F_PHI0 + ns; i < nfp; ++i) o[i] = 0.0f;
}

// ---------------------------------------------------------------- learned-surrogate inputs
// nearest wall point of every geometric node: distance, wall edge and position on it (the edges
// in order, each with its images one period to the left, in place and to the right; the first
// strictly nearest point wins)
__global__ void wall_distance_kernel(int N, const double* __restrict__ xy, const double* __restrict__ seg,
                                     const int* __restrict__ seg_off, const int* __restrict__ ncomp, double period,
                                     double* __restrict__ dist, int* __restrict__ wseg, double* __restrict__ wt)
{
    const int nd = blockIdx.x * blockDim.x + threadIdx.x;
    if (nd >= N) return;
    const double px = xy[2 * nd], py = xy[2 * nd + 1];
    double best = 1e300, bt = 0.0;
    const int c = ncomp[nd], s0 = seg_off[c], s1 = seg_off[c + 1];
    int bs = s0;
    const int ni = period > 0.0 ? 1 : 0;
    for (int s = s0; s < s1; ++s) {
        const double ax = seg[4 * s], ay = seg[4 * s + 1], tx = seg[4 * s + 2] - ax, ty = seg[4 * s + 3] - ay;
        const double tt = tx * tx + ty * ty;
        for (int im = -ni; im <= ni; ++im) {
            const double qx = px - ax - im * period, qy = py - ay;
            const double t = fmin(1.0, fmax(0.0, (qx * tx + qy * ty) / tt));
            const double dx = qx - t * tx, dy = qy - t * ty;
            const double d2 = dx * dx + dy * dy;
            if (d2 < best) {
                best = d2;
                bs = s;
                bt = t;
            }
        }
    }
    dist[nd] = s1 > s0 ? sqrt(best) : 0.0;
    wseg[nd] = bs;
    wt[nd] = bt;
}

// inputs: wall distance, log k, log <omega>, b11, b22, b12, II_b = b_ij b_ij with the anisotropy
// b_ij = <u_i u_j> / (2 k) - delta_ij / 3, and log(eps_w / eps) with eps_w the dissipation
// k <omega> interpolated linearly along the wall edge to the nearest wall point; targets (from node fields): G11, G12, G21,
// G22, G33 over <omega>, C_0 epsilon / (k <omega>) and the relaxed trace wp_ii over its local value
// -9/4 C_0 epsilon (wp_ii = k G_ii + 3 epsilon / 2)
__global__ void features_kernel(const Fem F, const double* __restrict__ stats, int nq,
                                const float* __restrict__ fields, int nfp, double C0, float* __restrict__ feat,
                                float* __restrict__ tgt)
{
    const int nd = blockIdx.x * blockDim.x + threadIdx.x;
    if (nd >= F.N) return;
    const double* st = stats + (size_t)F.dof_node[F.dof[nd]] * nq;
    const double uu = st[4], uv = st[5], uw = st[6], vv = st[7], vw = st[8], ww = st[9], Om = st[10];
    const double k = 0.5 * (uu + vv + ww);
    double eps_w = 0.0;
    const int comp = F.ncomp[nd];
    const bool walls = F.seg_off[comp + 1] > F.seg_off[comp];
    if (walls) {
        const int s = F.wseg[nd];
        const double t = F.wt[nd];
        const double* sa = stats + (size_t)F.dof_node[F.dof[F.segn[2 * s]]] * nq;
        const double* sb = stats + (size_t)F.dof_node[F.dof[F.segn[2 * s + 1]]] * nq;
        const double ea = 0.5 * (sa[4] + sa[7] + sa[9]) * sa[10], eb = 0.5 * (sb[4] + sb[7] + sb[9]) * sb[10];
        eps_w = (1.0 - t) * ea + t * eb;
    }
    double b11 = 0.0, b22 = 0.0, b33 = 0.0, b12 = 0.0, b13 = 0.0, b23 = 0.0;
    if (k > 1e-12) {
        const double ik = 0.5 / k;
        b11 = uu * ik - 1.0 / 3.0;
        b22 = vv * ik - 1.0 / 3.0;
        b33 = ww * ik - 1.0 / 3.0;
        b12 = uv * ik;
        b13 = uw * ik;
        b23 = vw * ik;
    }
    float* f = feat + (size_t)nd * mlp::kIn;
    f[0] = (float)F.wdist[nd];
    f[1] = (float)log(fmax(k, 1e-12));
    f[2] = (float)log(fmax(Om, 1e-12));
    f[3] = (float)b11;
    f[4] = (float)b22;
    f[5] = (float)b12;
    f[6] = (float)(b11 * b11 + b22 * b22 + b33 * b33 + 2.0 * (b12 * b12 + b13 * b13 + b23 * b23));
    f[7] = (float)(walls ? log(fmax(eps_w, 1e-12) / fmax(k * Om, 1e-12)) : 0.0);
    if (!tgt) return;
    const float* o = fields + (size_t)nd * nfp;
    const double Omc = fmax(Om, 1e-12), kc = fmax(k, 1e-12), e = k * Om;
    float* y = tgt + (size_t)nd * mlp::kOut;
    for (int j = 0; j < 5; ++j) y[j] = (float)((double)o[LPDF_F_G11 + j] / Omc);
    y[5] = (float)((double)o[LPDF_F_C0EPS] / (kc * Omc));
    const double tr = k * ((double)o[LPDF_F_G11] + (double)o[LPDF_F_G11 + 3] + (double)o[LPDF_F_G11 + 4]) + 1.5 * e;
    y[6] = (float)(e > 1e-12 ? tr / (-2.25 * C0 * e) : 1.0);
}

// {sum (a - b)^2, sum b^2} over the G_ij and C_0 epsilon columns (one block)
__global__ void fields_compare_kernel(const float* __restrict__ a, const float* __restrict__ b, int N, int nfp,
                                      double* __restrict__ out)
{
    __shared__ double sh[2][1024];
    double d2 = 0.0, b2 = 0.0;
    for (int i = threadIdx.x; i < N * 6; i += blockDim.x) {
        const size_t at = (size_t)(i / 6) * nfp + LPDF_F_G11 + i % 6;
        const double x = a[at], y = b[at];
        d2 += (x - y) * (x - y);
        b2 += y * y;
    }
    sh[0][threadIdx.x] = d2;
    sh[1][threadIdx.x] = b2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sh[0][0];
        out[1] = sh[1][0];
    }
}

}  // namespace

// ------------------------------------------------------------------------- host side

cudaError_t fem_build(const double* node_xy, int N, const int32_t* tri, int E, const int32_t* tag,
                      const std::vector<int32_t>& master, const std::vector<int32_t>& node_comp, double period,
                      Fem** out)
{
    *out = nullptr;
    std::vector<int> dof(N), dof_node;
    std::vector<int> dof_of(N, -1);
    int ndof = 0;
    for (int i = 0; i < N; ++i)
        if (master[i] == i) {
            dof_of[i] = ndof++;
            dof_node.push_back(i);
        }
    for (int i = 0; i < N; ++i) dof[i] = dof_of[master[i]];
    std::vector<int> edof(3 * (size_t)E);
    std::vector<double> area(E), grad(6 * (size_t)E);
    for (int e = 0; e < E; ++e) {
        double x[3], y[3];
        for (int a = 0; a < 3; ++a) {
            edof[3 * e + a] = dof[tri[3 * e + a]];
            x[a] = node_xy[2 * tri[3 * e + a]];
            y[a] = node_xy[2 * tri[3 * e + a] + 1];
        }
        const double det = (x[1] - x[0]) * (y[2] - y[0]) - (y[1] - y[0]) * (x[2] - x[0]);
        area[e] = 0.5 * det;
        for (int a = 0; a < 3; ++a) {
            const int b = (a + 1) % 3, c = (a + 2) % 3;
            grad[6 * e + 2 * a] = (y[b] - y[c]) / det;
            grad[6 * e + 2 * a + 1] = (x[c] - x[b]) / det;
        }
    }
    // DOF -> incident (element, corner) pairs, in element order
    std::vector<int> de_ptr(ndof + 1, 0), de_el(3 * (size_t)E);
    for (int e = 0; e < E; ++e)
        for (int a = 0; a < 3; ++a) ++de_ptr[edof[3 * e + a] + 1];
    for (int d = 0; d < ndof; ++d) de_ptr[d + 1] += de_ptr[d];
    std::vector<double> darea(ndof, 0.0);
    {
        std::vector<int> cur(de_ptr.begin(), de_ptr.end() - 1);
        for (int e = 0; e < E; ++e)
            for (int a = 0; a < 3; ++a) {
                const int d = edof[3 * e + a];
                de_el[cur[d]++] = 3 * e + a;
                darea[d] += area[e];
            }
    }
    // matrix pattern, mass and stiffness matrices, and per-entry contribution lists
    std::vector<std::map<int, std::vector<int>>> rows(ndof);
    for (int e = 0; e < E; ++e)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) rows[edof[3 * e + a]][edof[3 * e + b]].push_back(9 * e + 3 * a + b);
    std::vector<int> row(ndof + 1, 0), col, cptr(1, 0), cel;
    std::vector<double> Mval, Kval;
    for (int i = 0; i < ndof; ++i) {
        for (const auto& kv : rows[i]) {
            col.push_back(kv.first);
            double m = 0.0, kk = 0.0;
            for (int c : kv.second) {
                const int e = c / 9, a = (c / 3) % 3, b = c % 3;
                const double* g = &grad[6 * (size_t)e];
                m += area[e] / 12.0 * (a == b ? 2.0 : 1.0);
                kk += area[e] * (g[2 * a] * g[2 * b] + g[2 * a + 1] * g[2 * b + 1]);
                cel.push_back(c);
            }
            cptr.push_back((int)cel.size());
            Mval.push_back(m);
            Kval.push_back(kk);
        }
        row[i + 1] = (int)col.size();
    }
    // wall DOFs with the averaged inward unit normal (left of each CCW boundary edge)
    std::vector<unsigned char> wall(ndof, 0);
    std::vector<double> normal(2 * (size_t)ndof, 0.0);
    for (int e = 0; e < E; ++e)
        for (int k = 0; k < 3; ++k) {
            const int t = tag[3 * e + k];
            if (t != LPDF_EDGE_WALL && t != LPDF_EDGE_MOVING_WALL) continue;
            const int a = tri[3 * e + k], b = tri[3 * e + (k + 1) % 3];
            const double tx = node_xy[2 * b] - node_xy[2 * a], ty = node_xy[2 * b + 1] - node_xy[2 * a + 1];
            const double len = std::hypot(tx, ty);
            for (int v : {a, b}) {
                const int d = dof[v];
                wall[d] = 1;
                normal[2 * d] += -ty / len;
                normal[2 * d + 1] += tx / len;
            }
        }
    // wall edges grouped by component (components own contiguous element ranges, in order)
    const int n_comp = node_comp.empty() ? 1 : *std::max_element(node_comp.begin(), node_comp.end()) + 1;
    std::vector<double> seg;
    std::vector<int> segn, seg_off(n_comp + 1, 0);
    for (int e = 0; e < E; ++e)
        for (int k = 0; k < 3; ++k) {
            const int t = tag[3 * e + k];
            if (t != LPDF_EDGE_WALL && t != LPDF_EDGE_MOVING_WALL) continue;
            const int a = tri[3 * e + k], b = tri[3 * e + (k + 1) % 3];
            seg.insert(seg.end(), {node_xy[2 * a], node_xy[2 * a + 1], node_xy[2 * b], node_xy[2 * b + 1]});
            segn.insert(segn.end(), {a, b});
            ++seg_off[(node_comp.empty() ? 0 : node_comp[a]) + 1];
        }
    for (int c = 0; c < n_comp; ++c) seg_off[c + 1] += seg_off[c];
    std::vector<int> ncomp_v(N, 0);
    for (int i = 0; i < N && !node_comp.empty(); ++i) ncomp_v[i] = node_comp[i];
    const std::vector<double> xy(node_xy, node_xy + 2 * (size_t)N);
    for (int d = 0; d < ndof; ++d)
        if (wall[d]) {
            const double l = std::hypot(normal[2 * d], normal[2 * d + 1]);
            normal[2 * d] /= l;
            normal[2 * d + 1] /= l;
        }
    Fem* F = new Fem();
    F->ndof = ndof;
    F->nnz = (int)col.size();
    F->E = E;
    F->N = N;
    F->nseg = (int)(seg.size() / 4);
    F->n_comp = n_comp;
    F->period = period;
    if (seg.empty()) {
        seg.assign(4, 0.0);
        segn.assign(2, 0);
    }
    cudaError_t e = cudaSuccess;
    if ((e = upload(&F->dof, dof)) || (e = upload(&F->dof_node, dof_node)) || (e = upload(&F->edof, edof)) ||
        (e = upload(&F->area, area)) || (e = upload(&F->grad, grad)) || (e = upload(&F->de_ptr, de_ptr)) ||
        (e = upload(&F->de_el, de_el)) || (e = upload(&F->darea, darea)) || (e = upload(&F->row, row)) ||
        (e = upload(&F->col, col)) || (e = upload(&F->cptr, cptr)) || (e = upload(&F->cel, cel)) ||
        (e = upload(&F->Mval, Mval)) || (e = upload(&F->Kval, Kval)) || (e = upload(&F->wall, wall)) ||
        (e = upload(&F->normal, normal)) || (e = upload(&F->xy, xy)) || (e = upload(&F->seg, seg)) ||
        (e = upload(&F->segn, segn)) || (e = upload(&F->seg_off, seg_off)) || (e = upload(&F->ncomp, ncomp_v)) || (e = cudaMalloc((void**)&F->wdist, sizeof(double) * std::max(1, N))) ||
        (e = cudaMalloc((void**)&F->wseg, sizeof(int) * std::max(1, N))) ||
        (e = cudaMalloc((void**)&F->wt, sizeof(double) * std::max(1, N))) ||
        (e = cudaMalloc((void**)&F->Aval, sizeof(double) * std::max(1, F->nnz))) ||
        (e = cudaMalloc((void**)&F->work, sizeof(double) * (Fem::kWorkPerDof * (size_t)ndof + 16 * (size_t)E))) ||
        (e = cudaMalloc((void**)&F->part, sizeof(double) * 12 * Fem::kDotBlocks)) ||
        (e = cudaMalloc((void**)&F->scal, sizeof(double) * kNScal)) ||
        (e = cudaMallocHost((void**)&F->scal_host, sizeof(double) * kNScal))) {
        fem_free(F);
        return e;
    }
    *out = F;
    return cudaSuccess;
}

void fem_free(Fem* F)
{
    if (!F) return;
    void* ps[] = {F->dof, F->dof_node, F->edof, F->area, F->grad, F->de_ptr, F->de_el, F->darea, F->row, F->col,
                  F->cptr, F->cel, F->Mval, F->Kval, F->Aval, F->wall, F->normal, F->work, F->part, F->scal,
                  F->xy, F->seg, F->segn, F->seg_off, F->ncomp, F->wdist, F->wseg, F->wt};
    for (void* p : ps) cudaFree(p);
    cudaFreeHost(F->scal_host);
    for (auto& g : F->cg_graphs) cudaGraphExecDestroy(g.exec);
    if (F->capture_stream) cudaStreamDestroy(F->capture_stream);
    delete F;
}

namespace {

void launch_dot(const Fem& F, const double* x, const double* y, int nv, int slot, int mode, cudaStream_t st)
{
    const int nb = (int)std::min<unsigned>(Fem::kDotBlocks, blocks(F.ndof, kDotThreads));
    dot_kernel<<<nb, kDotThreads, 0, st>>>(x, y, F.ndof, nv, F.part + 8 * Fem::kDotBlocks);
    scalar_kernel<<<1, 32, 0, st>>>(F.part + 8 * Fem::kDotBlocks, nb, nv, slot, mode, F.scal);
}

// Jacobi-preconditioned CG on nv <= 4 systems with the same matrix A (diagonal `diag`).
// x holds the start vector, with the fixed values in place on the wall rows when `mask` is set
// (those rows are not solved for). Converged when ||r_c|| <= tol ||r_c(xref)|| for every c, the
// residual of the reference start xref (xref = NULL: x itself); tested on the host every
// kCheckEvery iterations. Five launches per iteration: q = A p with p.q, alpha, the update with
// r.z and r.r, beta, the new direction. Returns cudaErrorNotReady if not converged.
cudaError_t pcg(const Fem& F, const double* A, const double* diag, const double* b, double* x, const double* xref,
                int nv, int mask, double tol, int maxit, int* iters, double* scratch, cudaStream_t st)
{
    const size_t n = F.ndof;
    double* r = scratch;
    double* z = r + 4 * n;
    double* p = z + 4 * n;
    double* q = p + 4 * n;
    const unsigned g = blocks((int64_t)n);
    const int nb = (int)std::min<unsigned>(Fem::kDotBlocks, blocks(F.ndof, kDotThreads));
    double* part_rz = F.part;
    double* part_rr = F.part + 4 * Fem::kDotBlocks;
    if (xref) {
        spmv_kernel<<<g, 256, 0, st>>>(F, A, xref, q, mask, nv);
        cg_start_kernel<<<g, 256, 0, st>>>(F, b, q, diag, r, z, p, mask, nv);
        launch_dot(F, r, r, nv, kR0, 0, st);
    }
    spmv_kernel<<<g, 256, 0, st>>>(F, A, x, q, mask, nv);
    cg_start_kernel<<<g, 256, 0, st>>>(F, b, q, diag, r, z, p, mask, nv);
    if (!xref) launch_dot(F, r, r, nv, kR0, 0, st);
    launch_dot(F, r, r, nv, kRR, 0, st);
    launch_dot(F, r, z, nv, kRZ, 0, st);
    // one CG iteration: five launches (SpMV with the p.q dot, alpha, update with the r.z and r.r
    // dots, beta, new direction)
    auto iteration = [&](cudaStream_t s) {
        spmv_dot_kernel<<<nb, kDotThreads, 0, s>>>(F, A, p, q, mask, nv, F.part);
        scalar_kernel<<<1, 32, 0, s>>>(F.part, nb, nv, kDot, 1, F.scal);          // alpha = rz / pq
        update_dot_kernel<<<nb, kDotThreads, 0, s>>>((int)n, nv, F.scal, diag, p, q, x, r, z, part_rz, part_rr);
        scalar_beta_kernel<<<1, 32, 0, s>>>(part_rz, part_rr, nb, nv, F.scal);    // beta, rz, rr
        cg_direction_kernel<<<g, 256, 0, s>>>((int)n, nv, F.scal, z, p);
    };
    // kCheckEvery iterations between two convergence tests replay one CUDA graph, captured once per
    // call site (the scalars live on the device, so a replay needs no host work)
    cudaGraphExec_t exec = nullptr;
    for (const auto& cg : F.cg_graphs)
        if (cg.key[0] == A && cg.key[1] == diag && cg.key[2] == x && cg.key[3] == scratch && cg.nv == nv &&
            cg.mask == mask)
            exec = cg.exec;
    if (!exec) {
        Fem& Fm = const_cast<Fem&>(F);
        cudaError_t e = cudaSuccess;
        if (!Fm.capture_stream) e = cudaStreamCreateWithFlags(&Fm.capture_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(Fm.capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int k = 0; k < kCheckEvery; ++k) iteration(Fm.capture_stream);
            cudaGraph_t graph = nullptr;
            e = cudaStreamEndCapture(Fm.capture_stream, &graph);
            if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
        }
        if (e != cudaSuccess) return e;
        Fm.cg_graphs.push_back({{A, diag, x, scratch}, nv, mask, exec});
    }
    double r0[4] = {0, 0, 0, 0};
    int it = 0;
    bool done = false;
    for (;;) {
        if (it % kCheckEvery == 0 || it >= maxit) {
            cudaError_t e = cudaMemcpyAsync(F.scal_host, F.scal, sizeof(double) * kNScal, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return e;
            if (it == 0)
                for (int c = 0; c < nv; ++c) r0[c] = std::sqrt(F.scal_host[kR0 + c]);
            done = true;
            for (int c = 0; c < nv; ++c)
                if (std::sqrt(F.scal_host[kRR + c]) > tol * r0[c]) done = false;
            if (done || it >= maxit) break;
        }
        if (it % kCheckEvery == 0 && it + kCheckEvery <= maxit) {
            const cudaError_t e = cudaGraphLaunch(exec, st);
            if (e != cudaSuccess) return e;
            it += kCheckEvery;
        } else {
            iteration(st);
            ++it;
        }
    }
    *iters = it;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return done ? cudaSuccess : cudaErrorNotReady;
}

}  // namespace

cudaError_t node_fields_solve(Fem& F, const double* stats, const lpdf_params& P, float* out, double tol,
                              int maxit, int* iters, cudaStream_t st, const float* surr, const float* surr_norm)
{
    const int ns = P.ns;
    const size_t n = F.ndof;
    const int nq = nquant(ns);
    const int nfp = nfields_padded(ns);
    double* w = F.work;
    double* U = w;      w += 3 * n;
    double* R = w;      w += 6 * n;
    double* om = w;     w += n;
    double* phi = w;    w += (size_t)kMaxNS * n;
    double* k = w;      w += n;
    double* eps = w;    w += n;
    double* gU = w;     w += 6 * n;
    double* lapU = w;   w += 3 * n;
    double* gp = w;     w += 2 * n;
    double* wp = w;     w += 4 * n;
    double* diag = w;   w += n;
    double* rhs = w;    w += 4 * n;
    double* tmp = w;    w += 4 * n;
    double* cgs = w;    w += 16 * n;      // r, z, p, q of the CG
    double* xref = w;   w += 4 * n;       // the zero-interior start (reference of the test)
    double* wp_prev = w; w += 4 * n;      // previous solutions (warm start)
    double* p_prev = w; w += n;
    double* ew = F.work + Fem::kWorkPerDof * n;   // element scratch, 16 per element
    const unsigned gd = blocks((int64_t)n), ge = blocks(F.E);
    iters[0] = iters[1] = 0;
    dof_stats_kernel<<<gd, 256, 0, st>>>(F, stats, nq, ns, U, R, om, phi, k, eps);
    // recovered gradients of the mean velocity, then their recovered divergences
    elem_grad_kernel<<<ge, 256, 0, st>>>(F, U, 3, 3, ew);
    recover_kernel<<<gd, 256, 0, st>>>(F, ew, 6, gU, 6);
    for (int i = 0; i < 3; ++i) {
        elem_div_kernel<<<ge, 256, 0, st>>>(F, gU + 2 * i, 6, ew);
        recover_kernel<<<gd, 256, 0, st>>>(F, ew, 1, lapU + i, 3);
    }
    if (P.gmodel == 0 && !surr) {
        elem_L2_kernel<<<ge, 256, 0, st>>>(F, k, eps, P.CL, P.Ceta, P.nu, ew);
        assemble_kernel<<<gd, 256, 0, st>>>(F, ew, F.Aval, diag);
        const bool warm = P.cg_warm_start && F.has_wp;
        er_setup_kernel<<<gd, 256, 0, st>>>(F, eps, P.C0, tmp, wp, warm ? wp_prev : nullptr, xref);
        spmv_kernel<<<gd, 256, 0, st>>>(F, F.Mval, tmp, rhs, 0, 4);     // b = M wp^h
        cudaError_t e = pcg(F, F.Aval, diag, rhs, wp, xref, 4, 1, tol, maxit, &iters[0], cgs, st);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(wp_prev, wp, sizeof(double) * 4 * n, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        F.has_wp = true;
    }
    if (P.pressure_solve) {
        pressure_T_kernel<<<gd, 256, 0, st>>>(F, U, R, tmp);
        elem_grad_kernel<<<ge, 256, 0, st>>>(F, tmp, 4, 4, ew);
        pressure_rhs_kernel<<<gd, 256, 0, st>>>(F, ew, rhs);
        diag_kernel<<<gd, 256, 0, st>>>(F, F.Kval, diag);
        double* p = tmp;
        const bool warm = P.cg_warm_start && F.has_p;
        if (warm) {
            cudaError_t e = cudaMemcpyAsync(p, p_prev, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return e;
        } else {
            fill_kernel<<<gd, 256, 0, st>>>((int)n, 0.0, p);
        }
        // consistent singular system (the right-hand side sums to zero): CG stays in the range up
        // to rounding; the constant is removed afterwards. Reference start: zero.
        fill_kernel<<<gd, 256, 0, st>>>((int)n, 0.0, xref);
        cudaError_t e = pcg(F, F.Kval, diag, rhs, p, warm ? xref : nullptr, 1, 0, tol, maxit, &iters[1], cgs, st);
        if (e != cudaSuccess) return e;
        double* ones = rhs + n;
        fill_kernel<<<gd, 256, 0, st>>>((int)n, 1.0, ones);
        launch_dot(F, p, ones, 1, kDot, 0, st);
        subtract_mean_kernel<<<gd, 256, 0, st>>>((int)n, F.scal + kDot, p);
        e = cudaMemcpyAsync(p_prev, p, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        F.has_p = true;
        elem_grad_kernel<<<ge, 256, 0, st>>>(F, p, 1, 1, ew);
        recover_kernel<<<gd, 256, 0, st>>>(F, ew, 2, gp, 2);
    } else {
        fill_kernel<<<blocks(2 * (int64_t)n), 256, 0, st>>>(2 * (int)n, 0.0, gp);
    }
    fields_kernel<<<blocks(F.N), 256, 0, st>>>(F, ns, nfp, U, R, om, phi, k, eps, gU, lapU, gp, wp, P.gmodel, P.C0,
                                               P.Comega1, P.Comega2, P.dpdx0, P.dpdy0, surr, surr_norm, out);
    return cudaGetLastError();
}

cudaError_t surrogate_features(Fem& F, const double* stats, int ns, const float* fields, double C0, float* feat,
                               float* tgt, cudaStream_t st)
{
    if (!F.has_wdist) {
        wall_distance_kernel<<<blocks(F.N), 256, 0, st>>>(F.N, F.xy, F.seg, F.seg_off, F.ncomp, F.period, F.wdist,
                                                          F.wseg, F.wt);
        F.has_wdist = true;
    }
    features_kernel<<<blocks(F.N), 256, 0, st>>>(F, stats, nquant(ns), fields, nfields_padded(ns), C0, feat,
                                                 fields ? tgt : nullptr);
    return cudaGetLastError();
}

cudaError_t fields_compare(const float* a, const float* b, int n_nodes, int nfp, double* out2, cudaStream_t st)
{
    fields_compare_kernel<<<1, 1024, 0, st>>>(a, b, n_nodes, nfp, out2);
    return cudaGetLastError();
}

}  // namespace lpdf
