"""FP64 oracle of the gridpoint side: node fields from gridpoint statistics.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). numpy/scipy, no code shared with the CUDA
path. What it computes (arXiv:1006.0549):

* the grid solves for the Eulerian quantities (Introduction, item ii): the mean pressure by a
  projection on the grid (Section "Governing equations", summary paragraph);
* G_ij from an elliptic relaxation equation whose wall effect enters only through its boundary
  conditions and which blends into a local model away from walls (the paragraph after Eq. 4);
* epsilon = k <omega>, k = <u_i u_i>/2 (the paragraph before Eq. 5), P = -<u_i u_j> d<U_i>/dx_j
  and S_omega = C_omega2 - C_omega1 P/epsilon (Eq. 6).

Readings where the paper is silent (the cited works are not at hand):
* gradients of P1 fields are recovered at nodes by area-weighted averaging of the element
  gradients; the Laplacian is the recovered divergence of the recovered gradient;
* elliptic relaxation: wp_ij - L^2 lap(wp_ij) = wp^h_ij with the local (simplified-Langevin)
  model wp^h_ij = -3/4 C0 eps delta_ij, L = CL max(k^1.5/eps, Ceta nu^0.75/eps^0.25), wall values
  wp_ij = -4.5 eps n_i n_j; G_ij = (wp_ij - eps delta_ij / 2)/k; C0 eps from the k-consistency
  condition C0 eps = -2/3 (eps + <u_i u_j> G_ij) (clipped at 0). Discretised with P1 finite
  elements: (M + K_L) wp = M wp^h, L^2 averaged over each element's nodes;
* mean pressure: lap p = -d_i d_j (<U_i><U_j> + <u_i u_j>) in weak form with its natural boundary
  condition and zero mean; a fixed mean gradient (dpdx0, dpdy0) is added (the channel is driven
  by d<P>/dx = -1).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# statistics columns (lpdf_grid_statistics, raw = 0)
S0, MU, MV, MW, RUU, RUV, RUW, RVV, RVW, RWW, OM = range(11)
EPS_MIN = 1e-12
K_MIN = 1e-12


class Geometry:
    """Element areas and shape-function gradients, periodic DOF numbering, wall DOFs and normals."""

    def __init__(self, mesh):
        xy = mesh.node_xy
        tri = mesh.tri
        self.mesh = mesh
        N = xy.shape[0]
        master = np.arange(N)
        if mesh.period_x > 0:
            x0, x1 = mesh.box[0], mesh.box[1]
            left = {float(xy[i, 1]): i for i in np.nonzero(xy[:, 0] == x0)[0]}
            for i in np.nonzero(xy[:, 0] == x1)[0]:
                master[i] = left[float(xy[i, 1])]
        uniq = np.unique(master)
        self.dof_of_master = -np.ones(N, dtype=np.int64)
        self.dof_of_master[uniq] = np.arange(len(uniq))
        self.dof = self.dof_of_master[master]          # geometric node -> DOF
        self.ndof = len(uniq)
        self.master = master
        p0, p1, p2 = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
        det = (p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p1[:, 1] - p0[:, 1]) * (p2[:, 0] - p0[:, 0])
        self.area = 0.5 * det
        # grad lambda_a = (y_b - y_c, x_c - x_b) / det for (a, b, c) cyclic
        g = np.zeros((tri.shape[0], 3, 2))
        P = [p0, p1, p2]
        for a in range(3):
            b, c = P[(a + 1) % 3], P[(a + 2) % 3]
            g[:, a, 0] = (b[:, 1] - c[:, 1]) / det
            g[:, a, 1] = (c[:, 0] - b[:, 0]) / det
        self.grad = g
        self.edof = self.dof[tri]                       # (E, 3)
        # wall DOFs (edges tagged 1 or 2) with the averaged inward unit normal
        wall = np.zeros(self.ndof, dtype=bool)
        normal = np.zeros((self.ndof, 2))
        for e in range(tri.shape[0]):
            for k in range(3):
                if mesh.edge_tag[e, k] in (1, 2):
                    a, b = tri[e, k], tri[e, (k + 1) % 3]
                    t = xy[b] - xy[a]
                    n = np.array([-t[1], t[0]]) / np.hypot(*t)   # left of a->b = inward (CCW)
                    for v in (a, b):
                        wall[self.dof[v]] = True
                        normal[self.dof[v]] += n
        nn = np.linalg.norm(normal, axis=1)
        normal[wall] /= nn[wall, None]
        self.wall = wall
        self.normal = normal

    def dof_values(self, node_values):
        """Per-DOF values from per-geometric-node values (the master's row)."""
        out = np.zeros((self.ndof,) + node_values.shape[1:])
        out[self.dof] = node_values
        return out


def element_gradient(geo: Geometry, f):
    """Gradient of the P1 interpolant of DOF values f on every element: (E, 2)."""
    return np.einsum("ea,ead->ed", f[geo.edof], geo.grad)


def recover(geo: Geometry, elem_values):
    """Area-weighted average of element values to DOFs."""
    num = np.zeros((geo.ndof,) + elem_values.shape[1:])
    den = np.zeros(geo.ndof)
    for a in range(3):
        np.add.at(num, geo.edof[:, a], geo.area.reshape((-1,) + (1,) * (elem_values.ndim - 1)) * elem_values)
        np.add.at(den, geo.edof[:, a], geo.area)
    return num / den.reshape((-1,) + (1,) * (elem_values.ndim - 1))


def recover_gradient(geo: Geometry, f):
    return recover(geo, element_gradient(geo, f))


def recover_laplacian(geo: Geometry, f):
    g = recover_gradient(geo, f)
    div = element_gradient(geo, g[:, 0])[:, 0] + element_gradient(geo, g[:, 1])[:, 1]
    return recover(geo, div)


def assemble(geo: Geometry, coef_elem=None):
    """P1 mass matrix M and stiffness K (with an element coefficient for K), on the DOFs."""
    E = geo.edof.shape[0]
    rows, cols, mv, kv = [], [], [], []
    coef = np.ones(E) if coef_elem is None else coef_elem
    for a in range(3):
        for b in range(3):
            rows.append(geo.edof[:, a])
            cols.append(geo.edof[:, b])
            mv.append(geo.area / 12.0 * (2.0 if a == b else 1.0))
            kv.append(coef * geo.area * (geo.grad[:, a, 0] * geo.grad[:, b, 0] + geo.grad[:, a, 1] * geo.grad[:, b, 1]))
    r, c = np.concatenate(rows), np.concatenate(cols)
    M = sp.csr_matrix((np.concatenate(mv), (r, c)), shape=(geo.ndof, geo.ndof))
    K = sp.csr_matrix((np.concatenate(kv), (r, c)), shape=(geo.ndof, geo.ndof))
    return M, K


def solve_dirichlet(A, b, wall, g):
    """Solve A x = b with x = g on wall DOFs (symmetric elimination), sparse direct."""
    inner = ~wall
    x = np.zeros(A.shape[0])
    x[wall] = g[wall]
    rhs = b[inner] - A[inner][:, wall] @ g[wall]
    x[inner] = spla.spsolve(A[inner][:, inner].tocsc(), rhs)
    return x


def elliptic_relaxation(geo: Geometry, k, eps, C0, CL, Ceta, nu):
    """wp_ij for ij = 11, 12, 22, 33 (DOF arrays) from the P1 Helmholtz problem."""
    epsc = np.maximum(eps, EPS_MIN)
    L = CL * np.maximum(np.maximum(k, 0.0) ** 1.5 / epsc, Ceta * nu ** 0.75 / epsc ** 0.25)
    L2e = np.mean((L ** 2)[geo.edof], axis=1)
    M, K = assemble(geo, L2e)
    A = (M + K).tocsr()
    src = -0.75 * C0 * eps
    n1, n2 = geo.normal[:, 0], geo.normal[:, 1]
    out = {}
    for name, s, bc in (("11", src, -4.5 * eps * n1 * n1), ("12", 0.0 * src, -4.5 * eps * n1 * n2),
                        ("22", src, -4.5 * eps * n2 * n2), ("33", src, 0.0 * eps)):
        out[name] = solve_dirichlet(A, M @ s, geo.wall, bc)
    return out


def pressure(geo: Geometry, U, R):
    """Mean pressure (zero mean): weak form of lap p = -d_i d_j T_ij, T = <U><U> + <uu> (planar)."""
    T = np.zeros((geo.ndof, 2, 2))
    T[:, 0, 0] = U[:, 0] * U[:, 0] + R[:, 0]
    T[:, 0, 1] = T[:, 1, 0] = U[:, 0] * U[:, 1] + R[:, 1]
    T[:, 1, 1] = U[:, 1] * U[:, 1] + R[:, 3]
    # element divergence of the P1 tensor field: (div T)_i = sum_j d_j T_ij
    dT = np.zeros((geo.edof.shape[0], 2))
    for i in range(2):
        for j in range(2):
            dT[:, i] += element_gradient(geo, T[:, i, j])[:, j]
    b = np.zeros(geo.ndof)
    for a in range(3):
        np.add.at(b, geo.edof[:, a], -geo.area * (geo.grad[:, a, 0] * dT[:, 0] + geo.grad[:, a, 1] * dT[:, 1]))
    _, K = assemble(geo)
    # pure Neumann: pin DOF 0, then remove the mean
    inner = np.ones(geo.ndof, dtype=bool)
    inner[0] = False
    p = np.zeros(geo.ndof)
    p[inner] = spla.spsolve(K[inner][:, inner].tocsc(), b[inner])
    return p - p.mean()


def node_fields(mesh, stats, ns, C0=2.1, Comega1=0.5, Comega2=0.73, CL=0.134, Ceta=72.0, nu=1.0 / 180.0,
                gmodel=0, pressure_solve=0, dpdx0=0.0, dpdy0=0.0, return_parts=False):
    """(N, nfp) float64 node fields from per-node statistics (means and central moments)."""
    geo = Geometry(mesh)
    st = geo.dof_values(np.asarray(stats, dtype=np.float64))
    U = st[:, MU:MW + 1]
    R = st[:, RUU:RWW + 1]       # uu, uv, uw, vv, vw, ww
    Om = st[:, OM]
    k = 0.5 * (R[:, 0] + R[:, 3] + R[:, 5])
    eps = k * Om
    gU = [recover_gradient(geo, U[:, i]) for i in range(3)]
    lU = [recover_laplacian(geo, U[:, i]) for i in range(3)]
    prod = -(R[:, 0] * gU[0][:, 0] + R[:, 1] * gU[0][:, 1] + R[:, 1] * gU[1][:, 0] + R[:, 3] * gU[1][:, 1]
             + R[:, 2] * gU[2][:, 0] + R[:, 4] * gU[2][:, 1])
    Som = np.where(eps > EPS_MIN, Comega2 - Comega1 * prod / np.maximum(eps, EPS_MIN), Comega2)
    kc = np.maximum(k, K_MIN)
    if gmodel == 1:
        a = -(0.5 + 0.75 * C0) * Om
        G11 = G22 = G33 = a
        G12 = np.zeros_like(a)
        c0e = C0 * eps
        parts = {}
    else:
        wp = elliptic_relaxation(geo, k, eps, C0, CL, Ceta, nu)
        G11 = (wp["11"] - 0.5 * eps) / kc
        G22 = (wp["22"] - 0.5 * eps) / kc
        G33 = (wp["33"] - 0.5 * eps) / kc
        G12 = wp["12"] / kc
        c0e = np.maximum(0.0, -2.0 / 3.0 * (eps + R[:, 0] * G11 + 2.0 * R[:, 1] * G12 + R[:, 3] * G22 + R[:, 5] * G33))
        parts = wp
    if pressure_solve:
        p = pressure(geo, U, R)
        gp = recover_gradient(geo, p)
    else:
        p = np.zeros(geo.ndof)
        gp = np.zeros((geo.ndof, 2))
    nfp = (22 + ns + 3) // 4 * 4
    F = np.zeros((geo.ndof, nfp))
    F[:, 0:3] = U
    F[:, 3] = gU[0][:, 0]; F[:, 4] = gU[0][:, 1]
    F[:, 5] = gU[1][:, 0]; F[:, 6] = gU[1][:, 1]
    F[:, 7] = gU[2][:, 0]; F[:, 8] = gU[2][:, 1]
    F[:, 9] = lU[0]; F[:, 10] = lU[1]; F[:, 11] = lU[2]
    F[:, 12] = gp[:, 0] + dpdx0
    F[:, 13] = gp[:, 1] + dpdy0
    F[:, 14] = G11; F[:, 15] = G12; F[:, 16] = G12; F[:, 17] = G22; F[:, 18] = G33
    F[:, 19] = c0e
    F[:, 20] = Om
    F[:, 21] = Som
    for a in range(ns):
        F[:, 22 + a] = st[:, 11 + a]
    out = F[geo.dof]
    if return_parts:
        return out, dict(geo=geo, k=k, eps=eps, p=p, **parts)
    return out


# ---------------------------------------------------------------------------------- IECM (Eq. 9)

def flux_covariances(stats_raw, flux_raw, ns):
    """<u_i psi_a> - <u_i><psi_a> per node from raw sums (S_0, S_u, S_v, S_w, ..., S_psi) and the
    raw flux sums (u psi_a, v psi_a, w psi_a per scalar); zeros where S_0 = 0."""
    S = np.asarray(stats_raw, dtype=np.float64)
    Fx = np.asarray(flux_raw, dtype=np.float64)
    out = np.zeros_like(Fx)
    s0 = S[:, 0]
    ok = s0 != 0.0
    for a in range(ns):
        mpsi = np.where(ok, S[:, 11 + a] / np.where(ok, s0, 1.0), 0.0)
        for c in range(3):
            mu = np.where(ok, S[:, 1 + c] / np.where(ok, s0, 1.0), 0.0)
            out[:, 3 * a + c] = np.where(ok, Fx[:, 3 * a + c] / np.where(ok, s0, 1.0) - mu * mpsi, 0.0)
    return out


def iecm_coefficients(stats, flux, ns):
    """beta_a = R^-1 c_a per node: R the Reynolds-stress tensor (statistics columns uu, uv, uw, vv,
    vw, ww), c_a the scalar flux <u_i psi_a'>; beta = 0 where det R <= 1e-12 (trace R / 3)^3. The
    conditional mean of Eq. 9 is then read as <phi_a|V> = <phi_a> + beta_a . (V - <U>), the
    conditional expectation of jointly Gaussian velocity and scalar."""
    st = np.asarray(stats, dtype=np.float64)
    c = np.asarray(flux, dtype=np.float64)
    N = st.shape[0]
    R = np.empty((N, 3, 3))
    R[:, 0, 0], R[:, 0, 1], R[:, 0, 2] = st[:, RUU], st[:, RUV], st[:, RUW]
    R[:, 1, 0], R[:, 1, 1], R[:, 1, 2] = st[:, RUV], st[:, RVV], st[:, RVW]
    R[:, 2, 0], R[:, 2, 1], R[:, 2, 2] = st[:, RUW], st[:, RVW], st[:, RWW]
    det = np.linalg.det(R)
    tr = np.trace(R, axis1=1, axis2=2) / 3.0
    ok = det > 1e-12 * np.maximum(tr, 0.0) ** 3
    beta = np.zeros((N, 3 * ns))
    for a in range(ns):
        rhs = c[:, 3 * a:3 * a + 3]
        sol = np.zeros((N, 3))
        if ok.any():
            sol[ok] = np.linalg.solve(R[ok], rhs[ok][:, :, None])[:, :, 0]
        beta[:, 3 * a:3 * a + 3] = sol
    return beta

