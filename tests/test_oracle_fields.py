"""Pins of the gridpoint-side oracle (oracle/fields.py) against closed forms."""

import numpy as np

from oracle import fields as of
from paper_1006_0549_gb300 import workloads as wl


def _stats(mesh, U=None, R=None, Om=1.0, phi=0.0, ns=1):
    N = mesh.n_nodes
    st = np.zeros((N, 11 + 2 * ns))
    st[:, 0] = 1.0
    if U is not None:
        st[:, 1:4] = U
    if R is not None:
        st[:, 4:10] = R
    st[:, 10] = Om
    st[:, 11:11 + ns] = phi
    return st


def test_recovered_gradient_and_laplacian_of_linear_fields_are_exact():
    mesh = wl.cavity_mesh(14, 11, 3)
    geo = of.Geometry(mesh)
    xy = geo.dof_values(mesh.node_xy)
    f = 2.0 - 3.0 * xy[:, 0] + 0.5 * xy[:, 1]
    g = of.recover_gradient(geo, f)
    assert np.allclose(g[:, 0], -3.0, atol=1e-10) and np.allclose(g[:, 1], 0.5, atol=1e-10)
    assert np.allclose(of.recover_laplacian(geo, f), 0.0, atol=1e-8)


def test_recovered_laplacian_of_a_quadratic_converges_to_4_in_the_mean():
    """lap(x^2 + y^2) = 4. Averaging recovery is not pointwise consistent on meshes with mixed
    diagonals (about 10 % scatter), but its area-weighted mean over the interior converges."""
    means = []
    for n in (16, 32, 64):
        mesh = wl.cavity_mesh(n, n, 5, jitter=0.1)
        geo = of.Geometry(mesh)
        xy = geo.dof_values(mesh.node_xy)
        lap = of.recover_laplacian(geo, xy[:, 0] ** 2 + xy[:, 1] ** 2)
        interior = (xy[:, 0] > 0.2) & (xy[:, 0] < 0.8) & (xy[:, 1] > 0.2) & (xy[:, 1] < 0.8)
        w = np.zeros(geo.ndof)
        for a in range(3):
            np.add.at(w, geo.edof[:, a], geo.area / 3.0)
        means.append(np.sum(lap[interior] * w[interior]) / np.sum(w[interior]))
    err = [abs(m - 4.0) for m in means]
    assert err[2] < err[1] < err[0] and err[2] < 0.01


def test_elliptic_relaxation_matches_the_1d_closed_form_in_the_channel():
    """k = eps = 1 everywhere gives a constant L = C_L; the x-independent problem
    psi - L^2 psi'' = f, psi(0) = psi(2) = psi_w, has psi = f + (psi_w - f) cosh((y-1)/L)/cosh(1/L)."""
    mesh = wl.channel_mesh(60, 80, 2, jitter=0.0)
    geo = of.Geometry(mesh)
    k = np.ones(geo.ndof)
    eps = np.ones(geo.ndof)
    C0, CL = 2.1, 0.134
    wp = of.elliptic_relaxation(geo, k, eps, C0, CL, 72.0, 1e-6)
    y = geo.dof_values(mesh.node_xy)[:, 1]
    f = -0.75 * C0
    for name, psi_w in (("22", -4.5), ("11", 0.0), ("33", 0.0)):
        exact = f + (psi_w - f) * np.cosh((y - 1.0) / CL) / np.cosh(1.0 / CL)
        assert np.max(np.abs(wp[name] - exact)) < 0.02 * abs(psi_w - f) + 1e-12, name
    assert np.max(np.abs(wp["12"])) < 1e-12


def test_vanishing_length_scale_gives_the_simplified_langevin_model():
    """C_L = 0: wp = wp^h = -3/4 C0 eps away from the walls, so G_ij = -(1/2 + 3/4 C0) <omega> delta_ij
    (the simplified Langevin model) and, for isotropic stresses <u_i u_j> = 2k/3 delta_ij, the
    k-consistency condition returns C0 eps."""
    mesh = wl.channel_mesh(20, 24, 3)
    N = mesh.n_nodes
    k0, Om, C0 = 1.5, 4.0, 2.1
    R = np.zeros((N, 6))
    R[:, 0] = R[:, 3] = R[:, 5] = 2.0 * k0 / 3.0
    st = _stats(mesh, U=np.zeros((N, 3)), R=R, Om=Om)
    F, parts = of.node_fields(mesh, st, 1, C0=C0, CL=0.0, gmodel=0, return_parts=True)
    y = mesh.node_xy[:, 1]
    far = (y > 0.3) & (y < 1.7)
    a = -(0.5 + 0.75 * C0) * Om
    # the wall values reach the interior only through the (exponentially decaying) inverse of the
    # consistent mass matrix
    assert np.allclose(F[far, wl.F_G11], a, rtol=1e-3) and np.allclose(F[far, wl.F_G33], a, rtol=1e-3)
    assert np.allclose(F[far, wl.F_G12], 0.0, atol=1e-3 * abs(a))
    assert np.allclose(F[far, wl.F_C0EPS], C0 * k0 * Om, rtol=1e-3)


def test_pressure_of_an_isotropic_stress_field_is_its_negative():
    """U = 0, <u_i u_j> = g delta_ij: div T = grad g, so the weak Poisson problem gives p = -g + c
    exactly in the P1 space."""
    mesh = wl.cavity_mesh(20, 18, 7)
    geo = of.Geometry(mesh)
    xy = geo.dof_values(mesh.node_xy)
    g = np.sin(3 * xy[:, 0]) * np.cos(2 * xy[:, 1]) + xy[:, 0] * xy[:, 1]
    R = np.zeros((geo.ndof, 6))
    R[:, 0] = R[:, 3] = g
    p = of.pressure(geo, np.zeros((geo.ndof, 3)), R)
    d = p + g
    assert np.max(np.abs(d - d.mean())) < 1e-9


def test_production_and_frequency_source_of_a_linear_shear():
    """U = (gamma y, 0, 0), <u v> = -tau: P = tau gamma, S_omega = C_omega2 - C_omega1 P / eps."""
    mesh = wl.cavity_mesh(10, 10, 1)
    N = mesh.n_nodes
    gamma, tau, Om = 3.0, 0.4, 2.0
    U = np.zeros((N, 3))
    U[:, 0] = gamma * mesh.node_xy[:, 1]
    R = np.zeros((N, 6))
    R[:, 0], R[:, 1], R[:, 3], R[:, 5] = 1.0, -tau, 0.8, 0.6
    st = _stats(mesh, U=U, R=R, Om=Om)
    F = of.node_fields(mesh, st, 1, gmodel=1)
    eps = 0.5 * (1.0 + 0.8 + 0.6) * Om
    assert np.allclose(F[:, wl.F_DUDY], gamma, atol=1e-10)
    assert np.allclose(F[:, wl.F_SOMEGA], 0.73 - 0.5 * tau * gamma / eps, atol=1e-10)
    assert np.allclose(F[:, wl.F_LAPU], 0.0, atol=1e-8)


def test_periodic_duplicates_carry_identical_fields():
    mesh = wl.channel_mesh(12, 10, 4)
    rng = np.random.default_rng(0)
    geo = of.Geometry(mesh)
    st_dof = np.abs(rng.standard_normal((geo.ndof, 13))) + 0.5
    st = st_dof[geo.dof]
    F = of.node_fields(mesh, st, 1, gmodel=0)
    right = np.nonzero(mesh.node_xy[:, 0] == mesh.period_x)[0]
    assert np.array_equal(F[right], F[geo.master[right]])
