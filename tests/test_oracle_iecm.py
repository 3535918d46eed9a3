"""Pins of the oracle's IECM micromixing and reactive source (Eq. 9) and of its gridpoint
estimate of the conditional mean (the linear, joint-Gaussian reading)."""
import numpy as np
import pytest

import oracle
from oracle import fields as of
from paper_1006_0549_gb300 import workloads as wl


def _uniform_fields(mesh, ns, U=(1.0, -0.5, 0.25), phi=0.3, omega=1.0):
    F = np.zeros((mesh.n_nodes, wl.n_fields_padded(ns)), dtype=np.float32)
    F[:, wl.F_U], F[:, wl.F_V], F[:, wl.F_W] = U
    F[:, wl.F_OMEGA] = omega
    for a in range(ns):
        F[:, wl.F_PHI0 + a] = phi + 0.1 * a
    return F


def _state(mesh, ns, seed, n_per_elem=20):
    st = wl.synthetic_state(mesh, n_per_elem, ns, seed=seed)
    return st


def test_iecm_with_zero_coefficients_is_iem():
    mesh = wl.cavity_mesh(6, 6, 1)
    om = oracle.OracleMesh(mesh)
    st = _state(mesh, 2, 3)
    F = wl.synthetic_node_fields(mesh, 2, seed=4)
    p = oracle.make_params(nu=1e-4, dt=1e-3, seed=5, ns=2)
    r0, e0, _, _ = oracle.pdf_step(om, p, F, st, 1)
    r1, e1, _, _ = oracle.pdf_step(om, p, F, st, 1, beta=np.zeros((mesh.n_nodes, 6), np.float32))
    assert np.array_equal(e0, e1)
    for k in r0:
        assert np.array_equal(r0[k], r1[k]), k


def test_iecm_keeps_a_scalar_that_is_linear_in_the_velocity():
    """psi = <phi> + gamma . (U - <U>) for every particle: it already equals its conditional mean,
    so IECM with beta = gamma leaves it in place while IEM pulls it toward <phi>."""
    mesh = wl.cavity_mesh(6, 6, 2)
    om = oracle.OracleMesh(mesh)
    st = _state(mesh, 1, 6)
    Ubar = np.array([1.0, -0.5, 0.25])
    gamma = np.array([0.2, -0.35, 0.1])
    F = _uniform_fields(mesh, 1, U=tuple(Ubar), phi=0.3)
    Ud = np.stack([st.u, st.v, st.w], axis=1).astype(np.float64) - Ubar
    st.psi[0] = (0.3 + Ud @ gamma).astype(np.float32)
    beta = np.tile(gamma.astype(np.float32), (mesh.n_nodes, 1))
    p = oracle.make_params(nu=1e-4, dt=1e-3, seed=7, ns=1, Cphi=2.0)
    r_iecm, _, _, _ = oracle.pdf_step(om, p, F, st, 1, beta=beta)
    r_iem, _, _, _ = oracle.pdf_step(om, p, F, st, 1)
    psi0 = st.psi[0].astype(np.float64)
    mix = 0.5 * 2.0 * 1.0 * 1e-3
    assert np.max(np.abs(r_iecm["psi"][0] - psi0)) < 1e-9
    phibar = float(np.float32(0.3))
    assert np.allclose(r_iem["psi"][0], psi0 - (psi0 - phibar) * mix, rtol=1e-12, atol=1e-12)


def test_coefficients_recover_the_slope_of_a_linear_scalar():
    rng = np.random.default_rng(1)
    N = 50
    A = rng.standard_normal((N, 3, 3))
    R = A @ np.transpose(A, (0, 2, 1)) + 0.1 * np.eye(3)
    gamma = rng.standard_normal((N, 2, 3))
    st = np.zeros((N, 11 + 2 * 2))
    st[:, 4], st[:, 5], st[:, 6] = R[:, 0, 0], R[:, 0, 1], R[:, 0, 2]
    st[:, 7], st[:, 8], st[:, 9] = R[:, 1, 1], R[:, 1, 2], R[:, 2, 2]
    c = np.einsum("nij,naj->nai", R, gamma).reshape(N, 6)
    beta = of.iecm_coefficients(st, c, 2)
    assert np.allclose(beta, gamma.reshape(N, 6), rtol=1e-10, atol=1e-12)
    # a degenerate (zero) stress tensor gives no correlation
    st[0, 4:10] = 0.0
    assert np.all(of.iecm_coefficients(st, c, 2)[0] == 0.0)


def test_flux_covariance_of_a_scalar_linear_in_u():
    """psi = a + b u on every particle: cov(u, psi) = b var(u) and cov(v, psi) = b cov(u, v) at
    every node, from the oracle's moment sums and flux sums (two independent reductions)."""
    mesh = wl.channel_mesh(8, 6, 3)
    om = oracle.OracleMesh(mesh)
    st = _state(mesh, 1, 9, n_per_elem=12)
    b = 0.7
    psi = (0.2 + b * st.u.astype(np.float64))
    x, y, u, v, w = (getattr(st, k).astype(np.float64) for k in ("x", "y", "u", "v", "w"))
    S, _ = oracle.moments(om, 1, x, y, u, v, w, st.omega.astype(np.float64), psi[None, :], st.elem)
    Fx = oracle.flux_moments(om, 1, x, y, u, v, w, psi[None, :], st.elem)
    cov = of.flux_covariances(S, Fx, 1)
    stats = oracle.grid_statistics(S, 1)
    assert np.allclose(cov[:, 0], b * stats[:, 4], rtol=1e-9, atol=1e-12)
    assert np.allclose(cov[:, 1], b * stats[:, 5], rtol=1e-9, atol=1e-12)
    assert np.allclose(cov[:, 2], b * stats[:, 6], rtol=1e-9, atol=1e-12)


def test_second_order_reaction_follows_the_euler_map():
    """psi_0 + psi_1 -> psi_2 at rate k without mixing: every particle follows
    c_{n+1} = c_n - k c_n^2 dt from c_0, with psi_0 + psi_2 conserved; the map converges to the
    exact c_0 / (1 + k c_0 t) as dt -> 0."""
    mesh = wl.cavity_mesh(5, 5, 4)
    om = oracle.OracleMesh(mesh)
    st = _state(mesh, 3, 10, n_per_elem=4)
    c0, k, dt = 0.8, 5.0, 1e-3
    st.psi[:] = np.array([[c0], [c0], [0.0]], dtype=np.float32)
    F = _uniform_fields(mesh, 3)
    p = oracle.make_params(nu=1e-4, dt=dt, seed=11, ns=3, Cphi=0.0, react=(k, 0, 1, 2))
    c = c0
    for n in range(20):
        res, elem, _, _ = oracle.pdf_step(om, p, F, st, n)
        c = np.float32(c - k * c * c * dt)        # the FP32 state carried from step to step
        assert np.allclose(res["psi"][0], c, rtol=2e-6)
        assert np.allclose(res["psi"][0] + res["psi"][2], c0, rtol=2e-6)
        st = wl.State(*(res[q].astype(np.float32) for q in ("x", "y", "u", "v", "w", "omega")),
                      res["psi"].astype(np.float32), elem, st.pid)
    t = 20 * dt
    assert abs(float(c) - c0 / (1 + k * c0 * t)) < 2 * k * c0 * c0 * dt
