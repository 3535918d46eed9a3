"""Taylor dispersion in stationary homogeneous turbulence under the simplified Langevin model: a
whole-method check of Eq. 4 and Eq. 2 together.

Uniform node fields: <U> = 0, no gradients, G_ij = -a delta_ij with a = (1/2 + 3/4 C0) <omega>,
C0 eps = C0 k <omega>, nu = 0. Each velocity component is then an Ornstein-Uhlenbeck process and
Eq. 2 integrates it with the velocity at t_n. Started from the discrete stationary variance
sigma^2 = b^2 dt / (1 - rho^2) (b^2 = C0 eps, rho = 1 - a dt), the displacement variance after n
steps is exactly dt^2 sigma^2 sum_{i,j<n} rho^|i-j|, which tends to Taylor's
2 <v^2> T_L^2 (t/T_L - 1 + exp(-t/T_L)), T_L = 1/a, as dt -> 0. Particles start in a band
away from the walls (no reflection within the test time); the tolerance is five standard errors
of a sample variance, sqrt(2/N)."""
import numpy as np
import pytest

import oracle
from paper_1006_0549_gb300 import lpdf, workloads as wl
from tests import gpu_common as gc

C0, K, OMEGA, DT = 2.1, 1.5, 5.0, 1e-3
A = (0.5 + 0.75 * C0) * OMEGA
B2 = C0 * K * OMEGA
RHO = 1.0 - A * DT
SIGMA2 = B2 * DT / (1.0 - RHO * RHO)


def exact_discrete(n):
    k = np.arange(1, n)
    return DT * DT * SIGMA2 * (n + 2.0 * np.sum((n - k) * RHO ** k))


def taylor(t):
    TL = 1.0 / A
    return 2.0 * SIGMA2 * TL * TL * (t / TL - 1.0 + np.exp(-t / TL))


def uniform_fields(mesh):
    F = np.zeros((mesh.n_nodes, wl.n_fields_padded(1)), dtype=np.float32)
    F[:, wl.F_G11] = F[:, wl.F_G22] = F[:, wl.F_G33] = -A
    F[:, wl.F_C0EPS] = B2
    F[:, wl.F_OMEGA] = OMEGA
    F[:, wl.F_SOMEGA] = 0.73
    return F


def band_state(mesh, n_per_elem, seed):
    """Particles of the elements whose centroid lies in 0.75 < y < 1.25, with stationary OU
    velocities (numpy's generator: the initial state is an input, not part of the method)."""
    st = wl.synthetic_state(mesh, n_per_elem, 1, seed=seed)
    cy = mesh.node_xy[mesh.tri, 1].mean(axis=1)
    keep = np.nonzero(np.abs(cy[st.elem] - 1.0) < 0.25)[0]
    st = gc.reorder(st, keep)
    rng = np.random.default_rng(seed + 1)
    s = np.sqrt(SIGMA2)
    st.u[:] = s * rng.standard_normal(st.n)
    st.v[:] = s * rng.standard_normal(st.n)
    st.w[:] = s * rng.standard_normal(st.n)
    st.omega[:] = OMEGA
    st.psi[:] = 0.0
    return st


def check(steps, var, n):
    for m, v in zip(steps, var):
        ex = exact_discrete(m)
        assert abs(v - ex) <= 5.0 * np.sqrt(2.0 / n) * ex, (m, v, ex, taylor(m * DT))


def test_oracle_taylor_dispersion():
    mesh = wl.channel_mesh(25, 20, 1006054901)
    om = oracle.OracleMesh(mesh)
    st = band_state(mesh, 150, seed=5)
    y0 = st.y.astype(np.float64)
    p = oracle.make_params(nu=0.0, dt=DT, seed=17, ns=1, sources=[])
    F = uniform_fields(mesh)
    record, var = (10, 40, 80), []
    for step in range(80):
        res, elem, aux, lost = oracle.pdf_step(om, p, F, st, step)
        assert lost == 0
        st = wl.State(*(res[k].astype(np.float32) for k in gc.FIELDS), res["psi"].astype(np.float32), elem, st.pid)
        if step + 1 in record:
            var.append(float(np.var(st.y.astype(np.float64) - y0)))
    check(record, var, st.n)


@pytest.mark.gpu
def test_gpu_taylor_dispersion():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_0549_gb300 import _build
    _build.build()
    mesh = wl.channel_mesh(25, 20, 1006054901)
    st = band_state(mesh, 2000, seed=6)
    gm = lpdf.Mesh(mesh)
    params = lpdf.make_params(nu=0.0, dt=DT, seed=18, ns=1)
    ctx = lpdf.Context(gm, params, st.n)
    ctx.set_state(gc.torch_state(st))
    Fd = torch.from_numpy(uniform_fields(mesh)).cuda()
    order = np.argsort(st.pid)
    y0 = st.y.astype(np.float64)[order]
    record, var = (10, 50, 100, 200, 300), []
    for step in range(300):
        ctx.pdf_step(Fd, step)
        if step + 1 in record:
            rc, status = ctx.status(raise_on_error=False)
            assert rc == lpdf.LPDF_OK, status
            g = gc.host_state(ctx.get_state(), 1)
            y = g.y.astype(np.float64)[np.argsort(g.pid)]
            var.append(float(np.var(y - y0)))
    check(record, var, st.n)
    # the continuous limit: Taylor's formula within the O(dt) discretisation error
    t = 300 * DT
    assert abs(exact_discrete(300) - taylor(t)) < 0.05 * taylor(t)
