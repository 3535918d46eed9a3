"""IECM micromixing and the reactive source (Eq. 9) on the GPU against the FP64 oracle: one step
with both, the scalar-flux sums at the gridpoints, the conditional-mean slopes, and the loop
statistics -> fluxes -> slopes -> steps."""
import numpy as np
import pytest

import oracle
from oracle import fields as of
from paper_1006_0549_gb300 import lpdf, workloads as wl
from tests import gpu_common as gc

pytestmark = pytest.mark.gpu
NS = 3


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_0549_gb300 import _build
    _build.build()
    return torch


def _case():
    mesh = wl.channel_mesh(20, 12, 31)
    params = lpdf.make_params(ns=NS, seed=8, sources=[(0.25, 0.67, 0.05, 0)], mixing=1, react_k=4.0,
                              react_a=0, react_b=1, react_p=2)
    st = wl.synthetic_state(mesh, 10, NS, seed=32)
    F = wl.synthetic_node_fields(mesh, NS, seed=33)
    beta = (0.2 * np.random.default_rng(34).standard_normal((mesh.n_nodes, 3 * NS))).astype(np.float32)
    master = oracle.OracleMesh(mesh).masters()
    beta = beta[master]                        # periodic partners carry the same slopes
    return mesh, params, st, F, beta


def test_one_step_with_iecm_and_reaction(torch_cuda):
    torch = torch_cuda
    mesh, params, st, F, beta = _case()
    gm = lpdf.Mesh(mesh)
    om = oracle.OracleMesh(mesh)
    ctx = lpdf.Context(gm, params, st.n + 128)
    b = torch.from_numpy(beta).cuda()
    ctx.set_iecm(b)
    g, S, rc, status = gc.gpu_step(ctx, torch.from_numpy(F).cuda(), st, step=4)
    assert rc == lpdf.LPDF_OK, status
    diag, res, _ = gc.compare_step(mesh, om, params, F, st, 4, g, beta=beta)
    # the conditional mean and the reaction changed the scalars compared with plain IEM
    p_iem = gc.oracle_params(params)
    p_iem.react_k = 0.0
    r_iem, _, _, _ = oracle.pdf_step(om, p_iem, F, st, 4)
    assert np.max(np.abs(res["psi"] - r_iem["psi"])) > 1e-4
    gc.compare_moments(om, g, S, NS)


@pytest.mark.parametrize("ms", [0, 1])
def test_flux_sums_and_covariances_match_the_oracle(torch_cuda, ms):
    torch = torch_cuda
    mesh, params, st, F, beta = _case()
    params.moment_sums = ms
    gm = lpdf.Mesh(mesh)
    om = oracle.OracleMesh(mesh)
    ctx = lpdf.Context(gm, params, st.n + 128)
    ctx.set_state(gc.torch_state(st))
    ctx.pdf_step(torch.from_numpy(F).cuda(), 1)
    ctx.status()
    g = gc.host_state(ctx.get_state(), NS)
    Fr = torch.empty((mesh.n_nodes, 3 * NS), dtype=torch.float64, device="cuda")
    Fc = torch.empty_like(Fr)
    S = torch.empty((mesh.n_nodes, 11 + 2 * NS), dtype=torch.float64, device="cuda")
    ctx.grid_flux_statistics(Fr, raw=True)
    ctx.grid_flux_statistics(Fc, raw=False)
    ctx.grid_statistics(S, raw=True)
    torch.cuda.synchronize()
    x, y, u, v, w = (getattr(g, k).astype(np.float64) for k in ("x", "y", "u", "v", "w"))
    psi = g.psi.astype(np.float64)
    want = oracle.flux_moments(om, NS, x, y, u, v, w, psi, g.elem)
    scale = oracle.flux_moments(om, NS, x, y, np.abs(u), np.abs(v), np.abs(w), np.abs(psi), g.elem)
    # the flux sums go through the reduction of the plain statistics, in its precision
    bound = "compensated" if params.moment_sums == 1 else "fp32"
    assert np.all(np.abs(Fr.cpu().numpy() - want) <= gc.MOMENT_RTOL[bound] * scale + 2.0 ** -30)
    cov = of.flux_covariances(S.cpu().numpy(), Fr.cpu().numpy(), NS)
    assert np.allclose(Fc.cpu().numpy(), cov, rtol=1e-12, atol=1e-12)


def test_coefficients_match_the_oracle(torch_cuda):
    torch = torch_cuda
    mesh = wl.channel_mesh(12, 8, 35)
    st = wl.synthetic_statistics(mesh, NS, 36)
    rng = np.random.default_rng(37)
    flux = 0.05 * rng.standard_normal((mesh.n_nodes, 3 * NS))
    gm = lpdf.Mesh(mesh)
    b = torch.empty((mesh.n_nodes, 3 * NS), dtype=torch.float32, device="cuda")
    gm.iecm_coefficients(NS, torch.from_numpy(st).cuda(), torch.from_numpy(flux).cuda(), b)
    torch.cuda.synchronize()
    want = of.iecm_coefficients(st, flux, NS)
    assert np.allclose(b.cpu().numpy(), want, rtol=1e-5, atol=1e-6 * np.abs(want).max())


def test_iecm_time_loop_runs(torch_cuda):
    """statistics -> scalar fluxes -> slopes -> steps, with graph replays."""
    torch = torch_cuda
    wk = wl.channel_small()
    params = lpdf.params_for(wk, mixing=1)
    gm = lpdf.Mesh(wk.mesh)
    ctx = lpdf.Context(gm, params, wk.n_particles + 128)
    ctx.particles_init(wk.n_per_elem, torch.from_numpy(wl.node_init_fields(wk.mesh)).cuda())
    F = torch.from_numpy(wl.synthetic_node_fields(wk.mesh, 1, seed=5)).cuda()
    N = wk.mesh.n_nodes
    S = torch.empty((N, 13), dtype=torch.float64, device="cuda")
    Fx = torch.empty((N, 3), dtype=torch.float64, device="cuda")
    beta = torch.zeros((N, 3), dtype=torch.float32, device="cuda")
    ctx.set_iecm(beta)
    step = 0
    for _ in range(4):
        ctx.pdf_steps(F, step, 2)
        step += 2
        ctx.grid_statistics(S, raw=False)
        ctx.grid_flux_statistics(Fx, raw=False)
        gm.iecm_coefficients(1, S, Fx, beta)
    ctx.status()
    assert torch.isfinite(beta).all()
    assert float(beta.abs().max()) > 0.0
