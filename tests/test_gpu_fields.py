"""Parity of the CUDA gridpoint solve (lpdf_elliptic_relax_solve, through the C-ABI) with the
FP64 oracle of oracle/fields.py: gradient recovery, elliptic relaxation, mean pressure, node fields."""
import numpy as np
import pytest

import oracle
from oracle import fields as of
from paper_1006_0549_gb300 import lpdf, workloads as wl
from tests import gpu_common as gc

pytestmark = pytest.mark.gpu

# FP64 on both sides, CG to a relative residual of 1e-12, output rounded to FP32: per column,
# |gpu - oracle| <= RTOL * max(|oracle|, rms of the column)
RTOL = 2e-5
CG_TOL = 1e-12


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_0549_gb300 import _build
    _build.build()
    return torch


def _solve(torch, gm, params, stats, tol=CG_TOL, maxit=20000):
    nfp = wl.n_fields_padded(params.ns)
    out = torch.full((gm.n_nodes, nfp), float("nan"), dtype=torch.float32, device="cuda")
    its = gm.elliptic_relax_solve(params, torch.from_numpy(np.ascontiguousarray(stats)).cuda(), out, tol, maxit)
    torch.cuda.synchronize()
    return out.cpu().numpy(), its


def _compare(F, O, ns, label):
    cols = list(range(22 + ns))
    worst = 0.0
    for c in cols:
        o = O[:, c]
        scale = np.maximum(np.abs(o), np.sqrt(np.mean(o ** 2)))
        err = np.abs(F[:, c].astype(np.float64) - o)
        bad = err > RTOL * scale + 1e-30
        if bad.any():
            i = int(np.argmax(err / np.maximum(scale, 1e-300)))
            raise AssertionError(f"{label}: column {c}: {int(bad.sum())} nodes off, worst node {i}: gpu {F[i, c]!r} "
                                 f"oracle {o[i]!r}")
        worst = max(worst, float(np.max(err / np.maximum(scale, 1e-300))))
    assert np.isfinite(F[:, :22 + ns]).all()
    assert np.all(F[:, 22 + ns:] == 0.0)
    return worst


CASES = [
    ("channel", 1, 0, 1),     # mesh, ns, gmodel, pressure_solve
    ("channel", 2, 1, 0),
    ("cavity", 4, 0, 1),
    ("cavity", 1, 1, 1),
]


@pytest.mark.parametrize("kind,ns,gmodel,psolve", CASES)
def test_node_fields_parity(torch_cuda, kind, ns, gmodel, psolve):
    mesh = wl.channel_mesh(25, 20, 1006054901) if kind == "channel" else wl.cavity_mesh(32, 32, 1006054903)
    stats = wl.synthetic_statistics(mesh, ns, seed=11)
    dpdx0 = -1.0 if kind == "channel" else 0.0
    params = lpdf.make_params(ns=ns, gmodel=gmodel, pressure_solve=psolve, dpdx0=dpdx0)
    gm = lpdf.Mesh(mesh)
    F, its = _solve(torch_cuda, gm, params, stats)
    O = of.node_fields(mesh, stats, ns, C0=params.C0, Comega1=params.Comega1, Comega2=params.Comega2, CL=params.CL,
                       Ceta=params.Ceta, nu=params.nu, gmodel=gmodel, pressure_solve=psolve, dpdx0=dpdx0)
    worst = _compare(F, O, ns, f"{kind} ns={ns} gmodel={gmodel} pressure={psolve}")
    assert (its[0] > 0) == (gmodel == 0) and (its[1] > 0) == bool(psolve)
    print(kind, ns, gmodel, psolve, "CG iterations", its, "worst error / scale", worst)


def test_node_fields_parity_full_size_channel_mesh(torch_cuda):
    """The 250 x 100 channel mesh of the 25M-particle workload (25,351 nodes)."""
    wk = wl.channel_25m()
    stats = wl.synthetic_statistics(wk.mesh, 1, seed=12)
    params = lpdf.make_params(ns=1, gmodel=0, pressure_solve=1, dpdx0=-1.0)
    gm = lpdf.Mesh(wk.mesh)
    F, its = _solve(torch_cuda, gm, params, stats)
    O = of.node_fields(wk.mesh, stats, 1, gmodel=0, pressure_solve=1, dpdx0=-1.0)
    worst = _compare(F, O, 1, "channel 250x100")
    print("CG iterations", its, "worst error / scale", worst)


def test_solve_is_bit_reproducible_and_periodic(torch_cuda):
    mesh = wl.channel_mesh(25, 20, 3)
    stats = wl.synthetic_statistics(mesh, 1, seed=13)
    params = lpdf.make_params(ns=1, gmodel=0, pressure_solve=1)
    gm = lpdf.Mesh(mesh)
    F1, it1 = _solve(torch_cuda, gm, params, stats)
    F2, it2 = _solve(torch_cuda, gm, params, stats)
    assert it1 == it2 and np.array_equal(F1.view(np.uint32), F2.view(np.uint32))
    m = gm.masters()
    assert np.array_equal(F1, F1[m])


def test_nonconvergence_is_reported_and_the_mesh_stays_usable(torch_cuda):
    mesh = wl.cavity_mesh(20, 20, 4)
    stats = wl.synthetic_statistics(mesh, 1, seed=14)
    params = lpdf.make_params(ns=1, gmodel=0, pressure_solve=0)
    gm = lpdf.Mesh(mesh)
    with pytest.raises(lpdf.LpdfError) as ei:
        _solve(torch_cuda, gm, params, stats, maxit=2)
    assert ei.value.code == lpdf.LPDF_ERR_CG_NOCONV
    F, its = _solve(torch_cuda, gm, params, stats)
    O = of.node_fields(mesh, stats, 1, gmodel=0)
    _compare(F, O, 1, "after a failed solve")


def test_statistics_to_fields_chain(torch_cuda):
    """pdf_step -> grid_statistics -> elliptic_relax_solve on the GPU; the raw sums agree with the
    oracle's reduction of the GPU's particles, and the oracle solves from the same statistics."""
    torch = torch_cuda
    wk = wl.channel_small()
    mesh = wk.mesh
    gm = lpdf.Mesh(mesh)
    om = oracle.OracleMesh(mesh)
    params = lpdf.params_for(wk, gmodel=0, pressure_solve=1, dpdx0=-1.0)
    F0 = wl.synthetic_node_fields(mesh, wk.ns, seed=5)
    ctx = lpdf.Context(gm, params, mesh.n_tri * 20 + 100)
    st = wl.synthetic_state(mesh, 20, wk.ns, seed=7)
    ctx.set_state(gc.torch_state(st))
    ctx.pdf_step(torch.from_numpy(F0).cuda(), 1)
    ctx.status()
    nq = 11 + 2 * wk.ns
    S = torch.zeros((mesh.n_nodes, nq), dtype=torch.float64, device="cuda")
    ctx.grid_statistics(S, raw=True)
    torch.cuda.synchronize()
    # the raw sums agree with the oracle's reduction of the GPU's new particle state
    gc.compare_moments(om, gc.host_state(ctx.get_state(), wk.ns), S.cpu().numpy(), wk.ns)
    ctx.grid_statistics(S, raw=False)
    torch.cuda.synchronize()
    stats = S.cpu().numpy()
    F, its = _solve(torch, gm, params, stats)
    O = of.node_fields(mesh, stats, wk.ns, nu=params.nu, gmodel=0, pressure_solve=1, dpdx0=-1.0)
    _compare(F, O, wk.ns, "chain")


def test_warm_start_converges_to_the_same_fields_in_fewer_iterations(torch_cuda):
    """cg_warm_start: the CGs start from the previous solution on the mesh; on slightly changed
    statistics they reach the cold solution's accuracy in fewer iterations."""
    mesh = wl.channel_mesh(40, 30, 1006054901)
    stats = wl.synthetic_statistics(mesh, 1, seed=21)
    params = lpdf.make_params(ns=1, gmodel=0, pressure_solve=1, dpdx0=-1.0)
    gm = lpdf.Mesh(mesh)
    _solve(torch_cuda, gm, params, stats)                     # previous solution on this mesh
    stats2 = stats.copy()
    stats2[:, 4:11] *= 1.0 + 1e-3 * np.random.default_rng(3).standard_normal((mesh.n_nodes, 7))
    stats2[gm.masters() != np.arange(mesh.n_nodes)] = stats2[gm.masters()[gm.masters() != np.arange(mesh.n_nodes)]]
    cold, it_cold = _solve(torch_cuda, gm, params, stats2)
    params.cg_warm_start = 1
    _solve(torch_cuda, gm, params, stats)                     # previous solution: the first statistics
    warm, it_warm = _solve(torch_cuda, gm, params, stats2)
    assert it_warm[0] < it_cold[0] and it_warm[1] < it_cold[1], (it_warm, it_cold)
    O = of.node_fields(mesh, stats2, 1, gmodel=0, pressure_solve=1, dpdx0=-1.0)
    _compare(warm, O, 1, "warm start")
    _compare(cold, O, 1, "cold start")
