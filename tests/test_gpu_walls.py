"""Walls of any shape on the GPU: one step on a channel with a curved (non-convex) bottom wall and
on a quadrilateral with slanted walls, against the FP64 oracle (positions and velocities within
the step tolerance, element ids exactly the owners of the GPU positions), and several steps in
which no particle is lost."""
import numpy as np
import pytest

import oracle
from paper_1006_0549_gb300 import lpdf, workloads as wl
from tests import gpu_common as gc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_0549_gb300 import _build
    _build.build()
    return torch


def _case(kind):
    if kind == "bump":
        mesh = wl.bump_channel_mesh(40, 14, 21, amp=0.3)
        params = lpdf.make_params(ns=1, seed=5, sources=[(0.25, 0.67, 0.05, 0)])
    else:
        mesh = wl.trapezoid_mesh(24, 24, 22)
        params = lpdf.make_params(nu=1e-4, ns=1, seed=6, lid_u=1.0, sources=[(0.5, 0.5, 0.05, 0)])
    st = wl.synthetic_state(mesh, 8, 1, seed=23)
    # fast wall-normal motion, so that many particles meet a wall in one step
    st.u = (st.u * 3.0).astype(np.float32)
    st.v = (st.v * 30.0).astype(np.float32)
    F = wl.synthetic_node_fields(mesh, 1, seed=24)
    return mesh, params, st, F


@pytest.mark.parametrize("kind", ["bump", "trapezoid"])
def test_one_step_with_walls_of_any_shape(torch_cuda, kind):
    torch = torch_cuda
    mesh, params, st, F = _case(kind)
    gm = lpdf.Mesh(mesh)
    om = oracle.OracleMesh(mesh)
    assert om.edge_walls
    ctx = lpdf.Context(gm, params, st.n + 128)
    g, S, rc, status = gc.gpu_step(ctx, torch.from_numpy(F).cuda(), st, step=3)
    assert rc == lpdf.LPDF_OK, status
    diag, res, oelem = gc.compare_step(mesh, om, params, F, st, 3, g)
    _, _, aux, _ = oracle.pdf_step(om, gc.oracle_params(params), F, st, 3)
    assert (aux[:, 2] > 0).sum() > 50                     # the walls were met
    gc.compare_moments(om, g, S, 1)


@pytest.mark.parametrize("kind", ["bump", "trapezoid"])
def test_no_particle_leaves_through_a_wall(torch_cuda, kind):
    torch = torch_cuda
    mesh, params, st, F = _case(kind)
    gm = lpdf.Mesh(mesh)
    om = oracle.OracleMesh(mesh)
    ctx = lpdf.Context(gm, params, st.n + 128)
    ctx.set_state(gc.torch_state(st))
    Fd = torch.from_numpy(F).cuda()
    for s in range(10):
        ctx.pdf_step(Fd, s)
    rc, status = ctx.status(raise_on_error=False)
    assert rc == lpdf.LPDF_OK, status
    g = gc.host_state(ctx.get_state(), 1)
    assert g.n == st.n
    for i in range(0, g.n, 7):
        assert om.locate_brute(float(g.x[i]), float(g.y[i])) == g.elem[i]
