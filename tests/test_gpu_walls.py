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


def test_corner_of_the_seam_and_the_top_wall(torch_cuda):
    """Particles near the top-left corner of the 50,000-triangle bump channel moving up and to the
    left: each step wraps them across the periodic seam and beyond the top wall at once. The GPU
    step equals the oracle's (the walk crosses the periodic edge, then mirrors), nothing is lost."""
    from tests.test_oracle_walls import _corner_state
    torch = torch_cuda
    mesh = wl.bump_channel_mesh(250, 100, 1006054905)
    om = oracle.OracleMesh(mesh)
    st = _corner_state(mesh, om, 4000, np.random.default_rng(41))
    params = lpdf.make_params(nu=1.0 / 180.0, ns=1, seed=42)
    F = np.zeros((mesh.n_nodes, wl.n_fields_padded(1)), dtype=np.float32)
    F[:, wl.F_OMEGA] = 1.0
    ctx = lpdf.Context(lpdf.Mesh(mesh), params, st.n + 128)
    g, _, rc, status = gc.gpu_step(ctx, torch.from_numpy(F).cuda(), st, 3)
    assert rc == lpdf.LPDF_OK, status
    gc.compare_step(mesh, om, params, F, st, 3, g)


def test_mirror_image_that_rounds_back_onto_the_point(torch_cuda):
    """A particle of the 25M bump-channel run whose move ends within about an ulp beyond the curved
    bottom wall: mirrored in FP32, its image rounded back onto the point itself and eight
    mirrorings made no progress (the particle was lost). The mirror is taken in FP64 as in the
    oracle, and an image that still rounds onto the point steps one ulp along the inward normal:
    the GPU finds the owner the oracle finds, after one mirroring."""
    torch = torch_cuda
    mesh = wl.bump_channel_mesh(250, 100, 1006054905)
    om = oracle.OracleMesh(mesh)
    f = lambda v: np.array([v], dtype=np.float32)
    st = wl.State(f(4.090161), f(0.12242391), f(1.5177567), f(-0.53100747), f(0.0), f(1.0),
                  np.zeros((1, 1), np.float32), np.array([32402], np.int32), np.array([16201350], np.uint32))
    params = lpdf.make_params(nu=1.0 / 180.0, dt=1e-3, seed=wl.channel_25m().seed, ns=1)
    F = np.zeros((mesh.n_nodes, wl.n_fields_padded(1)), dtype=np.float32)
    F[:, wl.F_OMEGA] = 1.0
    ctx = lpdf.Context(lpdf.Mesh(mesh), params, 128)
    g, _, rc, status = gc.gpu_step(ctx, torch.from_numpy(F).cuda(), st, 0)
    assert rc == lpdf.LPDF_OK, status
    res, oelem, aux, lost = oracle.pdf_step(om, gc.oracle_params(params), F, st, 0, locate_mode=2)
    assert lost == 0 and aux[0, 2] == 1
    assert g.x[0] == np.float32(res["x"][0]) and g.y[0] == np.float32(res["y"][0])
    assert g.elem[0] == oelem[0] == om.locate_brute(float(g.x[0]), float(g.y[0])) >= 0


def test_image_across_a_sloped_wall_is_wrapped_into_the_frame(torch_cuda):
    """The same particle on the GPU: the image below the seam's first wall edge leaves the frame
    in x and is wrapped; the GPU step equals the oracle's and nothing is lost."""
    torch = torch_cuda
    mesh = wl.bump_channel_mesh(250, 100, 1006054905)
    om = oracle.OracleMesh(mesh)
    f = lambda v: np.array([v], dtype=np.float32)
    st = wl.State(f(0.00021887), f(0.00056443), f(-0.12476623), f(1.2149805), f(0.0), f(1.0),
                  np.zeros((1, 1), np.float32), np.array([0], np.int32), np.array([1810], np.uint32))
    params = lpdf.make_params(nu=1.0 / 180.0, dt=1e-3, seed=wl.channel_25m().seed, ns=1)
    F = np.zeros((mesh.n_nodes, wl.n_fields_padded(1)), dtype=np.float32)
    F[:, wl.F_OMEGA] = 1.0
    ctx = lpdf.Context(lpdf.Mesh(mesh), params, 128)
    g, _, rc, status = gc.gpu_step(ctx, torch.from_numpy(F).cuda(), st, 1)
    assert rc == lpdf.LPDF_OK, status
    res, oelem, aux, lost = oracle.pdf_step(om, gc.oracle_params(params), F, st, 1, locate_mode=2)
    assert lost == 0
    assert g.x[0] == np.float32(res["x"][0]) and g.y[0] == np.float32(res["y"][0])
    assert g.elem[0] == oelem[0] == om.locate_brute(float(g.x[0]), float(g.y[0])) >= 0


def test_hand_worked_moves_on_the_lshape(torch_cuda):
    """The hand-worked moves of the L-shaped mesh, made by one GPU step with no diffusion and still
    fields: the walk round the reentrant corner takes the interior exit (4 hops, no mirroring,
    although the wall's barycentric coordinate is the more negative one in the second element),
    and the two moves into the notch are mirrored across the wall they cross. Positions,
    velocities and owners are exactly the hand-worked ones; the hop count is their sum."""
    from tests.test_oracle_walls import LSHAPE_MOVES, lshape_mesh, lshape_state
    torch = torch_cuda
    mesh = lshape_mesh()
    st = lshape_state()
    params = lpdf.make_params(nu=1e-30, dt=0.5, ns=1, seed=31)
    F = np.zeros((mesh.n_nodes, wl.n_fields_padded(1)), dtype=np.float32)
    F[:, wl.F_OMEGA] = 1.0
    ctx = lpdf.Context(lpdf.Mesh(mesh), params, 128)
    g, _, rc, status = gc.gpu_step(ctx, torch.from_numpy(F).cuda(), st, 0)
    assert rc == lpdf.LPDF_OK, status
    k = gc.match_pids(np.arange(st.n), g.pid)
    for row, (_, _, _, e1, (x1, y1), (u1, v1), _, _) in enumerate(LSHAPE_MOVES):
        j = k[row]
        assert (g.elem[j], g.x[j], g.y[j], g.u[j], g.v[j]) == (e1, x1, y1, u1, v1), row
    assert status[3] == sum(m[6] for m in LSHAPE_MOVES)


def _three_triangle_mesh():
    """The triangle (0,0), (2,0), (0,2) split at the interior point (0.5, 0.5) into three elements;
    every boundary edge is a wall (the hypotenuse is off the sides of the bounding box). An odd
    number of elements: the moments kernel's last warp has an element in one half only."""
    xy = np.array([(0, 0), (2, 0), (0, 2), (0.5, 0.5)], dtype=np.float64)
    tri = np.array([(0, 1, 3), (1, 2, 3), (2, 0, 3)], dtype=np.int32)
    tag = np.zeros((3, 3), dtype=np.int32)
    tag[:, 0] = wl.EDGE_WALL                          # edge 0 of each element is a boundary edge
    return wl.Mesh(xy, tri, tag, 0.0, (0.0, 2.0, 0.0, 2.0), "tri3", 0, 0)


def test_three_element_mesh_step_and_moments(torch_cuda):
    torch = torch_cuda
    mesh = _three_triangle_mesh()
    om = oracle.OracleMesh(mesh)
    assert om.edge_walls
    params = lpdf.make_params(nu=1e-4, ns=2, seed=8)
    st = wl.synthetic_state(mesh, 40, 2, seed=9)
    F = wl.synthetic_node_fields(mesh, 2, seed=10)
    ctx = lpdf.Context(lpdf.Mesh(mesh), params, st.n + 64)
    g, S, rc, status = gc.gpu_step(ctx, torch.from_numpy(F).cuda(), st, 1)
    assert rc == lpdf.LPDF_OK, status
    gc.compare_step(mesh, om, params, F, st, 1, g)
    gc.compare_moments(om, g, S, 2)
