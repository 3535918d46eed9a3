"""Ownership at exact hits on the GPU (tracking through the grid, Introduction item iii; the
top-left rule on CCW elements, walls of any shape closed).

A step with nu = 0 and particle velocities U = V = 0 leaves every position where it is (Eq. 2:
X' = X + U dt + (2 nu)^1/2 dW = X), apart from the boundary rules (the half-open frame, the
periodic wrap, the mirroring of a position beyond a wall). The particles sit exactly on interior,
wall and periodic edges, exactly at vertices, and 1-3 FP32 ulps either side of both
(tests/exact_points.py decides exactness by rational arithmetic), and each starts its walk in
every element that shares its edge or vertex. So the step's certified fast test, its FP32
orientation filter and its exact FP64 expansion all decide ties, and the walk has to leave an
element through the very edge a point lies on. Every GPU element id must equal the oracle's
brute-force owner of the GPU position; the state and the moment sums must match the oracle's
step as in the other parity tests."""
import numpy as np
import pytest

import oracle
from paper_1006_0549_gb300 import lpdf, workloads as wl
from tests import exact_points as ep
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


def _case(name):
    if name == "channel":
        return wl.channel_mesh(25, 20, 1006054901), 1, 0.0
    if name == "cavity":
        return wl.cavity_mesh(32, 32, 1006054903), 4, 1.0
    return wl.bump_channel_mesh(25, 20, 7), 1, 0.0


def _still_state(mesh, ns, seed):
    X, Y, S, K = ep.exact_points(mesh)
    rng = np.random.default_rng(seed)
    n = X.size
    z = np.zeros(n, dtype=np.float32)
    st = wl.State(X.copy(), Y.copy(), z.copy(), z.copy(), rng.standard_normal(n).astype(np.float32),
                  rng.gamma(4.0, 0.25, n).astype(np.float32), rng.uniform(0, 1, (ns, n)).astype(np.float32),
                  S.copy(), np.arange(n, dtype=np.uint32))
    return st, K


@pytest.mark.parametrize("name", ["channel", "cavity", "bump"])
def test_exact_edge_and_vertex_hits(torch_cuda, name):
    torch = torch_cuda
    mesh, ns, lid_u = _case(name)
    st, K = _still_state(mesh, ns, seed=41)
    gm = lpdf.Mesh(mesh)
    om = oracle.OracleMesh(mesh)
    params = lpdf.make_params(nu=0.0, dt=1e-3, seed=77, ns=ns, lid_u=lid_u)
    F = wl.synthetic_node_fields(mesh, ns, seed=5)
    ctx = lpdf.Context(gm, params, st.n)
    g, S, rc, status = gc.gpu_step(ctx, torch.from_numpy(F).cuda(), st, step=2)
    assert rc == lpdf.LPDF_OK, status
    # state against the oracle's step, and every element id against the brute-force owner
    diag, res, oelem = gc.compare_step(mesh, om, params, F, st, 2, g)
    assert diag["explained_discrete_mismatches"] == 0
    assert diag["bitwise_equal_positions"] == 1.0
    # the positions are the inputs, except where a boundary rule moved them
    g = gc.reorder(g, gc.match_pids(st.pid, g.pid))
    moved = (g.x != st.x) | (g.y != st.y)
    inside = ep.in_box(mesh, st.x, st.y)
    x0, x1, y0, y1 = mesh.box
    on_open_side = (st.x == x1) | (st.y == y1)
    assert not np.any(moved & inside & ~on_open_side) or om.edge_walls
    gc.compare_moments(om, g, S, ns)
    print(name, st.n, "particles;", "exact vertex/edge/perturbed:", np.bincount(K), diag)
