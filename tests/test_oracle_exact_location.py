"""The oracle's neighbour walk at exact hits: positions exactly on edges (interior, wall, periodic)
and at vertices, and a few FP32 ulps either side, located by the walk from each element that
shares the edge or the vertex, against the oracle's brute-force owner (tracking through the grid,
Introduction item iii; the top-left rule makes the owner unique). On the periodic channels the
points of the seam at x = x1 are wrapped to x0 as the step does, so their walks start from
elements on the far side of the seam. Exactness of the inputs is decided by rational arithmetic
in tests/exact_points.py, not by the oracle."""
import numpy as np
import pytest

import oracle
from paper_1006_0549_gb300 import workloads as wl
from tests import exact_points as ep


def _meshes():
    return {
        "channel": wl.channel_mesh(25, 20, 1006054901),
        "cavity": wl.cavity_mesh(32, 32, 1006054903),
        "bump": wl.bump_channel_mesh(25, 20, 7),
    }


@pytest.mark.parametrize("name", ["channel", "cavity", "bump"])
def test_walk_equals_brute_force_at_exact_hits(name):
    mesh = _meshes()[name]
    om = oracle.OracleMesh(mesh)
    X, Y, S, K = ep.exact_points(mesh, max_edges=600)
    located = np.zeros(3, dtype=int)
    outside = 0
    if mesh.period_x > 0:
        # the periodic wrap puts x = x1 at x0 (half-open frame): those walks start on the far
        # side of the seam, in an image frame
        X = np.where(X == np.float32(mesh.period_x), np.float32(0.0), X)
    for x, y, s, k in zip(X, Y, S, K):
        b = om.locate_brute(float(x), float(y))
        assert b >= -1, ("several owners", x, y, b)
        if b < 0:
            outside += 1      # beyond a wall or outside the half-open frame
            continue
        w, _ = om.locate_walk(int(s), float(x), float(y))
        assert w == b, (name, float(x), float(y), int(s), w, b, int(k))
        located[k] += 1
    # every kind of hit is exercised many times
    assert located[0] > 300 and located[1] > 300 and located[2] > 3000, located
    assert outside > 0


def test_exact_points_are_on_their_edges():
    """The generator's on-edge points lie on an edge exactly: the oracle's exact orientation of the
    point against the edge is zero, and one FP32 ulp off it is not (where an ulp moves it off)."""
    mesh = wl.channel_mesh(25, 20, 1006054901)
    edges = ep.edge_elements(mesh)
    xy = mesh.node_xy
    X, Y, S, K = ep.exact_points(mesh, max_edges=200)
    on = np.nonzero(K == 1)[0]
    assert on.size > 100
    for i in on[:400]:
        e = int(S[i])
        hits = 0
        for k in range(3):
            a, b = int(mesh.tri[e, k]), int(mesh.tri[e, (k + 1) % 3])
            if (min(a, b), max(a, b)) in edges:
                s = oracle.orient2d_sign(xy[a, 0], xy[a, 1], xy[b, 0], xy[b, 1], float(X[i]), float(Y[i]))
                hits += s == 0
        assert hits == 1, (i, X[i], Y[i], e)
