"""The concentrated scalar sources at their edges (Section "Two testcases": psi_alpha = 1 for
the particles inside a source disc after the move). The kernel tests a position against the
discs only inside their bounding box, rounded outward to FP32; outside it the rounded distance
test cannot succeed. Particles placed within a few ulps of each disc's circle and of the box's
sides and corners, with a step that does not move them, must take exactly the decision of the
oracle's FP32 disc test on the same positions."""
import numpy as np
import pytest

import oracle
from paper_1006_0549_gb300 import lpdf, workloads as wl
from tests import gpu_common as gc

pytestmark = pytest.mark.gpu

SOURCES = [(0.25, 0.67, 0.02, 0), (1.0, 1.2, 0.05, 1), (1.3, 1.25, 0.03, 0)]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_0549_gb300 import _build
    _build.build()
    return torch


def _ulps(v, m):
    """v moved by m FP32 ulps (m may be negative)."""
    v = np.float32(v)
    for _ in range(abs(m)):
        v = np.nextafter(v, np.float32(np.inf if m > 0 else -np.inf), dtype=np.float32)
    return v


def _edge_points(rng):
    pts = []
    # around every circle: radius r (1 + m 2^-23) at many angles
    th = rng.uniform(0.0, 2.0 * np.pi, 300)
    for sx, sy, r, _ in SOURCES:
        for m in range(-4, 5):
            rr = r * (1.0 + m * 2.0 ** -23)
            pts.append(np.stack([sx + rr * np.cos(th), sy + rr * np.sin(th)], axis=1))
        # the four points of the circle on the box sides, nudged by a few ulps
        for dx, dy in ((-r, 0.0), (r, 0.0), (0.0, -r), (0.0, r)):
            for mx in range(-2, 3):
                for my in range(-2, 3):
                    pts.append(np.array([[_ulps(sx + dx, mx), _ulps(sy + dy, my)]]))
    # the sides and corners of the box around all discs (FP64 bounds, nudged in FP32)
    x0 = min(s[0] - s[2] for s in SOURCES)
    x1 = max(s[0] + s[2] for s in SOURCES)
    y0 = min(s[1] - s[2] for s in SOURCES)
    y1 = max(s[1] + s[2] for s in SOURCES)
    t = rng.uniform(0.0, 1.0, 200)
    for m in range(-3, 4):
        pts.append(np.stack([np.full(t.size, _ulps(x0, m)), y0 + t * (y1 - y0)], axis=1))
        pts.append(np.stack([np.full(t.size, _ulps(x1, m)), y0 + t * (y1 - y0)], axis=1))
        pts.append(np.stack([x0 + t * (x1 - x0), np.full(t.size, _ulps(y0, m))], axis=1))
        pts.append(np.stack([x0 + t * (x1 - x0), np.full(t.size, _ulps(y1, m))], axis=1))
        for cx in (x0, x1):
            for cy in (y0, y1):
                pts.append(np.array([[_ulps(cx, m), _ulps(cy, m)], [_ulps(cx, m), _ulps(cy, -m)]]))
    return np.concatenate(pts).astype(np.float32)


def test_source_decisions_at_the_disc_and_box_edges(torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(17)
    mesh = wl.channel_mesh(25, 20, 3)
    om = oracle.OracleMesh(mesh)
    pts = _edge_points(rng)
    elem = np.array([om.locate_brute(float(x), float(y)) for x, y in pts], dtype=np.int32)
    keep = elem >= 0
    pts, elem = pts[keep], elem[keep]
    n, ns = pts.shape[0], 2
    st = wl.State(pts[:, 0].copy(), pts[:, 1].copy(), np.zeros(n, np.float32), np.zeros(n, np.float32),
                  np.zeros(n, np.float32), np.ones(n, np.float32), np.zeros((ns, n), np.float32), elem,
                  np.arange(n, dtype=np.uint32))
    # no displacement: U = 0 and a vanishing viscosity leave every FP32 position unchanged
    params = lpdf.make_params(nu=1e-30, dt=1e-3, seed=5, ns=ns, sources=SOURCES)
    F = np.zeros((mesh.n_nodes, wl.n_fields_padded(ns)), dtype=np.float32)
    F[:, wl.F_OMEGA] = 1.0
    ctx = lpdf.Context(lpdf.Mesh(mesh), params, n + 128)
    g, _, rc, status = gc.gpu_step(ctx, torch.from_numpy(F).cuda(), st, 1)
    assert rc == lpdf.LPDF_OK, status
    g = gc.reorder(g, gc.match_pids(st.pid, g.pid))
    assert np.array_equal(g.x, st.x) and np.array_equal(g.y, st.y)
    res, _, _, lost = oracle.pdf_step(om, gc.oracle_params(params), F, st, 1)
    assert lost == 0
    assert np.array_equal(res["x"], st.x.astype(np.float64)) and np.array_equal(res["y"], st.y.astype(np.float64))
    for a in range(ns):
        want = res["psi"][a]
        assert set(np.unique(want)) <= {0.0, 1.0}
        assert np.array_equal(g.psi[a].astype(np.float64), want), (a, np.nonzero(g.psi[a] != want)[0][:10])
    # the placement straddles the circles: both decisions occur
    inside = res["psi"].max(axis=0) == 1.0
    assert 0.2 < inside.mean() < 0.8
