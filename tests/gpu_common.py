"""Helpers of the GPU parity tests: run the CUDA path through the C-ABI and compare with the oracle."""
import numpy as np

import oracle
from paper_1006_0549_gb300 import lpdf, workloads as wl

FIELDS = ("x", "y", "u", "v", "w", "omega")
EPS32 = 2.0 ** -24
# FP32 particle state, per step: |gpu - oracle| <= RTOL * max(|oracle|, rms of that field)
RTOL = 1e-5


def torch_state(st: wl.State):
    import torch
    d = torch.device("cuda")
    out = {k: torch.from_numpy(np.ascontiguousarray(getattr(st, k))).to(d) for k in FIELDS}
    out["psi"] = torch.from_numpy(np.ascontiguousarray(st.psi)).to(d)
    out["elem"] = torch.from_numpy(np.ascontiguousarray(st.elem, dtype=np.int32)).to(d)
    out["pid"] = torch.from_numpy(np.ascontiguousarray(st.pid).view(np.int32)).to(d)
    return out


def host_state(d, ns) -> wl.State:
    """State from get_state's dict (torch tensors or numpy arrays)."""
    g = {k: (v.cpu().numpy() if hasattr(v, "cpu") else np.asarray(v)) for k, v in d.items()}
    return wl.State(*(g[k].astype(np.float32) for k in FIELDS), g["psi"].reshape(ns, -1).astype(np.float32),
                    g["elem"].astype(np.int32), g["pid"].view(np.uint32))


def oracle_params(p: lpdf.Params):
    react = (p.react_k, p.react_a, p.react_b, p.react_p) if p.react_k > 0 else None
    return oracle.make_params(nu=p.nu, dt=p.dt, seed=p.seed, ns=p.ns,
                              sources=[(float(p.src_x[i]), float(p.src_y[i]), float(p.src_r[i]), int(p.src_alpha[i]))
                                       for i in range(p.n_sources)],
                              C3=p.C3, C4=p.C4, Cphi=p.Cphi, lid_u=p.lid_u, react=react)


def gpu_step(ctx: lpdf.Context, fields_dev, st: wl.State, step: int):
    """set_state -> pdf_step -> (new host state, raw moment sums, status)."""
    import torch
    ctx.set_state(torch_state(st))
    ctx.pdf_step(fields_dev, step)
    rc, status = ctx.status(raise_on_error=False)
    out = host_state(ctx.get_state(), ctx.ns)
    S = torch.empty((ctx.mesh.n_nodes, 11 + 2 * ctx.ns), dtype=torch.float64, device="cuda")
    ctx.grid_statistics(S, raw=True)
    torch.cuda.synchronize()
    return out, S.cpu().numpy(), rc, status


def match_pids(want, have):
    """Indices into `have` that list the same pids as `want` (both permutations of one set)."""
    want = np.asarray(want).astype(np.int64)
    have = np.asarray(have).astype(np.int64)
    ih = np.argsort(have, kind="stable")
    pos = np.searchsorted(have[ih], want)
    assert np.all(pos < have.size) and np.array_equal(have[ih][pos], want), "the step lost or invented particles"
    return ih[pos]


def reorder(st: wl.State, idx) -> wl.State:
    return wl.State(*(np.ascontiguousarray(getattr(st, k)[idx]) for k in FIELDS), np.ascontiguousarray(st.psi[:, idx]),
                    np.ascontiguousarray(st.elem[idx]), np.ascontiguousarray(st.pid[idx]))


def wall_distance_points(mesh: wl.Mesh, px, py):
    """Distance of points to the nearest wall edge (tags 1, 2; periodic images in x)."""
    xy = mesh.node_xy
    segs = [(xy[mesh.tri[e, k]], xy[mesh.tri[e, (k + 1) % 3]]) for e in range(mesh.n_tri) for k in range(3)
            if mesh.edge_tag[e, k] in (1, 2)]
    q = np.stack([np.asarray(px, dtype=np.float64), np.asarray(py, dtype=np.float64)], axis=1)
    best = np.full(q.shape[0], np.inf)
    shifts = [0.0] if not mesh.period_x > 0 else [-mesh.period_x, 0.0, mesh.period_x]
    for a, b in segs:
        t = b - a
        for sx in shifts:
            r = q - a - np.array([sx, 0.0])
            s = np.clip(r @ t / (t @ t), 0.0, 1.0)
            best = np.minimum(best, np.hypot(r[:, 0] - s * t[0], r[:, 1] - s * t[1]))
    return best


def compare_step(mesh: wl.Mesh, om: oracle.OracleMesh, params: lpdf.Params, F, st_in: wl.State, step: int,
                 g: wl.State, check_locate: bool = True, beta=None):
    """Per-stage parity of one step from the same input state.

    1. FP32 state within RTOL of the oracle's FP64 step, except for particles whose discrete
       outcome (reflection, wrap, source) legitimately differs because the FP32 positions of the
       two sides straddle the decision boundary by a rounding error;
    2. the GPU's element of every particle equals the oracle's exact owner of the GPU's FP32
       position (bit-exact): by the oracle's brute force over every element, or, with
       check_locate="walk" (meshes too large for brute force on many particles), by the oracle's
       neighbour walk from the particle's input element, which its own pins tie to brute force;
       where the two sides' positions are bit-equal, the elements are equal too.
    Returns a dict of diagnostics."""
    ns = params.ns
    # the step may list its output in another order (it keeps the ensemble in element order):
    # match the particles by pid
    g = reorder(g, match_pids(st_in.pid, g.pid))
    op = oracle_params(params)
    res, oelem, aux, lost = oracle.pdf_step(om, op, F, st_in, step, beta=beta)
    assert lost == 0
    diag = {}
    x0, x1, y0, y1 = mesh.box
    pre_x, pre_y = aux[:, 0], aux[:, 1]
    # straddling a wall or the periodic seam within rounding distance
    if om.edge_walls:
        near_wall = wall_distance_points(mesh, pre_x, pre_y) < 1e-5
    else:
        near_wall = (np.abs(pre_y - y0) < 1e-5) | (np.abs(pre_y - y1) < 1e-5)
        if mesh.period_x == 0.0:
            near_wall |= (np.abs(pre_x - x0) < 1e-5) | (np.abs(pre_x - x1) < 1e-5)
    ok_any = np.zeros(st_in.n, dtype=bool)
    for k in FIELDS:
        o = res[k]
        gv = getattr(g, k).astype(np.float64)
        rms = float(np.sqrt(np.mean(o * o))) or 1.0
        d = np.abs(gv - o)
        if k == "x" and mesh.period_x > 0:
            d = np.minimum(d, np.abs(d - mesh.period_x))
        bad = d > RTOL * np.maximum(np.abs(o), rms)
        diag[f"max_rel_{k}"] = float(np.max(d / np.maximum(np.abs(o), rms)))
        unexplained = bad & ~near_wall
        assert not unexplained.any(), (k, np.nonzero(unexplained)[0][:10], gv[unexplained][:5], o[unexplained][:5])
        ok_any |= bad
    diag["explained_discrete_mismatches"] = int(ok_any.sum())
    assert ok_any.sum() <= max(3, st_in.n // 10000)
    # scalars: the source disc decision is taken on each side's own FP32 position
    srcd = np.full(st_in.n, np.inf)
    for i in range(params.n_sources):
        srcd = np.minimum(srcd, np.abs(np.hypot(res["x"] - params.src_x[i], res["y"] - params.src_y[i]) - params.src_r[i]))
    for a in range(ns):
        o = res["psi"][a]
        gv = g.psi[a].astype(np.float64)
        d = np.abs(gv - o)
        rms = float(np.sqrt(np.mean(o * o))) or 1.0
        bad = d > RTOL * np.maximum(np.abs(o), rms)
        diag[f"max_rel_psi{a}"] = float(np.max(d / np.maximum(np.abs(o), rms)))
        unexplained = bad & ~(srcd < 1e-5) & ~near_wall
        assert not unexplained.any(), ("psi", a, np.nonzero(unexplained)[0][:10])
    # element ids: exact owner of the GPU position, by the oracle's brute force location
    if check_locate:
        for i in range(st_in.n):
            if check_locate == "walk" and not om.edge_walls:
                e, _ = om.locate_walk(int(st_in.elem[i]), float(g.x[i]), float(g.y[i]))
            else:
                e = om.locate_brute(float(g.x[i]), float(g.y[i]))
            assert e == g.elem[i], (i, g.x[i], g.y[i], g.elem[i], e)
        same = (g.x.astype(np.float64) == res["x"]) & (g.y.astype(np.float64) == res["y"])
        assert np.array_equal(g.elem[same], oelem[same])
        diag["bitwise_equal_positions"] = float(same.mean())
    assert np.array_equal(g.pid, st_in.pid)
    return diag, res, oelem


# Gridpoint moment sums against the oracle's FP64 reduction of the same FP32 state, relative to
# sum_p |lambda_a q_k| (the oracle's absolute sum), plus 2^-33 per fixed-point conversion.
# lpdf_params.moment_sums = 1 (compensated): the sums of q, dx q and dy q ((dx, dy) from vertex 0, formed exactly) in
#   compensated FP32 (error-free products and additions, double-float accumulators over at most 16
#   particles of a lane and 5 levels of the warp reduction: relative error of order 21 (2 eps32^2),
#   about 1e-13), combined in FP64 with the element's FP64 barycentric coefficients (relative error
#   of order eps64 times (|b dx| + |g dy|) / |lambda|); 1e-9 leaves three orders of magnitude for
#   elements whose weights cancel.
# moment_sums = 0 (lpdf_pdf_step's default) and lpdf_pdf_step_static's fused kernel: each term lambda_a q_k formed in FP32 (barycentric
#   determinants with one FMA-compensated rounding, the division, the products) and summed in FP32
#   over at most 8 particles of a lane and 5 levels of the warp reduction (the fused kernel: units
#   of at most 6 particles, column sums of at most 32 units): 48 eps32.
MOMENT_RTOL = {"compensated": 1e-9, "fp32": 48 * EPS32}
LAMBDA_RTOL = 8 * EPS32   # FP32 barycentric weights: per unit of kappa (lambda_rounding_sums)


def lambda_rounding_sums(om: oracle.OracleMesh, g: wl.State, ns: int):
    """Per node and quantity, sum over the particles of kappa_n(p) |q_k(p)|, where
    kappa_n = (|dx_b dy_c| + |dy_b dx_c|) / |2A| with (dx_v, dy_v) = vertex v - the particle, b and c
    the element's other two vertices. The FP32 moments kernel forms lambda_n as the determinant of
    those four FP32 differences (each rounded once) times the rounded 1/2A, so its absolute error is
    at most about 2 eps32 kappa_n + 2 eps32 |lambda_n|: for a particle far from node n on a long thin
    element kappa_n is of the order of the aspect ratio while lambda_n is near 0, and a bound
    relative to |lambda_n q| alone does not cover it. Folded onto master nodes like the sums."""
    xy, tri = om.node_xy, om.tri[g.elem]
    X, Y = xy[tri, 0], xy[tri, 1]                      # (n, 3) vertex coordinates, exact
    dx = X - g.x.astype(np.float64)[:, None]
    dy = Y - g.y.astype(np.float64)[:, None]
    A2 = np.abs((X[:, 1] - X[:, 0]) * (Y[:, 2] - Y[:, 0]) - (Y[:, 1] - Y[:, 0]) * (X[:, 2] - X[:, 0]))
    kappa = np.empty_like(X)
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        kappa[:, a] = (np.abs(dx[:, b] * dy[:, c]) + np.abs(dy[:, b] * dx[:, c])) / A2
    u, v, w = (getattr(g, k).astype(np.float64) for k in ("u", "v", "w"))
    psi = np.asarray(g.psi, dtype=np.float64).reshape(ns, g.n)
    q = np.stack([np.ones(g.n), u, v, w, u * u, u * v, u * w, v * v, v * w, w * w, g.omega.astype(np.float64)]
                 + [psi[a] for a in range(ns)] + [psi[a] ** 2 for a in range(ns)], axis=1)
    masters = om.masters()
    K = np.zeros((om.n_nodes, q.shape[1]))
    for a in range(3):
        np.add.at(K, masters[tri[:, a]], kappa[:, a:a + 1] * np.abs(q))
    return K[masters]


def moment_tolerance(S_o, Sabs, bound: str = "fp32", K=None):
    """The bound of the kernel that formed the sums: MOMENT_RTOL of sum |lambda q|, with FP32 partial
    sums also LAMBDA_RTOL of sum kappa |q| (K, lambda_rounding_sums), plus 2^-33 per fixed-point
    conversion (at most 8 per unit of particle weight)."""
    count = np.maximum(S_o[:, :1], 1.0) * 8.0
    tol = MOMENT_RTOL[bound] * Sabs + count * 2.0 ** -33
    if bound == "fp32" and K is not None:
        tol = tol + LAMBDA_RTOL * K
    return tol


def compare_moments(om: oracle.OracleMesh, g: wl.State, S_gpu, ns: int, bound: str = "fp32"):
    """GPU fixed-point sums against the oracle's FP64 reduction of the same FP32 state, within the
    bound of the kernel that formed them (MOMENT_RTOL). Returns (max error / sum|lambda q|, S_oracle)."""
    f = lambda a: a.astype(np.float64)
    S_o, Sabs = oracle.moments(om, ns, f(g.x), f(g.y), f(g.u), f(g.v), f(g.w), f(g.omega), f(g.psi), g.elem)
    tol = moment_tolerance(S_o, Sabs, bound, lambda_rounding_sums(om, g, ns) if bound == "fp32" else None)
    err = np.abs(S_gpu - S_o)
    ratio = float(np.max(err / np.maximum(Sabs, 1e-300)))
    assert np.all(err <= tol), (np.argwhere(err > tol)[:5], err[err > tol][:5], tol[err > tol][:5])
    return ratio, S_o
