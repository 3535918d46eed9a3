"""Seeded synthetic inputs for the particle time step: meshes, node fields, particle states.

This module generates *inputs* only. It holds none of the method's arithmetic (no SDE, no
barycentric location, no statistics), so the CUDA path and the CPU oracle can both consume
what it produces without sharing any of the method's code.

Workloads (the paper's two testcases, Section "Two testcases"):
  * channel: fully developed 2D channel, x periodic with period L = fl32(2*pi), walls at
    y = 0 and y = 2 (half-height 1), Re_tau = 180 (nu = 1/180, u_tau = h = 1); unstructured
    triangles refined toward both walls (tanh stretching), interior nodes jittered, each cell
    split along a seeded random diagonal.
  * cavity: lid-driven unit square, walls on all sides, lid (y = 1) moving with U_w = (1, 0, 0),
    Re = 1e4 (nu = 1e-4); cosine clustering toward all four walls, jittered interior.

All node coordinates are FP32 values (stored as float64 that are exactly FP32), because the
particle state is FP32 and exact point location works on those exact values.

Edge tags (per element, edge k runs from vertex k to vertex (k+1) % 3):
  0 interior, 1 wall (U_w = 0), 2 moving wall (lid), 3 periodic boundary.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

EDGE_INTERIOR = 0
EDGE_WALL = 1
EDGE_MOVING_WALL = 2
EDGE_PERIODIC = 3

PERIOD_CHANNEL = float(np.float32(2.0 * math.pi))  # 6.2831854820251465

# Node-field layout on the hot path (per node, FP32). Index names follow Eq. 4, 5, 6, 9.
F_U, F_V, F_W = 0, 1, 2                          # <U_i>
F_DUDX, F_DUDY, F_DVDX, F_DVDY, F_DWDX, F_DWDY = 3, 4, 5, 6, 7, 8   # d<U_i>/dx_j
F_LAPU, F_LAPV, F_LAPW = 9, 10, 11               # laplacian of <U_i>
F_DPDX, F_DPDY = 12, 13                          # d<P>/dx_j / rho
F_G11, F_G12, F_G21, F_G22, F_G33 = 14, 15, 16, 17, 18   # G_ij (planar)
F_C0EPS = 19                                     # C_0 * epsilon
F_OMEGA = 20                                     # <omega>
F_SOMEGA = 21                                    # S_omega, Eq. 6
F_PHI0 = 22                                      # <phi_alpha>, alpha = 0..ns-1


def n_fields(ns: int) -> int:
    """Number of meaningful node fields for ns scalars."""
    return 22 + ns


def n_fields_padded(ns: int) -> int:
    """Row stride of the node-field table (multiple of 4 floats = 16 bytes)."""
    return (n_fields(ns) + 3) // 4 * 4


@dataclasses.dataclass
class Mesh:
    """A 2D triangle mesh in the form the library and the oracle both accept."""
    node_xy: np.ndarray      # (N, 2) float64, every value exactly representable in FP32
    tri: np.ndarray          # (E, 3) int32, counter-clockwise
    edge_tag: np.ndarray     # (E, 3) int32
    period_x: float          # 0.0 when not periodic
    box: tuple               # (x0, x1, y0, y1) domain bounds (FP32 values)
    kind: str
    nx: int
    ny: int

    @property
    def n_nodes(self) -> int:
        return int(self.node_xy.shape[0])

    @property
    def n_tri(self) -> int:
        return int(self.tri.shape[0])


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _triangulate(X: np.ndarray, Y: np.ndarray, rng: np.random.Generator):
    """Split each cell of an (nx+1) x (ny+1) node grid into two CCW triangles.

    Node (i, j) has index i*(ny+1) + j; element (i, j, d) has index 2*(i*ny + j) + d, so
    elements of one column are contiguous and neighbours are close in index.
    """
    nx, ny = X.shape[0] - 1, X.shape[1] - 1
    nid = lambda i, j: i * (ny + 1) + j
    diag = rng.integers(0, 2, size=(nx, ny))
    tri = np.empty((2 * nx * ny, 3), dtype=np.int64)
    for i in range(nx):
        for j in range(ny):
            a, b, c, d = nid(i, j), nid(i + 1, j), nid(i + 1, j + 1), nid(i, j + 1)
            e = 2 * (i * ny + j)
            if diag[i, j] == 0:      # diagonal a-c
                tri[e] = (a, b, c)
                tri[e + 1] = (a, c, d)
            else:                     # diagonal b-d
                tri[e] = (a, b, d)
                tri[e + 1] = (b, c, d)
    xy = np.stack([X.reshape(-1), Y.reshape(-1)], axis=1)
    # orientation check (CCW, strictly positive area)
    p0, p1, p2 = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    area2 = (p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p1[:, 1] - p0[:, 1]) * (p2[:, 0] - p0[:, 0])
    if not np.all(area2 > 0):
        raise ValueError("mesh generator produced a non-CCW or degenerate triangle")
    return xy, tri.astype(np.int32)


def _edge_tags(xy, tri, box, periodic_x: bool, lid: bool):
    x0, x1, y0, y1 = box
    E = tri.shape[0]
    tags = np.zeros((E, 3), dtype=np.int32)
    for k in range(3):
        a = xy[tri[:, k]]
        b = xy[tri[:, (k + 1) % 3]]
        bottom = (a[:, 1] == y0) & (b[:, 1] == y0)
        top = (a[:, 1] == y1) & (b[:, 1] == y1)
        left = (a[:, 0] == x0) & (b[:, 0] == x0)
        right = (a[:, 0] == x1) & (b[:, 0] == x1)
        tags[bottom, k] = EDGE_WALL
        tags[top, k] = EDGE_MOVING_WALL if lid else EDGE_WALL
        if periodic_x:
            tags[left | right, k] = EDGE_PERIODIC
        else:
            tags[left | right, k] = EDGE_WALL
    return tags


def channel_mesh(nx: int, ny: int, seed: int, gamma: float = 2.0, jitter: float = 0.2) -> Mesh:
    """Wall-refined channel [0, L) x [0, 2], L = fl32(2 pi), x periodic.

    nx*ny cells, E = 2*nx*ny triangles. Rows are tanh-clustered toward both walls; interior
    nodes are moved by up to +-jitter of the local spacing. The two periodic columns
    (x = 0 and x = L) carry identical y values so their edges pair exactly.
    """
    rng = np.random.default_rng(seed)
    L = PERIOD_CHANNEL
    s = np.linspace(-1.0, 1.0, ny + 1)
    yrow = 1.0 + np.tanh(gamma * s) / np.tanh(gamma)
    yrow[0], yrow[-1] = 0.0, 2.0
    xcol = np.linspace(0.0, L, nx + 1)
    X = np.repeat(xcol[:, None], ny + 1, axis=1).astype(np.float64)
    Y = np.repeat(yrow[None, :], nx + 1, axis=0).astype(np.float64)
    dx = L / nx
    dy = np.diff(yrow)
    dyloc = np.minimum(np.r_[dy[0], dy], np.r_[dy, dy[-1]])  # local row spacing
    jx = rng.uniform(-jitter, jitter, size=X.shape) * dx
    jy = rng.uniform(-jitter, jitter, size=Y.shape) * dyloc[None, :]
    jx[0, :] = 0.0
    jx[-1, :] = 0.0
    jy[:, 0] = 0.0
    jy[:, -1] = 0.0
    jy[-1, :] = jy[0, :]          # periodic pair columns share y
    X = X + jx
    Y = Y + jy
    X[-1, :] = L
    X, Y = _f32(X), _f32(Y)
    xy, tri = _triangulate(X, Y, rng)
    box = (0.0, L, 0.0, 2.0)
    tags = _edge_tags(xy, tri, box, periodic_x=True, lid=False)
    return Mesh(xy, tri, tags, L, box, "channel", nx, ny)


def cavity_mesh(nx: int, ny: int, seed: int, jitter: float = 0.2) -> Mesh:
    """Lid-driven unit cavity [0, 1] x [0, 1]; cosine clustering toward all walls; lid on top."""
    rng = np.random.default_rng(seed)
    xs = 0.5 * (1.0 - np.cos(np.pi * np.arange(nx + 1) / nx))
    ys = 0.5 * (1.0 - np.cos(np.pi * np.arange(ny + 1) / ny))
    xs[0], xs[-1], ys[0], ys[-1] = 0.0, 1.0, 0.0, 1.0
    X = np.repeat(xs[:, None], ny + 1, axis=1).astype(np.float64)
    Y = np.repeat(ys[None, :], nx + 1, axis=0).astype(np.float64)
    dxs, dys = np.diff(xs), np.diff(ys)
    dxl = np.minimum(np.r_[dxs[0], dxs], np.r_[dxs, dxs[-1]])
    dyl = np.minimum(np.r_[dys[0], dys], np.r_[dys, dys[-1]])
    jx = rng.uniform(-jitter, jitter, size=X.shape) * dxl[:, None]
    jy = rng.uniform(-jitter, jitter, size=Y.shape) * dyl[None, :]
    jx[0, :] = jx[-1, :] = 0.0
    jy[:, 0] = jy[:, -1] = 0.0
    jx[:, 0] = jx[:, -1] = 0.0     # keep boundary rows straight
    jy[0, :] = jy[-1, :] = 0.0
    X, Y = _f32(X + jx), _f32(Y + jy)
    xy, tri = _triangulate(X, Y, rng)
    box = (0.0, 1.0, 0.0, 1.0)
    tags = _edge_tags(xy, tri, box, periodic_x=False, lid=True)
    return Mesh(xy, tri, tags, 0.0, box, "cavity", nx, ny)


# --------------------------------------------------------------------------------------
# Synthetic node fields. They have the structure of the channel / cavity fields (log-law
# mean profile, wall-damped gradients, negative-definite G_ij, positive C_0 eps and <omega>)
# but are not a solution of anything; they are inputs for parity and throughput runs.
# --------------------------------------------------------------------------------------

def _loglaw(yw, re_tau=180.0):
    yp = re_tau * yw
    return np.where(yp < 11.0, yp, np.log(np.maximum(yp, 1e-30)) / 0.41 + 5.2)


def channel_wall_distance(mesh: Mesh) -> np.ndarray:
    """Distance of every node to the channel's walls: min(y, 2 - y) when both walls are flat
    (every wall node at y = 0 or y = 2), else the distance to the nearest wall edge (tags 1, 2;
    the x-periodic images included), e.g. over the bump of bump_channel_mesh."""
    xy = mesh.node_xy
    y = xy[:, 1]
    wall = [(e, k) for e in range(mesh.n_tri) for k in range(3) if mesh.edge_tag[e, k] in (1, 2)]
    wall_nodes = np.unique([mesh.tri[e, k] for e, k in wall] + [mesh.tri[e, (k + 1) % 3] for e, k in wall])
    if np.all((y[wall_nodes] == 0.0) | (y[wall_nodes] == 2.0)):
        return np.minimum(y, 2.0 - y)
    a = np.array([xy[mesh.tri[e, k]] for e, k in wall])
    d = np.array([xy[mesh.tri[e, (k + 1) % 3]] for e, k in wall]) - a
    best = np.full(len(xy), np.inf)
    for sx in ([-mesh.period_x, 0.0, mesh.period_x] if mesh.period_x > 0 else [0.0]):
        for i in range(len(a)):
            r = xy - a[i] - np.array([sx, 0.0])
            t = np.clip(r @ d[i] / (d[i] @ d[i]), 0.0, 1.0)
            best = np.minimum(best, np.hypot(r[:, 0] - t * d[i, 0], r[:, 1] - t * d[i, 1]))
    return best


def synthetic_node_fields(mesh: Mesh, ns: int, seed: int, noise: float = 0.05) -> np.ndarray:
    """(N, n_fields_padded(ns)) float32 node fields for parity / throughput runs."""
    rng = np.random.default_rng(seed)
    N = mesh.n_nodes
    nfp = n_fields_padded(ns)
    F = np.zeros((N, nfp), dtype=np.float64)
    x, y = mesh.node_xy[:, 0], mesh.node_xy[:, 1]
    if mesh.kind == "channel":
        yw = channel_wall_distance(mesh)
        U = _loglaw(yw)
        F[:, F_U] = U
        sgn = np.where(y < 1.0, 1.0, -1.0)
        F[:, F_DUDY] = sgn * np.where(180 * yw < 11.0, 180.0, 1.0 / (0.41 * np.maximum(yw, 1e-3)))
        F[:, F_LAPU] = -sgn * 0.0 + np.where(180 * yw < 11.0, 0.0, -1.0 / (0.41 * np.maximum(yw, 1e-2) ** 2)) * 1e-2
        F[:, F_DPDX] = -1.0                       # -d<P>/dx / rho = +1 drives the flow
        om = 1.0 / (0.3 * 0.41 * np.maximum(yw, 10.0 / 180.0))
        k = 1.0 + 3.0 * np.exp(-((180 * yw - 15.0) / 30.0) ** 2)
    else:
        F[:, F_U] = (y ** 3) * (1.0 - 0.5 * np.cos(2 * np.pi * x))
        F[:, F_V] = -0.2 * np.sin(np.pi * x) * np.sin(np.pi * y)
        F[:, F_DUDX] = np.pi * (y ** 3) * np.sin(2 * np.pi * x)
        F[:, F_DUDY] = 3 * y ** 2 * (1.0 - 0.5 * np.cos(2 * np.pi * x))
        F[:, F_DVDX] = -0.2 * np.pi * np.cos(np.pi * x) * np.sin(np.pi * y)
        F[:, F_DVDY] = -0.2 * np.pi * np.sin(np.pi * x) * np.cos(np.pi * y)
        F[:, F_LAPU] = 6 * y * (1.0 - 0.5 * np.cos(2 * np.pi * x)) + 2 * np.pi ** 2 * y ** 3 * np.cos(2 * np.pi * x)
        F[:, F_DPDX] = 0.05 * np.sin(np.pi * x)
        F[:, F_DPDY] = 0.05 * np.cos(np.pi * y)
        om = 1.0 + 2.0 * np.exp(-10 * np.minimum.reduce([x, 1 - x, y, 1 - y]))
        k = 0.01 * (1.0 + y)
    a = 0.5 + 0.75 * 2.1
    F[:, F_G11] = -a * om * (1.0 + noise * rng.standard_normal(N))
    F[:, F_G22] = -a * om * (1.0 + noise * rng.standard_normal(N))
    F[:, F_G33] = -a * om * (1.0 + noise * rng.standard_normal(N))
    F[:, F_G12] = 0.1 * om * noise * rng.standard_normal(N)
    F[:, F_G21] = 0.1 * om * noise * rng.standard_normal(N)
    F[:, F_C0EPS] = 2.1 * k * om
    F[:, F_OMEGA] = om
    F[:, F_SOMEGA] = 0.73 - 0.5 * np.clip(0.5 + 0.2 * rng.standard_normal(N), 0.0, 1.5)
    for a_ in range(ns):
        F[:, F_PHI0 + a_] = np.clip(0.1 + 0.05 * rng.standard_normal(N), 0.0, 1.0)
    # small smooth-ish noise on gradients so that every term of Eq. 4 is exercised
    for f in (F_DVDX, F_DVDY, F_DWDX, F_DWDY, F_LAPV, F_LAPW, F_V, F_W):
        F[:, f] += noise * rng.standard_normal(N)
    if mesh.period_x > 0.0:
        # periodic duplicate nodes (x = L) carry the same values as their x = 0 partners
        L = mesh.period_x
        right = np.nonzero(mesh.node_xy[:, 0] == L)[0]
        left = np.nonzero(mesh.node_xy[:, 0] == 0.0)[0]
        ly = {float(mesh.node_xy[i, 1]): i for i in left}
        for i in right:
            F[i] = F[ly[float(mesh.node_xy[i, 1])]]
    return F.astype(np.float32)


def synthetic_statistics(mesh: Mesh, ns: int, seed: int, noise: float = 0.02) -> np.ndarray:
    """(N, 11 + 2 ns) float64 gridpoint statistics in the layout of the statistics call (raw = 0):
    S0, <U>, <V>, <W>, <uu>, <uv>, <uw>, <vv>, <vw>, <ww>, <omega>, <phi_a> (ns), <phi_a'^2> (ns).

    Smooth wall-bounded profiles (channel: log-law mean, near-wall peak of the normal stresses,
    antisymmetric shear stress; cavity: a lid-driven vortex shape) with a little seeded noise,
    positive-definite stress tensors and positive frequency; periodic duplicates equal."""
    rng = np.random.default_rng(seed)
    N = mesh.n_nodes
    x, y = mesh.node_xy[:, 0], mesh.node_xy[:, 1]
    st = np.zeros((N, 11 + 2 * ns))
    st[:, 0] = 50.0 * (1.0 + 0.1 * rng.random(N))
    if mesh.kind == "channel":
        yw = np.minimum(y, 2.0 - y)
        sgn = np.where(y < 1.0, 1.0, -1.0)
        st[:, 1] = _loglaw(yw) / 20.0
        st[:, 2] = 0.05 * np.sin(x) * np.sin(np.pi * y / 2.0)
        bump = np.exp(-((180.0 * yw - 15.0) / 30.0) ** 2)
        uu = 0.5 + 3.0 * bump
        vv = 0.3 + 0.5 * bump
        ww = 0.4 + 1.0 * bump
        uv = -0.4 * sgn * np.sqrt(uu * vv) * np.tanh(10.0 * yw)
        om = 1.0 / (0.3 * 0.41 * np.maximum(yw, 10.0 / 180.0)) / 20.0 + 1.0
    else:
        st[:, 1] = (y ** 3) * (1.0 - 0.5 * np.cos(2 * np.pi * x))
        st[:, 2] = -0.2 * np.sin(np.pi * x) * np.sin(np.pi * y)
        uu = 0.02 * (1.0 + y)
        vv = 0.015 * (1.0 + x * y)
        ww = 0.01 * (1.5 - 0.5 * x)
        uv = -0.3 * np.sqrt(uu * vv) * np.sin(np.pi * x) * y
        om = 1.0 + 2.0 * np.exp(-10 * np.minimum.reduce([x, 1 - x, y, 1 - y]))
    st[:, 3] = 0.01 * rng.standard_normal(N)
    st[:, 1] += noise * rng.standard_normal(N) * np.abs(st[:, 1]).max()
    st[:, 2] += noise * 0.1 * rng.standard_normal(N)
    st[:, 4] = uu * (1.0 + noise * rng.standard_normal(N))
    st[:, 5] = uv
    st[:, 6] = 0.05 * np.sqrt(uu * ww) * rng.standard_normal(N) * noise
    st[:, 7] = vv * (1.0 + noise * rng.standard_normal(N))
    st[:, 8] = 0.05 * np.sqrt(vv * ww) * rng.standard_normal(N) * noise
    st[:, 9] = ww * (1.0 + noise * rng.standard_normal(N))
    st[:, 10] = om * (1.0 + noise * rng.standard_normal(N))
    for a in range(ns):
        st[:, 11 + a] = np.clip(0.1 + 0.05 * rng.standard_normal(N), 0.0, 1.0)
        st[:, 11 + ns + a] = 0.01 * rng.random(N)
    if mesh.period_x > 0.0:
        right = np.nonzero(x == mesh.period_x)[0]
        left = np.nonzero(x == 0.0)[0]
        ly = {float(y[i]): i for i in left}
        for i in right:
            st[i] = st[ly[float(y[i])]]
    return st


def node_init_fields(mesh: Mesh, sigma: float = 1.0, re_tau: float = 180.0) -> np.ndarray:
    """(N, 8) float32 initial-condition fields per node: <U>, <V>, <W>, sigma_u, <omega>, pad.

    Channel: log-law mean (U = y+ for y+ < 11, else ln(y+)/0.41 + 5.2, y+ = Re_tau * y_wall),
    sigma = 1, <omega> = 1/(0.3 * 0.41 * max(y_wall, 10/Re_tau)).
    Cavity: U = 0, sigma = 0.1, <omega> = 1.
    """
    N = mesh.n_nodes
    out = np.zeros((N, 8), dtype=np.float64)
    y = mesh.node_xy[:, 1]
    if mesh.kind == "channel":
        yw = channel_wall_distance(mesh)
        out[:, 0] = _loglaw(yw, re_tau)
        out[:, 3] = sigma
        out[:, 4] = 1.0 / (0.3 * 0.41 * np.maximum(yw, 10.0 / re_tau))
    else:
        out[:, 3] = 0.1
        out[:, 4] = 1.0
    return out.astype(np.float32)


@dataclasses.dataclass
class State:
    """SoA particle state (host copy). Positions and all fields are FP32."""
    x: np.ndarray
    y: np.ndarray
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    omega: np.ndarray
    psi: np.ndarray          # (ns, P)
    elem: np.ndarray         # int32
    pid: np.ndarray          # uint32

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def copy(self) -> "State":
        return State(*(np.array(getattr(self, f.name), copy=True) for f in dataclasses.fields(self)))


def synthetic_state(mesh: Mesh, n_per_elem: int, ns: int, seed: int, margin: float = 0.01,
                    speed: float = 1.0) -> State:
    """Particles strictly inside their elements (every barycentric >= margin), sorted by element.

    Velocities are N(interpolation-free guess, 1): U from a log-law in the channel, small in the
    cavity; omega ~ Gamma(4, 1/4) * <omega> guess; psi ~ U[0, 1]. Strict interiority makes the
    owning element known by construction, so no point location is needed to build the input.
    """
    rng = np.random.default_rng(seed)
    E = mesh.n_tri
    P = E * n_per_elem
    elem = np.repeat(np.arange(E, dtype=np.int32), n_per_elem)
    r = rng.uniform(margin, 1.0 - 2 * margin, size=(P, 3))
    r = r / r.sum(axis=1, keepdims=True)
    r = np.clip(r, margin, None)
    r = r / r.sum(axis=1, keepdims=True)
    v = mesh.node_xy[mesh.tri[elem]]          # (P, 3, 2)
    xy = np.einsum("pk,pkd->pd", r, v)
    x = xy[:, 0].astype(np.float32)
    y = xy[:, 1].astype(np.float32)
    if mesh.kind == "channel":
        yw = np.minimum(y, 2.0 - y).astype(np.float64)
        U0 = _loglaw(yw)
        om0 = 1.0 / (0.3 * 0.41 * np.maximum(yw, 10.0 / 180.0))
    else:
        U0 = np.zeros(P)
        om0 = np.ones(P)
    u = (speed * U0 + rng.standard_normal(P)).astype(np.float32)
    vv = rng.standard_normal(P).astype(np.float32)
    w = rng.standard_normal(P).astype(np.float32)
    omega = (om0 * rng.gamma(4.0, 0.25, size=P)).astype(np.float32)
    psi = rng.uniform(0.0, 1.0, size=(ns, P)).astype(np.float32)
    pid = np.arange(P, dtype=np.uint32)
    return State(x, y, u, vv, w, omega, psi, elem, pid)


# --------------------------------------------------------------------------------------
# Named workloads (sizes of the channel and cavity configurations).
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    mesh: Mesh
    n_per_elem: int
    ns: int
    nu: float
    dt: float
    seed: int
    lid_u: float
    sources: list            # [(x, y, r, alpha), ...]

    @property
    def n_particles(self) -> int:
        return self.mesh.n_tri * self.n_per_elem


def channel_small(seed: int = 1006054901) -> Workload:
    """~1,000-triangle channel, 50 particles per element (~50k particles), one scalar."""
    m = channel_mesh(25, 20, seed)
    return Workload("channel-1k-50k", m, 50, 1, 1.0 / 180.0, 1e-3, seed, 0.0, [(0.25, 0.67, 0.02, 0)])


def channel_25m(seed: int = 1006054902) -> Workload:
    """50,000-triangle wall-refined channel, 500 particles per element (25M particles), one scalar."""
    m = channel_mesh(250, 100, seed)
    return Workload("channel-50k-25M", m, 500, 1, 1.0 / 180.0, 1e-3, seed, 0.0, [(0.25, 0.67, 0.02, 0)])


def cavity_20m(seed: int = 1006054903) -> Workload:
    """~200,000-triangle lid-driven cavity, 100 particles per element (~20M), four scalars."""
    m = cavity_mesh(316, 316, seed)
    src = [(0.25, 0.25, 0.01, 0), (0.75, 0.25, 0.01, 1), (0.5, 0.5, 0.01, 2), (0.5, 0.8, 0.01, 3)]
    return Workload("cavity-200k-20M", m, 100, 4, 1e-4, 1e-3, seed, 1.0, src)


def cavity_small(seed: int = 1006054903) -> Workload:
    """Small cavity (2,048 triangles, 50 per element) with the cavity's physics, for parity."""
    m = cavity_mesh(32, 32, seed)
    src = [(0.25, 0.25, 0.02, 0), (0.75, 0.25, 0.02, 1), (0.5, 0.5, 0.02, 2), (0.5, 0.8, 0.02, 3)]
    return Workload("cavity-2k-100k", m, 50, 4, 1e-4, 1e-3, seed, 1.0, src)


def mlp_init_params(seed: int, n_in: int = 8, hidden: int = 128, n_out: int = 7) -> np.ndarray:
    """Seeded starting parameters of the surrogate network (ABI order W1, b1, W2, b2, W3, b3, W4, b4;
    W [out][in]): weights uniform in +-sqrt(6 / (fan_in + fan_out)) (Glorot), biases zero."""
    rng = np.random.default_rng(seed)
    parts = []
    for fi, fo in ((n_in, hidden), (hidden, hidden), (hidden, hidden), (hidden, n_out)):
        a = np.sqrt(6.0 / (fi + fo))
        parts.append(rng.uniform(-a, a, size=fo * fi))
        parts.append(np.zeros(fo))
    return np.concatenate(parts).astype(np.float32)


def mlp_random_data(n: int, seed: int, n_in: int = 8, n_out: int = 7):
    """Seeded regression data for the network alone: features with unequal scales and offsets and
    smooth nonlinear targets of them (float32 arrays n x n_in and n x n_out)."""
    rng = np.random.default_rng(seed)
    scale = np.linspace(0.5, 3.0, n_in)
    shift = np.linspace(-1.0, 2.0, n_in)
    feat = shift + scale * rng.standard_normal((n, n_in))
    z = (feat - shift) / scale
    mix = rng.standard_normal((n_in, n_out)) / np.sqrt(n_in)
    tgt = np.sin(z @ mix) + 0.3 * (z[:, :n_out] ** 2 if n_out <= n_in else 0.0) + np.arange(n_out)
    return feat.astype(np.float32), tgt.astype(np.float32)


@dataclasses.dataclass
class MultiMesh(Mesh):
    """Several independent meshes held as one (lpdf_mesh_load_multi): nodes and elements of
    component c are [node_off[c], node_off[c + 1]) and [tri_off[c], tri_off[c + 1])."""
    node_off: np.ndarray = None
    tri_off: np.ndarray = None
    parts: list = None


def union_mesh(meshes) -> MultiMesh:
    """The disjoint union of meshes that share one x period (or none): node ids offset per part."""
    period = meshes[0].period_x
    assert all(m.period_x == period for m in meshes), "components must share the x period"
    node_off = np.zeros(len(meshes) + 1, dtype=np.int64)
    tri_off = np.zeros(len(meshes) + 1, dtype=np.int64)
    for k, m in enumerate(meshes):
        node_off[k + 1] = node_off[k] + m.n_nodes
        tri_off[k + 1] = tri_off[k] + m.n_tri
    xy = np.concatenate([m.node_xy for m in meshes])
    tri = np.concatenate([m.tri + node_off[k] for k, m in enumerate(meshes)]).astype(np.int32)
    tag = np.concatenate([m.edge_tag for m in meshes]).astype(np.int32)
    box = (min(m.box[0] for m in meshes), max(m.box[1] for m in meshes),
           min(m.box[2] for m in meshes), max(m.box[3] for m in meshes))
    return MultiMesh(xy, tri, tag, period, box, meshes[0].kind, 0, 0, node_off, tri_off, list(meshes))


def stack_node_arrays(parts) -> np.ndarray:
    """Per-node arrays of the components, one after the other (the union's node order)."""
    return np.ascontiguousarray(np.concatenate(parts))


@dataclasses.dataclass
class BatchedWorkload:
    name: str
    mesh: MultiMesh
    n_per_elem: list          # per component
    seeds: list               # per component
    sources: list             # per component: [(x, y, r, alpha)]
    ns: int
    nu: float
    dt: float

    @property
    def n_particles(self) -> int:
        return int(sum((self.mesh.tri_off[k + 1] - self.mesh.tri_off[k]) * p
                       for k, p in enumerate(self.n_per_elem)))


def batched_channels(n: int = 64, tri_range=(2000, 40000), ppe_range=(50, 400), seed: int = 1006054904,
                     source_y=(0.2, 1.8)) -> BatchedWorkload:
    """n independent channel ensembles of uneven size: component k has about E_k ~ U[tri_range]
    triangles (nx : ny = 5 : 2, so E = 2 nx ny = 5 ny^2), ppe_k ~ U{ppe_range} particles per
    element, seed = seed + k and one scalar line source (a disc of radius 0.02 at x = 0.25) at a
    height ~ U[source_y]; the draws come from one generator seeded with `seed`."""
    rng = np.random.default_rng(seed)
    meshes, ppe, seeds, srcs = [], [], [], []
    for k in range(n):
        E = rng.uniform(*tri_range)
        ny = max(2, int(round(np.sqrt(E / 5.0))))
        nx = max(3, int(round(2.5 * ny)))
        meshes.append(channel_mesh(nx, ny, seed + k))
        ppe.append(int(rng.integers(ppe_range[0], ppe_range[1] + 1)))
        seeds.append(seed + k)
        srcs.append([(0.25, float(np.float32(rng.uniform(*source_y))), 0.02, 0)])
    return BatchedWorkload(f"channels-x{n}", union_mesh(meshes), ppe, seeds, srcs, 1, 1.0 / 180.0, 1e-3)


def bump_channel_mesh(nx: int, ny: int, seed: int, amp: float = 0.15, jitter: float = 0.2) -> Mesh:
    """The periodic channel of channel_mesh with a smooth bump on the bottom wall: every node moves
    up by h(s) (1 - y / 2), h(s) = amp (1 - cos 2 pi s) / 2, s = the node column's position along
    the channel (0 and 1 at the periodic columns, which therefore keep their y values and their
    pairing). The bottom wall is curved and the fluid side of it is non-convex; the top wall stays
    flat. Coordinates are rounded to FP32."""
    m = channel_mesh(nx, ny, seed, jitter=jitter)
    x, y = m.node_xy[:, 0], m.node_xy[:, 1]
    s = x / m.period_x
    h = amp * 0.5 * (1.0 - np.cos(2.0 * np.pi * s))
    h[(x == 0.0) | (x == m.period_x)] = 0.0
    xy = np.stack([x, _f32(y + h * (1.0 - 0.5 * y))], axis=1)
    box = (0.0, m.period_x, float(xy[:, 1].min()), float(xy[:, 1].max()))
    return Mesh(xy, m.tri, m.edge_tag, m.period_x, box, "channel", nx, ny)


def trapezoid_mesh(nx: int, ny: int, seed: int, jitter: float = 0.2) -> Mesh:
    """The cavity mesh mapped to the convex quadrilateral with corners (0, 0), (1, 0), (1.3, 1.2)
    and (0.3, 0.8) by x' = x + 0.3 y, y' = y (0.8 + 0.4 x): three slanted walls (the top one
    keeps the lid tag) and a flat bottom. Coordinates are rounded to FP32."""
    m = cavity_mesh(nx, ny, seed, jitter=jitter)
    x, y = m.node_xy[:, 0], m.node_xy[:, 1]
    xy = np.stack([_f32(x + 0.3 * y), _f32(y * (0.8 + 0.4 * x))], axis=1)
    box = (float(xy[:, 0].min()), float(xy[:, 0].max()), float(xy[:, 1].min()), float(xy[:, 1].max()))
    return Mesh(xy, m.tri, m.edge_tag, 0.0, box, "cavity", nx, ny)
