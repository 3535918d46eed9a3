"""FP64 oracle of the learned surrogate of the elliptic-relaxation solve.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). numpy, no code shared with the CUDA path.

The paper obtains G_ij from an elliptic relaxation equation (the paragraph after Eq. 4); it has
no learned part. What is stated here is the definition of the network that stands in for that
solve and of its training:

* inputs per gridpoint: wall distance, ln k, ln <omega>, the anisotropy b_ij = <u_i u_j>/(2k) -
  delta_ij/3 (b11, b22, b12; b33 = -b11 - b22 is implied) and its second invariant II_b =
  b_ij b_ij, with k = <u_i u_i>/2 (the paragraph before Eq. 5), and the wall effect
  ln(eps_w / eps): eps = k <omega> (the paragraph before Eq. 5), eps_w its value at the nearest
  wall point, interpolated linearly along that wall edge (the wall enters the relaxation only
  through its boundary values, which scale with the wall's eps);
* targets: G11, G12, G21, G22, G33 over <omega>, C0 eps/(k <omega>) and the relaxed trace
  wp_ii = k G_ii + 3 eps/2 over its local value -9/4 C0 eps (eps = k <omega>);
* network 8 -> 128 -> 128 -> 128 -> 7, tanh on the hidden layers, standardised inputs and
  targets, mean squared error with per-output weights;
* the tensor-core arithmetic: inputs, weights, activations and, in the backward pass, the error
  signals of the matrix products are rounded to bfloat16 (round to nearest even); sums are
  exact here (FP64), FP32 on the GPU; biases, tanh and the bias gradients use unrounded values;
* Adam (Kingma & Ba) with bias correction.

With ``bf16=False`` every rounding is skipped: that is the plain FP64 network, whose gradient is
pinned by finite differences.
"""
from __future__ import annotations

import numpy as np

IN, H, OUT = 8, 128, 7
NPARAMS = H * IN + H + 2 * (H * H + H) + OUT * H + OUT      # 35,079
NNORM = 2 * IN + 3 * OUT                                      # 37
K_MIN = 1e-12
OM_MIN = 1e-12
EPS_MIN = 1e-12


def bf16(x):
    """Round to bfloat16, nearest even (the value as float64). x is first taken as float32."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if np.any(nan):
        out = np.where(nan, np.nan, out)
    return out


def unpack(p):
    """Parameter vector (ABI order) -> [(W1, b1), (W2, b2), (W3, b3), (W4, b4)], W [out][in]."""
    p = np.asarray(p, dtype=np.float64)
    assert p.size == NPARAMS
    shapes = [(H, IN), (H,), (H, H), (H,), (H, H), (H,), (OUT, H), (OUT,)]
    out, at = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(p[at:at + n].reshape(s))
        at += n
    return [(out[0], out[1]), (out[2], out[3]), (out[4], out[5]), (out[6], out[7])]


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def norm_parts(norm):
    n = np.asarray(norm, dtype=np.float64)
    assert n.size == NNORM
    return dict(fm=n[0:8], fs=n[8:16], w=n[16:23], tm=n[23:30], ts=n[30:37])


def identity_norm():
    n = np.zeros(NNORM)
    n[8:16] = 1.0
    n[16:23] = 1.0
    n[30:37] = 1.0
    return n


def standardised_inputs(norm, feat, rounding=True):
    """x = (feature - mean) / deviation, in FP32 as the kernel forms it (then BF16 if rounding)."""
    nm = norm_parts(norm)
    f = np.asarray(feat, dtype=np.float32)
    x = ((f - nm["fm"].astype(np.float32)) / nm["fs"].astype(np.float32)).astype(np.float64)
    return bf16(x) if rounding else x


def forward(params, norm, feat, bf16_ops=True):
    """Standardised outputs (B x 7) and the hidden activations [a1, a2, a3] (as rounded)."""
    r = bf16 if bf16_ops else (lambda v: np.asarray(v, dtype=np.float64))
    layers = unpack(params)
    a = standardised_inputs(norm, feat, bf16_ops)
    acts = []
    for W, b in layers[:3]:
        z = a @ r(W).T + b
        a = r(np.tanh(z))
        acts.append(a)
    W4, b4 = layers[3]
    y = a @ r(W4).T + b4
    return y, acts


def forward_user(params, norm, feat, bf16_ops=True):
    """Outputs in target units: standardised output x target deviation + target mean."""
    nm = norm_parts(norm)
    y, _ = forward(params, norm, feat, bf16_ops)
    return y * nm["ts"] + nm["tm"]


def standardised_targets(norm, tgt):
    nm = norm_parts(norm)
    return (np.asarray(tgt, dtype=np.float64) - nm["tm"]) / nm["ts"]


def loss(params, norm, feat, tgt, bf16_ops=True):
    """Sum over rows and outputs of w_j (y_j - t_j)^2 / (7 B), y and t standardised."""
    y, _ = forward(params, norm, feat, bf16_ops)
    t = standardised_targets(norm, tgt)
    w = norm_parts(norm)["w"]
    return float(np.sum(w * (y - t) ** 2) / (OUT * y.shape[0]))


def gradient(params, norm, feat, tgt, bf16_ops=True):
    """(d loss / d params in ABI order, loss) by back-propagation through the network above.

    With bf16_ops the error signals entering the matrix products are rounded as on the tensor
    cores; the rounding of weights and activations is treated as the identity for the derivative
    (the gradient of the rounded network with respect to its unrounded parameters)."""
    r = bf16 if bf16_ops else (lambda v: np.asarray(v, dtype=np.float64))
    layers = unpack(params)
    x = standardised_inputs(norm, feat, bf16_ops)
    y, acts = forward(params, norm, feat, bf16_ops)
    B = y.shape[0]
    t = standardised_targets(norm, tgt)
    w = norm_parts(norm)["w"]
    dz = 2.0 * (y - t) * w / (OUT * B)                  # d loss / d z4
    ins = [x] + acts[:-1]                               # input of layers 1..3
    grads = [None] * 4
    # output layer
    grads[3] = (r(dz).T @ acts[2], dz.sum(axis=0))
    dh = r(dz) @ r(layers[3][0])                        # d loss / d a3
    for l in (2, 1, 0):
        dz = dh * (1.0 - acts[l] ** 2)                 # tanh' = 1 - a^2 (a as stored)
        grads[l] = (r(dz).T @ ins[l], dz.sum(axis=0))
        if l > 0:
            dh = r(dz) @ r(layers[l][0])
    L = float(np.sum(w * (y - t) ** 2) / (OUT * B))
    return pack(grads), L


def adam(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (step counts from 1): returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# ------------------------------------------------------------------ inputs and targets per node

def wall_edges(mesh):
    """(n, 2) end nodes of the wall edges (tags 1, 2), in element order."""
    return np.array([(mesh.tri[e, k], mesh.tri[e, (k + 1) % 3]) for e in range(mesh.tri.shape[0])
                     for k in range(3) if mesh.edge_tag[e, k] in (1, 2)], dtype=np.int64).reshape(-1, 2)


def nearest_wall_point(mesh):
    """Per node: distance to the nearest wall point, its wall edge and its position t on the edge
    (0 at the first end node). Edges in element order, each tried at x - period, x, x + period; the
    first strictly nearest point wins."""
    xy = np.asarray(mesh.node_xy, dtype=np.float64)
    edges = wall_edges(mesh)
    n = xy.shape[0]
    best, bs, bt = np.full(n, np.inf), np.zeros(n, dtype=np.int64), np.zeros(n)
    shifts = [0.0] if not mesh.period_x > 0 else [-mesh.period_x, 0.0, mesh.period_x]
    for i, (a, b) in enumerate(edges):
        t = xy[b] - xy[a]
        for sx in shifts:
            q = xy - xy[a] - np.array([sx, 0.0])
            s = np.clip(q @ t / (t @ t), 0.0, 1.0)
            d2 = (q[:, 0] - s * t[0]) ** 2 + (q[:, 1] - s * t[1]) ** 2
            closer = d2 < best
            best[closer], bs[closer], bt[closer] = d2[closer], i, s[closer]
    if len(edges) == 0:
        best[:] = 0.0
    return np.sqrt(best), bs, bt


def wall_distance(mesh):
    """Distance of every node to the nearest wall edge (tags 1, 2), periodic images included."""
    return nearest_wall_point(mesh)[0]


def features(mesh, stats):
    """(n_nodes, 8) inputs from statistics rows (lpdf_grid_statistics raw = 0 layout)."""
    st = np.asarray(stats, dtype=np.float64)
    uu, uv, uw, vv, vw, ww, om = (st[:, i] for i in (4, 5, 6, 7, 8, 9, 10))
    k = 0.5 * (uu + vv + ww)
    R = np.zeros((st.shape[0], 3, 3))
    R[:, 0, 0], R[:, 0, 1], R[:, 0, 2] = uu, uv, uw
    R[:, 1, 0], R[:, 1, 1], R[:, 1, 2] = uv, vv, vw
    R[:, 2, 0], R[:, 2, 1], R[:, 2, 2] = uw, vw, ww
    live = k > K_MIN
    b = np.zeros_like(R)
    b[live] = R[live] / (2.0 * k[live, None, None]) - np.eye(3) / 3.0
    eps = k * om
    dist, edge, t = nearest_wall_point(mesh)
    f = np.zeros((st.shape[0], IN))
    f[:, 0] = dist
    f[:, 1] = np.log(np.maximum(k, K_MIN))
    f[:, 2] = np.log(np.maximum(om, OM_MIN))
    f[:, 3] = b[:, 0, 0]
    f[:, 4] = b[:, 1, 1]
    f[:, 5] = b[:, 0, 1]
    f[:, 6] = np.einsum("nij,nij->n", b, b)
    edges = wall_edges(mesh)
    if len(edges):
        eps_w = (1.0 - t) * eps[edges[edge, 0]] + t * eps[edges[edge, 1]]
        f[:, 7] = np.log(np.maximum(eps_w, EPS_MIN) / np.maximum(eps, EPS_MIN))
    return f


def targets(stats, fields, C0):
    """(n_nodes, 7) targets from statistics rows and node fields (LPDF_F_* columns)."""
    st = np.asarray(stats, dtype=np.float64)
    F = np.asarray(fields, dtype=np.float64)
    k = 0.5 * (st[:, 4] + st[:, 7] + st[:, 9])
    om = st[:, 10]
    omc, kc, eps = np.maximum(om, OM_MIN), np.maximum(k, K_MIN), k * om
    G = F[:, 14:19]                              # G11, G12, G21, G22, G33
    y = np.zeros((st.shape[0], OUT))
    y[:, 0:5] = G / omc[:, None]
    y[:, 5] = F[:, 19] / (kc * omc)
    trace = k * (G[:, 0] + G[:, 3] + G[:, 4]) + 1.5 * eps
    safe = np.where(eps > EPS_MIN, eps, 1.0)
    y[:, 6] = np.where(eps > EPS_MIN, trace / (-2.25 * C0 * safe), 1.0)
    return y


def fields_from_outputs(stats, y_user):
    """G11, G12, G21, G22, G33 and C0 eps from network outputs in target units."""
    st = np.asarray(stats, dtype=np.float64)
    k = 0.5 * (st[:, 4] + st[:, 7] + st[:, 9])
    om = st[:, 10]
    G = om[:, None] * y_user[:, 0:5]
    c0e = np.maximum(0.0, k * om * y_user[:, 5])
    return G, c0e
