"""Positions exactly on the edges and at the vertices of a mesh, and a few FP32 ulps either side.

These are the inputs of the ownership tests at exact hits (the top-left rule, Introduction item
iii: tracking through the grid). Whether an FP32 point lies exactly on an edge is decided here by
rational arithmetic (``fractions.Fraction`` of the float values), independently of the oracle and
of the CUDA path. Each point comes with start elements for the walk: the elements that share the
edge (or the vertex), so that a walk that starts in the element that does not own the point must
leave it through the very edge the point lies on.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

# parameters along an edge whose FP32 images are tried as exact points (dyadic, so the FP64 value
# of a + t (b - a) is often an FP32 number)
_T = (0.5, 0.25, 0.75, 0.125, 0.375, 0.625, 0.875)
# ulp offsets (in x, in y) of the perturbed copies of every exact point
OFFSETS = ((1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (1, -1), (-1, 1), (3, 0), (0, -3), (2, -2), (-2, 3))


def _step(v: np.float32, k: int) -> np.float32:
    d = np.float32(np.inf) if k > 0 else np.float32(-np.inf)
    for _ in range(abs(k)):
        v = np.nextafter(v, d)
    return v


def _on_segment(ax, ay, bx, by, px, py) -> bool:
    """Exactly on the closed segment a-b, excluding its end points (rational arithmetic)."""
    A, B, P = (Fraction(ax), Fraction(ay)), (Fraction(bx), Fraction(by)), (Fraction(px), Fraction(py))
    cross = (B[0] - A[0]) * (P[1] - A[1]) - (B[1] - A[1]) * (P[0] - A[0])
    if cross != 0 or (px, py) == (ax, ay) or (px, py) == (bx, by):
        return False
    return min(A[0], B[0]) <= P[0] <= max(A[0], B[0]) and min(A[1], B[1]) <= P[1] <= max(A[1], B[1])


def edge_elements(mesh):
    """{(lo node, hi node): [(element, local edge k)]} over every edge of the mesh."""
    out = {}
    for e in range(mesh.n_tri):
        for k in range(3):
            a, b = int(mesh.tri[e, k]), int(mesh.tri[e, (k + 1) % 3])
            out.setdefault((min(a, b), max(a, b)), []).append((e, k))
    return out


def exact_points(mesh, max_edges: int | None = None, seed: int = 0):
    """(px, py, start, kind) arrays: kind 0 = a vertex, 1 = exactly on an edge (interior, wall or
    periodic), 2 = a perturbed copy (OFFSETS ulps away) of one of those. Every point is listed once
    per start element (the elements around the vertex, or the two sharing the edge)."""
    xy = mesh.node_xy
    pts = []          # (x32, y32, [starts], kind)
    # vertices and the elements around them
    around = [[] for _ in range(mesh.n_nodes)]
    for e in range(mesh.n_tri):
        for k in range(3):
            around[int(mesh.tri[e, k])].append(e)
    for nd in range(mesh.n_nodes):
        if around[nd]:
            # at most three starts per vertex: the first, a middle and the last element around it
            s = around[nd]
            starts = sorted({s[0], s[len(s) // 2], s[-1]})
            pts.append((np.float32(xy[nd, 0]), np.float32(xy[nd, 1]), starts, 0))
    # exact points on edges
    edges = edge_elements(mesh)
    keys = sorted(edges)
    if max_edges is not None and len(keys) > max_edges:
        rng = np.random.default_rng(seed)
        keys = [keys[i] for i in sorted(rng.choice(len(keys), max_edges, replace=False))]
    for a, b in keys:
        ax, ay, bx, by = (float(xy[a, 0]), float(xy[a, 1]), float(xy[b, 0]), float(xy[b, 1]))
        starts = sorted({e for e, _ in edges[(a, b)]})
        found = set()
        for t in _T:
            mx, my = np.float32(ax + t * (bx - ax)), np.float32(ay + t * (by - ay))
            for i in (-1, 0, 1):
                for j in (-1, 0, 1):
                    px, py = _step(mx, i), _step(my, j)
                    key = (float(px), float(py))
                    if key not in found and _on_segment(ax, ay, bx, by, *key):
                        found.add(key)
        for px, py in sorted(found)[:3]:
            pts.append((np.float32(px), np.float32(py), starts, 1))
    # perturbed copies
    base = list(pts)
    for px, py, starts, _ in base:
        for i, j in OFFSETS:
            pts.append((_step(px, i), _step(py, j), starts, 2))
    X, Y, S, K = [], [], [], []
    for px, py, starts, kind in pts:
        for s in starts:
            X.append(px)
            Y.append(py)
            S.append(s)
            K.append(kind)
    return (np.asarray(X, dtype=np.float32), np.asarray(Y, dtype=np.float32), np.asarray(S, dtype=np.int32),
            np.asarray(K, dtype=np.int8))


def in_box(mesh, px, py):
    x0, x1, y0, y1 = mesh.box
    return (px >= x0) & (px <= x1) & (py >= y0) & (py <= y1)
