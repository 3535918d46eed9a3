"""The certified fast walk test (affine barycentrics relative to vertex 0, FP32, with a rounding
bound): whenever it decides "inside" or "outside through edge k", the exact orientation of the
FP32 point agrees. Emulated here in numpy float32 (with and without the fused multiply-add the
compiler may use), on the elements of both workload meshes and points placed at the rounding
distance of their edges and vertices."""
from fractions import Fraction

import numpy as np

from paper_1006_0549_gb300 import workloads as wl

U = 2.0 ** -24


def coefficients(xy):
    a, b, c = xy
    A = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
    f = np.float32
    return (f(a[0]), f(a[1]), f((c[1] - a[1]) / A), f(-(c[0] - a[0]) / A), f(-(b[1] - a[1]) / A), f((b[0] - a[0]) / A))


def fast(coef, px, py, fma):
    f = np.float32
    x0, y0, b1, g1, b2, g2 = coef
    dx, dy = f(f(px) - x0), f(f(py) - y0)
    t1, s1, t2, s2 = f(b1 * dx), f(g1 * dy), f(b2 * dx), f(g2 * dy)
    if fma:   # one rounding of b*dx + s
        l1 = f(float(b1) * float(dx) + float(s1))
        l2 = f(float(b2) * float(dx) + float(s2))
    else:
        l1, l2 = f(t1 + s1), f(t2 + s2)
    l0 = f(f(f(1.0) - l1) - l2)
    E1 = f(f(3.0e-7) * f(abs(t1) + abs(s1))) + f(1e-30)
    E2 = f(f(3.0e-7) * f(abs(t2) + abs(s2))) + f(1e-30)
    E0 = f(E1 + E2 + f(1.5e-7) * f(1.0 + abs(l1) + abs(l2)))
    if l0 > E0 and l1 > E1 and l2 > E2:
        return "in", None
    lam = [l0, l1, l2]
    a = int(np.argmin(lam))
    if lam[a] < -[E0, E1, E2][a]:
        return "out", a
    return "undecided", None


def exact_signs(xy, px, py):
    """Signs of the exact barycentrics of the FP32 point (px, py): orientation of the point
    against the edge opposite each vertex."""
    P = [(Fraction(float(x)), Fraction(float(y))) for x, y in xy]
    q = (Fraction(float(px)), Fraction(float(py)))
    out = []
    for a in range(3):
        u, v = P[(a + 1) % 3], P[(a + 2) % 3]
        d = (v[0] - u[0]) * (q[1] - u[1]) - (v[1] - u[1]) * (q[0] - u[0])
        out.append((d > 0) - (d < 0))
    return out


def test_fast_walk_decisions_are_certified():
    rng = np.random.default_rng(7)
    checked = decided = 0
    for mesh in (wl.channel_mesh(250, 100, 1006054902), wl.cavity_mesh(64, 64, 3)):
        for e in rng.choice(mesh.n_tri, 300, replace=False):
            xy = mesh.node_xy[mesh.tri[e]].astype(np.float64)
            coef = coefficients(xy)
            for _ in range(12):
                # a point on an edge or at a vertex, then nudged by a few ulps either way
                k = rng.integers(3)
                t = rng.choice([0.0, 1.0, rng.random()])
                p = xy[k] + t * (xy[(k + 1) % 3] - xy[k])
                px, py = np.float32(p[0]), np.float32(p[1])
                for _ in range(int(rng.integers(0, 4))):
                    px = np.nextafter(px, np.float32(rng.choice([-1e9, 1e9])), dtype=np.float32)
                    py = np.nextafter(py, np.float32(rng.choice([-1e9, 1e9])), dtype=np.float32)
                signs = exact_signs(xy, px, py)
                for fma in (False, True):
                    decision, a = fast(coef, px, py, fma)
                    checked += 1
                    if decision == "in":
                        decided += 1
                        assert min(signs) > 0, (e, px, py, signs)
                    elif decision == "out":
                        decided += 1
                        assert signs[a] < 0, (e, px, py, signs, a)
            # and clearly interior points are decided
            px, py = np.float32(xy.mean(0)[0]), np.float32(xy.mean(0)[1])
            assert fast(coef, px, py, False)[0] == "in"
    assert decided > checked // 4    # the filter decides a good share even at the edges
