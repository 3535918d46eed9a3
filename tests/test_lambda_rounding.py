"""The rounding bound of the FP32 barycentric weights that the moments kernel forms (the term
LAMBDA_RTOL * sum kappa |q| of the FP32 moment-sum tolerance): an emulation of the kernel's
arithmetic in numpy, against exact FP64 weights, on elements of aspect ratio up to 1000.

The kernel computes lambda_a = det2(x_b - p_x, y_b - p_y, x_c - p_x, y_c - p_y) * fl32(1 / 2A) with
every difference rounded to FP32 and det2 by Kahan's FMA scheme (w = fl(b c), e = fma(-b, c, w),
f = fma(a, d, -w), f + e). A product of two FP32 numbers is exact in FP64, so each FMA is
emulated exactly by the FP64 expression rounded once to FP32 (the FP64 sum of an exact product
and an FP32 number carries at most one FP64 rounding, far below the FP32 one)."""
import numpy as np

from tests.gpu_common import EPS32, LAMBDA_RTOL

f32 = np.float32


def _det2(a, b, c, d):
    a, b, c, d = (np.asarray(t, dtype=np.float32).astype(np.float64) for t in (a, b, c, d))
    w = (b * c).astype(np.float32).astype(np.float64)
    e = (-(b * c) + w).astype(np.float32).astype(np.float64)
    f = (a * d - w).astype(np.float32).astype(np.float64)
    return (f + e).astype(np.float32)


def _lambda_fp32(X, Y, px, py, inv2a):
    """The kernel's barycentric(): vertex a's weight from the other two vertices b, c."""
    out = []
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        d = _det2(f32(X[b] - px), f32(Y[b] - py), f32(X[c] - px), f32(Y[c] - py))
        out.append((d.astype(np.float64) * np.float64(inv2a)).astype(np.float32))
    return np.stack(out)


def test_fp32_weights_stay_within_the_kappa_bound():
    rng = np.random.default_rng(17)
    worst = 0.0
    for trial in range(400):
        L = 10.0 ** rng.uniform(-4, 0)                   # element size
        ar = 10.0 ** rng.uniform(0, 3)                   # aspect ratio up to 1000
        x0, y0 = rng.uniform(0, 6), rng.uniform(0, 2)
        ang = rng.uniform(0, 2 * np.pi)
        P = np.array([[0.0, 0.0], [L, 0.0], [rng.uniform(0.1, 0.9) * L, L / ar]])
        R = np.array([[np.cos(ang), -np.sin(ang)], [np.sin(ang), np.cos(ang)]])
        P = (P @ R.T + [x0, y0]).astype(np.float32).astype(np.float64)   # FP32 vertices, as meshes give
        X, Y = P[:, 0], P[:, 1]
        A2 = (X[1] - X[0]) * (Y[2] - Y[0]) - (Y[1] - Y[0]) * (X[2] - X[0])
        if A2 <= 0:
            X, Y = X[[0, 2, 1]], Y[[0, 2, 1]]
            A2 = -A2
        if A2 == 0:
            continue
        r = rng.dirichlet([0.3, 0.3, 0.3], size=64)     # many points near the edges and vertices
        px = (r @ X).astype(np.float32).astype(np.float64)
        py = (r @ Y).astype(np.float32).astype(np.float64)
        lam_exact = np.stack([((X[(a + 1) % 3] - px) * (Y[(a + 2) % 3] - py)
                               - (Y[(a + 1) % 3] - py) * (X[(a + 2) % 3] - px)) / A2 for a in range(3)])
        kappa = np.stack([(np.abs((X[(a + 1) % 3] - px) * (Y[(a + 2) % 3] - py))
                           + np.abs((Y[(a + 1) % 3] - py) * (X[(a + 2) % 3] - px))) / A2 for a in range(3)])
        lam32 = _lambda_fp32(X, Y, px, py, np.float32(1.0 / A2)).astype(np.float64)
        err = np.abs(lam32 - lam_exact)
        bound = 2 * EPS32 * kappa + 2 * EPS32 * np.abs(lam_exact) + 1e-300
        worst = max(worst, float(np.max(err / bound)))
        # the tolerance the tests use: LAMBDA_RTOL kappa (the |lambda| part sits in MOMENT_RTOL)
        assert np.all(err <= LAMBDA_RTOL * kappa + 4 * EPS32 * np.abs(lam_exact)), trial
    assert worst <= 1.0, worst
    print("max error / (2 eps kappa + 2 eps |lambda|) =", worst)


def test_kappa_grows_with_the_aspect_ratio_on_rotated_elements():
    """On a long thin element that is not aligned with the axes, the determinant behind the weight
    of the vertex opposite the long edge is the difference of two products of the element's length:
    at the midpoint of that edge the weight is 0 and kappa = 1 / (4 h) for an element of length 1
    and height h, so the FP32 weight can be off by about 2 eps / (4 h) there, which no bound
    relative to |lambda q| covers."""
    c, s = np.cos(np.pi / 4), np.sin(np.pi / 4)
    for h in (1e-1, 1e-2, 1e-3):
        P = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, h]]) @ np.array([[c, -s], [s, c]]).T
        X, Y = P[:, 0], P[:, 1]
        A2 = (X[1] - X[0]) * (Y[2] - Y[0]) - (Y[1] - Y[0]) * (X[2] - X[0])
        px, py = 0.5 * (X[0] + X[1]), 0.5 * (Y[0] + Y[1])     # on the long edge, opposite vertex 2
        b, cc = 0, 1
        lam = ((X[b] - px) * (Y[cc] - py) - (Y[b] - py) * (X[cc] - px)) / A2
        kappa = (abs((X[b] - px) * (Y[cc] - py)) + abs((Y[b] - py) * (X[cc] - px))) / A2
        assert abs(lam) < 1e-12 and np.isclose(A2, h) and np.isclose(kappa, 0.25 / h, rtol=1e-9)
