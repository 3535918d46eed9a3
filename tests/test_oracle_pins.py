"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: an independent library (cuRAND's host Philox
generator, exact rational arithmetic, scipy distributions, numpy's weighted covariance), a
closed form of the model (Ornstein-Uhlenbeck variance, simplified-Langevin decay, the
Cox-Ingersoll-Ross stationary gamma law of Eq. 5, the exact IEM decay), or brute force.
"""
import ctypes
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1006_0549_gb300 import workloads as wl
from tests.helpers import state_from, uniform_fields


# ------------------------------------------------------------------ Philox / normals
def _curand_host_words(seed, n):
    path = "/usr/local/cuda/lib64/libcurand.so"
    if not os.path.exists(path):
        pytest.skip("libcurand not present")
    lib = ctypes.CDLL(path)
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:   # CURAND_RNG_PSEUDO_PHILOX4_32_10
        pytest.skip("cuRAND host generator unavailable")
    assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
    buf = np.zeros(n, dtype=np.uint32)
    assert lib.curandGenerate(gen, buf.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    lib.curandDestroyGenerator(gen)
    return buf


@pytest.mark.parametrize("seed", [0, 0x0123456789ABCDEF, 1006054902])
def test_philox_matches_curand_host_generator(seed):
    """cuRAND's host Philox4x32-10 emits block g of its stream from counter (0, 0, g, 0) and
    key (seed_lo, seed_hi); an independent implementation of the same SC'11 generator."""
    G = 512
    ref = _curand_host_words(seed, 4 * G).reshape(G, 4)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    got = np.stack([oracle.philox4x32_10([0, 0, g, 0], key) for g in range(G)])
    assert np.array_equal(got, ref)


def test_philox_counter_words_all_matter():
    key = [0x12345678, 0x9ABCDEF0]
    base = oracle.philox4x32_10([1, 2, 3, 4], key)
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        out = oracle.philox4x32_10(c, key)
        # one flipped input bit changes about half of the 128 output bits
        flips = sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(base, out))
        assert 30 < flips < 98
    out = oracle.philox4x32_10([1, 2, 3, 4], [key[0], key[1] ^ 1])
    assert not np.array_equal(out, base)


def test_normals_are_standard_gaussian_and_independent():
    """Box-Muller normals keyed by (seed, pid, step): N(0,1) marginals (KS), no correlation
    between the six components of one update, none between consecutive steps."""
    n = 12000
    Z = np.array([oracle.normals6(77, pid, 5) for pid in range(n)])
    Z2 = np.array([oracle.normals6(77, pid, 6) for pid in range(n)])
    allz = Z.ravel()
    assert abs(allz.mean()) < 4.0 / math.sqrt(allz.size)
    assert abs(allz.var() - 1.0) < 4.0 * math.sqrt(2.0 / allz.size)
    assert stats.kstest(allz, "norm").pvalue > 1e-3
    C = np.corrcoef(Z.T)
    assert np.max(np.abs(C - np.eye(6))) < 4.0 / math.sqrt(n)
    lag = np.corrcoef(Z.ravel(), Z2.ravel())[0, 1]
    assert abs(lag) < 4.0 / math.sqrt(allz.size)
    # the tag separates the initialisation stream from the step stream
    assert not np.allclose(oracle.normals6(77, 3, 5, 0), oracle.normals6(77, 3, 5, 1))


# ------------------------------------------------------------------ exact orient2d
def _exact_sign(ax, ay, bx, by, cx, cy):
    F = Fraction
    d = (F(ax) - F(cx)) * (F(by) - F(cy)) - (F(ay) - F(cy)) * (F(bx) - F(cx))
    return (d > 0) - (d < 0)


def test_orient2d_exact_against_rationals():
    rng = np.random.default_rng(3)
    pts = []
    for _ in range(3000):  # generic
        pts.append(tuple(float(np.float32(v)) for v in rng.uniform(-7, 7, 6)))
    for _ in range(3000):  # nearly collinear FP32 triples
        a = rng.uniform(0, 6.3, 2)
        b = rng.uniform(0, 6.3, 2)
        t = rng.uniform(-0.5, 1.5)
        c = a + t * (b - a)
        c = c + rng.integers(-2, 3, 2) * np.spacing(np.float32(c)).astype(np.float64)
        pts.append(tuple(float(np.float32(v)) for v in (*a, *b, *c)))
    for _ in range(500):  # exactly collinear on axis-aligned and diagonal lines
        y = float(np.float32(rng.uniform(0, 2)))
        xs = [float(np.float32(v)) for v in rng.uniform(0, 6.3, 3)]
        pts.append((xs[0], y, xs[1], y, xs[2], y))
        v = float(np.float32(rng.uniform(0, 1)))
        pts.append((0.0, 0.0, 1.0, 1.0, v, v))
    for p in pts:
        assert oracle.orient2d_sign(*p) == _exact_sign(*p), p


# ------------------------------------------------------------------ point location
def _probe_points(mesh, rng, n_random=400):
    """Random points, nodes, edge midpoints and points exactly on axis-aligned edges (FP32)."""
    x0, x1, y0, y1 = mesh.box
    P = [(float(np.float32(rng.uniform(x0, x1))), float(np.float32(rng.uniform(y0, y1)))) for _ in range(n_random)]
    P += [tuple(p) for p in mesh.node_xy]
    for t in mesh.tri[:200]:
        for k in range(3):
            a, b = mesh.node_xy[t[k]], mesh.node_xy[t[(k + 1) % 3]]
            m = 0.5 * (a + b)
            P.append((float(np.float32(m[0])), float(np.float32(m[1]))))
    for _ in range(100):
        P.append((float(np.float32(rng.uniform(x0, x1))), y0))
        P.append((x0, float(np.float32(rng.uniform(y0, y1)))))
    return P


def _in_half_open_domain(mesh, x, y):
    x0, x1, y0, y1 = mesh.box
    return x0 <= x < x1 and y0 <= y < y1


@pytest.mark.parametrize("kind", ["channel", "cavity"])
def test_every_point_of_the_domain_has_exactly_one_owner(kind):
    """Brute force over all elements with the exact predicate and the top-left tie rule."""
    mesh = wl.channel_mesh(6, 5, 11) if kind == "channel" else wl.cavity_mesh(5, 6, 12)
    om = oracle.OracleMesh(mesh)
    rng = np.random.default_rng(5)
    for (x, y) in _probe_points(mesh, rng):
        owner = om.locate_brute(x, y)
        if _in_half_open_domain(mesh, x, y):
            assert owner >= 0, (x, y, owner)
        else:
            assert owner == -1, (x, y, owner)
    # points on the excluded sides (x = x1 or y = y1) have no owner
    x0, x1, y0, y1 = mesh.box
    assert om.locate_brute(0.5 * (x0 + x1), y1) == -1
    assert om.locate_brute(x1, 0.5 * (y0 + y1)) == -1


@pytest.mark.parametrize("kind", ["channel", "cavity"])
def test_walk_agrees_with_brute_force(kind):
    mesh = wl.channel_mesh(12, 8, 21) if kind == "channel" else wl.cavity_mesh(10, 9, 22)
    om = oracle.OracleMesh(mesh)
    rng = np.random.default_rng(9)
    pts = _probe_points(mesh, rng, 600)
    for (x, y) in pts:
        if not _in_half_open_domain(mesh, x, y):
            continue
        start = int(rng.integers(0, mesh.n_tri))
        e, hops = om.locate_walk(start, x, y)
        assert e == om.locate_brute(x, y), (x, y, start, e, hops)


def test_periodic_neighbours_and_node_pairing():
    mesh = wl.channel_mesh(7, 4, 3)
    om = oracle.OracleMesh(mesh)
    nb = om.neighbors()
    tags = mesh.edge_tag
    assert np.all((nb < 0) == (tags == wl.EDGE_WALL))
    # neighbour relation is symmetric
    for e in range(mesh.n_tri):
        for k in range(3):
            f = nb[e, k]
            if f >= 0:
                assert e in nb[f]
    ma = om.masters()
    right = np.nonzero(mesh.node_xy[:, 0] == mesh.period_x)[0]
    assert np.all(mesh.node_xy[ma[right], 0] == 0.0)
    assert np.all(mesh.node_xy[ma[right], 1] == mesh.node_xy[right, 1])


# ------------------------------------------------------------------ shape functions
def test_barycentric_partition_of_unity_and_kronecker():
    mesh = wl.cavity_mesh(6, 6, 4)
    om = oracle.OracleMesh(mesh)
    rng = np.random.default_rng(1)
    for e in range(mesh.n_tri):
        t = mesh.tri[e]
        for a in range(3):
            lam = om.barycentric(e, *mesh.node_xy[t[a]])
            assert np.allclose(lam, np.eye(3)[a], atol=1e-12)
        r = rng.dirichlet([1, 1, 1])
        p = r @ mesh.node_xy[t]
        lam = om.barycentric(e, *p)
        assert abs(lam.sum() - 1.0) < 1e-12
        assert np.allclose(lam, r, atol=1e-10)
        # a linear field is interpolated exactly
        f = 2.0 + 3.0 * mesh.node_xy[t, 0] - 1.5 * mesh.node_xy[t, 1]
        assert abs(lam @ f - (2.0 + 3.0 * p[0] - 1.5 * p[1])) < 1e-10


# ------------------------------------------------------------------ model closed forms
def _run(om, params, fields_fn, st, nsteps, step0=0):
    hist = []
    for n in range(nsteps):
        F = fields_fn(st)
        res, elem, aux, lost = oracle.pdf_step(om, params, F, st, step0 + n)
        assert lost == 0
        st = state_from(res, elem, st.pid, params.ns)
        hist.append(res)
    return st, hist


def _homogeneous_state(mesh, P, ns, rng, u=0.0, omega=1.0, psi=None):
    base = wl.synthetic_state(mesh, max(1, P // mesh.n_tri), ns, seed=int(rng.integers(1 << 30)))
    n = base.n
    z = np.zeros(n, dtype=np.float32)
    base.u, base.v, base.w = z + u, z.copy(), z.copy()
    base.omega = np.full(n, omega, dtype=np.float32)
    if psi is not None:
        base.psi = psi.astype(np.float32)
    return base


def test_ornstein_uhlenbeck_variance_exact_in_expectation():
    """G_ij = -a delta_ij, C_0 eps = b^2, <U> = 0, nu = 0: Eq. 4 is the OU process
    U' = (1 - a dt) U + b dW'. From U_0 = 0: Var_n = b^2 dt (1 - r^(2n)) / (1 - r^2), r = 1 - a dt;
    stationary b^2 / (a (2 - a dt)) (continuous limit b^2 / (2a))."""
    mesh = wl.channel_mesh(8, 6, 2)
    om = oracle.OracleMesh(mesh)
    a, b, dt = 40.0, 3.0, 2e-3
    params = oracle.make_params(nu=0.0, dt=dt, seed=99, ns=1)
    F = uniform_fields(mesh, 1, g11=-a, g22=-a, g33=-a, c0eps=b * b, omega=1.0)
    rng = np.random.default_rng(2)
    st = _homogeneous_state(mesh, 60000, 1, rng)
    r = 1.0 - a * dt
    st, hist = _run(om, params, lambda s: F, st, 40)
    for n in (5, 20, 40):
        res = hist[n - 1]
        expect = b * b * dt * (1 - r ** (2 * n)) / (1 - r * r)
        for comp in ("u", "v", "w"):
            var = np.mean(res[comp] ** 2)
            assert abs(var / expect - 1.0) < 4.0 * math.sqrt(2.0 / res[comp].size), (n, comp, var, expect)
            assert abs(np.mean(res[comp])) < 4.0 * math.sqrt(expect / res[comp].size)
    stationary = b * b / (a * (2 - a * dt))
    assert abs(np.mean(hist[-1]["u"] ** 2) / stationary - 1.0) < 0.03


def test_simplified_langevin_kinetic_energy_decay():
    """SLM in homogeneous turbulence: G = -(1/2 + 3/4 C_0) <omega>, C_0 eps = C_0 k <omega>,
    <omega> held fixed. Per step E[k'] = k (1 - <omega> dt + G^2 dt^2) exactly, so
    k_n = k_0 (1 - <omega> dt + G^2 dt^2)^n -> k_0 exp(-<omega> t)."""
    mesh = wl.channel_mesh(8, 6, 3)
    om = oracle.OracleMesh(mesh)
    C0, Om, dt = 2.1, 20.0, 1e-3
    G = -(0.5 + 0.75 * C0) * Om
    params = oracle.make_params(nu=0.0, dt=dt, seed=7, ns=1)
    rng = np.random.default_rng(4)
    st = _homogeneous_state(mesh, 60000, 1, rng)
    st.u = rng.standard_normal(st.n).astype(np.float32)
    st.v = rng.standard_normal(st.n).astype(np.float32)
    st.w = rng.standard_normal(st.n).astype(np.float32)
    k = lambda s: 0.5 * float(np.mean(s.u.astype(np.float64) ** 2 + s.v.astype(np.float64) ** 2 + s.w.astype(np.float64) ** 2))
    k0 = k(st)
    ratios = []

    def fields(s):
        return uniform_fields(mesh, 1, g11=G, g22=G, g33=G, c0eps=C0 * k(s) * Om, omega=Om)

    nsteps = 60
    kk = [k0]
    for n in range(nsteps):
        res, elem, aux, lost = oracle.pdf_step(om, params, fields(st), st, n)
        st = state_from(res, elem, st.pid, 1)
        kk.append(k(st))
        ratios.append(kk[-1] / kk[-2])
    q = 1.0 - Om * dt + G * G * dt * dt
    # mean per-step ratio: exact expectation q; noise of one ratio ~ sqrt(2/(3P)) * (noise share)
    assert abs(np.mean(ratios) - q) < 3e-3
    kn = k0 * q ** nsteps
    assert abs(kk[-1] / kn - 1.0) < 0.03
    t = nsteps * dt
    assert abs(kn / (k0 * math.exp(-Om * t)) - 1.0) < 2 * (G * G * dt * dt + Om * Om * dt * dt) * nsteps


def test_frequency_mean_decay_with_constant_source():
    """Eq. 5 with S_omega = C_omega2 and <omega> taken from the particles each step:
    E[<omega>'] = <omega>(1 - C_omega2 <omega> dt), the Euler form of d<omega>/dt = -C_omega2 <omega>^2
    whose solution is omega_0 / (1 + C_omega2 omega_0 t)."""
    mesh = wl.channel_mesh(8, 6, 5)
    om = oracle.OracleMesh(mesh)
    Cw2, dt, w0 = 0.73, 2e-4, 30.0      # noise / omega ~ 12% per step: no reflections of omega
    params = oracle.make_params(nu=0.0, dt=dt, seed=11, ns=1)
    rng = np.random.default_rng(6)
    st = _homogeneous_state(mesh, 60000, 1, rng, omega=w0)
    Wm = [w0]
    pred = [w0]
    for n in range(100):
        Om = float(np.mean(st.omega.astype(np.float64)))
        F = uniform_fields(mesh, 1, omega=Om, somega=Cw2)
        res, elem, aux, lost = oracle.pdf_step(om, params, F, st, n)
        st = state_from(res, elem, st.pid, 1)
        Wm.append(float(np.mean(res["omega"])))
        pred.append(Om * (1.0 - Cw2 * Om * dt))
        assert abs(Wm[-1] / pred[-1] - 1.0) < 2e-3, (n, Wm[-1], pred[-1])
    t = 100 * dt
    assert abs(Wm[-1] / (w0 / (1.0 + Cw2 * w0 * t)) - 1.0) < 0.02


@pytest.mark.slow
def test_frequency_stationary_law_is_gamma():
    """Eq. 5 with S_omega = 0 and fixed <omega> = W is a CIR process whose stationary law is
    Gamma(shape 1/C_4, scale C_4 W): mean W, variance C_4 W^2."""
    mesh = wl.channel_mesh(8, 6, 6)
    om = oracle.OracleMesh(mesh)
    C3, C4, W, dt = 5.0, 0.25, 10.0, 1e-3
    params = oracle.make_params(nu=0.0, dt=dt, seed=13, ns=1, C3=C3, C4=C4)
    rng = np.random.default_rng(8)
    st = _homogeneous_state(mesh, 40000, 1, rng, omega=W)
    F = uniform_fields(mesh, 1, omega=W, somega=0.0)
    st, hist = _run(om, params, lambda s: F, st, 120)   # 6 relaxation times of C_3 W
    w = hist[-1]["omega"]
    assert abs(w.mean() / W - 1.0) < 0.01
    assert abs(w.var() / (C4 * W * W) - 1.0) < 0.05
    assert stats.kstest(w, stats.gamma(a=1.0 / C4, scale=C4 * W).cdf).statistic < 0.02


def test_iem_decay_exact_per_step_and_exponential_limit():
    """Eq. 9 (IEM form) with uniform <phi> and <omega>: psi' - <phi> = (psi - <phi>)(1 - C_phi <omega> dt/2)
    for every particle, so the scalar variance decays by (1 - C_phi<omega>dt/2)^2 per step and
    -> exp(-C_phi <omega> t) as dt -> 0."""
    mesh = wl.channel_mesh(8, 6, 7)
    om = oracle.OracleMesh(mesh)
    Cphi, W, dt, phi = 2.0, 8.0, 1e-3, float(np.float32(0.3))   # node fields are FP32 values
    params = oracle.make_params(nu=1e-3, dt=dt, seed=17, ns=1, Cphi=Cphi)
    rng = np.random.default_rng(10)
    st = _homogeneous_state(mesh, 20000, 1, rng, omega=W, psi=rng.uniform(0, 1, (1, 20000 // mesh.n_tri * mesh.n_tri)))
    F = uniform_fields(mesh, 1, omega=W, phi0=phi, c0eps=1.0, g11=-1.0, g22=-1.0, g33=-1.0)
    psi0 = st.psi[0].astype(np.float64)
    var0 = np.mean((psi0 - phi) ** 2)
    st1, hist = _run(om, params, lambda s: F, st, 100)
    d = 1.0 - Cphi * W * dt / 2.0
    assert np.allclose(hist[0]["psi"][0], phi + (psi0 - phi) * d, rtol=0, atol=1e-12)
    var = np.mean((hist[-1]["psi"][0] - phi) ** 2)
    assert abs(var / (var0 * d ** 200) - 1.0) < 1e-5      # FP32 storage between steps
    assert abs(var / (var0 * math.exp(-Cphi * W * 100 * dt)) - 1.0) < 100 * (Cphi * W * dt) ** 2


# ------------------------------------------------------------------ boundaries
def test_wall_reflection_is_the_mirror_image():
    """nu = 0 and zero fields: X' = X + U dt; a crossing of y = 0 or y = 2 is mirrored and U <- -U;
    a crossing of x = L wraps by L. Cavity lid (y = 1): U <- 2 (1,0,0) - U."""
    mesh = wl.channel_mesh(10, 6, 8)
    om = oracle.OracleMesh(mesh)
    dt = 0.01
    params = oracle.make_params(nu=0.0, dt=dt, seed=1, ns=1)
    F = uniform_fields(mesh, 1)
    st = wl.synthetic_state(mesh, 1, 1, seed=3)
    n = st.n
    rng = np.random.default_rng(0)
    st.v = rng.uniform(-30, 30, n).astype(np.float32)
    st.u = rng.uniform(-80, 80, n).astype(np.float32)
    st.w = rng.uniform(-1, 1, n).astype(np.float32)
    st.omega[:] = 1.0
    res, elem, aux, lost = oracle.pdf_step(om, params, F, st, 0)
    assert lost == 0
    L = mesh.period_x
    for i in range(n):
        qx = float(st.x[i]) + float(st.u[i]) * dt
        qy = float(st.y[i]) + float(st.v[i]) * dt
        qx -= L * math.floor(qx / L)
        flips = 0
        while qy < 0 or qy > 2:
            qy = -qy if qy < 0 else 4.0 - qy
            flips += 1
        sgn = -1.0 if flips % 2 else 1.0
        assert res["x"][i] == float(np.float32(qx)) or (qx >= float(np.float32(L)) and res["x"][i] == 0.0)
        assert res["y"][i] == float(np.float32(qy))
        assert res["v"][i] == sgn * float(st.v[i]) and res["u"][i] == sgn * float(st.u[i])
        assert aux[i, 2] == flips
        assert om.inside(elem[i], res["x"][i], res["y"][i])
    # lid
    cav = wl.cavity_mesh(8, 8, 9)
    oc = oracle.OracleMesh(cav)
    pc = oracle.make_params(nu=0.0, dt=dt, seed=1, ns=1, lid_u=1.0)
    sc = wl.synthetic_state(cav, 1, 1, seed=4)
    top = sc.y > 0.9
    sc.v = np.where(top, 30.0, 0.0).astype(np.float32)
    sc.u = np.full(sc.n, 0.25, dtype=np.float32)
    sc.w[:] = 0.0
    rc, ec, ac, lc = oracle.pdf_step(oc, pc, uniform_fields(cav, 1), sc, 0)
    hit = ac[:, 2] > 0
    assert hit.sum() > 0
    assert np.all(rc["u"][hit] == 2.0 - 0.25) and np.all(rc["v"][hit] == -30.0)


def test_scalar_source_sets_psi_inside_the_disc():
    mesh = wl.channel_mesh(25, 20, 1)
    om = oracle.OracleMesh(mesh)
    params = oracle.make_params(nu=0.0, dt=1e-6, seed=1, ns=1, sources=[(0.25, 0.67, 0.15, 0)])
    st = wl.synthetic_state(mesh, 20, 1, seed=3)
    st.u[:] = 0.0; st.v[:] = 0.0; st.w[:] = 0.0
    st.psi[:] = 0.0
    res, elem, aux, lost = oracle.pdf_step(om, params, uniform_fields(mesh, 1), st, 0)
    d = np.hypot(res["x"] - 0.25, res["y"] - 0.67)
    inside = res["psi"][0] == 1.0
    assert inside.sum() > 10
    assert np.all(d[inside] < 0.15 + 1e-6) and np.all(d[~inside] > 0.15 - 1e-6)


# ------------------------------------------------------------------ whole-step invariants and moments
def test_count_conservation_domain_and_total_weight():
    """Every particle stays located and inside the half-open domain; sum over distinct nodes of
    S_0 equals the particle count (partition of unity of the shape functions)."""
    wk = wl.channel_small()
    mesh = wk.mesh
    om = oracle.OracleMesh(mesh)
    params = oracle.make_params(nu=wk.nu, dt=wk.dt, seed=wk.seed, ns=1, sources=wk.sources)
    F = wl.synthetic_node_fields(mesh, 1, seed=5)
    st = wl.synthetic_state(mesh, 10, 1, seed=6)
    masters = om.masters()
    for n in range(3):
        res, elem, aux, lost = oracle.pdf_step(om, params, F, st, n, locate_mode=2 if n == 0 else 0)
        assert lost == 0
        assert np.all((res["x"] >= 0) & (res["x"] < mesh.period_x) & (res["y"] >= 0) & (res["y"] < 2))
        st = state_from(res, elem, st.pid, 1)
        S, _ = oracle.moments(om, 1, res["x"], res["y"], res["u"], res["v"], res["w"], res["omega"], res["psi"], elem)
        uniq = masters == np.arange(mesh.n_nodes)
        assert abs(S[uniq, 0].sum() - st.n) < 1e-8 * st.n


def test_moments_match_numpy_weighted_covariance():
    """The node statistics equal numpy's weighted mean and (biased) covariance with the
    shape-function weights lambda_n(X_p)."""
    mesh = wl.cavity_mesh(5, 5, 2)
    om = oracle.OracleMesh(mesh)
    st = wl.synthetic_state(mesh, 40, 2, seed=12)
    P = st.n
    f = lambda a: a.astype(np.float64)
    S, _ = oracle.moments(om, 2, f(st.x), f(st.y), f(st.u), f(st.v), f(st.w), f(st.omega), f(st.psi), st.elem)
    out = oracle.grid_statistics(S, 2)
    # shape-function weights of every particle for every node
    Wn = np.zeros((mesh.n_nodes, P))
    for i in range(P):
        lam = om.barycentric(st.elem[i], st.x[i], st.y[i])
        Wn[mesh.tri[st.elem[i]], i] += lam
    for n in range(mesh.n_nodes):
        wts = Wn[n]
        sel = wts != 0
        if sel.sum() < 3:
            continue
        X = np.stack([f(st.u), f(st.v), f(st.w), f(st.omega), f(st.psi[0]), f(st.psi[1])])[:, sel]
        w = wts[sel]
        mean = np.average(X, axis=1, weights=w)
        cov = np.cov(X, aweights=w, bias=True)
        assert abs(out[n, 0] - w.sum()) < 1e-12 * w.sum()
        assert np.allclose(out[n, 1:4], mean[:3], rtol=1e-10, atol=1e-12)
        iu = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
        assert np.allclose(out[n, 4:10], [cov[a, b] for a, b in iu], rtol=1e-8, atol=1e-11)
        assert np.isclose(out[n, 10], mean[3], rtol=1e-10)
        assert np.allclose(out[n, 11:13], mean[4:6], rtol=1e-10)
        assert np.allclose(out[n, 13:15], [cov[4, 4], cov[5, 5]], rtol=1e-8, atol=1e-11)


def test_moments_of_a_constant_field():
    mesh = wl.channel_mesh(6, 4, 1)
    om = oracle.OracleMesh(mesh)
    st = wl.synthetic_state(mesh, 30, 1, seed=2)
    c = np.full(st.n, 1.75)
    S, _ = oracle.moments(om, 1, st.x, st.y, c, -c, 0 * c, 2 * c, [0.5 * c], st.elem)
    out = oracle.grid_statistics(S, 1)
    live = out[:, 0] > 0
    assert np.allclose(out[live, 1], 1.75) and np.allclose(out[live, 2], -1.75)
    assert np.allclose(out[live, 4:10], 0.0, atol=1e-12)
    assert np.allclose(out[live, 10], 3.5) and np.allclose(out[live, 11], 0.875)
    assert np.allclose(out[live, 12], 0.0, atol=1e-12)


def test_particles_init_distribution():
    """Initialisation: positions uniform inside each element (mean barycentric 1/3, and
    lambda_0 = 1 - sqrt(r1) has CDF 1 - (1 - t)^2), every particle owned by its element,
    U ~ N(<U>, sigma^2), omega ~ Erlang(m) with mean <omega> (variance <omega>^2 / m)."""
    mesh = wl.cavity_mesh(6, 6, 1)
    om = oracle.OracleMesh(mesh)
    init = wl.node_init_fields(mesh)
    init[:, 0] = 0.5
    init[:, 3] = 0.2
    init[:, 4] = 3.0
    params = oracle.make_params(nu=1e-4, dt=1e-3, seed=21, ns=1)
    res, elem, pid, lost = oracle.particles_init(om, params, 400, init, 4)
    assert lost == 0
    P = mesh.n_tri * 400
    assert np.array_equal(pid, np.arange(P, dtype=np.uint32))
    lam0 = []
    for i in range(0, P, 7):
        assert om.inside(elem[i], res["x"][i], res["y"][i])
        e0 = i // 400
        lam0.append(om.barycentric(e0, res["x"][i], res["y"][i])[0])
    lam0 = np.array(lam0)
    assert abs(lam0.mean() - 1.0 / 3.0) < 0.01
    assert stats.kstest(lam0, lambda t: 1 - (1 - np.clip(t, 0, 1)) ** 2).pvalue > 1e-3
    assert abs(res["u"].mean() - 0.5) < 0.002 and abs(res["u"].std() - 0.2) < 0.002
    assert abs(res["w"].mean()) < 0.002
    w = res["omega"]
    assert abs(w.mean() / 3.0 - 1.0) < 0.01 and abs(w.var() / (9.0 / 4.0) - 1.0) < 0.03
    assert stats.kstest(w, stats.gamma(a=4, scale=0.75).cdf).pvalue > 1e-3


def test_position_diffusion_is_brownian():
    """U = 0, no forcing: Eq. 2 reduces to dX = (2 nu)^(1/2) dW, so the displacement after n steps
    has variance 2 nu n dt per component (Einstein) and zero mean."""
    mesh = wl.channel_mesh(10, 8, 12)
    om = oracle.OracleMesh(mesh)
    nu, dt = 1e-3, 1e-3
    params = oracle.make_params(nu=nu, dt=dt, seed=23, ns=1)
    st = wl.synthetic_state(mesh, 60, 1, seed=13)
    keep = (st.y > 0.5) & (st.y < 1.5)
    x0, y0 = st.x.astype(np.float64), st.y.astype(np.float64)
    st.u[:] = 0; st.v[:] = 0; st.w[:] = 0
    F = uniform_fields(mesh, 1, omega=1.0)
    st, hist = _run(om, params, lambda s: F, st, 20)
    dx = hist[-1]["x"] - x0
    dx = (dx + 0.5 * mesh.period_x) % mesh.period_x - 0.5 * mesh.period_x
    dy = hist[-1]["y"] - y0
    var = 2 * nu * 20 * dt
    n = keep.sum()
    for d in (dx[keep], dy[keep]):
        assert abs(d.var() / var - 1.0) < 4 * math.sqrt(2.0 / n)
        assert abs(d.mean()) < 4 * math.sqrt(var / n)


def test_glm_drift_coefficients_and_shared_wiener_increment():
    """One Euler step of Eq. 4 from U = (1, 0, 0) with uniform fields. The expected increments are
    the drift: E[du] = (-dP/dx + 2 nu lap<U> + G11 (1 - <U>)) dt, E[dv] = (-dP/dy + 2 nu lap<V> + G21 (1 - <U>)) dt,
    E[dw] = 2 nu lap<W> dt. The paper requires the same dW_j in Eq. 2 and Eq. 4, so
    Cov(du, dy) = 2 nu (d<U>/dy) dt and Cov(dv, dx) = 2 nu (d<V>/dx) dt, while the independent
    dW'_i add C_0 eps dt to each velocity variance."""
    mesh = wl.channel_mesh(10, 8, 14)
    om = oracle.OracleMesh(mesh)
    nu, dt = 0.05, 1e-2
    params = oracle.make_params(nu=nu, dt=dt, seed=29, ns=1)
    st = wl.synthetic_state(mesh, 150, 1, seed=15)
    keep = (st.y > 0.5) & (st.y < 1.5)
    st.u[:] = 1.0; st.v[:] = 0.0; st.w[:] = 0.0
    g = dict(u=0.25, dpdx=-3.0, dpdy=1.5, lapu=4.0, lapv=-2.0, lapw=6.0, g11=-7.0, g12=2.0, g21=5.0,
             g22=-6.0, g33=-4.0, dudy=3.0, dvdx=-2.5, c0eps=0.8, omega=1.0)
    F = uniform_fields(mesh, 1, **g)
    res, elem, aux, lost = oracle.pdf_step(om, params, F, st, 0)
    k = keep & (aux[:, 2] == 0)
    n = k.sum()
    du, dv, dw = res["u"][k] - 1.0, res["v"][k], res["w"][k]
    dx = aux[k, 0] - st.x[k]
    dy = aux[k, 1] - st.y[k]
    Eu = (3.0 + 2 * nu * 4.0 + (-7.0) * (1 - 0.25)) * dt
    Ev = (-1.5 + 2 * nu * (-2.0) + 5.0 * (1 - 0.25)) * dt
    Ew = (2 * nu * 6.0) * dt
    for d, E_, sd in ((du, Eu, math.sqrt((2 * nu * 9.0 + 0.8) * dt)),
                      (dv, Ev, math.sqrt((2 * nu * 6.25 + 0.8) * dt)),
                      (dw, Ew, math.sqrt(0.8 * dt))):
        assert abs(d.mean() - E_) < 4 * sd / math.sqrt(n), (d.mean(), E_)
        assert abs(d.std() / sd - 1.0) < 4 * math.sqrt(0.5 / n)
    assert abs(np.cov(du, dy)[0, 1] / (2 * nu * 3.0 * dt) - 1.0) < 0.05
    assert abs(np.cov(dv, dx)[0, 1] / (2 * nu * -2.5 * dt) - 1.0) < 0.05
    assert abs(np.corrcoef(dw, dx)[0, 1]) < 4 / math.sqrt(n)
