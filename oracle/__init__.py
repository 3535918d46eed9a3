"""ctypes front end of the FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: the oracle is the plain, slow statement of what the particle step
computes. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import it. It never imports the CUDA package, and the CUDA package never
imports it; the two meet only in tests, on inputs from ``paper_1006_0549_gb300.workloads``.

Every function cites the part of the paper (arXiv:1006.0549) it follows; see ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
MAX_SOURCES = 8
HOP_CAP = 64


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no FMA contraction, so FP32 decisions match the kernel)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        vp = ctypes.c_void_p
        L.oracle_mesh_new.restype = vp
        L.oracle_mesh_new.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, vp, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.oracle_mesh_free.argtypes = [vp]
        L.oracle_mesh_neighbors.argtypes = [vp, vp]
        L.oracle_mesh_edge_walls.restype = ctypes.c_int
        L.oracle_mesh_edge_walls.argtypes = [vp]
        L.oracle_mesh_masters.argtypes = [vp, vp]
        L.oracle_philox4x32_10.argtypes = [vp, vp, vp]
        L.oracle_normals6.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, vp]
        L.oracle_orient2d_sign.restype = ctypes.c_int
        L.oracle_orient2d_sign.argtypes = [ctypes.c_double] * 6
        L.oracle_inside.restype = ctypes.c_int
        L.oracle_inside.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.oracle_locate_brute.restype = ctypes.c_int
        L.oracle_locate_brute.argtypes = [vp, ctypes.c_double, ctypes.c_double]
        L.oracle_locate_walk.restype = ctypes.c_int
        L.oracle_locate_walk.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, vp]
        L.oracle_barycentric.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, vp]
        L.oracle_locate_walk_reflect.restype = ctypes.c_int
        L.oracle_locate_walk_reflect.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, vp, ctypes.c_double, vp, vp]
        L.oracle_pdf_step.restype = ctypes.c_long
        L.oracle_flux_moments.argtypes = [vp, ctypes.c_int, ctypes.c_long] + [vp] * 8
        L.oracle_pdf_step.argtypes = [vp, vp, vp, ctypes.c_int, vp, ctypes.c_long] + [vp] * 9 + \
            [ctypes.c_uint64, ctypes.c_int] + [vp] * 9
        L.oracle_moments.argtypes = [vp, ctypes.c_int, ctypes.c_long] + [vp] * 10
        L.oracle_grid_statistics.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp]
        L.oracle_particles_init.restype = ctypes.c_long
        L.oracle_particles_init.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.c_int] + [vp] * 9
        _lib = L
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


class OParams(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("dt", ctypes.c_double), ("C3", ctypes.c_double),
                ("C4", ctypes.c_double), ("Cphi", ctypes.c_double), ("lid_u", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("ns", ctypes.c_int32), ("n_sources", ctypes.c_int32),
                ("src_x", ctypes.c_double * MAX_SOURCES), ("src_y", ctypes.c_double * MAX_SOURCES),
                ("src_r", ctypes.c_double * MAX_SOURCES), ("src_alpha", ctypes.c_int32 * MAX_SOURCES),
                ("react_k", ctypes.c_double), ("react_a", ctypes.c_int32), ("react_b", ctypes.c_int32),
                ("react_p", ctypes.c_int32)]


def make_params(nu, dt, seed, ns, sources=(), C3=5.0, C4=0.25, Cphi=2.0, lid_u=0.0, react=None) -> OParams:
    """Model constants: C_3, C_4 (Eq. 5), C_phi (IEM time scale); the paper prints no values,
    so the defaults are the literature values recalled for the cited models. react = (k, a, b, p):
    the reactive source of Eq. 9 for psi_a + psi_b -> psi_p at rate k."""
    p = OParams()
    p.nu, p.dt, p.C3, p.C4, p.Cphi, p.lid_u = nu, dt, C3, C4, Cphi, lid_u
    if react is not None:
        p.react_k, p.react_a, p.react_b, p.react_p = react
    p.seed, p.ns, p.n_sources = seed, ns, len(sources)
    for i, (sx, sy, sr, sa) in enumerate(sources):
        p.src_x[i], p.src_y[i], p.src_r[i], p.src_alpha[i] = sx, sy, sr, sa
    return p


class OracleMesh:
    """The oracle's own mesh (adjacency and periodic pairing built independently)."""

    def __init__(self, mesh):
        L = lib()
        self.node_xy = np.ascontiguousarray(mesh.node_xy, dtype=np.float64)
        self.tri = np.ascontiguousarray(mesh.tri, dtype=np.int32)
        self.tag = np.ascontiguousarray(mesh.edge_tag, dtype=np.int32)
        x0, x1, y0, y1 = mesh.box
        self.n_nodes, self.n_tri = self.node_xy.shape[0], self.tri.shape[0]
        self.ptr = L.oracle_mesh_new(_p(self.node_xy), self.n_nodes, _p(self.tri), self.n_tri, _p(self.tag),
                                     float(mesh.period_x), x0, x1, y0, y1)
        self.mesh = mesh

    def __del__(self):
        try:
            lib().oracle_mesh_free(self.ptr)
        except Exception:
            pass

    @property
    def edge_walls(self) -> bool:
        """True when some wall edge is off the sides of the bounding box (walls mirrored in the walk)."""
        return bool(lib().oracle_mesh_edge_walls(self.ptr))

    def neighbors(self):
        out = np.empty((self.n_tri, 3), dtype=np.int32)
        lib().oracle_mesh_neighbors(self.ptr, _p(out))
        return out

    def masters(self):
        out = np.empty(self.n_nodes, dtype=np.int32)
        lib().oracle_mesh_masters(self.ptr, _p(out))
        return out

    def locate_brute(self, px, py) -> int:
        return lib().oracle_locate_brute(self.ptr, float(px), float(py))

    def locate_walk(self, start, px, py):
        h = ctypes.c_int(0)
        e = lib().oracle_locate_walk(self.ptr, int(start), float(px), float(py), ctypes.byref(h))
        return e, h.value

    def locate_walk_reflect(self, start, px, py, u=0.0, v=0.0, w=0.0, lid_u=0.0):
        """The walk that mirrors the FP32 position across the wall edges it meets (walls of any
        shape): returns (owner or a negative code, x, y, u, v, w, hops, mirrorings)."""
        x, y = ctypes.c_float(px), ctypes.c_float(py)
        U, V, W = ctypes.c_double(u), ctypes.c_double(v), ctypes.c_double(w)
        h, n = ctypes.c_int(0), ctypes.c_int(0)
        e = lib().oracle_locate_walk_reflect(self.ptr, int(start), ctypes.byref(x), ctypes.byref(y), ctypes.byref(U),
                                             ctypes.byref(V), ctypes.byref(W), float(lid_u), ctypes.byref(h),
                                             ctypes.byref(n))
        return e, x.value, y.value, U.value, V.value, W.value, h.value, n.value

    def inside(self, e, px, py) -> bool:
        return bool(lib().oracle_inside(self.ptr, int(e), float(px), float(py)))

    def barycentric(self, e, px, py):
        out = np.empty(3, dtype=np.float64)
        lib().oracle_barycentric(self.ptr, int(e), float(px), float(py), _p(out))
        return out


def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.empty(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def normals6(seed, pid, step, tag=0):
    z = np.empty(6, dtype=np.float64)
    lib().oracle_normals6(seed, pid, step, tag, _p(z))
    return z


def orient2d_sign(ax, ay, bx, by, cx, cy) -> int:
    return lib().oracle_orient2d_sign(ax, ay, bx, by, cx, cy)


def _f32c(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def pdf_step(om: OracleMesh, params: OParams, fields, state, step: int, locate_mode: int = 0, beta=None):
    """One forward-Euler step of every particle (Eq. 2, 4, 5, 9; tracking; reflection; sources).

    `state` is a workloads.State (FP32); beta (n_nodes x 3 ns) switches Eq. 9 to IECM. Returns
    (dict of FP64 arrays, elem, aux, lost)."""
    P, ns = state.n, params.ns
    fields = _f32c(fields)
    nfp = fields.shape[1]
    beta = None if beta is None else _f32c(beta)
    ins = [_f32c(a) for a in (state.x, state.y, state.u, state.v, state.w, state.omega)]
    psi = _f32c(state.psi.reshape(ns, P))
    elem = np.ascontiguousarray(state.elem, dtype=np.int32)
    pid = np.ascontiguousarray(state.pid, dtype=np.uint32)
    outs = [np.empty(P) for _ in range(6)]
    opsi = np.empty((ns, P))
    oelem = np.empty(P, dtype=np.int32)
    aux = np.empty((P, 4))
    lost = lib().oracle_pdf_step(om.ptr, ctypes.byref(params), _p(fields), nfp, _p(beta), P,
                                 *[_p(a) for a in ins], _p(psi), _p(elem), _p(pid), step, locate_mode,
                                 *[_p(a) for a in outs], _p(opsi), _p(oelem), _p(aux))
    names = ("x", "y", "u", "v", "w", "omega")
    res = {n: a for n, a in zip(names, outs)}
    res["psi"] = opsi
    return res, oelem, aux, int(lost)


def moments(om: OracleMesh, ns: int, x, y, u, v, w, omega, psi, elem, with_abs: bool = True):
    """Gridpoint raw sums S_k(n) = sum_p lambda_n(X_p) q_k(p) (FP64) and sum |lambda||q|."""
    P = len(x)
    arrs = [_f64c(a) for a in (x, y, u, v, w, omega)]
    psi = _f64c(np.asarray(psi).reshape(ns, P))
    elem = np.ascontiguousarray(elem, dtype=np.int32)
    nq = 11 + 2 * ns
    S = np.empty((om.n_nodes, nq))
    Sabs = np.empty((om.n_nodes, nq)) if with_abs else None
    lib().oracle_moments(om.ptr, ns, P, *[_p(a) for a in arrs], _p(psi), _p(elem), _p(S), _p(Sabs))
    return S, Sabs


def flux_moments(om: OracleMesh, ns: int, x, y, u, v, w, psi, elem):
    """Raw scalar-flux sums per node: sum_p lambda_n (u psi_a, v psi_a, w psi_a), FP64."""
    P = len(x)
    F = np.empty((om.n_nodes, 3 * ns))
    lib().oracle_flux_moments(om.ptr, ns, P, *[_p(_f64c(a)) for a in (x, y, u, v, w)],
                              _p(_f64c(np.asarray(psi).reshape(ns, P))), _p(np.ascontiguousarray(elem, dtype=np.int32)),
                              _p(F))
    return F


def grid_statistics(S, ns: int):
    S = _f64c(S)
    out = np.empty_like(S)
    lib().oracle_grid_statistics(S.shape[0], ns, _p(S), _p(out))
    return out


def particles_init(om: OracleMesh, params: OParams, n_per_elem: int, node_init, m_erlang: int = 4):
    P = om.n_tri * n_per_elem
    ns = params.ns
    node_init = _f32c(node_init)
    outs = [np.empty(P) for _ in range(6)]
    opsi = np.empty((ns, P))
    oelem = np.empty(P, dtype=np.int32)
    opid = np.empty(P, dtype=np.uint32)
    lost = lib().oracle_particles_init(om.ptr, ctypes.byref(params), n_per_elem, _p(node_init), m_erlang,
                                       *[_p(a) for a in outs], _p(opsi), _p(oelem), _p(opid))
    names = ("x", "y", "u", "v", "w", "omega")
    res = {n: a for n, a in zip(names, outs)}
    res["psi"] = opsi
    return res, oelem, opid, int(lost)
