"""Thin ctypes binding of liblpdf (include/lpdf.h): argument marshalling only.

Every numerical step runs in the CUDA library. There is no CPU fallback: if liblpdf.so is
missing or cannot be loaded, every call raises. Device buffers are torch CUDA tensors (the
binding passes their data pointers) and streams are torch CUDA streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import workloads as wl

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblpdf.so")

LPDF_OK = 0
LPDF_ERR_ARG = -1
LPDF_ERR_MESH = -2
LPDF_ERR_LOST_PARTICLE = -3
LPDF_ERR_NONFINITE = -4
LPDF_ERR_CG_NOCONV = -5
LPDF_ERR_CUDA = -6
LPDF_ERR_OVERFLOW = -7
LPDF_ERR_UNSUPPORTED = -8
ERRORS = {-1: "LPDF_ERR_ARG", -2: "LPDF_ERR_MESH", -3: "LPDF_ERR_LOST_PARTICLE", -4: "LPDF_ERR_NONFINITE",
          -5: "LPDF_ERR_CG_NOCONV", -6: "LPDF_ERR_CUDA", -7: "LPDF_ERR_OVERFLOW", -8: "LPDF_ERR_UNSUPPORTED"}
MAX_SOURCES = 8
MAX_SCALARS = 4

# every symbol include/lpdf.h declares
EXPORTS = ("lpdf_params_default", "lpdf_last_error", "lpdf_version", "lpdf_mesh_load", "lpdf_mesh_free",
           "lpdf_mesh_info", "lpdf_mesh_neighbors", "lpdf_mesh_masters", "lpdf_ctx_create", "lpdf_ctx_free",
           "lpdf_ctx_set_params", "lpdf_ctx_size", "lpdf_particles_init", "lpdf_set_state", "lpdf_get_state",
           "lpdf_pdf_step", "lpdf_status", "lpdf_grid_statistics", "lpdf_pdf_step_static", "lpdf_sort",
           "lpdf_elliptic_relax_solve", "lpdf_ctx_set_timing", "lpdf_ctx_timings", "lpdf_tc_gemm_bf16",
           "lpdf_mlp_create", "lpdf_mlp_free", "lpdf_mlp_set_params", "lpdf_mlp_get_params", "lpdf_mlp_fit_norm",
           "lpdf_mlp_forward", "lpdf_mlp_gradient", "lpdf_mlp_train", "lpdf_surrogate_features",
           "lpdf_mlp_set_policy", "lpdf_surrogate_relax_solve", "lpdf_mesh_load_multi", "lpdf_ctx_set_components",
           "lpdf_particles_init_multi", "lpdf_pdf_steps", "lpdf_ctx_set_tune", "lpdf_ctx_autotune",
           "lpdf_grid_flux_statistics", "lpdf_iecm_coefficients", "lpdf_ctx_set_iecm", "lpdf_mlp_request_check")

N_ADV_VARIANTS, N_MOM_VARIANTS = 6, 4

MLP_IN, MLP_OUT, MLP_HIDDEN = 8, 7, 128
MLP_NPARAMS = 35079
MLP_NNORM = 37


class LpdfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Component(ctypes.Structure):
    """lpdf_component: per-component seed and scalar sources of a multi-component mesh."""
    _fields_ = [("seed", ctypes.c_uint64), ("n_sources", ctypes.c_int32),
                ("src_x", ctypes.c_float * 8), ("src_y", ctypes.c_float * 8), ("src_r", ctypes.c_float * 8),
                ("src_alpha", ctypes.c_int32 * 8)]


class Params(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("dt", ctypes.c_double), ("C3", ctypes.c_double), ("C4", ctypes.c_double),
                ("Cphi", ctypes.c_double), ("C0", ctypes.c_double), ("Comega1", ctypes.c_double),
                ("Comega2", ctypes.c_double), ("CL", ctypes.c_double), ("Ceta", ctypes.c_double),
                ("lid_u", ctypes.c_double), ("seed", ctypes.c_uint64), ("ns", ctypes.c_int32),
                ("n_sources", ctypes.c_int32), ("src_x", ctypes.c_float * MAX_SOURCES),
                ("src_y", ctypes.c_float * MAX_SOURCES), ("src_r", ctypes.c_float * MAX_SOURCES),
                ("src_alpha", ctypes.c_int32 * MAX_SOURCES),
                ("gmodel", ctypes.c_int32), ("pressure_solve", ctypes.c_int32), ("cg_warm_start", ctypes.c_int32),
                ("dpdx0", ctypes.c_double), ("dpdy0", ctypes.c_double),
                ("mixing", ctypes.c_int32), ("react_a", ctypes.c_int32), ("react_b", ctypes.c_int32),
                ("react_p", ctypes.c_int32), ("react_k", ctypes.c_double), ("moment_sums", ctypes.c_int32)]


_lib = None


def lib():
    """Load liblpdf.so (built by paper_1006_0549_gb300._build.build()); raise if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1006_0549_gb300._build.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    L.lpdf_params_default.argtypes = [vp]
    L.lpdf_params_default.restype = None
    L.lpdf_last_error.restype = ctypes.c_char_p
    L.lpdf_version.restype = ctypes.c_char_p
    L.lpdf_mesh_load.argtypes = [vp, i32, vp, i32, vp, ctypes.c_double, vp]
    L.lpdf_mesh_free.argtypes = [vp]
    L.lpdf_mesh_free.restype = None
    L.lpdf_mesh_info.argtypes = [vp, vp, vp, vp]
    L.lpdf_mesh_neighbors.argtypes = [vp, vp]
    L.lpdf_mesh_masters.argtypes = [vp, vp]
    L.lpdf_ctx_create.argtypes = [vp, vp, i64, vp]
    L.lpdf_ctx_free.argtypes = [vp]
    L.lpdf_ctx_free.restype = None
    L.lpdf_ctx_set_params.argtypes = [vp, vp]
    L.lpdf_ctx_size.argtypes = [vp]
    L.lpdf_ctx_size.restype = i64
    L.lpdf_particles_init.argtypes = [vp, i32, vp, i32, vp]
    L.lpdf_set_state.argtypes = [vp, i64] + [vp] * 9 + [ctypes.c_int, vp]
    L.lpdf_get_state.argtypes = [vp] + [vp] * 9 + [ctypes.c_int, vp]
    L.lpdf_pdf_step.argtypes = [vp, vp, u64, vp]
    L.lpdf_sort.argtypes = [vp, vp]
    L.lpdf_status.argtypes = [vp, vp, vp]
    L.lpdf_grid_statistics.argtypes = [vp, vp, ctypes.c_int, vp]
    L.lpdf_pdf_step_static.argtypes = [vp, vp, i64] + [vp] * 9 + [vp, u64, vp, vp, vp]
    L.lpdf_tc_gemm_bf16.argtypes = [vp, vp, vp, i32, i32, i32, vp]
    L.lpdf_ctx_set_timing.argtypes = [vp, ctypes.c_int]
    L.lpdf_ctx_timings.argtypes = [vp, vp, vp]
    L.lpdf_elliptic_relax_solve.argtypes = [vp, vp, vp, vp, ctypes.c_double, i32, vp, vp]
    L.lpdf_mlp_create.argtypes = [i64, vp]
    L.lpdf_mlp_free.argtypes = [vp]
    L.lpdf_mlp_free.restype = None
    L.lpdf_mlp_set_params.argtypes = [vp, vp, vp]
    L.lpdf_mlp_get_params.argtypes = [vp, vp, vp]
    L.lpdf_mlp_fit_norm.argtypes = [vp, vp, vp, i64, vp]
    L.lpdf_mlp_forward.argtypes = [vp, vp, i64, vp, vp]
    L.lpdf_mlp_gradient.argtypes = [vp, vp, vp, i64, vp, vp, vp]
    L.lpdf_mlp_train.argtypes = [vp, vp, vp, i64, i64, i32, ctypes.c_float, vp, vp]
    L.lpdf_surrogate_features.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.lpdf_mlp_set_policy.argtypes = [vp, i32, ctypes.c_double]
    L.lpdf_mlp_request_check.argtypes = [vp]
    L.lpdf_surrogate_relax_solve.argtypes = [vp, vp, vp, vp, vp, ctypes.c_double, i32, vp, vp]
    L.lpdf_mesh_load_multi.argtypes = [vp, i32, vp, i32, vp, i32, vp, vp, ctypes.c_double, vp]
    L.lpdf_ctx_set_components.argtypes = [vp, vp, i32]
    L.lpdf_particles_init_multi.argtypes = [vp, vp, vp, i32, vp]
    L.lpdf_pdf_steps.argtypes = [vp, vp, u64, i32, vp]
    L.lpdf_ctx_set_tune.argtypes = [vp, i32, i32]
    L.lpdf_grid_flux_statistics.argtypes = [vp, vp, ctypes.c_int, vp]
    L.lpdf_iecm_coefficients.argtypes = [vp, i32, vp, vp, vp, vp]
    L.lpdf_ctx_set_iecm.argtypes = [vp, vp]
    L.lpdf_ctx_autotune.argtypes = [vp, vp, u64, i32, i32, vp, vp, vp, vp]
    for name in EXPORTS:
        f = getattr(L, name)
        if f.restype is ctypes.c_int or (name not in ("lpdf_params_default", "lpdf_mesh_free", "lpdf_ctx_free",
                                                      "lpdf_last_error", "lpdf_version", "lpdf_ctx_size",
                                                      "lpdf_mlp_free")):
            f.restype = ctypes.c_int
    _lib = L
    return L


def _check(rc):
    if rc != LPDF_OK:
        raise LpdfError(rc, lib().lpdf_last_error().decode())
    return rc


def _ptr(t):
    """Data pointer of a torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return ctypes.c_void_p(t.ctypes.data)
    return ctypes.c_void_p(t.data_ptr())


def _stream(s):
    import torch
    if s is None:
        s = torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_params(nu=1.0 / 180.0, dt=1e-3, seed=1, ns=1, sources=(), lid_u=0.0, **consts) -> Params:
    p = Params()
    lib().lpdf_params_default(ctypes.byref(p))
    p.nu, p.dt, p.seed, p.ns, p.lid_u = nu, dt, seed, ns, lid_u
    p.n_sources = len(sources)
    for i, (sx, sy, sr, sa) in enumerate(sources):
        p.src_x[i], p.src_y[i], p.src_r[i], p.src_alpha[i] = sx, sy, sr, sa
    for k, v in consts.items():
        setattr(p, k, v)
    return p


def params_for(wk: "wl.Workload", **consts) -> Params:
    return make_params(nu=wk.nu, dt=wk.dt, seed=wk.seed, ns=wk.ns, sources=wk.sources, lid_u=wk.lid_u, **consts)


class Mesh:
    """lpdf_mesh_load (or lpdf_mesh_load_multi for a wl.MultiMesh) / lpdf_mesh_free."""

    def __init__(self, mesh: "wl.Mesh"):
        L = lib()
        xy = np.ascontiguousarray(mesh.node_xy, dtype=np.float64)
        tri = np.ascontiguousarray(mesh.tri, dtype=np.int32)
        tag = np.ascontiguousarray(mesh.edge_tag, dtype=np.int32)
        h = ctypes.c_void_p()
        node_off = getattr(mesh, "node_off", None)
        if node_off is None:
            _check(L.lpdf_mesh_load(_ptr(xy), xy.shape[0], _ptr(tri), tri.shape[0], _ptr(tag), float(mesh.period_x),
                                    ctypes.byref(h)))
            self.n_comp = 1
        else:
            no = np.ascontiguousarray(node_off, dtype=np.int32)
            to = np.ascontiguousarray(mesh.tri_off, dtype=np.int32)
            _check(L.lpdf_mesh_load_multi(_ptr(xy), xy.shape[0], _ptr(tri), tri.shape[0], _ptr(tag), len(no) - 1,
                                          _ptr(no), _ptr(to), float(mesh.period_x), ctypes.byref(h)))
            self.n_comp = len(no) - 1
        self.h = h
        self.mesh = mesh
        self.n_nodes, self.n_tri = xy.shape[0], tri.shape[0]

    def neighbors(self):
        out = np.empty((self.n_tri, 3), dtype=np.int32)
        _check(lib().lpdf_mesh_neighbors(self.h, _ptr(out)))
        return out

    def masters(self):
        out = np.empty(self.n_nodes, dtype=np.int32)
        _check(lib().lpdf_mesh_masters(self.h, _ptr(out)))
        return out

    def info(self):
        n = ctypes.c_int32()
        e = ctypes.c_int32()
        box = np.empty(4)
        _check(lib().lpdf_mesh_info(self.h, ctypes.byref(n), ctypes.byref(e), _ptr(box)))
        return n.value, e.value, tuple(box)

    def elliptic_relax_solve(self, params: Params, stats, out, tol: float = 1e-10, maxit: int = 20000, stream=None):
        """lpdf_elliptic_relax_solve: node fields (out, n_nodes x nfp float32, CUDA) from gridpoint
        statistics (stats, n_nodes x (11 + 2 ns) float64, CUDA). Returns the CG iteration counts."""
        it = np.zeros(2, dtype=np.int32)
        _check(lib().lpdf_elliptic_relax_solve(self.h, ctypes.byref(params), _ptr(stats), _ptr(out), float(tol),
                                               int(maxit), _ptr(it), _stream(stream)))
        return int(it[0]), int(it[1])

    def iecm_coefficients(self, ns: int, stats, flux, beta, stream=None):
        """lpdf_iecm_coefficients: beta (n_nodes x 3 ns FP32) from statistics and flux covariances."""
        _check(lib().lpdf_iecm_coefficients(self.h, int(ns), _ptr(stats), _ptr(flux), _ptr(beta), _stream(stream)))
        return beta

    def surrogate_features(self, params: Params, stats, feat, fields=None, tgt=None, stream=None):
        """lpdf_surrogate_features: per-node network inputs (feat, n_nodes x 8 float32, CUDA) and,
        with fields given, the targets taken from them (tgt, n_nodes x 7 float32, CUDA)."""
        _check(lib().lpdf_surrogate_features(self.h, ctypes.byref(params), _ptr(stats), _ptr(fields), _ptr(feat),
                                             _ptr(tgt), _stream(stream)))
        return feat, tgt

    def surrogate_relax_solve(self, net: "MLP", params: Params, stats, out, tol: float = 1e-10, maxit: int = 20000,
                              stream=None):
        """lpdf_surrogate_relax_solve: node fields with G_ij and C0 eps from the network, checked
        against the plain solve at the network's cadence. Returns (checked, error, used_plain, calls)."""
        info = np.zeros(4, dtype=np.float64)
        _check(lib().lpdf_surrogate_relax_solve(self.h, net.h, ctypes.byref(params), _ptr(stats), _ptr(out),
                                                float(tol), int(maxit), _ptr(info), _stream(stream)))
        return bool(info[0]), float(info[1]), bool(info[2]), int(info[3])

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().lpdf_mesh_free(self.h)
                self.h = None
        except Exception:
            pass


class Context:
    """lpdf_ctx_create and the per-ensemble calls."""

    def __init__(self, mesh: Mesh, params: Params, capacity: int):
        self.mesh = mesh
        self.params = params
        self.ns = params.ns
        h = ctypes.c_void_p()
        _check(lib().lpdf_ctx_create(mesh.h, ctypes.byref(params), int(capacity), ctypes.byref(h)))
        self.h = h

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().lpdf_ctx_free(self.h)
                self.h = None
        except Exception:
            pass

    @property
    def n(self) -> int:
        return int(lib().lpdf_ctx_size(self.h))

    def set_params(self, params: Params):
        _check(lib().lpdf_ctx_set_params(self.h, ctypes.byref(params)))
        self.params = params

    def particles_init(self, n_per_elem: int, node_init, m_erlang: int = 4, stream=None):
        _check(lib().lpdf_particles_init(self.h, int(n_per_elem), _ptr(node_init), int(m_erlang), _stream(stream)))

    def particles_init_multi(self, n_per_elem, node_init, m_erlang: int = 4, stream=None):
        """lpdf_particles_init_multi: n_per_elem[c] particles per element of component c."""
        ppe = np.ascontiguousarray(n_per_elem, dtype=np.int32)
        _check(lib().lpdf_particles_init_multi(self.h, _ptr(ppe), _ptr(node_init), int(m_erlang), _stream(stream)))

    def set_components(self, comps):
        """lpdf_ctx_set_components: comps = [(seed, [(x, y, r, alpha), ...]), ...], one per component."""
        arr = (Component * len(comps))()
        for k, (seed, sources) in enumerate(comps):
            arr[k].seed = int(seed)
            arr[k].n_sources = len(sources)
            for i, (sx, sy, sr, sa) in enumerate(sources):
                arr[k].src_x[i], arr[k].src_y[i], arr[k].src_r[i], arr[k].src_alpha[i] = sx, sy, sr, sa
        _check(lib().lpdf_ctx_set_components(self.h, arr, len(comps)))

    def pdf_steps(self, node_fields, step0: int, nsteps: int, stream=None):
        """lpdf_pdf_steps: nsteps steps from step0, pairs of steps replayed from a CUDA graph."""
        _check(lib().lpdf_pdf_steps(self.h, _ptr(node_fields), int(step0), int(nsteps), _stream(stream)))

    def grid_flux_statistics(self, out, raw: bool = False, stream=None):
        """lpdf_grid_flux_statistics: per node (u psi_a, v psi_a, w psi_a) sums or covariances (FP64)."""
        _check(lib().lpdf_grid_flux_statistics(self.h, _ptr(out), int(raw), _stream(stream)))
        return out

    def set_iecm(self, beta):
        """lpdf_ctx_set_iecm: the conditional-mean slopes (n_nodes x 3 ns FP32, CUDA) or None."""
        self._iecm_beta = beta            # the context reads it at every step: keep it alive
        _check(lib().lpdf_ctx_set_iecm(self.h, _ptr(beta)))

    def set_tune(self, adv: int, mom: int):
        _check(lib().lpdf_ctx_set_tune(self.h, int(adv), int(mom)))

    def autotune(self, node_fields, step0: int, steps_per_trial: int = 3, rounds: int = 2, stream=None):
        """lpdf_ctx_autotune: returns ((adv, mom), per-variant milliseconds per step, steps used)."""
        choice = np.zeros(2, dtype=np.int32)
        ms = np.zeros(N_ADV_VARIANTS + N_MOM_VARIANTS, dtype=np.float64)
        used = ctypes.c_int32()
        _check(lib().lpdf_ctx_autotune(self.h, _ptr(node_fields), int(step0), int(steps_per_trial), int(rounds),
                                       _ptr(choice), _ptr(ms), ctypes.byref(used), _stream(stream)))
        return (int(choice[0]), int(choice[1])), ms, used.value

    def set_state(self, st, stream=None):
        """st: dict/State of torch CUDA tensors (on_device=1) or numpy arrays (host)."""
        get = (lambda k: st[k]) if isinstance(st, dict) else (lambda k: getattr(st, k))
        x = get("x")
        on_dev = 0 if isinstance(x, np.ndarray) else 1
        n = int(x.shape[0])
        arrs = [get(k) for k in ("x", "y", "u", "v", "w", "omega", "psi", "elem", "pid")]
        if not on_dev:
            arrs = [np.ascontiguousarray(a) for a in arrs]
        self._keep = arrs
        _check(lib().lpdf_set_state(self.h, n, *[_ptr(a) for a in arrs], on_dev, _stream(stream)))

    def get_state(self, stream=None, device: bool = True):
        """Returns a dict of torch CUDA tensors (device=True) or numpy arrays."""
        import torch
        n, ns = self.n, self.ns
        if device:
            dev = torch.device("cuda")
            out = {k: torch.empty(n, dtype=torch.float32, device=dev) for k in ("x", "y", "u", "v", "w", "omega")}
            out["psi"] = torch.empty((ns, n), dtype=torch.float32, device=dev)
            out["elem"] = torch.empty(n, dtype=torch.int32, device=dev)
            out["pid"] = torch.empty(n, dtype=torch.int32, device=dev)
        else:
            out = {k: np.empty(n, dtype=np.float32) for k in ("x", "y", "u", "v", "w", "omega")}
            out["psi"] = np.empty((ns, n), dtype=np.float32)
            out["elem"] = np.empty(n, dtype=np.int32)
            out["pid"] = np.empty(n, dtype=np.uint32)
        _check(lib().lpdf_get_state(self.h, *[_ptr(out[k]) for k in ("x", "y", "u", "v", "w", "omega", "psi",
                                                                      "elem", "pid")], 1 if device else 0,
                                    _stream(stream)))
        if not device:
            torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        return out

    def sort(self, stream=None):
        """lpdf_sort: re-bucket the particles by element (deterministic order)."""
        _check(lib().lpdf_sort(self.h, _stream(stream)))

    def pdf_step(self, node_fields, step: int, stream=None):
        _check(lib().lpdf_pdf_step(self.h, _ptr(node_fields), int(step), _stream(stream)))

    def status(self, stream=None, raise_on_error: bool = True):
        out = np.zeros(4, dtype=np.int64)
        rc = lib().lpdf_status(self.h, _ptr(out), _stream(stream))
        if raise_on_error:
            _check(rc)
        return rc, out

    def set_timing(self, enable: bool = True):
        """lpdf_ctx_set_timing: record the device time of the step's kernels."""
        _check(lib().lpdf_ctx_set_timing(self.h, 1 if enable else 0))

    def timings(self):
        """lpdf_ctx_timings: (ms of the advance kernel, of the re-bucketing kernels, of the moments
        kernel) summed over the steps recorded since the previous call, and their number."""
        out = np.zeros(3)
        n = ctypes.c_int64()
        _check(lib().lpdf_ctx_timings(self.h, _ptr(out), ctypes.byref(n)))
        return out, n.value

    def grid_statistics(self, out, raw: bool = False, stream=None):
        _check(lib().lpdf_grid_statistics(self.h, _ptr(out), 1 if raw else 0, _stream(stream)))
        return out


def check_static_args(n_nodes: int, ns: int, state: dict, node_fields, moments) -> int:
    """The buffers of lpdf_pdf_step_static, checked before any launch: the library receives bare
    pointers and cannot size them, so a wrong dtype, shape or layout would become out-of-bounds
    device accesses. Raises ValueError; returns the particle count n."""
    import torch

    def need(name, t, dtypes, shape):
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if t.dtype not in dtypes:
            raise ValueError(f"{name} must be {' or '.join(str(d) for d in dtypes)}, not {t.dtype}")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} must have shape {tuple(shape)}, not {tuple(t.shape)}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")

    if not (1 <= ns <= MAX_SCALARS):
        raise ValueError(f"ns must be in 1..{MAX_SCALARS}, not {ns}")
    missing = [k for k in ("x", "y", "u", "v", "w", "omega", "psi", "elem", "pid") if k not in state]
    if missing:
        raise ValueError(f"state lacks {missing}")
    x = state["x"]
    if not isinstance(x, torch.Tensor) or x.dim() != 1:
        raise ValueError("state['x'] must be a 1-D torch tensor")
    n = int(x.shape[0])
    for k in ("x", "y", "u", "v", "w", "omega"):
        need(f"state[{k!r}]", state[k], (torch.float32,), (n,))
    need("state['psi']", state["psi"], (torch.float32,), (ns, n))
    need("state['elem']", state["elem"], (torch.int32,), (n,))
    need("state['pid']", state["pid"], (torch.int32, getattr(torch, "uint32", torch.int32)), (n,))
    need("node_fields", node_fields, (torch.float32,), (n_nodes, wl.n_fields_padded(ns)))
    need("moments", moments, (torch.float64,), (n_nodes, 11 + 2 * ns))
    tensors = [state[k] for k in ("x", "y", "u", "v", "w", "omega", "psi", "elem", "pid")] + [node_fields, moments]
    dev = {t.device for t in tensors}
    if len(dev) != 1 or next(iter(dev)).type != "cuda":
        raise ValueError(f"every buffer must be on one CUDA device, not {sorted(str(d) for d in dev)}")
    return n


def pdf_step_static(mesh: Mesh, params: Params, state: dict, node_fields, step: int, moments,
                    read_status: bool = True, stream=None):
    """lpdf_pdf_step_static: the step on caller-owned device buffers; allocates nothing.

    `state` holds torch CUDA tensors x, y, u, v, w, omega (float32, n), psi (float32, ns x n),
    elem and pid (int32, n), advanced in place; node_fields is n_nodes x n_fields_padded(ns)
    float32; `moments` (n_nodes x (11 + 2 ns) float64) receives the raw gridpoint sums. All on one
    CUDA device and contiguous (checked: ValueError)."""
    n = check_static_args(mesh.n_nodes, int(params.ns), state, node_fields, moments)
    st = np.zeros(4, dtype=np.int64) if read_status else None
    rc = lib().lpdf_pdf_step_static(mesh.h, ctypes.byref(params), n,
                                    *[_ptr(state[k]) for k in ("x", "y", "u", "v", "w", "omega", "psi", "elem",
                                                               "pid")],
                                    _ptr(node_fields), int(step), _ptr(moments), _ptr(st), _stream(stream))
    return rc, st


def tc_gemm_bf16(A, B, D, stream=None):
    """lpdf_tc_gemm_bf16: D = A B^T on the tensor cores (A: M x K, B: N x K BF16; D: M x N FP32;
    torch CUDA tensors)."""
    M, K = A.shape
    N = B.shape[0]
    _check(lib().lpdf_tc_gemm_bf16(_ptr(A), _ptr(B), _ptr(D), int(M), int(N), int(K), _stream(stream)))
    return D


class MLP:
    """lpdf_mlp: the learned surrogate network (8 -> 128 -> 128 -> 128 -> 7, BF16 tensor cores)."""

    def __init__(self, max_batch: int):
        h = ctypes.c_void_p()
        _check(lib().lpdf_mlp_create(int(max_batch), ctypes.byref(h)))
        self.h = h
        self.max_batch = int(max_batch)
        self.check_every, self.threshold = 50, 0.02

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().lpdf_mlp_free(self.h)
                self.h = None
        except Exception:
            pass

    def set_params(self, params, norm=None):
        """params: MLP_NPARAMS float32 (host); norm: MLP_NNORM float32 (host) or None."""
        p = np.ascontiguousarray(params, dtype=np.float32)
        n = None if norm is None else np.ascontiguousarray(norm, dtype=np.float32)
        if p.size != MLP_NPARAMS or (n is not None and n.size != MLP_NNORM):
            raise ValueError("parameter or standardisation block of the wrong size")
        _check(lib().lpdf_mlp_set_params(self.h, _ptr(p), _ptr(n)))

    def get_params(self):
        p = np.zeros(MLP_NPARAMS, dtype=np.float32)
        n = np.zeros(MLP_NNORM, dtype=np.float32)
        _check(lib().lpdf_mlp_get_params(self.h, _ptr(p), _ptr(n)))
        return p, n

    def fit_norm(self, feat, tgt, stream=None):
        _check(lib().lpdf_mlp_fit_norm(self.h, _ptr(feat), _ptr(tgt), int(feat.shape[0]), _stream(stream)))

    def forward(self, feat, out, stream=None):
        """out (B x 7 float32, CUDA) = the network on feat (B x 8 float32, CUDA), in target units."""
        _check(lib().lpdf_mlp_forward(self.h, _ptr(feat), int(feat.shape[0]), _ptr(out), _stream(stream)))
        return out

    def gradient(self, feat, tgt, stream=None):
        """(gradient (MLP_NPARAMS float32, host), loss) on the batch (feat, tgt)."""
        g = np.zeros(MLP_NPARAMS, dtype=np.float32)
        loss = ctypes.c_double()
        _check(lib().lpdf_mlp_gradient(self.h, _ptr(feat), _ptr(tgt), int(feat.shape[0]), _ptr(g),
                                       ctypes.byref(loss), _stream(stream)))
        return g, loss.value

    def train(self, feat, tgt, batch: int, steps: int, lr: float, stream=None):
        """Adam steps on minibatches; returns the minibatch losses (before each step)."""
        losses = np.zeros(max(int(steps), 1), dtype=np.float64)
        _check(lib().lpdf_mlp_train(self.h, _ptr(feat), _ptr(tgt), int(feat.shape[0]), int(batch), int(steps),
                                    float(lr), _ptr(losses), _stream(stream)))
        return losses[:int(steps)]

    def set_policy(self, check_every: int = 50, threshold: float = 0.02):
        _check(lib().lpdf_mlp_set_policy(self.h, int(check_every), float(threshold)))
        self.check_every, self.threshold = int(check_every), float(threshold)

    def request_check(self):
        """lpdf_mlp_request_check: the next surrogate solve checks against the plain solve."""
        _check(lib().lpdf_mlp_request_check(self.h))


def version() -> str:
    return lib().lpdf_version().decode()
