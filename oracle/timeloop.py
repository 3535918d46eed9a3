"""FP64 oracle of the coupled time loop: particle step, gridpoint statistics, gridpoint solve.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): tests/ and the CPU-baseline legs of bench.py
call it; the CUDA package never does.

What it follows (arXiv:1006.0549): the particles are advanced by forward Euler with the node
fields of the previous solve (Section "Governing equations", summary paragraph: Eq. 2, 4, 5, 9);
their statistics are extracted at the gridpoints (Introduction, item i); the Eulerian fields are
solved on the grid from those statistics -- G_ij by the elliptic relaxation of the paragraph after
Eq. 4, S_omega from Eq. 6, and the mean pressure by a projection (Introduction, item ii) -- and
interpolated back to the particles by the next step. Each step is a call of the oracle's own
functions in that order: oracle.pdf_step, oracle.moments, oracle.grid_statistics and
oracle.fields.node_fields.

Precision: every computation is FP64. Between steps the particle state is held in FP32, the
precision of the step's interface (positions must be FP32 values for exact point location, and
the other fields follow the state layout of the method's hot path); node fields passed to the
next step are rounded to FP32 likewise.
"""
from __future__ import annotations

import time

import numpy as np

from . import fields as of
from . import grid_statistics, moments, pdf_step, OracleMesh


def _f32_state(res, elem, pid, cls):
    f = lambda a: np.asarray(a, dtype=np.float32)
    return cls(f(res["x"]), f(res["y"]), f(res["u"]), f(res["v"]), f(res["w"]), f(res["omega"]),
                 f(res["psi"]), np.asarray(elem, dtype=np.int32).copy(), pid.copy())


def run_coupled(mesh, params, state, fields0, steps: int, record=(), solve=None, om: OracleMesh | None = None,
                step0: int = 1, timings: dict | None = None):
    """Run `steps` coupled steps from `state` (FP32 SoA fields x, y, u, v, w, omega, psi, elem, pid;
    the state after each step has the input's class) with the first step's node
    fields `fields0` (n_nodes x nfp FP32). `params` is an oracle.OParams; `solve` holds the keyword
    arguments of oracle.fields.node_fields (nu, gmodel, pressure_solve, dpdx0, ...). Step n uses
    Philox step number step0 + n - 1. Returns (statistics at the steps listed in `record` as
    {n: (N x (11 + 2 ns)) means and central moments}, final state, particle losses); `timings`
    (a dict, optional) receives the host seconds spent in the particle steps with their statistics
    (step_s) and in the gridpoint solves (solve_s)."""
    om = om or OracleMesh(mesh)
    ns = params.ns
    solve = dict(solve or {})
    F = np.ascontiguousarray(fields0, dtype=np.float32)
    st = state
    out, lost_total = {}, 0
    t_step = t_solve = 0.0
    for n in range(1, steps + 1):
        t0 = time.perf_counter()
        res, elem, aux, lost = pdf_step(om, params, F, st, step0 + n - 1)
        lost_total += lost
        st = _f32_state(res, elem, st.pid, type(st))
        S, _ = moments(om, ns, *[getattr(st, k).astype(np.float64) for k in ("x", "y", "u", "v", "w", "omega")],
                       st.psi.astype(np.float64), st.elem, with_abs=False)
        stats = grid_statistics(S, ns)
        t1 = time.perf_counter()
        t_step += t1 - t0
        if n in record:
            out[n] = stats
        if n < steps:
            F = of.node_fields(mesh, stats, ns, **solve).astype(np.float32)
            t_solve += time.perf_counter() - t1
    if timings is not None:
        timings.update(step_s=t_step, solve_s=t_solve)
    return out, st, lost_total
