"""lpdf_pdf_step_static: the step for callers that cannot allocate device memory.

Some host codes own every device buffer through their own pool and forbid cudaMalloc in their
time loop; they call lpdf_pdf_step_static on their own buffers. Its scratch lives in a static
device array inside the library. This test drives it through the C-ABI on two calls in a row
and checks each against the ordinary context-based path (lpdf_pdf_step + raw grid statistics)
from the same input (particles matched by pid), and checks each path's moment sums against the
oracle's reduction of its own new state, within the parity tolerances of the other GPU tests. Collected last on
purpose (file name), so a failure here comes after every other test has run.
"""
import numpy as np
import pytest

import oracle
from paper_1006_0549_gb300 import lpdf, workloads as wl

pytestmark = pytest.mark.gpu

RTOL = 1e-5          # FP32 particle state, as in the parity tests
EPS32 = 2.0 ** -24


def _dev(st, torch):
    d = torch.device("cuda")
    out = {k: torch.from_numpy(np.ascontiguousarray(getattr(st, k))).to(d)
           for k in ("x", "y", "u", "v", "w", "omega")}
    out["psi"] = torch.from_numpy(np.ascontiguousarray(st.psi)).to(d)
    out["elem"] = torch.from_numpy(np.ascontiguousarray(st.elem, dtype=np.int32)).to(d)
    out["pid"] = torch.from_numpy(np.ascontiguousarray(st.pid).view(np.int32)).to(d)
    return out


def test_static_entry_point_matches_context_path():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_0549_gb300 import _build
    _build.build()
    wk = wl.cavity_small()
    mesh = lpdf.Mesh(wk.mesh)
    params = lpdf.params_for(wk)
    F = torch.from_numpy(wl.synthetic_node_fields(wk.mesh, wk.ns, seed=5)).cuda()
    st0 = wl.synthetic_state(wk.mesh, 25, wk.ns, seed=31)
    nq = 11 + 2 * wk.ns

    # reference: the context path (allocates its own state and accumulators)
    ctx = lpdf.Context(mesh, params, st0.n)
    ctx.set_state(_dev(st0, torch))
    ref_states, ref_moments = [], []
    for step in (0, 1):
        ctx.pdf_step(F, step)
        rc, _ = ctx.status(raise_on_error=False)
        assert rc == lpdf.LPDF_OK
        S = torch.empty((mesh.n_nodes, nq), dtype=torch.float64, device="cuda")
        ctx.grid_statistics(S, raw=True)
        ref_states.append({k: v.cpu().numpy() for k, v in ctx.get_state().items()})
        ref_moments.append(S.cpu().numpy())

    # caller-owned buffers, two calls in a row
    from tests import gpu_common as gc
    om = oracle.OracleMesh(wk.mesh)
    state = _dev(st0, torch)
    for step in (0, 1):
        moments = torch.full((mesh.n_nodes, nq), np.nan, dtype=torch.float64, device="cuda")
        rc, status = lpdf.pdf_step_static(mesh, params, state, F, step, moments)
        assert rc == lpdf.LPDF_OK, (rc, status)
        torch.cuda.synchronize()
        # the context path keeps its ensemble in element order: match the particles by pid
        ref = ref_states[step]
        mine = {k: v.cpu().numpy() for k, v in state.items()}
        idx = gc.match_pids(mine["pid"].view(np.uint32), ref["pid"].view(np.uint32))
        for k in ("x", "y", "u", "v", "w", "omega"):
            o = ref[k][idx].astype(np.float64)
            g = mine[k].astype(np.float64)
            rms = float(np.sqrt(np.mean(o * o))) or 1.0
            assert np.all(np.abs(g - o) <= RTOL * np.maximum(np.abs(o), rms)), (step, k)
        o = ref["psi"].reshape(wk.ns, -1)[:, idx].astype(np.float64)
        g = mine["psi"].reshape(wk.ns, -1).astype(np.float64)
        assert np.all(np.abs(g - o) <= RTOL * np.maximum(np.abs(o), float(np.sqrt(np.mean(o * o))) or 1.0)), step
        assert np.array_equal(mine["elem"], ref["elem"][idx])
        S = moments.cpu().numpy()
        assert np.all(np.isfinite(S))
        # the sums of the static path against the oracle's reduction of its own new state, with
        # the bound of the parity tests (the two paths group the FP32 partials differently)
        gc.compare_moments(om, gc.host_state(state, wk.ns), S, wk.ns)
        # and the context path's sums against the oracle's reduction of its state
        gc.compare_moments(om, gc.host_state({k: torch.from_numpy(v) for k, v in ref.items()}, wk.ns),
                           ref_moments[step], wk.ns)


def test_static_entry_point_rejects_oversized_mesh():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    big = wl.cavity_mesh(400, 400, 1)          # 160,801 nodes x 19 > 2^21 accumulators
    mesh = lpdf.Mesh(big)
    params = lpdf.make_params(nu=1e-4, dt=1e-3, seed=1, ns=4)
    F = torch.zeros((big.n_nodes, wl.n_fields_padded(4)), dtype=torch.float32, device="cuda")
    moments = torch.zeros((big.n_nodes, 19), dtype=torch.float64, device="cuda")
    st = wl.synthetic_state(wl.cavity_mesh(4, 4, 1), 1, 4, seed=1)
    rc, _ = lpdf.pdf_step_static(mesh, params, _dev(st, torch), F, 0, moments)
    assert rc == lpdf.LPDF_ERR_ARG
    assert "static maximum" in lpdf.lib().lpdf_last_error().decode()


def test_static_entry_point_rejects_iecm_and_reactions():
    """The static entry point's fused kernel mixes with IEM only: IECM and a reactive source are
    refused (they need a context), not silently dropped."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    small = wl.cavity_mesh(4, 4, 1)
    mesh = lpdf.Mesh(small)
    F = torch.zeros((small.n_nodes, wl.n_fields_padded(3)), dtype=torch.float32, device="cuda")
    moments = torch.zeros((small.n_nodes, 17), dtype=torch.float64, device="cuda")
    st = wl.synthetic_state(small, 1, 3, seed=1)
    for kw in ({"mixing": 1}, {"react_k": 5.0, "react_a": 0, "react_b": 1, "react_p": 2}):
        params = lpdf.make_params(nu=1e-4, dt=1e-3, seed=1, ns=3)
        for k, v in kw.items():
            setattr(params, k, v)
        rc, _ = lpdf.pdf_step_static(mesh, params, _dev(st, torch), F, 0, moments)
        assert rc == lpdf.LPDF_ERR_UNSUPPORTED, kw
        assert "need a context" in lpdf.lib().lpdf_last_error().decode()
