"""lpdf_pdf_step_static: the step for callers that cannot allocate device memory.

Some host codes own every device buffer through their own pool and forbid cudaMalloc in their
time loop; they call lpdf_pdf_step_static on their own buffers. Its scratch lives in a static
device array inside the library. This test drives it through the C-ABI on two calls in a row,
the first without reading the status back (asynchronous), on the periodic channel and on the
cavity with one and with four scalars. Each call's new state is checked against the FP64
oracle's step from the same input (the per-step parity of the other GPU tests: FP32 state within
the tolerance, every element id the oracle's brute-force owner), its moment sums against the
oracle's reduction of that state, and both against the ordinary context-based path (lpdf_pdf_step
+ raw grid statistics; particles matched by pid). Collected last on purpose (file name), so a
failure here comes after every other test has run.
"""
import numpy as np
import pytest

import oracle
from paper_1006_0549_gb300 import lpdf, workloads as wl

pytestmark = pytest.mark.gpu

RTOL = 1e-5          # FP32 particle state, as in the parity tests


def _dev(st, torch):
    d = torch.device("cuda")
    out = {k: torch.from_numpy(np.ascontiguousarray(getattr(st, k))).to(d)
           for k in ("x", "y", "u", "v", "w", "omega")}
    out["psi"] = torch.from_numpy(np.ascontiguousarray(st.psi)).to(d)
    out["elem"] = torch.from_numpy(np.ascontiguousarray(st.elem, dtype=np.int32)).to(d)
    out["pid"] = torch.from_numpy(np.ascontiguousarray(st.pid).view(np.int32)).to(d)
    return out


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_0549_gb300 import _build
    _build.build()
    return torch


@pytest.mark.parametrize("name,ns", [("channel", 1), ("channel", 4), ("cavity", 1), ("cavity", 4)])
def test_static_entry_point_matches_oracle_and_context_path(name, ns):
    torch = _cuda()
    from tests import gpu_common as gc
    wk = wl.channel_small() if name == "channel" else wl.cavity_small()
    src = [(x, y, r, a % ns) for (x, y, r, a) in wk.sources]
    params = lpdf.make_params(nu=wk.nu, dt=wk.dt, seed=wk.seed, ns=ns, sources=src, lid_u=wk.lid_u)
    mesh = lpdf.Mesh(wk.mesh)
    om = oracle.OracleMesh(wk.mesh)
    Fh = wl.synthetic_node_fields(wk.mesh, ns, seed=5)
    F = torch.from_numpy(Fh).cuda()
    st0 = wl.synthetic_state(wk.mesh, 25, ns, seed=31)
    nq = 11 + 2 * ns

    # the context path (allocates its own state and accumulators)
    ctx = lpdf.Context(mesh, params, st0.n)
    ctx.set_state(_dev(st0, torch))
    ref_states, ref_moments = [], []
    for step in (0, 1):
        ctx.pdf_step(F, step)
        rc, _ = ctx.status(raise_on_error=False)
        assert rc == lpdf.LPDF_OK
        S = torch.empty((mesh.n_nodes, nq), dtype=torch.float64, device="cuda")
        ctx.grid_statistics(S, raw=True)
        ref_states.append(gc.host_state(ctx.get_state(), ns))
        ref_moments.append(S.cpu().numpy())

    # caller-owned buffers, two calls in a row; the first does not read the status back
    state = _dev(st0, torch)
    st_in = st0
    for step in (0, 1):
        moments = torch.full((mesh.n_nodes, nq), np.nan, dtype=torch.float64, device="cuda")
        rc, status = lpdf.pdf_step_static(mesh, params, state, F, step, moments, read_status=(step == 1))
        assert rc == lpdf.LPDF_OK, (rc, status)
        if step == 1:
            assert status[0] == 0 and status[1] == 0 and status[2] == -1, status
        torch.cuda.synchronize()
        mine = gc.host_state(state, ns)
        # against the oracle's step from the same input
        gc.compare_step(wk.mesh, om, params, Fh, st_in, step, mine)
        S = moments.cpu().numpy()
        assert np.all(np.isfinite(S))
        gc.compare_moments(om, mine, S, ns)
        # against the context path (the fused kernel and the pipeline round and group differently)
        ref = ref_states[step]
        idx = gc.match_pids(mine.pid, ref.pid)
        for k in gc.FIELDS:
            o = getattr(ref, k)[idx].astype(np.float64)
            g = getattr(mine, k).astype(np.float64)
            rms = float(np.sqrt(np.mean(o * o))) or 1.0
            assert np.all(np.abs(g - o) <= RTOL * np.maximum(np.abs(o), rms)), (step, k)
        o = ref.psi[:, idx].astype(np.float64)
        g = mine.psi.astype(np.float64)
        assert np.all(np.abs(g - o) <= RTOL * np.maximum(np.abs(o), float(np.sqrt(np.mean(o * o))) or 1.0)), step
        assert np.array_equal(mine.elem, ref.elem[idx])
        # the second call starts from cleared accumulators: its sums are its own step's, as the
        # context path's (both against the oracle's reduction of the context path's state)
        gc.compare_moments(om, ref, ref_moments[step], ns)
        _, Sabs = oracle.moments(om, ns, *[getattr(ref, k).astype(np.float64) for k in gc.FIELDS],
                                 ref.psi.astype(np.float64), ref.elem)
        # the two states differ by at most RTOL per particle: 4 RTOL covers the products
        assert np.all(np.abs(S - ref_moments[step]) <= 4 * RTOL * Sabs + 1e-9), step
        st_in = mine


def test_static_entry_point_rejects_oversized_mesh():
    torch = _cuda()
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
    """The static entry point's fused kernel mixes with IEM only and sums the moments in FP32
    partials: IECM, a reactive source and compensated moment sums are refused (they need a
    context), not silently dropped."""
    torch = _cuda()
    small = wl.cavity_mesh(4, 4, 1)
    mesh = lpdf.Mesh(small)
    F = torch.zeros((small.n_nodes, wl.n_fields_padded(3)), dtype=torch.float32, device="cuda")
    moments = torch.zeros((small.n_nodes, 17), dtype=torch.float64, device="cuda")
    st = wl.synthetic_state(small, 1, 3, seed=1)
    for kw in ({"mixing": 1}, {"react_k": 5.0, "react_a": 0, "react_b": 1, "react_p": 2}, {"moment_sums": 1}):
        params = lpdf.make_params(nu=1e-4, dt=1e-3, seed=1, ns=3)
        for k, v in kw.items():
            setattr(params, k, v)
        rc, _ = lpdf.pdf_step_static(mesh, params, _dev(st, torch), F, 0, moments)
        assert rc == lpdf.LPDF_ERR_UNSUPPORTED, kw
        assert "need a context" in lpdf.lib().lpdf_last_error().decode()
