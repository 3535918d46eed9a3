"""Parity at the full workload sizes, in the launch configuration the bench times.

The 50,000-triangle channel with 25M particles (one scalar) and the 199,712-triangle cavity with
~20M particles (four scalars, moving lid): the ensemble is initialised on the device, the launch
configuration is chosen by the autotuner on it (as bench.py does), and it is stepped once more,
so it is in the pipeline's element order; the next step is checked on samples the FP64 oracle
can compute one by one:
  * 20,000 sampled particles re-run by the oracle from the GPU's input state (matched by pid):
    FP32 state within the per-step tolerance;
  * 300 of them located by the oracle's brute force: element ids bit-exact;
  * the moment sums at 300 sampled gridpoints against the oracle's reduction of every particle
    whose new element touches them.
Then the same step, from the same input state, in the autotuner's configuration and in another
one: bit-identical state and moment sums at full size."""
import numpy as np
import pytest

import oracle
from paper_1006_0549_gb300 import lpdf, workloads as wl
from tests import gpu_common as gc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_0549_gb300 import _build
    _build.build()
    return torch


@pytest.mark.parametrize("name", ["channel-50k-25M", "cavity-200k-20M"])
def test_full_size_sampled_parity(torch_cuda, name):
    torch = torch_cuda
    wk = wl.channel_25m() if name.startswith("channel") else wl.cavity_20m()
    mesh = wk.mesh
    gm = lpdf.Mesh(mesh)
    om = oracle.OracleMesh(mesh)
    params = lpdf.params_for(wk)
    ctx = lpdf.Context(gm, params, wk.n_particles)
    ctx.particles_init(wk.n_per_elem, torch.from_numpy(wl.node_init_fields(mesh)).cuda(), m_erlang=4)
    F = wl.synthetic_node_fields(mesh, wk.ns, seed=5)
    Fd = torch.from_numpy(F).cuda()
    choice, _, used = ctx.autotune(Fd, 0, steps_per_trial=2, rounds=1)
    ctx.pdf_step(Fd, used)
    rc, status = ctx.status(raise_on_error=False)
    assert rc == lpdf.LPDF_OK, status
    before = gc.host_state(ctx.get_state(device=False), wk.ns)
    s1 = used + 1
    ctx.pdf_step(Fd, s1)
    rc, status = ctx.status(raise_on_error=False)
    assert rc == lpdf.LPDF_OK, status
    after = gc.host_state(ctx.get_state(device=False), wk.ns)
    nq = 11 + 2 * wk.ns
    S = torch.empty((mesh.n_nodes, nq), dtype=torch.float64, device="cuda")
    ctx.grid_statistics(S, raw=True)
    torch.cuda.synchronize()
    S = S.cpu().numpy()
    assert before.n == after.n == wk.n_particles
    assert abs(S[gm.masters() == np.arange(mesh.n_nodes), 0].sum() - after.n) < 1e-6 * after.n

    rng = np.random.default_rng(20260)
    # sampled particles: the oracle's step from the GPU's input state
    sel = np.sort(rng.choice(before.n, 20000, replace=False))
    st = gc.reorder(before, sel)
    g = gc.reorder(after, gc.match_pids(st.pid, after.pid))
    gc.compare_step(mesh, om, params, F, st, s1, g, check_locate=False)
    for i in rng.choice(st.n, 300, replace=False):
        assert om.locate_brute(float(g.x[i]), float(g.y[i])) == g.elem[i]

    # sampled gridpoints: every particle whose new element touches them
    masters = gm.masters()
    em = masters[mesh.tri]
    nodes = rng.choice(np.unique(masters), 300, replace=False)
    touch = np.isin(em, nodes).any(axis=1)
    sub = gc.reorder(after, np.nonzero(touch[after.elem])[0])
    f = lambda a: a.astype(np.float64)
    So, Sabs = oracle.moments(om, wk.ns, f(sub.x), f(sub.y), f(sub.u), f(sub.v), f(sub.w), f(sub.omega),
                              f(sub.psi), sub.elem)
    tol = 48 * gc.EPS32 * Sabs[nodes] + np.maximum(So[nodes, :1], 1.0) * 8.0 * 2.0 ** -33
    err = np.abs(S[nodes] - So[nodes])
    assert np.all(err <= tol), (nodes[np.argwhere(err > tol)[:5, 0]], err[err > tol][:5], tol[err > tol][:5])

    # the tuned configuration and another one, from the same input state: the same bits
    other = (0, 0) if tuple(choice) != (0, 0) else (3, 2)
    outs = []
    for tune in (tuple(choice), other):
        ctx.set_state(gc.torch_state(before))
        ctx.set_tune(*tune)
        ctx.pdf_step(Fd, s1)
        rc, status = ctx.status(raise_on_error=False)
        assert rc == lpdf.LPDF_OK, status
        S2 = torch.empty((mesh.n_nodes, nq), dtype=torch.float64, device="cuda")
        ctx.grid_statistics(S2, raw=True)
        torch.cuda.synchronize()
        outs.append((gc.host_state(ctx.get_state(device=False), wk.ns), S2.cpu().numpy()))
    (a, Sa), (b, Sb) = outs
    for k in gc.FIELDS + ("elem", "pid"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), (tune, k)
    assert np.array_equal(a.psi, b.psi)
    assert np.array_equal(Sa, Sb)
