"""Parity at the full workload sizes, in the launch configuration the bench times.

The 50,000-triangle channel with 25M particles (one scalar) and the 199,712-triangle cavity with
~20M particles (four scalars, moving lid): the ensemble is initialised on the device, the launch
configuration is chosen by the autotuner on it (as bench.py does), and it is stepped once more,
so it is in the pipeline's element order; the next step is checked on samples the FP64 oracle
can compute one by one:
  * 20,000 sampled particles re-run by the oracle from the GPU's input state (matched by pid):
    FP32 state within the per-step tolerance;
  * all of them located by the oracle's neighbour walk from their input element (pinned against
    brute force by the oracle tests), and 300 by the oracle's brute force: element ids
    bit-exact; where the GPU position equals the oracle's bit for bit, the element does too;
  * the moment sums at 300 sampled gridpoints against the oracle's reduction of every particle
    whose new element touches them: FP32 partial sums within 48 eps32 and, from the same input
    state with compensated sums, within 1e-9 of sum |lambda q|.
Then the same step, from the same input state, in the autotuner's configuration and in another
one: bit-identical state and moment sums at full size. The 64-channel batch (268M particles) is
checked per component (last test)."""
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
    diag, _, _ = gc.compare_step(mesh, om, params, F, st, s1, g, check_locate="walk")
    assert diag["bitwise_equal_positions"] > 0.1, diag
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
    tol = gc.moment_tolerance(So[nodes], Sabs[nodes], "fp32", gc.lambda_rounding_sums(om, sub, wk.ns)[nodes])
    err = np.abs(S[nodes] - So[nodes])
    assert np.all(err <= tol), (nodes[np.argwhere(err > tol)[:5, 0]], err[err > tol][:5], tol[err > tol][:5])

    # the same step with compensated moment sums: the same new state, sums within 1e-9
    params.moment_sums = 1
    ctx.set_params(params)
    ctx.set_state(gc.torch_state(before))
    ctx.pdf_step(Fd, s1)
    rc, status = ctx.status(raise_on_error=False)
    assert rc == lpdf.LPDF_OK, status
    S1 = torch.empty((mesh.n_nodes, nq), dtype=torch.float64, device="cuda")
    ctx.grid_statistics(S1, raw=True)
    after1 = gc.host_state(ctx.get_state(device=False), wk.ns)
    torch.cuda.synchronize()
    after1 = gc.reorder(after1, gc.match_pids(after.pid, after1.pid))   # set_state restarts the order
    for k in gc.FIELDS + ("elem",):
        assert np.array_equal(getattr(after1, k), getattr(after, k)), k
    S1 = S1.cpu().numpy()
    tol1 = gc.moment_tolerance(So[nodes], Sabs[nodes], "compensated")
    err1 = np.abs(S1[nodes] - So[nodes])
    assert np.all(err1 <= tol1), (nodes[np.argwhere(err1 > tol1)[:5, 0]], err1[err1 > tol1][:5])
    print(name, "sampled node sums, max error / sum|lambda q|:", float(np.max(err / np.maximum(Sabs[nodes], 1e-300))),
          "(FP32 partials),", float(np.max(err1 / np.maximum(Sabs[nodes], 1e-300))), "(compensated)")
    params.moment_sums = 0
    ctx.set_params(params)

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


def _subset(d, idx, ns):
    """The particles `idx` (a device index tensor) of a device state dict, on the host."""
    sub = {k: v[idx] for k, v in d.items() if k != "psi"}
    sub["psi"] = d["psi"][:, idx]
    return gc.host_state(sub, ns)


def test_full_size_batched_sampled_parity(torch_cuda):
    """The 64 channel ensembles of uneven size (268M particles) in one multi-component mesh, set up
    and autotuned as the bench's batched run. For the smallest, a middle and the largest component,
    4,000 sampled particles of one step are re-run by the oracle on that component's own mesh with
    its own seed, source and node fields (particles matched by their per-component pid): FP32 state
    within the per-step tolerance, every element id against the oracle's walk from the input
    element, and 200 of them located by the oracle's brute force."""
    torch = torch_cuda
    wk = wl.batched_channels()
    parts = wk.mesh.parts
    gm = lpdf.Mesh(wk.mesh)
    ctx = lpdf.Context(gm, lpdf.make_params(nu=wk.nu, dt=wk.dt, seed=wk.seeds[0], ns=wk.ns), wk.n_particles)
    ctx.set_components(list(zip(wk.seeds, wk.sources)))
    ctx.particles_init_multi(wk.n_per_elem,
                             torch.from_numpy(wl.stack_node_arrays([wl.node_init_fields(m) for m in parts])).cuda())
    Fs = [wl.synthetic_node_fields(m, wk.ns, seed=5 + k) for k, m in enumerate(parts)]
    F = torch.from_numpy(wl.stack_node_arrays(Fs)).cuda()
    _, _, used = ctx.autotune(F, 0, steps_per_trial=1, rounds=1)
    ctx.pdf_step(F, used)
    rc, status = ctx.status(raise_on_error=False)
    assert rc == lpdf.LPDF_OK, status
    tri_off = torch.from_numpy(np.asarray(wk.mesh.tri_off, dtype=np.int64)).cuda()
    sizes = [m.n_tri for m in parts]
    comps = [int(np.argmin(sizes)), int(np.argsort(sizes)[len(sizes) // 2]), int(np.argmax(sizes))]
    rng = np.random.default_rng(31)
    before = ctx.get_state()
    cb = torch.searchsorted(tri_off, before["elem"].long(), right=True) - 1
    picked = {}
    for k in comps:
        idx = torch.nonzero(cb == k).squeeze(1)
        sel = torch.from_numpy(np.sort(rng.choice(idx.numel(), 4000, replace=False))).cuda()
        st = _subset(before, idx[sel], wk.ns)
        st.elem = (st.elem - wk.mesh.tri_off[k]).astype(np.int32)
        picked[k] = st
    del before
    s1 = used + 1
    ctx.pdf_step(F, s1)
    rc, status = ctx.status(raise_on_error=False)
    assert rc == lpdf.LPDF_OK, status
    after = ctx.get_state()
    ca = torch.searchsorted(tri_off, after["elem"].long(), right=True) - 1
    for k in comps:
        st = picked[k]
        idx = torch.nonzero(ca == k).squeeze(1)
        pid_k = after["pid"][idx].long()
        order = torch.argsort(pid_k)
        want = torch.from_numpy(st.pid.astype(np.int64)).cuda()
        pos = torch.searchsorted(pid_k[order], want).clamp(max=pid_k.numel() - 1)
        assert torch.equal(pid_k[order][pos], want), "the step lost or invented particles"
        g = _subset(after, idx[order][pos], wk.ns)
        g.elem = (g.elem - wk.mesh.tri_off[k]).astype(np.int32)
        mesh_k = parts[k]
        om = oracle.OracleMesh(mesh_k)
        p_k = lpdf.make_params(nu=wk.nu, dt=wk.dt, seed=wk.seeds[k], ns=wk.ns, sources=wk.sources[k])
        gc.compare_step(mesh_k, om, p_k, Fs[k], st, s1, g, check_locate="walk")
        for i in rng.choice(st.n, 200, replace=False):
            assert om.locate_brute(float(g.x[i]), float(g.y[i])) == g.elem[i]
