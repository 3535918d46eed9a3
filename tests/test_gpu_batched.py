"""Batched ensembles: several independent channels of uneven size in one multi-component mesh,
stepped by the same kernel launches (and by CUDA-graph replays), under every launch
configuration the autotuner chooses from. Each component must evolve bit-identically to the same
ensemble stepped alone (whose parity with the FP64 oracle the single-mesh tests establish)."""
import numpy as np
import pytest

from paper_1006_0549_gb300 import lpdf, workloads as wl
from tests import gpu_common as gc

pytestmark = pytest.mark.gpu

SIZES = [(10, 6), (17, 9), (7, 5)]          # (nx, ny) of the components
PPE = [12, 30, 7]
STEPS = 3


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_0549_gb300 import _build
    _build.build()
    return torch


def _components():
    meshes = [wl.channel_mesh(nx, ny, 500 + k) for k, (nx, ny) in enumerate(SIZES)]
    seeds = [77 + 1000 * k for k in range(len(meshes))]
    sources = [[(0.25, 0.3 + 0.6 * k, 0.05, 0)] for k in range(len(meshes))]
    fields = [wl.synthetic_node_fields(m, 1, seed=40 + k) for k, m in enumerate(meshes)]
    inits = [wl.node_init_fields(m) for m in meshes]
    return meshes, seeds, sources, fields, inits


def _run_single(torch, mesh, seed, sources, F, init, ppe, steps):
    gm = lpdf.Mesh(mesh)
    p = lpdf.make_params(seed=seed, ns=1, sources=sources)
    ctx = lpdf.Context(gm, p, mesh.n_tri * ppe + 128)
    ctx.particles_init(ppe, torch.from_numpy(init).cuda())
    Fd = torch.from_numpy(F).cuda()
    for s in range(steps):
        ctx.pdf_step(Fd, s)
    ctx.status()
    S = torch.empty((mesh.n_nodes, 13), dtype=torch.float64, device="cuda")
    ctx.grid_statistics(S, raw=True)
    torch.cuda.synchronize()
    return gc.host_state(ctx.get_state(), 1), S.cpu().numpy()


def _batched_ctx(torch, um, seeds, sources, inits):
    gm = lpdf.Mesh(um)
    assert gm.n_comp == len(seeds)
    p = lpdf.make_params(seed=1, ns=1)
    n = sum((um.tri_off[k + 1] - um.tri_off[k]) * PPE[k] for k in range(len(PPE)))
    ctx = lpdf.Context(gm, p, int(n) + 128)
    ctx.set_components(list(zip(seeds, sources)))
    ctx.particles_init_multi(PPE, torch.from_numpy(wl.stack_node_arrays(inits)).cuda())
    return gm, ctx


def _component_states(um, g: wl.State):
    """The union's state split by component: (state sorted by pid, local element ids)."""
    comp = np.searchsorted(um.tri_off, g.elem, side="right") - 1
    out = []
    for k in range(len(um.tri_off) - 1):
        idx = np.nonzero(comp == k)[0]
        idx = idx[np.argsort(g.pid[idx], kind="stable")]
        st = gc.reorder(g, idx)
        st.elem = st.elem - um.tri_off[k]
        out.append(st)
    return out


def _same(a: wl.State, b: wl.State):
    for k in gc.FIELDS + ("elem", "pid"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
    assert np.array_equal(a.psi, b.psi)


def _by_pid(st: wl.State):
    return gc.reorder(st, np.argsort(st.pid, kind="stable"))


def test_components_evolve_as_if_alone(torch_cuda):
    torch = torch_cuda
    meshes, seeds, sources, fields, inits = _components()
    um = wl.union_mesh(meshes)
    gm, ctx = _batched_ctx(torch, um, seeds, sources, inits)
    Fd = torch.from_numpy(wl.stack_node_arrays(fields)).cuda()
    for s in range(STEPS):
        ctx.pdf_step(Fd, s)
    ctx.status()
    S = torch.empty((um.n_nodes, 13), dtype=torch.float64, device="cuda")
    ctx.grid_statistics(S, raw=True)
    torch.cuda.synchronize()
    parts = _component_states(um, gc.host_state(ctx.get_state(), 1))
    S = S.cpu().numpy()
    for k, m in enumerate(meshes):
        alone, S_alone = _run_single(torch, m, seeds[k], sources[k], fields[k], inits[k], PPE[k], STEPS)
        assert parts[k].n == m.n_tri * PPE[k]
        _same(parts[k], _by_pid(alone))
        assert np.array_equal(S[um.node_off[k]:um.node_off[k + 1]], S_alone)


def test_graph_replayed_steps_equal_single_steps(torch_cuda):
    torch = torch_cuda
    meshes, seeds, sources, fields, inits = _components()
    um = wl.union_mesh(meshes)
    Fd = torch.from_numpy(wl.stack_node_arrays(fields)).cuda()
    results = []
    for graphs in (False, True):
        gm, ctx = _batched_ctx(torch, um, seeds, sources, inits)
        if graphs:
            ctx.pdf_steps(Fd, 0, 4)      # two graph replays
            ctx.pdf_steps(Fd, 4, 3)      # one replay (the graph of the other buffer) and a single step
        else:
            for s in range(7):
                ctx.pdf_step(Fd, s)
        ctx.status()
        S = torch.empty((um.n_nodes, 13), dtype=torch.float64, device="cuda")
        ctx.grid_statistics(S, raw=True)
        torch.cuda.synchronize()
        results.append((_by_pid_union(gc.host_state(ctx.get_state(), 1), um), S.cpu().numpy()))
    _same(results[0][0], results[1][0])
    assert np.array_equal(results[0][1], results[1][1])


def _by_pid_union(g: wl.State, um):
    comp = np.searchsorted(um.tri_off, g.elem, side="right") - 1
    return gc.reorder(g, np.lexsort((g.pid, comp)))


@pytest.mark.parametrize("adv,mom", [(a, m) for a in range(lpdf.N_ADV_VARIANTS) for m in (0,)] +
                         [(0, m) for m in range(1, lpdf.N_MOM_VARIANTS)])
def test_every_launch_configuration_gives_the_same_step(torch_cuda, adv, mom):
    torch = torch_cuda
    meshes, seeds, sources, fields, inits = _components()
    um = wl.union_mesh(meshes)
    Fd = torch.from_numpy(wl.stack_node_arrays(fields)).cuda()
    out = []
    for tune in ((0, 0), (adv, mom)):
        gm, ctx = _batched_ctx(torch, um, seeds, sources, inits)
        ctx.set_tune(*tune)
        for s in range(2):
            ctx.pdf_step(Fd, s)
        ctx.status()
        S = torch.empty((um.n_nodes, 13), dtype=torch.float64, device="cuda")
        ctx.grid_statistics(S, raw=True)
        torch.cuda.synchronize()
        out.append((gc.host_state(ctx.get_state(), 1), S.cpu().numpy()))
    # the step writes position i from thread i in every configuration: even the order agrees
    _same(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_autotune_picks_a_valid_configuration(torch_cuda):
    torch = torch_cuda
    meshes, seeds, sources, fields, inits = _components()
    um = wl.union_mesh(meshes)
    Fd = torch.from_numpy(wl.stack_node_arrays(fields)).cuda()
    gm, ctx = _batched_ctx(torch, um, seeds, sources, inits)
    (adv, mom), ms, used = ctx.autotune(Fd, 0, steps_per_trial=2, rounds=2)
    assert 0 <= adv < lpdf.N_ADV_VARIANTS and 0 <= mom < lpdf.N_MOM_VARIANTS
    assert used == (lpdf.N_ADV_VARIANTS + lpdf.N_MOM_VARIANTS) * 3 * 2
    assert np.all(ms > 0.0)
    assert ms[adv] == ms[:lpdf.N_ADV_VARIANTS].min()
    assert ms[lpdf.N_ADV_VARIANTS + mom] == ms[lpdf.N_ADV_VARIANTS:].min()
    ctx.status()
    # the tuned context keeps stepping
    ctx.pdf_steps(Fd, used, 2)
    ctx.status()
