"""Parity of the CUDA particle step (through the C-ABI) with the FP64 oracle."""
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


def _setup(wk: wl.Workload, n_per_elem=None, fields_seed=5, moment_sums=0):
    import torch
    mesh = wk.mesh
    gm = lpdf.Mesh(mesh)
    om = oracle.OracleMesh(mesh)
    params = lpdf.params_for(wk, moment_sums=moment_sums)
    F = wl.synthetic_node_fields(mesh, wk.ns, seed=fields_seed)
    Fd = torch.from_numpy(F).cuda()
    npe = n_per_elem or wk.n_per_elem
    ctx = lpdf.Context(gm, params, mesh.n_tri * npe + 1000)
    return mesh, gm, om, params, F, Fd, ctx, npe


def test_mesh_adjacency_matches_oracle(torch_cuda):
    for mesh in (wl.channel_mesh(25, 20, 1), wl.cavity_mesh(20, 17, 2)):
        gm = lpdf.Mesh(mesh)
        om = oracle.OracleMesh(mesh)
        assert np.array_equal(gm.neighbors(), om.neighbors())
        assert np.array_equal(gm.masters(), om.masters())
        n, e, box = gm.info()
        assert (n, e) == (mesh.n_nodes, mesh.n_tri) and box == tuple(mesh.box)


BOUND = {0: "fp32", 1: "compensated"}


@pytest.mark.parametrize("workload,ms", [("channel", 0), ("cavity", 0), ("channel", 1), ("cavity", 1)])
def test_one_step_parity(torch_cuda, workload, ms):
    """One step from the same state on both sides; moment sums in either precision against the
    oracle's FP64 reduction of the GPU's new state (moment_sums = 1: within 1e-9 of sum |lambda q|)."""
    wk = wl.channel_small() if workload == "channel" else wl.cavity_small()
    mesh, gm, om, params, F, Fd, ctx, npe = _setup(wk, n_per_elem=20, moment_sums=ms)
    st = wl.synthetic_state(mesh, npe, wk.ns, seed=7)
    g, S, rc, status = gc.gpu_step(ctx, Fd, st, step=3)
    assert rc == lpdf.LPDF_OK, status
    diag, res, oelem = gc.compare_step(mesh, om, params, F, st, 3, g)
    ratio, _ = gc.compare_moments(om, g, S, wk.ns, BOUND[ms])
    print(workload, ms, diag, "moment error / sum|lambda q| max =", ratio)


def test_three_chained_steps_channel(torch_cuda):
    """Each step: the GPU advances its own state; the oracle re-runs that step from the GPU's input."""
    wk = wl.channel_small()
    mesh, gm, om, params, F, Fd, ctx, npe = _setup(wk, n_per_elem=30)
    st = wl.synthetic_state(mesh, npe, wk.ns, seed=8)
    for step in range(3):
        g, S, rc, status = gc.gpu_step(ctx, Fd, st, step)
        assert rc == lpdf.LPDF_OK
        gc.compare_step(mesh, om, params, F, st, step, g, check_locate=(step == 2))
        st = g


@pytest.mark.parametrize("ms", [0, 1])
def test_ragged_and_tiny_ensembles(torch_cuda, ms):
    """Sizes that are not multiples of the 8-particle lane chunk, 128-particle tile or 4096 CTA range."""
    wk = wl.channel_small()
    mesh, gm, om, params, F, Fd, ctx, npe = _setup(wk, n_per_elem=10, moment_sums=ms)
    full = wl.synthetic_state(mesh, 10, wk.ns, seed=9)
    for n in (1, 3, 127, 129, 4097, 9999):
        sel = np.sort(np.random.default_rng(n).choice(full.n, size=n, replace=False))
        st = wl.State(*(np.ascontiguousarray(getattr(full, k)[sel]) for k in gc.FIELDS),
                      np.ascontiguousarray(full.psi[:, sel]), full.elem[sel], full.pid[sel])
        g, S, rc, status = gc.gpu_step(ctx, Fd, st, 1)
        assert rc == lpdf.LPDF_OK
        gc.compare_step(mesh, om, params, F, st, 1, g)
        gc.compare_moments(om, g, S, wk.ns, BOUND[ms])


@pytest.mark.parametrize("workload,adv,mom", [("channel", a, 0) for a in range(lpdf.N_ADV_VARIANTS)] +
                         [(w, 0, m) for w in ("channel", "cavity") for m in range(1, lpdf.N_MOM_VARIANTS)])
def test_every_launch_variant_on_ragged_ensembles(torch_cuda, workload, adv, mom):
    """Each advance-kernel launch variant (one CTA per tile, persistent strides, the chunk queue)
    and each moments-kernel variant on sizes around the 64-particle chunks, 64- to 256-particle
    tiles and persistent grids, at up to 10 particles per element (the moments kernel's half-warp
    form): the oracle's step and moment sums, and the same bits as variant (0, 0)."""
    wk = wl.channel_small() if workload == "channel" else wl.cavity_small()
    mesh, gm, om, params, F, Fd, ctx, npe = _setup(wk, n_per_elem=10)
    full = wl.synthetic_state(mesh, 10, wk.ns, seed=19)
    for n in (1, 63, 64, 65, 129, 257, 5003):
        sel = np.sort(np.random.default_rng(n + 7).choice(full.n, size=n, replace=False))
        st = wl.State(*(np.ascontiguousarray(getattr(full, k)[sel]) for k in gc.FIELDS),
                      np.ascontiguousarray(full.psi[:, sel]), full.elem[sel], full.pid[sel])
        out = []
        for v in ((0, 0), (adv, mom)):
            ctx.set_tune(*v)
            g, S, rc, status = gc.gpu_step(ctx, Fd, st, 2)
            assert rc == lpdf.LPDF_OK, status
            out.append((g, S))
        for k in gc.FIELDS + ("elem", "pid"):
            assert np.array_equal(getattr(out[0][0], k), getattr(out[1][0], k)), (n, k)
        assert np.array_equal(out[0][0].psi, out[1][0].psi) and np.array_equal(out[0][1], out[1][1]), n
        gc.compare_step(mesh, om, params, F, st, 2, out[1][0])
        gc.compare_moments(om, out[1][0], out[1][1], wk.ns)


@pytest.mark.parametrize("npe", [200, 384, 385, 500])
def test_moments_on_both_sides_of_the_half_warp_threshold(torch_cuda, npe):
    """The moments kernel takes a half-warp per element when the ensemble averages at most 384
    particles per element, a warp otherwise: both forms against the oracle's FP64 reduction of the
    GPU's new state, within the FP32 partial-sum bound."""
    wk = wl.channel_small()
    mesh, gm, om, params, F, Fd, ctx, _ = _setup(wk, n_per_elem=npe)
    st = wl.synthetic_state(mesh, npe, wk.ns, seed=23)
    g, S, rc, status = gc.gpu_step(ctx, Fd, st, 4)
    assert rc == lpdf.LPDF_OK, status
    ratio, _ = gc.compare_moments(om, g, S, wk.ns)
    print(npe, "moment error / sum|lambda q| max =", ratio)


def test_empty_ensemble(torch_cuda):
    import torch
    wk = wl.channel_small()
    mesh, gm, om, params, F, Fd, ctx, npe = _setup(wk, n_per_elem=1)
    st = wl.synthetic_state(mesh, 1, wk.ns, seed=1)
    empty = wl.State(*(getattr(st, k)[:0].copy() for k in gc.FIELDS), st.psi[:, :0].copy(), st.elem[:0].copy(),
                     st.pid[:0].copy())
    g, S, rc, status = gc.gpu_step(ctx, Fd, empty, 0)
    assert rc == lpdf.LPDF_OK and g.n == 0 and np.all(S == 0.0)


@pytest.mark.parametrize("ms", [0, 1])
def test_step_is_bit_reproducible(torch_cuda, ms):
    wk = wl.cavity_small()
    mesh, gm, om, params, F, Fd, ctx, npe = _setup(wk, n_per_elem=40, moment_sums=ms)
    st = wl.synthetic_state(mesh, npe, wk.ns, seed=11)
    g1, S1, _, _ = gc.gpu_step(ctx, Fd, st, 5)
    g2, S2, _, _ = gc.gpu_step(ctx, Fd, st, 5)
    for k in gc.FIELDS:
        assert np.array_equal(getattr(g1, k), getattr(g2, k))
    assert np.array_equal(g1.elem, g2.elem) and np.array_equal(S1, S2)
    # a permutation of the particles changes nothing but the order (pid keys the noise)
    perm = np.random.default_rng(0).permutation(st.n)
    sp = wl.State(*(np.ascontiguousarray(getattr(st, k)[perm]) for k in gc.FIELDS),
                  np.ascontiguousarray(st.psi[:, perm]), st.elem[perm], st.pid[perm])
    g3, S3, _, _ = gc.gpu_step(ctx, Fd, sp, 5)
    inv = np.argsort(perm)
    for k in gc.FIELDS:
        assert np.array_equal(getattr(g3, k)[inv], getattr(g1, k))
    # the partial sums group different particles, so only the oracle tolerance applies
    gc.compare_moments(om, g3, S3, wk.ns, BOUND[ms])


def test_grid_statistics_means_and_central_moments(torch_cuda):
    import torch
    wk = wl.channel_small()
    mesh, gm, om, params, F, Fd, ctx, npe = _setup(wk, n_per_elem=20)
    st = wl.synthetic_state(mesh, npe, wk.ns, seed=12)
    g, S, rc, _ = gc.gpu_step(ctx, Fd, st, 0)
    out = torch.empty_like(torch.from_numpy(S)).cuda()
    ctx.grid_statistics(out, raw=False)
    stats_gpu = out.cpu().numpy()
    stats_ref = oracle.grid_statistics(S, wk.ns)    # same sums, oracle's formulas
    assert np.allclose(stats_gpu, stats_ref, rtol=1e-12, atol=1e-12)
    masters = gm.masters()
    uniq = masters == np.arange(mesh.n_nodes)
    assert abs(S[uniq, 0].sum() - st.n) < 1e-6 * st.n


def test_particles_init_parity(torch_cuda):
    """GPU initialisation vs the oracle's: positions within FP32 rounding, exact ownership of the
    GPU positions, velocities and frequencies within RTOL."""
    import torch
    wk = wl.channel_small()
    mesh, gm, om, params, F, Fd, ctx, npe = _setup(wk, n_per_elem=8)
    init = torch.from_numpy(wl.node_init_fields(mesh)).cuda()
    ctx.particles_init(npe, init, m_erlang=4)
    rc, status = ctx.status(raise_on_error=False)
    assert rc == lpdf.LPDF_OK
    g = gc.host_state(ctx.get_state(), wk.ns)
    res, oelem, opid, lost = oracle.particles_init(om, gc.oracle_params(params), npe, wl.node_init_fields(mesh), 4)
    assert lost == 0
    assert np.array_equal(g.pid, opid)
    for k in gc.FIELDS:
        o = res[k]
        rms = float(np.sqrt(np.mean(o * o)))
        assert np.all(np.abs(getattr(g, k) - o) <= 1e-5 * np.maximum(np.abs(o), rms)), k
    for i in range(g.n):
        assert om.locate_brute(float(g.x[i]), float(g.y[i])) == g.elem[i]
    assert np.all(g.psi == 0.0)


def test_lost_particle_is_reported_not_faulted(torch_cuda):
    """A particle whose element is > 64 hops from its position: the walk stops at its cap, the
    status reports the loss and the pid, and the context stays usable."""
    wk = wl.channel_25m()
    mesh = wk.mesh
    gm = lpdf.Mesh(mesh)
    params = lpdf.params_for(wk)
    import torch
    Fd = torch.from_numpy(wl.synthetic_node_fields(mesh, 1, seed=1)).cuda()
    ctx = lpdf.Context(gm, params, 4096)
    st = wl.synthetic_state(wl.channel_mesh(25, 20, 1), 1, 1, seed=1)
    st = wl.State(*(getattr(st, k)[:64].copy() for k in gc.FIELDS), st.psi[:, :64].copy(),
                  st.elem[:64].copy(), st.pid[:64].copy())
    # put every particle into a valid element of the big mesh first: x near 0.1 ...
    st.x[:] = 0.1
    st.y[:] = 1.0
    om = oracle.OracleMesh(mesh)
    e_true = om.locate_brute(0.1, 1.0)
    st.elem[:] = e_true
    st.elem[5] = (e_true + mesh.n_tri // 2) % mesh.n_tri      # ~125 columns away
    st.u[:] = 0.0; st.v[:] = 0.0
    g, S, rc, status = gc.gpu_step(ctx, Fd, st, 0)
    assert rc == lpdf.LPDF_ERR_LOST_PARTICLE
    assert status[1] == 1 and status[2] == st.pid[5]
    # the context still works
    st.elem[5] = e_true
    g, S, rc, status = gc.gpu_step(ctx, Fd, st, 1)
    assert rc == lpdf.LPDF_OK


def test_sort_rebuckets_deterministically(torch_cuda):
    """lpdf_sort: a permutation of the particles (every field travels with its pid), ordered by
    element and, within an element, by previous position."""
    wk = wl.channel_small()
    mesh, gm, om, params, F, Fd, ctx, npe = _setup(wk, n_per_elem=12)
    st = wl.synthetic_state(mesh, npe, wk.ns, seed=41)
    perm = np.random.default_rng(1).permutation(st.n)
    sp = wl.State(*(np.ascontiguousarray(getattr(st, k)[perm]) for k in gc.FIELDS),
                  np.ascontiguousarray(st.psi[:, perm]), st.elem[perm], st.pid[perm])
    ctx.set_state(gc.torch_state(sp))
    ctx.sort()
    g = gc.host_state(ctx.get_state(), wk.ns)
    assert np.all(np.diff(g.elem) >= 0)
    # within an element: previous positions ascending
    where = {int(p): i for i, p in enumerate(sp.pid)}
    prev = np.array([where[int(p)] for p in g.pid])
    same = g.elem[1:] == g.elem[:-1]
    assert np.all(prev[1:][same] > prev[:-1][same])
    idx = np.array([where[int(p)] for p in g.pid])
    for k in gc.FIELDS:
        assert np.array_equal(getattr(g, k), getattr(sp, k)[idx])
    assert np.array_equal(g.psi, sp.psi[:, idx])


def test_explicit_rebucketing_changes_only_the_order(torch_cuda):
    """lpdf_sort between steps changes only the order: per-pid state after 3 steps is bit-identical."""
    wk = wl.channel_small()
    mesh, gm, om, params, F, Fd, ctx, npe = _setup(wk, n_per_elem=10)
    st = wl.synthetic_state(mesh, npe, wk.ns, seed=42)
    ctx2 = lpdf.Context(gm, lpdf.params_for(wk), st.n)
    ctx.set_state(gc.torch_state(st))
    ctx2.set_state(gc.torch_state(st))
    for step in range(3):
        ctx.pdf_step(Fd, step)
        ctx2.sort()
        ctx2.pdf_step(Fd, step)
    a = gc.host_state(ctx.get_state(), wk.ns)
    b = gc.host_state(ctx2.get_state(), wk.ns)
    ia, ib = np.argsort(a.pid), np.argsort(b.pid)
    for k in gc.FIELDS:
        assert np.array_equal(getattr(a, k)[ia], getattr(b, k)[ib])
    assert np.array_equal(a.elem[ia], b.elem[ib])


@pytest.mark.parametrize("workload", ["channel", "cavity"])
def test_consecutive_steps_through_the_element_order(torch_cuda, workload):
    """Steps without set_state in between: each step gathers its input through the element order
    the previous step left behind. Every step matches the oracle run from that step's input
    (matched by pid), and the moments match the oracle's reduction of each new state."""
    import torch
    wk = wl.channel_small() if workload == "channel" else wl.cavity_small()
    mesh, gm, om, params, F, Fd, ctx, npe = _setup(wk, n_per_elem=25)
    st = wl.synthetic_state(mesh, npe, wk.ns, seed=43)
    ctx.set_state(gc.torch_state(st))
    for step in range(4):
        before = gc.host_state(ctx.get_state(), wk.ns)
        ctx.pdf_step(Fd, step)
        rc, status = ctx.status(raise_on_error=False)
        assert rc == lpdf.LPDF_OK, status
        after = gc.host_state(ctx.get_state(), wk.ns)
        S = torch.empty((mesh.n_nodes, 11 + 2 * wk.ns), dtype=torch.float64, device="cuda")
        ctx.grid_statistics(S, raw=True)
        torch.cuda.synchronize()
        gc.compare_step(mesh, om, params, F, before, step, after, check_locate=(step == 3))
        gc.compare_moments(om, after, S.cpu().numpy(), wk.ns)


@pytest.mark.parametrize("case", ["w_nan", "u_nan", "field_inf"])
def test_non_finite_state_is_reported_and_the_context_recovers(torch_cuda, case):
    """Non-finite values put in on the host: a NaN third velocity component of one particle (its
    position stays finite), a NaN streamwise velocity (the position becomes NaN too, so the walk
    cannot find an owner and the particle is also lost), and an Inf in one node's G11 (every
    particle of the elements around that node gets a non-finite velocity). The status word carries
    the non-finite bit (2); lpdf_status returns LPDF_ERR_NONFINITE, or LPDF_ERR_LOST_PARTICLE when
    the particle was lost as well; the next step from a clean state returns LPDF_OK."""
    import torch
    wk = wl.channel_small()
    mesh, gm, om, params, F, Fd, ctx, npe = _setup(wk, n_per_elem=10)
    st = wl.synthetic_state(mesh, npe, wk.ns, seed=44)
    bad_st = st.copy()
    bad_F = F.copy()
    if case == "w_nan":
        bad_st.w[17] = np.nan
    elif case == "u_nan":
        bad_st.u[17] = np.nan
    else:
        bad_F[int(mesh.tri[100, 0]), wl.F_G11] = np.inf
    g, S, rc, status = gc.gpu_step(ctx, torch.from_numpy(bad_F).cuda(), bad_st, 0)
    assert status[0] & 2, status
    if case == "u_nan":
        assert rc == lpdf.LPDF_ERR_LOST_PARTICLE and status[1] == 1 and status[2] == st.pid[17], (rc, status)
    else:
        assert rc == lpdf.LPDF_ERR_NONFINITE and status[1] == 0, (rc, status)
        assert not np.all(np.isfinite(g.w if case == "w_nan" else g.u))
    # the status was read and cleared; a clean step works and matches the oracle
    g, S, rc, status = gc.gpu_step(ctx, Fd, st, 1)
    assert rc == lpdf.LPDF_OK and status[0] == 0, status
    gc.compare_step(mesh, om, params, F, st, 1, g, check_locate=False)
