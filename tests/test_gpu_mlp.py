"""The BF16 tensor-core (tcgen05) kernels of the learned relaxation surrogate."""
import numpy as np
import pytest

from paper_1006_0549_gb300 import lpdf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_0549_gb300 import _build
    _build.build()
    return torch


@pytest.mark.parametrize("M,N,K", [(128, 128, 16), (300, 128, 128), (256, 256, 64), (1, 16, 16), (513, 16, 128)])
def test_tc_gemm_matches_fp32_product_of_the_bf16_values(torch_cuda, M, N, K):
    torch = torch_cuda
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    D = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    lpdf.tc_gemm_bf16(A.cuda(), B.cuda(), D)
    ref = A.double().numpy() @ B.double().numpy().T          # products of BF16 values are exact in FP32
    got = D.cpu().numpy().astype(np.float64)
    scale = np.abs(A.double().numpy()) @ np.abs(B.double().numpy()).T
    assert np.all(np.abs(got - ref) <= 1e-6 * scale + 1e-30), float(np.max(np.abs(got - ref) / scale))


# ---------------------------------------------------------------------------- surrogate network
from oracle import fields as of          # noqa: E402
from oracle import mlp as om             # noqa: E402
from paper_1006_0549_gb300 import workloads as wl   # noqa: E402

# Forward parity: both sides round the same operands to BF16; the GPU sums in FP32 (the oracle
# exactly), so a hidden activation can land on the other side of a BF16 rounding boundary now and
# then (one BF16 step, 2^-8 relative). Bound on the standardised outputs:
FWD_MAX = 2e-2
FWD_MEAN = 1e-3
# Gradient parity (the oracle rounds the same error signals to BF16): per block, relative L2
GRAD_REL = 1e-2


def _net(seed, bias=0.2):
    rng = np.random.default_rng(seed)
    p = wl.mlp_init_params(seed).astype(np.float64)
    layers = [(W, bias * rng.standard_normal(b.shape)) for W, b in om.unpack(p)]
    return om.pack(layers).astype(np.float32)


def _norm_for(feat, tgt):
    n = om.identity_norm()
    n[0:8] = feat.mean(axis=0)
    n[8:16] = feat.std(axis=0)
    n[23:30] = tgt.mean(axis=0)
    n[30:37] = tgt.std(axis=0)
    n[16:23] = np.linspace(0.5, 1.5, 7)
    return n.astype(np.float32)


@pytest.mark.parametrize("B", [1, 128, 300, 1031, 100489])   # 100,489: the nodes of the 20M cavity
def test_mlp_forward_matches_the_oracle(torch_cuda, B):
    torch = torch_cuda
    feat, tgt = wl.mlp_random_data(B, 10 + B)
    p = _net(B)
    norm = _norm_for(feat, tgt) if B > 1 else om.identity_norm().astype(np.float32)
    net = lpdf.MLP(1024)
    net.set_params(p, norm)
    out = torch.full((B, 7), float("nan"), dtype=torch.float32, device="cuda")
    net.forward(torch.from_numpy(feat).cuda(), out)
    got = out.cpu().numpy().astype(np.float64)
    want = om.forward_user(p.astype(np.float64), norm.astype(np.float64), feat)
    d = np.abs(got - want) / norm[30:37]
    assert np.all(np.isfinite(got))
    assert d.max() <= FWD_MAX and d.mean() <= FWD_MEAN, (d.max(), d.mean())


def _blocks():
    s = np.cumsum([0, 1024, 128, 16384, 128, 16384, 128, 896, 7])
    return list(zip(s[:-1], s[1:]))


@pytest.mark.parametrize("B", [300, 1024])
def test_mlp_gradient_matches_the_oracle_and_is_reproducible(torch_cuda, B):
    torch = torch_cuda
    feat, tgt = wl.mlp_random_data(B, 20 + B)
    p = _net(7 + B)
    norm = _norm_for(feat, tgt)
    net = lpdf.MLP(1024)
    net.set_params(p, norm)
    f, t = torch.from_numpy(feat).cuda(), torch.from_numpy(tgt).cuda()
    g, L = net.gradient(f, t)
    g2, L2 = net.gradient(f, t)
    assert np.array_equal(g, g2) and L == L2
    want, Lw = om.gradient(p.astype(np.float64), norm.astype(np.float64), feat, tgt, bf16_ops=True)
    exact, _ = om.gradient(p.astype(np.float64), norm.astype(np.float64), feat, tgt, bf16_ops=False)
    assert L == pytest.approx(Lw, rel=1e-3)
    for a, b in _blocks():
        e = np.linalg.norm(g[a:b] - want[a:b]) / np.linalg.norm(want[a:b])
        assert e <= GRAD_REL, (a, b, e)
        assert np.linalg.norm(g[a:b] - exact[a:b]) <= 5e-2 * np.linalg.norm(exact[a:b]), (a, b)


def test_mlp_adam_steps_match_the_oracle(torch_cuda):
    torch = torch_cuda
    B = 512
    feat, tgt = wl.mlp_random_data(B, 31)
    p = _net(31)
    norm = _norm_for(feat, tgt)
    net = lpdf.MLP(B)
    net.set_params(p, norm)
    f, t = torch.from_numpy(feat).cuda(), torch.from_numpy(tgt).cuda()
    P = p.astype(np.float64)
    m = np.zeros_like(P)
    v = np.zeros_like(P)
    lr = 1e-3
    for step in range(1, 4):
        g, _ = net.gradient(f, t)                     # the gradient the next train step uses
        net.train(f, t, batch=B, steps=1, lr=lr)
        P, m, v = om.adam(P, g.astype(np.float64), m, v, step, lr)
        got, _ = net.get_params()
        assert np.allclose(got, P, rtol=1e-5, atol=1e-7), step


def test_mlp_training_reduces_the_loss(torch_cuda):
    torch = torch_cuda
    feat, tgt = wl.mlp_random_data(8192, 41)
    net = lpdf.MLP(1024)
    net.set_params(wl.mlp_init_params(41))
    f, t = torch.from_numpy(feat).cuda(), torch.from_numpy(tgt).cuda()
    net.fit_norm(f, t)
    _, norm = net.get_params()
    assert np.allclose(norm[0:8], feat.mean(axis=0), rtol=1e-4, atol=1e-4)
    assert np.allclose(norm[8:16], feat.std(axis=0), rtol=1e-4)
    assert np.allclose(norm[23:30], tgt.mean(axis=0), rtol=1e-4, atol=1e-4)
    losses = net.train(f, t, batch=1024, steps=800, lr=2e-3)
    assert np.all(np.isfinite(losses))
    assert losses[-8:].mean() < 0.05 * losses[:8].mean(), (losses[:8].mean(), losses[-8:].mean())
    # the trained network, run forward, agrees with the oracle on held-out rows
    fe, te = wl.mlp_random_data(512, 42)
    out = torch.empty((512, 7), dtype=torch.float32, device="cuda")
    net.forward(torch.from_numpy(fe).cuda(), out)
    P, norm = net.get_params()
    want = om.forward_user(P.astype(np.float64), norm.astype(np.float64), fe)
    assert np.max(np.abs(out.cpu().numpy() - want) / norm[30:37]) <= FWD_MAX


def _channel(torch):
    mesh = wl.channel_mesh(24, 20, 5)
    gm = lpdf.Mesh(mesh)
    params = lpdf.make_params(ns=1)
    return mesh, gm, params


@pytest.mark.parametrize("case", ["channel-small", "cavity-200k"])
def test_surrogate_inputs_and_targets_match_the_oracle(torch_cuda, case):
    """The network's inputs and targets per node; the cavity case is the full 199,712-triangle mesh
    (100,489 nodes, four scalars) that the surrogate configuration runs on."""
    torch = torch_cuda
    if case == "channel-small":
        mesh, gm, params = _channel(torch)
        ns = 1
    else:
        wk = wl.cavity_20m()
        mesh, ns = wk.mesh, wk.ns
        gm = lpdf.Mesh(mesh)
        params = lpdf.params_for(wk)
    st = wl.synthetic_statistics(mesh, ns, 8)
    S = torch.from_numpy(st).cuda()
    nfp = wl.n_fields_padded(ns)
    F = torch.empty((mesh.n_nodes, nfp), dtype=torch.float32, device="cuda")
    gm.elliptic_relax_solve(params, S, F, 1e-10)
    feat = torch.empty((mesh.n_nodes, 8), dtype=torch.float32, device="cuda")
    tgt = torch.empty((mesh.n_nodes, 7), dtype=torch.float32, device="cuda")
    gm.surrogate_features(params, S, feat, F, tgt)
    torch.cuda.synchronize()
    want_f = om.features(mesh, st)
    got_f = feat.cpu().numpy()
    assert np.allclose(got_f, want_f, rtol=2e-6, atol=1e-6)
    want_t = om.targets(st, F.cpu().numpy(), params.C0)
    assert np.allclose(tgt.cpu().numpy(), want_t, rtol=2e-6, atol=1e-6)


def test_surrogate_solve_checks_falls_back_and_uses_the_network(torch_cuda):
    torch = torch_cuda
    mesh, gm, params = _channel(torch)
    st = wl.synthetic_statistics(mesh, 1, 9)
    S = torch.from_numpy(st).cuda()
    nfp = wl.n_fields_padded(1)
    plain = torch.empty((mesh.n_nodes, nfp), dtype=torch.float32, device="cuda")
    gm.elliptic_relax_solve(params, S, plain, 1e-10)
    plain = plain.cpu().numpy()
    net = lpdf.MLP(256)
    net.set_params(_net(3), None)
    out = torch.full((mesh.n_nodes, nfp), float("nan"), dtype=torch.float32, device="cuda")
    # an untrained network: the first (checking) call measures a large error and returns the plain
    # fields; the next call runs the plain solve because the check failed
    checked, err, used_plain, calls = gm.surrogate_relax_solve(net, params, S, out, 1e-10)
    assert checked and used_plain and err > 0.02 and calls == 1
    assert np.array_equal(out.cpu().numpy(), plain)
    checked, err, used_plain, calls = gm.surrogate_relax_solve(net, params, S, out, 1e-10)
    assert not checked and used_plain and err == -1.0 and calls == 2
    assert np.array_equal(out.cpu().numpy(), plain)
    # a threshold the network passes: the following unchecked call uses the network alone
    net.set_policy(check_every=3, threshold=1e30)
    checked, err, used_plain, _ = gm.surrogate_relax_solve(net, params, S, out, 1e-10)   # call 2: no check
    assert not checked and used_plain
    checked, err, used_plain, _ = gm.surrogate_relax_solve(net, params, S, out, 1e-10)   # call 3: check
    assert checked and used_plain and err > 0.02
    out.fill_(float("nan"))
    checked, err, used_plain, _ = gm.surrogate_relax_solve(net, params, S, out, 1e-10)   # network
    assert not checked and not used_plain
    got = out.cpu().numpy()
    P, norm = net.get_params()
    y = om.forward_user(P.astype(np.float64), norm.astype(np.float64), om.features(mesh, st))
    G, c0e = om.fields_from_outputs(st, y)
    scale = np.abs(G).max()
    assert np.max(np.abs(got[:, 14:19] - G)) <= 2e-2 * scale
    assert np.max(np.abs(got[:, 19] - c0e)) <= 2e-2 * max(np.abs(c0e).max(), 1e-30)
    # every other column is the plain solve's
    other = [c for c in range(22 + 1) if not 14 <= c <= 19]
    assert np.allclose(got[:, other], plain[:, other], rtol=1e-6, atol=1e-6)
    # a requested check runs on the next call whatever the cadence, once
    net.set_policy(check_every=1000, threshold=1e30)
    net.request_check()
    checked, err, used_plain, _ = gm.surrogate_relax_solve(net, params, S, out, 1e-10)
    assert checked and used_plain and err > 0.0
    checked, _, _, _ = gm.surrogate_relax_solve(net, params, S, out, 1e-10)
    assert not checked
