"""Pins of the surrogate-network oracle (oracle/mlp.py) against library routines, finite
differences, closed forms and invariants, so that a dropped term, a transposed operand or a
wrong sign in it fails here before it is used to judge the tensor-core kernels."""

import numpy as np
import pytest

from oracle import fields as of
from oracle import mlp as om
from paper_1006_0549_gb300 import workloads as wl


def _random_norm(rng):
    n = om.identity_norm()
    n[0:8] = rng.standard_normal(8)
    n[8:16] = rng.uniform(0.5, 2.0, 8)
    n[16:23] = rng.uniform(0.5, 1.5, 7)
    n[23:30] = rng.standard_normal(7)
    n[30:37] = rng.uniform(0.5, 2.0, 7)
    return n


def _params(seed, bias=0.3):
    rng = np.random.default_rng(seed)
    p = wl.mlp_init_params(seed).astype(np.float64)
    layers = om.unpack(p)
    layers = [(W, bias * rng.standard_normal(b.shape)) for W, b in layers]
    return om.pack(layers)


def test_parameter_count_matches_the_stated_size():
    assert om.NPARAMS == 35079 and om.NNORM == 37
    assert wl.mlp_init_params(1).size == om.NPARAMS


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-6, 6, 10000),
                        # exact ties: 1 + 2^-8 (to 1), 1 + 3 2^-8 (to 1 + 2^-6), their negatives
                        [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 0.0, -0.0, 65504.0]])
    want = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    got = om.bf16(x)
    assert np.array_equal(got, want)
    assert om.bf16(1.0 + 2.0 ** -8) == 1.0 and om.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6


def test_exact_gradient_matches_central_differences():
    rng = np.random.default_rng(11)
    p = _params(3)
    norm = _random_norm(rng)
    feat = rng.standard_normal((6, 8)) * norm[8:16] + norm[0:8]
    tgt = rng.standard_normal((6, 7)) * norm[30:37] + norm[23:30]
    g, L = om.gradient(p, norm, feat, tgt, bf16_ops=False)
    assert L == pytest.approx(om.loss(p, norm, feat, tgt, bf16_ops=False), rel=1e-14)
    # coordinates in every block: W1, b1, W2, b2, W3, b3, W4, b4
    starts = np.cumsum([0, 1024, 128, 16384, 128, 16384, 128, 896, 7])
    idx = np.concatenate([s + rng.choice(e - s, 6, replace=False) for s, e in zip(starts[:-1], starts[1:])])
    for i in idx:
        h = 1e-5 * max(1.0, abs(p[i]))
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (om.loss(pp, norm, feat, tgt, False) - om.loss(pm, norm, feat, tgt, False)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-10), i


def test_hidden_unit_permutation_leaves_the_output_unchanged():
    rng = np.random.default_rng(2)
    p = _params(4)
    norm = _random_norm(rng)
    feat = rng.standard_normal((9, 8))
    (W1, b1), (W2, b2), (W3, b3), (W4, b4) = om.unpack(p)
    pi1, pi2 = rng.permutation(128), rng.permutation(128)
    q = om.pack([(W1[pi1], b1[pi1]), (W2[pi2][:, pi1], b2[pi2]), (W3[:, pi2], b3), (W4, b4)])
    for rounding in (False, True):
        y0, _ = om.forward(p, norm, feat, rounding)
        y1, _ = om.forward(q, norm, feat, rounding)
        assert np.allclose(y0, y1, rtol=1e-12, atol=1e-12)


def test_zero_middle_layers_give_the_closed_form():
    rng = np.random.default_rng(7)
    (W1, b1), (W2, b2), (W3, b3), (W4, b4) = om.unpack(_params(5))
    W2 = np.zeros_like(W2)
    W3 = np.zeros_like(W3)
    p = om.pack([(W1, b1), (W2, b2), (W3, b3), (W4, b4)])
    feat = rng.standard_normal((4, 8))
    y, acts = om.forward(p, om.identity_norm(), feat, bf16_ops=False)
    assert np.allclose(acts[1], np.tanh(b2)) and np.allclose(acts[2], np.tanh(b3))
    assert np.allclose(y, W4 @ np.tanh(b3) + b4, rtol=1e-13)


def test_standardisation_of_targets_and_outputs():
    rng = np.random.default_rng(8)
    p = _params(6)
    norm = _random_norm(rng)
    feat = rng.standard_normal((5, 8))
    y, _ = om.forward(p, norm, feat, False)
    yu = om.forward_user(p, norm, feat, False)
    assert np.allclose((yu - norm[23:30]) / norm[30:37], y)
    # targets equal to the outputs: zero loss and zero gradient
    g, L = om.gradient(p, norm, feat, yu, bf16_ops=False)
    assert L < 1e-28 and np.abs(g).max() < 1e-14


def test_rounded_gradient_stays_close_to_the_exact_one():
    rng = np.random.default_rng(9)
    p = _params(7)
    norm = om.identity_norm()
    feat, tgt = wl.mlp_random_data(256, 3)
    g0, _ = om.gradient(p, norm, feat, tgt, bf16_ops=False)
    g1, _ = om.gradient(p, norm, feat, tgt, bf16_ops=True)
    assert np.linalg.norm(g1 - g0) <= 0.02 * np.linalg.norm(g0)


def test_adam_with_a_constant_gradient_moves_by_lr_per_step():
    rng = np.random.default_rng(1)
    p0 = rng.standard_normal(50)
    g = rng.standard_normal(50)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    lr = 1e-3
    for t in range(1, 8):
        p, m, v = om.adam(p, g, m, v, t, lr)
        # bias-corrected moments equal g and g^2 exactly, so each step is lr g / (|g| + eps)
        assert np.allclose(p, p0 - t * lr * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)


def test_wall_distance_closed_forms():
    ch = wl.channel_mesh(12, 9, 1)
    y = ch.node_xy[:, 1]
    assert np.allclose(om.wall_distance(ch), np.minimum(y, 2.0 - y), atol=1e-12)
    cav = wl.cavity_mesh(9, 8, 2)
    x, y = cav.node_xy[:, 0], cav.node_xy[:, 1]
    assert np.allclose(om.wall_distance(cav), np.minimum.reduce([x, 1 - x, y, 1 - y]), atol=1e-12)


def test_anisotropy_inputs_for_isotropic_and_one_component_stresses():
    mesh = wl.cavity_mesh(6, 5, 1)
    N = mesh.n_nodes
    st = np.zeros((N, 13))
    st[:, 4] = st[:, 7] = st[:, 9] = 0.3          # isotropic, k = 0.45
    st[:, 10] = 2.0
    f = om.features(mesh, st)
    assert np.allclose(f[:, 1], np.log(0.45)) and np.allclose(f[:, 2], np.log(2.0))
    assert np.allclose(f[:, 3:8], 0.0, atol=1e-15)   # uniform eps: the wall ratio is 1 too
    st[:, 4], st[:, 7], st[:, 9] = 0.8, 0.0, 0.0  # one component: b = diag(2/3, -1/3, -1/3)
    f = om.features(mesh, st)
    assert np.allclose(f[:, 3:6], [2 / 3, -1 / 3, 0.0]) and np.allclose(f[:, 6], 2.0 / 3.0)
    st[:, 4], st[:, 5], st[:, 7] = 0.4, 0.4, 0.4  # two-component, fully correlated shear
    f = om.features(mesh, st)
    # b = [[1/6, 1/2, 0], [1/2, 1/6, 0], [0, 0, -1/3]]
    assert np.allclose(f[:, 3:6], [1 / 6, 1 / 6, 1 / 2])
    assert np.allclose(f[:, 6], 1 / 36 + 1 / 36 + 1 / 9 + 2 * 1 / 4)


def test_wall_dissipation_input_follows_the_nearest_wall_point():
    # channel: eps = k <omega> varies with y only, so the nearest wall point of a node at height
    # y < 1 lies on the bottom wall (y = 0) and the input is ln(eps(0) / eps(y))
    mesh = wl.channel_mesh(12, 9, 4)
    y = mesh.node_xy[:, 1]
    st = np.zeros((mesh.n_nodes, 13))
    st[:, 4] = st[:, 7] = st[:, 9] = 2.0 / 3.0            # k = 1
    st[:, 10] = 1.0 + 3.0 * np.abs(y - 1.0)                 # eps = 4 at both walls, 1 at the centre
    f = om.features(mesh, st)
    assert np.allclose(f[:, 7], np.log(4.0 / st[:, 10]), atol=1e-12)
    # on the wall itself the input is 0
    assert np.allclose(f[(y == 0.0) | (y == 2.0), 7], 0.0)
    # cavity: linear eps along the bottom wall, interpolated to the foot of the perpendicular
    cav = wl.cavity_mesh(8, 8, 5)
    x, y = cav.node_xy[:, 0], cav.node_xy[:, 1]
    st = np.zeros((cav.n_nodes, 13))
    st[:, 4] = st[:, 7] = st[:, 9] = 2.0 / 3.0
    st[:, 10] = 1.0 + x                                      # eps = 1 + x everywhere
    f = om.features(cav, st)
    near_bottom = (y < x) & (y < 1 - x) & (y < 1 - y)
    assert np.allclose(f[near_bottom, 7], 0.0, atol=1e-12)   # foot of the perpendicular at the same x
    near_left = (x < y) & (x < 1 - y) & (x < 1 - x)
    assert np.allclose(f[near_left, 7], np.log(1.0 / (1.0 + x[near_left])), atol=1e-12)


def test_targets_of_the_simplified_langevin_model():
    mesh = wl.channel_mesh(10, 8, 3)
    st = wl.synthetic_statistics(mesh, 1, 4)
    C0 = 2.1
    F = of.node_fields(mesh, st, 1, C0=C0, gmodel=1)
    y = om.targets(st, F, C0)
    assert np.allclose(y[:, [0, 3, 4]], -(0.5 + 0.75 * C0))
    assert np.allclose(y[:, [1, 2]], 0.0)
    assert np.allclose(y[:, 5], C0)
    assert np.allclose(y[:, 6], 1.0)


def test_targets_round_trip_to_the_relaxation_fields():
    mesh = wl.channel_mesh(10, 8, 3)
    st = wl.synthetic_statistics(mesh, 1, 4)
    F = of.node_fields(mesh, st, 1, gmodel=0)
    y = om.targets(st, F, 2.1)
    G, c0e = om.fields_from_outputs(st, y)
    assert np.allclose(G, F[:, 14:19], rtol=1e-12, atol=1e-14)
    assert np.allclose(c0e, F[:, 19], rtol=1e-12, atol=1e-14)
