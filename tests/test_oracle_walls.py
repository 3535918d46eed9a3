"""Pins of the oracle's walls of any shape: the walk in a non-convex domain, and the mirroring of
a particle across a slanted or curved wall edge (reading 8 applied to each wall edge)."""
import numpy as np
import pytest

import oracle
from paper_1006_0549_gb300 import workloads as wl


def _inside_points(mesh, rng, n):
    """Random points strictly inside random elements (owner known by construction)."""
    e = rng.integers(0, mesh.n_tri, n)
    r = rng.uniform(0.02, 1.0, size=(n, 3))
    r /= r.sum(axis=1, keepdims=True)
    xy = np.einsum("pk,pkd->pd", r, mesh.node_xy[mesh.tri[e]]).astype(np.float32).astype(np.float64)
    return e, xy


def test_mesh_kinds():
    assert oracle.OracleMesh(wl.bump_channel_mesh(12, 8, 1)).edge_walls
    assert oracle.OracleMesh(wl.trapezoid_mesh(8, 8, 2)).edge_walls
    assert not oracle.OracleMesh(wl.channel_mesh(8, 6, 3)).edge_walls
    assert not oracle.OracleMesh(wl.cavity_mesh(6, 6, 4)).edge_walls


def test_walk_in_a_non_convex_domain_finds_the_owner_without_crossing_the_wall():
    """Points of the bump channel reached from elements a few hops away: the walk (interior exits
    first) ends at the brute-force owner, never at a wall."""
    mesh = wl.bump_channel_mesh(24, 10, 5, amp=0.3)
    om = oracle.OracleMesh(mesh)
    nbr = om.neighbors()
    rng = np.random.default_rng(1)
    e_true, xy = _inside_points(mesh, rng, 3000)
    for k in range(len(e_true)):
        start = int(e_true[k])
        for _ in range(int(rng.integers(0, 4))):          # a random nearby start
            cand = [n for n in nbr[start] if n >= 0]
            start = int(cand[rng.integers(0, len(cand))])
        e, _ = om.locate_walk(start, xy[k, 0], xy[k, 1])
        assert e == om.locate_brute(xy[k, 0], xy[k, 1]), (k, start, xy[k])


def _still_fields(mesh, ns):
    """Node fields that leave U unchanged (no pressure gradient, no drift, no diffusion)."""
    F = np.zeros((mesh.n_nodes, wl.n_fields_padded(ns)), dtype=np.float32)
    F[:, wl.F_OMEGA] = 1.0
    return F


def test_mirror_across_a_slanted_wall():
    """Particles near the trapezoid's left wall (the line from (0, 0) to (0.3, 0.8)) moving out
    through it: the final position is the mirror image of the moved position (checked with the
    unit-normal form p' = q - 2 ((q - a).n) n), the velocity is reversed, and the owner exists."""
    mesh = wl.trapezoid_mesh(12, 12, 7)
    om = oracle.OracleMesh(mesh)
    rng = np.random.default_rng(3)
    a = np.array([0.0, 0.0])
    d = np.array([0.3, 0.8]) / np.hypot(0.3, 0.8)
    n_in = np.array([d[1], -d[0]])                         # inward unit normal (the domain is to the right)
    # start points inside, 0.002 .. 0.01 from the wall, away from its ends
    P = 400
    t = rng.uniform(0.25, 0.75, P) * np.hypot(0.3, 0.8)
    dist = rng.uniform(0.002, 0.01, P)
    pts = (a + t[:, None] * d + dist[:, None] * n_in).astype(np.float32)
    elem = np.array([om.locate_brute(float(x), float(y)) for x, y in pts], dtype=np.int32)
    assert np.all(elem >= 0)
    speed = rng.uniform(15.0, 30.0, P)                     # dt = 1e-3: moves of 0.015 .. 0.03 outward
    U = (-speed[:, None] * n_in).astype(np.float32)
    st = wl.State(pts[:, 0].copy(), pts[:, 1].copy(), U[:, 0].copy(), U[:, 1].copy(),
                  np.zeros(P, np.float32), np.ones(P, np.float32), np.zeros((1, P), np.float32), elem,
                  np.arange(P, dtype=np.uint32))
    p = oracle.make_params(nu=1e-30, dt=1e-3, seed=9, ns=1)
    res, oelem, aux, lost = oracle.pdf_step(om, p, _still_fields(mesh, 1), st, 1, locate_mode=2)
    assert lost == 0
    q = aux[:, 0:2]                                        # moved position before the wall treatment
    beyond = (q - a) @ n_in < 0.0
    assert beyond.all()
    want = q - 2.0 * ((q - a) @ n_in)[:, None] * n_in[None, :]
    got = np.stack([res["x"], res["y"]], axis=1)
    assert np.allclose(got, want, atol=2e-7)
    assert np.all(aux[:, 2] == 1)                          # one mirroring each
    assert np.array_equal(res["u"], -st.u.astype(np.float64)) and np.array_equal(res["v"], -st.v.astype(np.float64))
    for i in range(P):
        assert om.locate_brute(res["x"][i], res["y"][i]) == oelem[i] >= 0


def test_particles_stay_in_the_bump_channel():
    """A step with fast random velocities: every particle ends owned, walk and brute force agree,
    and the ones that met the curved wall were mirrored back into the fluid."""
    mesh = wl.bump_channel_mesh(20, 8, 11, amp=0.3)
    om = oracle.OracleMesh(mesh)
    st = wl.synthetic_state(mesh, 6, 1, seed=12)
    st.u *= 4.0
    st.v = (st.v * 20.0).astype(np.float32)
    p = oracle.make_params(nu=1.0 / 180.0, dt=1e-3, seed=13, ns=1)
    F = wl.synthetic_node_fields(mesh, 1, seed=14)
    res, oelem, aux, lost = oracle.pdf_step(om, p, F, st, 1, locate_mode=2)
    assert lost == 0
    assert np.all(oelem >= 0)
    assert (aux[:, 2] > 0).sum() > 10                      # some particles met a wall


def _corner_state(mesh, om, n, rng):
    """Particles near the top-left corner (the periodic seam meets the top wall), moving up and
    to the left: the move crosses the seam and the top wall in the same step."""
    x = rng.uniform(0.0005, 0.004, n).astype(np.float32)
    y = (2.0 - rng.uniform(0.0005, 0.004, n)).astype(np.float32)
    elem = np.array([om.locate_brute(float(a), float(b)) for a, b in zip(x, y)], dtype=np.int32)
    assert np.all(elem >= 0)
    u = -rng.uniform(4.0, 8.0, n).astype(np.float32)
    v = rng.uniform(4.0, 8.0, n).astype(np.float32)
    return wl.State(x, y, u, v, np.zeros(n, np.float32), np.ones(n, np.float32), np.zeros((1, n), np.float32),
                    elem, np.arange(n, dtype=np.uint32))


def test_corner_of_the_seam_and_a_curved_walled_channel():
    """A step that wraps a particle across the periodic seam and carries it beyond the (flat) top
    wall: the walk starts in the image frame of the old element, crosses the periodic edge, mirrors
    the position across the top wall and finds the owner; nothing is lost. On this mesh the first
    element of such a walk can have the point beyond both its periodic edge and its diagonal, the
    diagonal more negative: a walk that took the diagonal reached a triangle with no periodic edge
    where the point lies beyond the wall only, and went round until the hop cap."""
    mesh = wl.bump_channel_mesh(250, 100, 1006054905)
    om = oracle.OracleMesh(mesh)
    # that walk: from element 198 to the wrapped position beyond the top wall
    e, hops = om.locate_walk(198, 6.2829685, 2.0009649)
    assert e == -1 and hops <= 2                  # it reaches the top wall, which the step mirrors
    rng = np.random.default_rng(21)
    st = _corner_state(mesh, om, 2000, rng)
    p = oracle.make_params(nu=1e-30, dt=1e-3, seed=22, ns=1)
    res, oelem, aux, lost = oracle.pdf_step(om, p, _still_fields(mesh, 1), st, 1, locate_mode=2)
    assert lost == 0
    pre_x, pre_y = aux[:, 0], aux[:, 1]
    assert np.all(pre_x < 0.0) and np.all(pre_y > 2.0)          # beyond the seam and the wall
    assert np.all(aux[:, 2] == 1)                                # one mirroring each
    L = np.float32(mesh.period_x)
    assert np.allclose(res["x"], np.float32(pre_x) + L, atol=4e-7)
    assert np.allclose(res["y"], 4.0 - pre_y, atol=4e-7)        # mirror across y = 2
    assert np.array_equal(res["v"], -st.v.astype(np.float64))
    for i in range(st.n):
        assert om.locate_brute(res["x"][i], res["y"][i]) == oelem[i] >= 0


def test_image_across_a_sloped_wall_is_wrapped_into_the_frame():
    """A particle at the bottom-left corner of the 50,000-triangle bump channel (pid 1810 of the
    25M run, its state at step 1) moves just below the bottom wall near the seam. The wall edge
    there rises slightly, so the mirror image lands at x = -1.5e-6, outside the periodic frame:
    it is wrapped to the other side, and the walk finds its owner instead of going back and forth
    across the seam until the hop cap."""
    mesh = wl.bump_channel_mesh(250, 100, 1006054905)
    om = oracle.OracleMesh(mesh)
    f = lambda v: np.array([v], dtype=np.float32)
    st = wl.State(f(0.00021887), f(0.00056443), f(-0.12476623), f(1.2149805), f(0.0), f(1.0),
                  np.zeros((1, 1), np.float32), np.array([0], np.int32), np.array([1810], np.uint32))
    p = oracle.make_params(nu=1.0 / 180.0, dt=1e-3, seed=wl.channel_25m().seed, ns=1)
    res, oelem, aux, lost = oracle.pdf_step(om, p, _still_fields(mesh, 1), st, 1, locate_mode=2)
    assert aux[0, 1] < 0.0 and aux[0, 2] == 1          # below the wall, one mirroring
    assert lost == 0
    L = mesh.period_x
    assert L - 1e-4 < res["x"][0] < L                  # wrapped to the right end of the frame
    assert om.locate_brute(res["x"][0], res["y"][0]) == oelem[0] >= 0


@pytest.mark.parametrize("seed", [16, 21])
def test_walks_across_the_seam_end_at_the_owner_or_at_a_wall(seed):
    """Points near the periodic seam of a curved-wall channel, walked from elements on the other
    side of the seam (so the walk starts in a periodic image frame): a point of the domain ends at
    its brute-force owner; a point just beyond the top or bottom wall near the seam ends at a wall
    (-1), never at the hop cap. (On these meshes the image-frame rule of taking the most negative
    interior edge first ran dozens of such walks into the hop cap.)"""
    mesh = wl.bump_channel_mesh(30, 10, seed, amp=0.3)
    om = oracle.OracleMesh(mesh)
    L = mesh.period_x
    cx = mesh.node_xy[mesh.tri].mean(axis=1)[:, 0]
    right = np.nonzero(cx > L - 0.5)[0]                 # starts on the far side of the seam
    left = np.nonzero(cx < 0.5)[0]
    rng = np.random.default_rng(17)
    # points of the domain near x = 0, walked from the right end
    e_true, xy = _inside_points(mesh, rng, 20000)
    near = np.nonzero(xy[:, 0] < 0.3)[0][:1500]
    for k in near:
        e, hops = om.locate_walk(int(rng.choice(right)), xy[k, 0], xy[k, 1])
        assert e == om.locate_brute(xy[k, 0], xy[k, 1]) and hops <= 64, (k, xy[k])
    # points just beyond the walls near the seam, on both sides of it
    for _ in range(1500):
        x = float(np.float32(rng.choice([rng.uniform(0.0, 0.05), rng.uniform(L - 0.05, L)])))
        top = rng.random() < 0.5
        y = float(np.float32(2.0 + rng.uniform(1e-6, 2e-3) if top else -rng.uniform(1e-6, 2e-3)))
        start = int(rng.choice(right if x < 0.5 else left))
        e, hops = om.locate_walk(start, min(x, np.nextafter(np.float32(L), np.float32(0))), y)
        assert e == -1 and hops <= 64, (x, y, start, e, hops)


def test_an_image_that_rounds_back_onto_the_point_steps_one_ulp_inward():
    """FP32 points just beyond a sloped wall edge of the bump whose FP64 mirror image rounds back
    onto the point itself (found by search): the reflecting walk moves each one FP32 step along
    the edge's inward normal (-d_y, d_x), with one mirroring, and ends at the owner of the result."""
    mesh = wl.bump_channel_mesh(250, 100, 1006054905)
    om = oracle.OracleMesh(mesh)
    xy = mesh.node_xy
    f32 = np.float32
    rng = np.random.default_rng(3)
    walls = [(e, k) for e in range(mesh.n_tri) for k in range(3)
             if mesh.edge_tag[e, k] == 1 and xy[mesh.tri[e, k], 1] < 0.5]
    found = []
    for e, k in walls[::7][:400]:
        a, b = xy[mesh.tri[e, k]], xy[mesh.tri[e, (k + 1) % 3]]
        d = b - a
        if abs(d[1]) < 1e-4:
            continue
        n_in = np.array([-d[1], d[0]]) / np.hypot(*d)
        for t in rng.uniform(0.2, 0.8, 30):
            q = a + t * d - 1e-9 * n_in
            px, py = f32(q[0]), f32(q[1])
            tt = ((float(px) - a[0]) * d[0] + (float(py) - a[1]) * d[1]) / (d[0] * d[0] + d[1] * d[1])
            mx, my = f32(2.0 * (a[0] + tt * d[0]) - float(px)), f32(2.0 * (a[1] + tt * d[1]) - float(py))
            beyond = (float(px) - a[0]) * n_in[0] + (float(py) - a[1]) * n_in[1] < 0.0
            if mx == px and my == py and beyond:
                found.append((e, d, px, py))
        if len(found) >= 5:
            break
    assert len(found) >= 3
    for e, d, px, py in found:
        assert om.locate_brute(float(px), float(py)) == -1           # the point is outside
        r, x, y, _, _, _, hops, nref = om.locate_walk_reflect(e, px, py)
        want_x = np.nextafter(px, f32(np.inf) if d[1] < 0 else f32(-np.inf), dtype=np.float32)
        want_y = np.nextafter(py, f32(np.inf) if d[0] > 0 else f32(-np.inf), dtype=np.float32)
        assert nref == 1 and f32(x) == want_x and f32(y) == want_y
        assert r == om.locate_brute(x, y) >= 0


def test_an_image_that_wraps_onto_x1_belongs_to_x0():
    """The corner of the seam and the flat top wall of a curved-wall channel, computed by hand: the
    point (2^-149, 2 + 2^-22) lies one FP32 ulp above the wall and one denormal step right of the
    seam. Its mirror image across y = 2 is (-2^-149, 2 - 2^-22); the wrap adds the period, and
    -2^-149 + L rounds to L = x1 exactly, outside the half-open frame [x0, x1), so the image is put
    at x0 = 0 (periodic wrap: a result equal to x1 becomes x0). The walk ends, after one mirroring,
    at the owner of (0, 2 - 2^-22); without the rule it walked to the hop cap."""
    mesh = wl.bump_channel_mesh(25, 20, 7)
    om = oracle.OracleMesh(mesh)
    f32 = np.float32
    px, py = f32(2.0 ** -149), f32(2.0 + 2.0 ** -22)
    want_y = f32(2.0 - 2.0 ** -22)
    owner = om.locate_brute(0.0, float(want_y))
    assert owner >= 0 and om.locate_brute(float(px), float(py)) == -1
    # from the owner, and from every element that touches the corner node (0, 2)
    corner = int(np.nonzero((mesh.node_xy[:, 0] == 0.0) & (mesh.node_xy[:, 1] == 2.0))[0][0])
    starts = sorted({owner} | {int(e) for e in np.nonzero((mesh.tri == corner).any(axis=1))[0]})
    for s in starts:
        r, x, y, u, v, w, hops, nref = om.locate_walk_reflect(s, px, py, 0.5, 0.25, 0.125)
        assert nref == 1 and x == 0.0 and f32(y) == want_y, (s, r, x, y, nref)
        assert r == owner and (u, v, w) == (-0.5, -0.25, -0.125)


def lshape_mesh():
    """A hand-built L-shaped domain, [0, 2] x [0, 1] joined to [0, 1] x [1, 2], with its reentrant
    corner at (1, 1); every boundary edge is a wall. Nodes 0..7 are (0,0) (1,0) (2,0) (0,1) (1,1)
    (2,1) (0,2) (1,2); elements, counter-clockwise (edge k runs from vertex k to vertex k + 1):
    T0 = (0,1,4) and T1 = (0,4,3) in the lower-left square, T2 = (1,2,5) and T3 = (1,5,4) in the
    lower-right one, T4 = (3,4,7) and T5 = (3,7,6) in the upper-left one. The walls at y = 1
    (x in [1, 2]) and x = 1 (y in [1, 2]) are off the sides of the bounding box."""
    xy = np.array([(0, 0), (1, 0), (2, 0), (0, 1), (1, 1), (2, 1), (0, 2), (1, 2)], dtype=np.float64)
    tri = np.array([(0, 1, 4), (0, 4, 3), (1, 2, 5), (1, 5, 4), (3, 4, 7), (3, 7, 6)], dtype=np.int32)
    count = {}
    for t in tri:
        for k in range(3):
            key = tuple(sorted((int(t[k]), int(t[(k + 1) % 3]))))
            count[key] = count.get(key, 0) + 1
    tag = np.zeros((len(tri), 3), dtype=np.int32)
    for e, t in enumerate(tri):
        for k in range(3):
            if count[tuple(sorted((int(t[k]), int(t[(k + 1) % 3]))))] == 1:
                tag[e, k] = wl.EDGE_WALL
    return wl.Mesh(xy, tri, tag, 0.0, (0.0, 2.0, 0.0, 2.0), "lshape", 0, 0)


# Hand-worked moves on the L-shaped mesh, all in exact binary fractions. Each row: start element,
# start (x, y), velocity (u, v), and after a move of dt = 0.5 the owner, the final (x, y) and
# (u, v), the hops and the mirrorings.
#  * From T2 to (0.8125, 1.3125), round the reentrant corner. In T2 only lambda_1 (of node 2,
#    across the diagonal) is negative: -1.5 -> T3. In T3 (nodes 1, 5, 4) lambda_0 = 1 - y =
#    -0.3125 lies across the wall y = 1 and lambda_1 = x - 1 = -0.1875 across the interior edge
#    x = 1: the walk takes the interior exit although the wall's lambda is the more negative one
#    -> T0, where lambda_1 = x - y = -0.5 -> T1, where lambda_0 = 1 - y = -0.3125 -> T4, where
#    lambda = (1 - x, x + 1 - y, y - 1) = (0.1875, 0.5, 0.3125): found after 4 hops, no mirroring.
#    A walk that always left by the most negative lambda would have mirrored at y = 1 and ended
#    in T0 at (0.8125, 0.6875).
#  * From T3 into the notch at (1.5, 1.25): in T3 only the wall's lambda_0 = -0.25 is negative, so
#    the position is mirrored across y = 1 to (1.5, 0.75) and the velocity reversed; T3 owns it.
#  * From T4 into the notch at (1.25, 1.5): only the wall x = 1 is crossed: mirrored to
#    (0.75, 1.5), velocity reversed, owned by T4.
LSHAPE_MOVES = [
    (2, (1.8125, 0.5), (-2.0, 1.625), 4, (0.8125, 1.3125), (-2.0, 1.625), 4, 0),
    (3, (1.25, 0.75), (0.5, 1.0), 3, (1.5, 0.75), (-0.5, -1.0), 0, 1),
    (4, (0.75, 1.5), (1.0, 0.0), 4, (0.75, 1.5), (-1.0, 0.0), 0, 1),
]


def lshape_state():
    """The start states of the hand-worked moves (pid = row)."""
    n = len(LSHAPE_MOVES)
    return wl.State(np.array([m[1][0] for m in LSHAPE_MOVES], np.float32),
                    np.array([m[1][1] for m in LSHAPE_MOVES], np.float32),
                    np.array([m[2][0] for m in LSHAPE_MOVES], np.float32),
                    np.array([m[2][1] for m in LSHAPE_MOVES], np.float32),
                    np.zeros(n, np.float32), np.ones(n, np.float32), np.zeros((1, n), np.float32),
                    np.array([m[0] for m in LSHAPE_MOVES], np.int32), np.arange(n, dtype=np.uint32))


def test_lshape_mesh_is_as_drawn():
    mesh = lshape_mesh()
    om = oracle.OracleMesh(mesh)
    assert om.edge_walls
    nbr = om.neighbors()
    assert sorted(n for n in nbr[3] if n >= 0) == [0, 2]          # T3: the diagonal and x = 1
    assert sorted(n for n in nbr[1] if n >= 0) == [0, 4]          # T1: the diagonal and y = 1
    for e, (x, y), *_ in LSHAPE_MOVES:
        assert om.locate_brute(x, y) == e


@pytest.mark.parametrize("row", range(len(LSHAPE_MOVES)))
def test_hand_worked_walks_on_the_lshape(row):
    """The walk with mirroring reproduces the hand-worked moves: the owner, the position, the
    velocity, the hops and the mirrorings."""
    om = oracle.OracleMesh(lshape_mesh())
    e0, (x, y), (u, v), e1, (x1, y1), (u1, v1), hops, mirrors = LSHAPE_MOVES[row]
    qx, qy = x + 0.5 * u, y + 0.5 * v
    e, px, py, U, V, W, h, n = om.locate_walk_reflect(e0, qx, qy, u, v, 0.0)
    assert (e, px, py, U, V, h, n) == (e1, x1, y1, u1, v1, hops, mirrors)
    assert om.locate_brute(px, py) == e1


def test_hand_worked_moves_through_a_step_on_the_lshape():
    """The same moves made by one oracle step with no diffusion and still fields (U, positions
    and the walk are then exact): every particle ends at its hand-worked owner and state."""
    mesh = lshape_mesh()
    om = oracle.OracleMesh(mesh)
    st = lshape_state()
    p = oracle.make_params(nu=1e-30, dt=0.5, seed=31, ns=1)
    res, oelem, aux, lost = oracle.pdf_step(om, p, _still_fields(mesh, 1), st, 0, locate_mode=2)
    assert lost == 0
    for k, (_, _, _, e1, (x1, y1), (u1, v1), _, mirrors) in enumerate(LSHAPE_MOVES):
        assert (oelem[k], res["x"][k], res["y"][k], res["u"][k], res["v"][k]) == (e1, x1, y1, u1, v1)
        assert aux[k, 2] == mirrors
