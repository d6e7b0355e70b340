"""Pins of the oracle's forward variants: the body-level smooth union of a
body's piece SDFs (Sec. 3.1, Eq. soft_union) and the isosurface projection of
contact points (Sec. 4.1).  Each pin is a bound, limit or closed form that a
dropped term, a wrong sign or a transposed operand would break."""
import numpy as np
import pytest

from paper_2604_17538_b300 import scenes

TAU = 5e-3


@pytest.fixture(scope="module")
def hull_body():
    return scenes.hull_env_scene(seed=5, n_envs=1, workers=1)


def test_union_lies_within_the_lse_bounds_of_the_smallest_piece_sdf(oracle_lib, hull_body):
    """min_s phi_s - tau log N <= phi_union <= min_s phi_s at every point, with
    phi_s each piece's own SDF (Sec. 3 smooth intersection)."""
    g = hull_body.geom
    rng = np.random.default_rng(0)
    body = 0
    pieces = list(g.pieces_of(body))
    for x in rng.normal(0.0, 0.15, size=(200, 3)):
        phis = [oracle_lib.sdf(g.piece(p)[1], x, TAU)[0] for p in pieces]
        phi, _ = oracle_lib.body_sdf(g, body, x, TAU)
        lo, hi = min(phis) - TAU * np.log(len(pieces)), min(phis)
        assert lo - 1e-12 <= phi <= hi + 1e-12


def test_union_gradient_is_its_derivative_and_a_softmin_mix(oracle_lib, hull_body):
    """Central differences of phi_union match its gradient, and the gradient
    is a convex combination of the pieces' gradients (norm <= 1)."""
    g = hull_body.geom
    rng = np.random.default_rng(1)
    h = 1e-6
    for x in rng.normal(0.0, 0.12, size=(40, 3)):
        _, gr = oracle_lib.body_sdf(g, 0, x, TAU)
        fd = np.array([(oracle_lib.body_sdf(g, 0, x + h * e, TAU)[0] -
                        oracle_lib.body_sdf(g, 0, x - h * e, TAU)[0]) / (2 * h)
                       for e in np.eye(3)])
        assert np.allclose(gr, fd, atol=1e-6)
        assert np.linalg.norm(gr) <= 1 + 1e-12


def test_union_of_far_apart_pieces_is_the_nearest_piece(oracle_lib):
    """Two unit cubes 10 apart: near one cube the other's term is e^{-10/tau},
    so the union equals that cube's own SDF to rounding."""
    geom = scenes.geometry_from_bodies([[scenes.unit_cube_piece(0.5),
                                         scenes.unit_cube_piece(0.5, center=(10.0, 0, 0))]])
    for x in ([0.1, 0.2, 0.3], [0.6, -0.1, 0.0], [9.7, 0.4, -0.45]):
        x = np.array(x)
        near = 0 if x[0] < 5 else 1
        phi_s, g_s = oracle_lib.sdf(geom.piece(near)[1], x, TAU)
        phi, gr = oracle_lib.body_sdf(geom, 0, x, TAU)
        assert abs(phi - phi_s) < 1e-12 and np.allclose(gr, g_s, atol=1e-12)


def test_union_forward_of_single_piece_bodies_is_the_per_piece_forward(oracle_lib):
    """With one piece per body the union of one SDF is that SDF, and a group's
    contacts are the same list: the outputs equal the default path's."""
    sc = scenes.cube_pair_scene(seed=1, n_poses=16)
    y0 = oracle_lib.forward(sc)
    y1 = oracle_lib.forward(sc, oracle_lib.params(flags=oracle_lib.FLAG_BODY_UNION))
    assert np.allclose(y1, y0, atol=1e-13, rtol=0)
    assert np.any(y0[:, 1] > 0)


def test_union_forward_is_invariant_and_symmetric(oracle_lib):
    """A common rigid motion leaves depths and weights unchanged and moves
    points and normals with it; swapping the bodies swaps the group blocks."""
    sc = scenes.hull_env_scene(seed=2, n_envs=4, workers=1)
    prm = oracle_lib.params(flags=oracle_lib.FLAG_BODY_UNION)
    y = oracle_lib.forward(sc, prm)
    assert np.any(y[:, 1] > 0)
    rng = np.random.default_rng(3)
    R = scenes.random_rotations(rng, 1)[0]
    t = rng.normal(size=3)
    moved = sc.take(np.arange(sc.n_pairs))
    for P in ("pose_a", "pose_b"):
        Rb, tb = scenes.unpack_pose(getattr(sc, P).astype(np.float64))
        setattr(moved, P, scenes.pack_pose(R[None] @ Rb, tb @ R.T + t))
    ym = oracle_lib.forward(moved, prm)
    # float32 storage of the moved poses limits agreement to ~1e-6
    act = y[:, 1] > 0
    assert np.abs(ym[:, 0] - y[:, 0]).max() < 2e-5
    assert np.abs(ym[:, 1] - y[:, 1]).max() < 2e-4
    assert np.abs(ym[act, 2:5] - (y[act, 2:5] @ R.T + t)).max() < 2e-5
    assert np.abs(ym[act, 5:8] - y[act, 5:8] @ R.T).max() < 2e-4
    sw = scenes.Scene(sc.geom, sc.pair_b, sc.pair_a, sc.pose_b, sc.pose_a)
    ys = oracle_lib.forward(sw, prm)
    off, offs = sc.group_offsets(), sw.group_offsets()
    npb = np.diff(sc.geom.body_piece_off)
    for i in range(sc.n_pairs):
        na, nb = npb[sc.pair_a[i]], npb[sc.pair_b[i]]
        blk = y[off[i]:off[i + 1]]
        sblk = ys[offs[i]:offs[i + 1]]
        assert np.allclose(sblk[:nb], blk[na:], atol=1e-12)
        assert np.allclose(sblk[nb:], blk[:na], atol=1e-12)


def test_projection_moves_contacts_onto_a_face_plane(oracle_lib):
    """Stacked cubes (Sec. 5.2): a vertex of B at depth delta under A's top
    face, away from A's other faces, has phi = -delta and grad phi = +z to
    rounding, so its projection p - phi grad phi lies on the face plane."""
    delta = 2.0 ** -8               # sizes exact in the float32 poses and vertices
    A = [scenes.unit_cube_piece(0.5)]
    B = [scenes.unit_cube_piece(0.125)]
    I = np.eye(3)[None]
    sc = scenes.Scene(scenes.geometry_from_bodies([A, B]), np.zeros(1, np.int64),
                      np.ones(1, np.int64), scenes.pack_pose(I, np.zeros((1, 3))),
                      scenes.pack_pose(I, np.array([[0.0, 0.0, 0.625 - delta]])))
    rows = oracle_lib.pair_contacts(sc, 0, oracle_lib.params(flags=oracle_lib.FLAG_PROJECT))
    base = oracle_lib.pair_contacts(sc, 0)
    deep = (rows[:, 0] == 1) & (rows[:, 2] > 0) & (np.abs(rows[:, 1] + delta) < 1e-9)
    assert deep.sum() >= 4                          # B's bottom corners and edges
    assert np.allclose(rows[deep, 6], 0.5, atol=1e-12)
    # depth, weight and normal are those of the unprojected contact
    assert np.array_equal(rows[:, 1:4], base[:, 1:4]) and np.array_equal(rows[:, 7:], base[:, 7:])
    assert np.allclose(base[deep, 6], 0.5 - delta, atol=1e-12)


def test_projection_of_a_single_half_space_lands_on_it(oracle_lib):
    """A piece with one face plane (a half-space, Sec. 3 phi = n.x + h) is
    linear with unit gradient: every projected contact point has phi = 0."""
    n = np.array([0.3, -0.5, 0.8])
    n /= np.linalg.norm(n)
    half = (np.zeros((1, 3), np.float32), np.array([[*n, 0.02]], np.float32),
            np.zeros((0, 2), np.int32))
    tri = np.random.default_rng(2).normal(0, 0.01, size=(4, 3))
    probe = scenes.hull_piece(tri)
    geom = scenes.geometry_from_bodies([[half], [probe]])
    I = np.eye(3)[None]
    sc = scenes.Scene(geom, np.zeros(1, np.int64), np.ones(1, np.int64),
                      scenes.pack_pose(I, np.zeros((1, 3))), scenes.pack_pose(I, np.zeros((1, 3))))
    rows = oracle_lib.pair_contacts(sc, 0, oracle_lib.params(flags=oracle_lib.FLAG_PROJECT))
    side_b = rows[rows[:, 0] == 1]                  # B's features against the half-space
    assert len(side_b) > 0
    plane = np.asarray(geom.planes[0], np.float64)
    assert np.allclose(side_b[:, 4:7] @ plane[:3] + plane[3], 0.0, atol=1e-9)


def test_union_is_the_softmin_of_its_pieces_definition(oracle_lib, hull_body):
    """Eq. soft_union evaluated here from its definition: every piece SDF as
    tau * logsumexp(plane values / tau) and the union as
    -tau * logsumexp(-phi_s / tau) over the pieces (scipy), its gradient the
    softmin-weighted mix of the pieces' softmax-weighted plane normals."""
    from scipy.special import logsumexp, softmax
    g = hull_body.geom
    rng = np.random.default_rng(4)
    body = 0
    planes = [np.asarray(g.piece(p)[1], np.float64) for p in g.pieces_of(body)]
    for x in rng.normal(0.0, 0.15, size=(100, 3)):
        vals = [(P[:, :3] @ x + P[:, 3]) / TAU for P in planes]
        phis = np.array([TAU * logsumexp(v) for v in vals])
        grads = np.array([softmax(v) @ P[:, :3] for v, P in zip(vals, planes)])
        ref = -TAU * logsumexp(-phis / TAU)
        ref_g = softmax(-phis / TAU) @ grads
        phi, grad = oracle_lib.body_sdf(g, body, x, TAU)
        assert abs(phi - ref) < 1e-12 and np.abs(grad - ref_g).max() < 1e-10


def test_projection_moves_every_contact_by_its_depth_along_its_normal(oracle_lib):
    """On random hulls at the default softness every projected contact point
    is the unprojected one moved by -phi along the contact normal (Sec. 4.1,
    p - phi(p) n(p), here in world frame, where the normal is the SDF body's
    rotated normal), and nothing else about the contact changes."""
    sc = scenes.hull_env_scene(seed=6, n_envs=3, workers=1)
    for i in range(sc.n_pairs):
        rows = oracle_lib.pair_contacts(sc, i, oracle_lib.params(flags=oracle_lib.FLAG_PROJECT))
        base = oracle_lib.pair_contacts(sc, i)
        assert np.array_equal(rows[:, :4], base[:, :4]) and np.array_equal(rows[:, 7:], base[:, 7:])
        moved = base[:, 4:7] - base[:, 1:2] * base[:, 7:10]
        assert np.abs(rows[:, 4:7] - moved).max() < 1e-12
