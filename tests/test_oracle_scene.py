"""Pins of the oracle's whole pipeline (Sec. 4: gate, narrow phase, blending)
against closed forms, hard limits and invariants of the geometry."""
import json
import os

import numpy as np
import pytest

from geom_util import cyrus_beck, rot
from paper_2604_17538_b300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _scene(bodies, RA, tA, RB, tB):
    geom = scenes.geometry_from_bodies(bodies)
    n = len(RA)
    return scenes.Scene(geom, np.zeros(n, np.int64), np.ones(n, np.int64),
                        scenes.pack_pose(RA, tA), scenes.pack_pose(RB, tB))


def _stacked(half_b, delta):
    """Unit cube A at the origin; cube B (half size half_b) resting on A's top
    face, axis aligned, penetrating by delta (Sec. 5.2 stacked boxes)."""
    A = [scenes.unit_cube_piece(0.5)]
    B = [scenes.unit_cube_piece(half_b)]
    I = np.eye(3)[None]
    return _scene([A, B], I, np.zeros((1, 3)), I, np.array([[0.0, 0.0, 0.5 + half_b - delta]]))


def test_cube_on_cube_hard_limit(oracle_lib):
    """All softness -> 0: the blended contact of B's piece is the 4-point
    manifold of its bottom face: 4 corners + 4 bottom-edge midpoints at depth
    -delta, centroid at the face centre, normal +z out of A, weight 1; A's
    features are all beyond d_max from B, so A's group is empty."""
    with open(os.path.join(GOLDEN, "stacked_cubes_hard_limit.json")) as f:
        gold = json.load(f)
    for case in gold["cases"]:
        sc = _stacked(case["half_b"], case["delta"])
        prm = oracle_lib.params(**gold["params"])
        y = oracle_lib.forward(sc, prm)
        assert np.allclose(y[0], case["group_A"], atol=1e-9), y[0]
        assert np.allclose(y[1], case["group_B"], atol=1e-7), y[1]


def test_cube_on_cube_default_softness_symmetry(oracle_lib):
    """At the default softness the 4-fold symmetry of the stacked scene about
    z still fixes p_x = p_y = 0 and n = +z; the depth lies between the
    deepest contact (-delta) and d_max, and the weight in (0, 1]."""
    for half_b, delta in ((0.25, 0.01), (0.5, 0.02), (0.5, 0.0)):
        sc = _stacked(half_b, delta)
        y = oracle_lib.forward(sc)
        g = y[1]
        assert abs(g[2]) < 1e-12 and abs(g[3]) < 1e-12
        assert np.allclose(g[5:8], [0, 0, 1], atol=1e-12)
        assert -delta - 1e-9 <= g[0] <= 0.01
        assert 0 < g[1] <= 1
        assert abs(g[4] - (0.5 - delta)) < 0.5 * delta + 0.02


def test_separated_bodies_are_empty_with_zero_gradient(oracle_lib):
    sc = scenes.hull_env_scene(seed=21, n_envs=4, workers=1)
    # move B far away along x: every contact is beyond d_max
    sc.pose_b[:, 9] += 5.0
    y = oracle_lib.forward(sc)
    assert np.all(y[:, 0] == 0.01) and np.all(y[:, 1:] == 0.0)
    yb = np.random.default_rng(0).normal(size=y.shape)
    g, _ = oracle_lib.gradient(sc, yb)
    assert np.all(g == 0.0)


@pytest.fixture(scope="module")
def small_hulls():
    return scenes.hull_env_scene(seed=2, n_envs=6, workers=1)


def test_common_rigid_motion_invariance(oracle_lib, small_hulls):
    sc = small_hulls
    y = oracle_lib.forward(sc)
    rng = np.random.default_rng(3)
    Rw = scenes.random_rotations(rng, 1)[0]
    tw = rng.uniform(-1, 1, 3)
    moved = sc.take(np.arange(sc.n_pairs))
    for P in (moved.pose_a, moved.pose_b):
        R, t = scenes.unpack_pose(P)
        P[:] = scenes.pack_pose(Rw @ R, t @ Rw.T + tw)
    y2 = oracle_lib.forward(moved)
    # float32 storage of the moved poses limits agreement to ~1e-6
    act = y[:, 1] > 0
    assert act.sum() > 5
    assert np.abs(y2[:, 0] - y[:, 0]).max() < 2e-5
    assert np.abs(y2[:, 1] - y[:, 1]).max() < 2e-4
    assert np.abs(y2[act, 2:5] - (y[act, 2:5] @ Rw.T + tw)).max() < 2e-5
    assert np.abs(y2[act, 5:8] - y[act, 5:8] @ Rw.T).max() < 2e-4


def test_body_swap_permutes_groups(oracle_lib, small_hulls):
    sc = small_hulls
    y = oracle_lib.forward(sc)
    sw = scenes.Scene(sc.geom, sc.pair_b, sc.pair_a, sc.pose_b, sc.pose_a)
    y2 = oracle_lib.forward(sw)
    off, off2 = sc.group_offsets(), sw.group_offsets()
    npb = np.diff(sc.geom.body_piece_off)
    for i in range(sc.n_pairs):
        na, nb = npb[sc.pair_a[i]], npb[sc.pair_b[i]]
        blk = y[off[i]:off[i + 1]]
        blk2 = y2[off2[i]:off2[i + 1]]
        assert np.array_equal(blk[:na], blk2[nb:])
        assert np.array_equal(blk[na:], blk2[:nb])


def test_blend_is_a_convex_combination(oracle_lib, small_hulls):
    """Sec. 4.4: sum w = 1, so the blended depth lies within the active
    contacts' depths, the point in their bounding box, a in (0, 1], |n| = 1."""
    sc = small_hulls
    y = oracle_lib.forward(sc)
    off = sc.group_offsets()
    seen = 0
    for i in range(sc.n_pairs):
        rows = oracle_lib.pair_contacts(sc, i)
        for g in range(off[i + 1] - off[i]):
            r = rows[(rows[:, 0] == g) & (rows[:, 2] > 0)]
            yy = y[off[i] + g]
            if len(r) == 0:
                assert yy[0] == 0.01 and np.all(yy[1:] == 0)
                continue
            seen += 1
            assert r[:, 3].min() - 1e-12 <= yy[0] <= r[:, 3].max() + 1e-12
            assert r[:, 2].min() - 1e-12 <= yy[1] <= r[:, 2].max() + 1e-12
            assert np.all(yy[2:5] >= r[:, 4:7].min(0) - 1e-12)
            assert np.all(yy[2:5] <= r[:, 4:7].max(0) + 1e-12)
            assert abs(np.linalg.norm(yy[5:8]) - 1) < 1e-12
    assert seen > 5


def test_blend_temperature_limit_is_argmax(oracle_lib, small_hulls):
    """tau_blend -> 0: the blend selects the deepest active contact."""
    sc = small_hulls
    prm = oracle_lib.params(tau_blend=1e-9)
    y = oracle_lib.forward(sc, prm)
    off = sc.group_offsets()
    for i in range(sc.n_pairs):
        rows = oracle_lib.pair_contacts(sc, i, prm)
        for g in range(off[i + 1] - off[i]):
            r = rows[(rows[:, 0] == g) & (rows[:, 2] > 0)]
            if len(r) == 0:
                continue
            k = np.argmin(r[:, 3])
            srt = np.sort(r[:, 3])
            if len(srt) > 1 and srt[1] - srt[0] < 1e-6:
                continue   # near tie
            yy = y[off[i] + g]
            assert abs(yy[0] - r[k, 3]) < 1e-9
            assert np.abs(yy[2:5] - r[k, 4:7]).max() < 1e-9


def _tetra_planes(c, s=0.05):
    n = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float) / np.sqrt(3)
    return np.concatenate([n, (-(n @ c) - s)[:, None]], 1)


def test_single_feature_group_reduces_to_its_contact(oracle_lib):
    """A piece with one vertex and no edges against one cube has exactly one
    contact: its group output is that contact (d_c, f, p, n/|n|)."""
    cube = scenes.unit_cube_piece(0.5)
    v = np.array([[0.1, -0.2, 0.5 - 0.004]])      # just below the top face
    single = (v.astype(np.float32), _tetra_planes(v[0]).astype(np.float32),
              np.zeros((0, 2), np.int32))
    I = np.eye(3)[None]
    R = rot([0.3, 1.0, 0.2], 0.7)[None]
    sc = _scene([[cube], [single]], R, np.array([[0.2, 0.1, -0.3]]), R, np.array([[0.2, 0.1, -0.3]]))
    y = oracle_lib.forward(sc)
    rows = oracle_lib.pair_contacts(sc, 0)
    r = rows[rows[:, 0] == 1]
    assert len(r) == 1 and r[0, 2] > 0
    g = y[1]
    assert abs(g[0] - r[0, 3]) < 1e-15 and abs(g[1] - r[0, 2]) < 1e-15
    assert np.abs(g[2:5] - r[0, 4:7]).max() < 1e-15
    n = r[0, 7:10] / np.linalg.norm(r[0, 7:10])
    assert np.abs(g[5:8] - n).max() < 1e-12
    # the contact is the vertex in world frame, its normal A's rotated top normal
    xw = R[0] @ v[0] + [0.2, 0.1, -0.3]
    assert np.abs(g[2:5] - xw).max() < 1e-6
    assert np.abs(g[5:8] - R[0] @ [0, 0, 1]).max() < 1e-6
    assert abs(r[0, 1] - (-0.004)) < 1e-6


def _hard_limit_contacts(sc, i):
    """Per group of pair i, the (phi, world point) of every contact in the
    hard limit, by brute force: a vertex's phi is its largest plane value in
    each SDF piece; an edge's contact is the midpoint of its Cyrus-Beck chord
    through the SDF piece (Sec. 4.2 traces tend to the chord's ends), with
    that point's largest plane value.  Groups: first A's pieces against B,
    then B's against A."""
    g = sc.geom
    RA, tA = scenes.unpack_pose(sc.pose_a[i:i + 1])
    RB, tB = scenes.unpack_pose(sc.pose_b[i:i + 1])
    sides = ((sc.pair_a[i], RA[0], tA[0], sc.pair_b[i], RB[0], tB[0]),
             (sc.pair_b[i], RB[0], tB[0], sc.pair_a[i], RA[0], tA[0]))
    groups = []
    for bF, RF, tF, bS, RS, tS in sides:
        for fp in range(g.body_piece_off[bF], g.body_piece_off[bF + 1]):
            V = g.verts[g.piece_v_off[fp]:g.piece_v_off[fp + 1]].astype(np.float64)
            E = g.edges[g.piece_e_off[fp]:g.piece_e_off[fp + 1]]
            X = (V @ RF.T + tF - tS) @ RS            # feature vertices in S's frame
            rows = []
            for sp in range(g.body_piece_off[bS], g.body_piece_off[bS + 1]):
                P = g.planes[g.piece_f_off[sp]:g.piece_f_off[sp + 1]].astype(np.float64)
                for x in X:
                    rows.append(((P[:, :3] @ x + P[:, 3]).max(), x))
                for i0, i1 in E:
                    iv = cyrus_beck(X[i0], X[i1], P)
                    if iv is not None:
                        m = X[i0] + 0.5 * (iv[0] + iv[1]) * (X[i1] - X[i0])
                        rows.append(((P[:, :3] @ m + P[:, 3]).max(), m))
            groups.append([(phi, RS @ x + tS) for phi, x in rows])
    return groups


def test_hard_limit_depth_is_the_deepest_brute_force_contact(oracle_lib):
    """Random hulls with every softness -> 0 and a long trace: a group whose
    deepest contact lies clearly inside (phi < -1e-3, so its gate is 1)
    returns that contact's depth, and its point when the minimum is unique."""
    sc = scenes.hull_env_scene(seed=5, n_envs=16, workers=1)
    prm = oracle_lib.params(tau_sdf=1e-8, tau_trace=1e-8, tau_clip=1e-8, tau_blend=1e-8,
                            trace_iters=400)
    y = oracle_lib.forward(sc, prm)
    off = sc.group_offsets()
    checked = points = 0
    for i in range(sc.n_pairs):
        for k, rows in enumerate(_hard_limit_contacts(sc, i)):
            if not rows:
                continue
            phis = np.array([r[0] for r in rows])
            j = int(np.argmin(phis))
            if phis[j] >= -1e-3:
                continue
            yy = y[off[i] + k]
            assert abs(yy[0] - phis[j]) < 1e-5, (i, k, yy[0], phis[j])
            assert abs(yy[1] - 1.0) < 1e-6
            checked += 1
            rest = np.delete(phis, j)
            if len(rest) == 0 or rest.min() - phis[j] > 1e-4:
                assert np.abs(yy[2:5] - rows[j][1]).max() < 1e-5, (i, k)
                points += 1
    assert checked >= 10 and points >= 5, (checked, points)
