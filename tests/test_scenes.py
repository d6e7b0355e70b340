"""The seeded input generators: every pose is a finite rigid motion, and each
pair sits at the depth its recipe asked for, checked by brute force over all
vertices and pieces (the deepest vertex-in-piece max-plane depth; positive =
penetration, negative = gap).  Parity tests rest on these scenes, so a broken
placement (a pair that no vertex line reaches) must fail here."""
import numpy as np
import pytest

from paper_2604_17538_b300 import scenes

# float32 geometry and poses of magnitude ~1: a depth computed from them
# differs from the float64 placement by a few float32 ulps of the coordinates
DEPTH_TOL = 2e-5


def _deepest(geom, bF, bS, PF, PS):
    RF, tF = scenes.unpack_pose(PF[None])
    RS, tS = scenes.unpack_pose(PS[None])
    best = -np.inf
    for pf in geom.pieces_of(bF):
        V = geom.piece(pf)[0].astype(np.float64)
        xs = ((V @ RF[0].T + tF[0]) - tS[0]) @ RS[0]
        for ps in geom.pieces_of(bS):
            P = geom.piece(ps)[1].astype(np.float64)
            m = (xs @ P[:, :3].T + P[:, 3]).max(1)
            best = max(best, -m.min())
    return best


def _check_scene(sc, n_check):
    assert np.isfinite(sc.pose_a).all() and np.isfinite(sc.pose_b).all()
    for P in (sc.pose_a, sc.pose_b):
        R, _ = scenes.unpack_pose(P)
        assert np.abs(R @ R.transpose(0, 2, 1) - np.eye(3)).max() < 1e-6
        assert np.all(np.linalg.det(R) > 0)
    target = sc.meta["target_depth"]
    sep = sc.meta["separated"]
    assert np.all((target < 0) == sep)
    for i in range(min(n_check, sc.n_pairs)):
        a, b = int(sc.pair_a[i]), int(sc.pair_b[i])
        d = max(_deepest(sc.geom, a, b, sc.pose_a[i], sc.pose_b[i]),
                _deepest(sc.geom, b, a, sc.pose_b[i], sc.pose_a[i]))
        assert abs(d - target[i]) < DEPTH_TOL, (i, d, target[i])


def test_hull_env_scene_places_every_pair_at_its_depth():
    sc = scenes.hull_env_scene(seed=2, n_envs=48)
    npb = np.diff(sc.geom.body_piece_off)
    assert np.all(npb == 8)
    nv = np.diff(sc.geom.piece_v_off)
    assert nv.min() >= 4 and nv.max() <= 64
    _check_scene(sc, 48)


@pytest.mark.parametrize("seed,n_pairs,pool", [(4, 96, 96), (9, 160, 48)])
def test_uneven_scene_places_every_pair_at_its_depth(seed, n_pairs, pool):
    # seed 9 (pool 48) has pairs whose vertex lines along the placement
    # direction miss the other body; they must be re-aimed, not left at inf
    sc = scenes.uneven_scene(seed=seed, n_pairs=n_pairs, pool_bodies=pool)
    npb = np.diff(sc.geom.body_piece_off)
    assert npb.min() >= 1 and npb.max() <= 64
    _check_scene(sc, n_pairs)


def test_cube_pair_scene_depth_is_the_box_depth():
    sc = scenes.cube_pair_scene(seed=1, n_poses=16)
    assert np.isfinite(sc.pose_a).all() and np.isfinite(sc.pose_b).all()
    RA, tA = scenes.unpack_pose(sc.pose_a)
    RB, tB = scenes.unpack_pose(sc.pose_b)
    for i in range(sc.n_pairs):
        d = scenes.box_penetration_depth(RA[i], tA[i], np.full(3, 0.5), RB[i], tB[i],
                                         np.full(3, 0.5))
        assert abs(d - sc.meta["depth"][i]) < DEPTH_TOL, (i, d, sc.meta["depth"][i])
