"""Pins of the oracle's ungated blend (FLAG_UNGATED): the literal reading of
Sec. 4.4's "softmax on {d_c}", a softmax of -d_c / tau_blend over every
contact of a group, the contacts with f = 0 (mollified depth exactly d_max)
included.  It sits beside the gated blend for comparison only; the GPU path
computes the gated one.

Each pin follows from the definition of a softmax average, not from the
oracle's code: equal logits give the plain mean, an infinite temperature the
plain mean, a zero temperature the deepest contact, and a group whose every
contact has f = 1 weighs its contacts exactly as the gated blend does."""
import numpy as np
import pytest

from paper_2604_17538_b300 import scenes


def _ungated(oracle_lib, **kw):
    return oracle_lib.params(flags=oracle_lib.FLAG_UNGATED, **kw)


def _groups(rows, g):
    return rows[rows[:, 0] == g]


def _unit(v):
    n = np.linalg.norm(v)
    return v / n if n > 0 else v


@pytest.fixture(scope="module")
def small_hulls():
    return scenes.hull_env_scene(seed=2, n_envs=6, workers=1)


def test_separated_bodies_average_every_contact_uniformly(oracle_lib):
    """Every contact beyond d_max: every logit is -d_max / tau_blend, so the
    weights are uniform -- d = d_max (to the rounding of the sums) and a = 0
    exactly, the point is the mean
    of the contact points and the normal the normalised mean of the contact
    normals (where the gated blend returns empty groups)."""
    sc = scenes.hull_env_scene(seed=21, n_envs=3, workers=1)
    sc.pose_b[:, 9] += 5.0
    prm = _ungated(oracle_lib)
    y = oracle_lib.forward(sc, prm)
    off = sc.group_offsets()
    assert np.abs(y[:, 0] - 0.01).max() < 1e-14 and np.all(y[:, 1] == 0.0)
    for i in range(sc.n_pairs):
        rows = oracle_lib.pair_contacts(sc, i, prm)
        assert np.all(rows[:, 2] == 0.0) and np.all(rows[:, 3] == 0.01)
        for g in range(off[i + 1] - off[i]):
            r = _groups(rows, g)
            yy = y[off[i] + g]
            assert np.allclose(yy[2:5], r[:, 4:7].mean(0), rtol=0, atol=1e-12)
            assert np.allclose(yy[5:8], _unit(r[:, 7:10].mean(0)), rtol=0, atol=1e-12)


def test_fully_immersed_body_blends_as_the_gated_blend(oracle_lib):
    """A cube of half size 0.1 at the centre of a unit cube: each of its
    vertices and edges lies at least 0.4 - tau log 3 inside, far past the
    transition band, so every contact of its group has f = 1 and the two
    blends weigh the same contacts by the same exp(-d_c / tau_blend).  The
    unit cube's own features are all far outside the small cube: gated, its
    group is empty; ungated, its contacts average uniformly at d_max."""
    geom = scenes.geometry_from_bodies([[scenes.unit_cube_piece(0.5)], [scenes.unit_cube_piece(0.1)]])
    I = np.eye(3)[None]
    sc = scenes.Scene(geom, np.zeros(1, np.int64), np.ones(1, np.int64),
                      scenes.pack_pose(I, np.zeros((1, 3))), scenes.pack_pose(I, np.full((1, 3), 0.013)))
    yg = oracle_lib.forward(sc)
    yu = oracle_lib.forward(sc, _ungated(oracle_lib))
    rows = oracle_lib.pair_contacts(sc, 0, _ungated(oracle_lib))
    assert np.all(_groups(rows, 1)[:, 2] == 1.0)
    assert np.array_equal(yg[1], yu[1])
    assert yu[1][0] < -0.3 and yu[1][1] == 1.0
    assert yg[0][0] == 0.01 and np.all(yg[0][1:] == 0.0)
    assert abs(yu[0][0] - 0.01) < 1e-14 and yu[0][1] == 0.0
    assert np.allclose(yu[0][2:5], _groups(rows, 0)[:, 4:7].mean(0), atol=1e-12)


def test_infinite_temperature_is_the_plain_mean(oracle_lib, small_hulls):
    """tau_blend -> infinity: every weight 1 / (number of contacts), so the
    group's depth, weight and point are the plain means over all its
    contacts, active or not."""
    sc = small_hulls
    prm = _ungated(oracle_lib, tau_blend=1e9)
    y = oracle_lib.forward(sc, prm)
    off = sc.group_offsets()
    for i in range(sc.n_pairs):
        rows = oracle_lib.pair_contacts(sc, i, prm)
        for g in range(off[i + 1] - off[i]):
            r = _groups(rows, g)
            yy = y[off[i] + g]
            assert abs(yy[0] - r[:, 3].mean()) < 1e-11
            assert abs(yy[1] - r[:, 2].mean()) < 1e-11
            assert np.abs(yy[2:5] - r[:, 4:7].mean(0)).max() < 1e-10


def test_zero_temperature_selects_the_deepest_contact(oracle_lib, small_hulls):
    """tau_blend -> 0: the softmax becomes the argmin of d_c over every
    contact; where the deepest is active (d_c < d_max) it is the gated blend's
    choice too."""
    sc = small_hulls
    prm = _ungated(oracle_lib, tau_blend=1e-9)
    y = oracle_lib.forward(sc, prm)
    yg = oracle_lib.forward(sc, oracle_lib.params(tau_blend=1e-9))
    off = sc.group_offsets()
    seen = 0
    for i in range(sc.n_pairs):
        rows = oracle_lib.pair_contacts(sc, i, prm)
        for g in range(off[i + 1] - off[i]):
            r = _groups(rows, g)
            srt = np.sort(r[:, 3])
            if srt[0] >= 0.01 or srt[1] - srt[0] < 1e-6:
                continue   # no active contact (all tie at d_max), or a near tie
            k = np.argmin(r[:, 3])
            yy = y[off[i] + g]
            assert abs(yy[0] - r[k, 3]) < 1e-9
            assert np.abs(yy[2:5] - r[k, 4:7]).max() < 1e-9
            assert np.abs(yy[:5] - yg[off[i] + g][:5]).max() < 1e-9
            seen += 1
    assert seen > 5
