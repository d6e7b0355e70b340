"""Pins of the oracle's pose derivatives: gradient, Hessian-vector product and
output tangents against central finite differences in FP64, plus the null
directions of a common rigid motion and the symmetry of the Hessian.

Twist chart per body: R <- Exp([w]x) R, t <- t + v; coordinates of a pair are
(w_A, v_A, w_B, v_B).  L = <ybar, y> with a random ybar."""
import numpy as np
import pytest

from paper_2604_17538_b300 import scenes

H = 1e-5


@pytest.fixture(scope="module")
def cases():
    cube = scenes.cube_pair_scene(seed=1).take(np.arange(8))
    hull = scenes.hull_env_scene(seed=2, n_envs=4, workers=1)
    return {"cube": cube, "hull": hull}


def _ybar(sc, seed=0):
    return np.random.default_rng(seed).normal(size=(int(sc.group_offsets()[-1]), 8))


def _dirs(n, seed=1):
    u = np.random.default_rng(seed).normal(size=(n, 12))
    return u / np.linalg.norm(u, axis=1, keepdims=True)


def _loss_per_pair(sc, y, yb):
    off = sc.group_offsets()
    return np.array([np.sum(y[off[i]:off[i + 1]] * yb[off[i]:off[i + 1]]) for i in range(sc.n_pairs)])


@pytest.mark.parametrize("name", ["cube", "hull"])
def test_gradient_matches_central_differences(oracle_lib, cases, name):
    sc = cases[name]
    yb = _ybar(sc)
    g, _ = oracle_lib.gradient(sc, yb)
    fd = np.zeros_like(g)
    for k in range(12):
        xi = np.zeros((sc.n_pairs, 12))
        xi[:, k] = H
        _, yp = oracle_lib.gradient(sc, yb, xi=xi)
        _, ym = oracle_lib.gradient(sc, yb, xi=-xi)
        fd[:, k] = (_loss_per_pair(sc, yp, yb) - _loss_per_pair(sc, ym, yb)) / (2 * H)
    scale = np.abs(fd).max(1, keepdims=True) + 1e-12
    assert np.all(np.abs(g - fd) <= 1e-4 * scale + 1e-9)


@pytest.mark.parametrize("name", ["cube", "hull"])
def test_hvp_and_jvp_match_central_differences(oracle_lib, cases, name):
    sc = cases[name]
    yb = _ybar(sc)
    u = _dirs(sc.n_pairs)
    g, hv, jv, y = oracle_lib.hvp(sc, yb, u)
    g0, y0 = oracle_lib.gradient(sc, yb)
    assert np.array_equal(y, y0)
    assert np.abs(g - g0).max() <= 1e-12 * (1 + np.abs(g0).max())
    gp, yp = oracle_lib.gradient(sc, yb, xi=H * u)
    gm, ym = oracle_lib.gradient(sc, yb, xi=-H * u)
    fd_h = (gp - gm) / (2 * H)
    scale = np.abs(fd_h).max(1, keepdims=True) + 1e-12
    assert np.all(np.abs(hv - fd_h) <= 1e-4 * scale + 1e-9)
    fd_j = (yp - ym) / (2 * H)
    assert np.abs(jv - fd_j).max() <= 1e-4 * (np.abs(fd_j).max() + 1e-9)


def test_hessian_is_symmetric(oracle_lib, cases):
    sc = cases["hull"]
    yb = _ybar(sc)
    u1, u2 = _dirs(sc.n_pairs, 5), _dirs(sc.n_pairs, 6)
    _, h1, _, _ = oracle_lib.hvp(sc, yb, u1)
    _, h2, _, _ = oracle_lib.hvp(sc, yb, u2)
    a = np.sum(u2 * h1, 1)
    b = np.sum(u1 * h2, 1)
    assert np.all(np.abs(a - b) <= 1e-9 * (np.abs(a) + np.abs(b) + 1e-9))


def test_common_rigid_motion_is_a_null_direction(oracle_lib, cases):
    """A rigid motion of the whole scene leaves depths and weights unchanged,
    so with ybar on (d, a) only the gradient is orthogonal to the 6 common-
    motion directions w_A = w_B = w, v_X = w x t_X + v."""
    for sc in cases.values():
        yb = _ybar(sc)
        yb[:, 2:] = 0.0
        g, _ = oracle_lib.gradient(sc, yb)
        for i in range(sc.n_pairs):
            tA = sc.pose_a[i, 9:].astype(np.float64)
            tB = sc.pose_b[i, 9:].astype(np.float64)
            for k in range(6):
                w = np.zeros(3)
                v = np.zeros(3)
                (w if k < 3 else v)[k % 3] = 1.0
                d = np.concatenate([w, np.cross(w, tA) + v, w, np.cross(w, tB) + v])
                assert abs(g[i] @ d) <= 1e-9 * (np.abs(g[i]).max() + 1)
