"""Pins of the oracle's piece SDF (Sec. 3: half-space SDF phi_k = n_k.x + h_k,
smooth intersection = LSE over the planes; Sec. 2: LSE and softmax).

The LSE with softness tau is bounded by the hard maximum m of its arguments,
m <= LSE <= m + tau log F, and tends to m as tau -> 0.  The hard maximum of the
plane values equals minus the exact distance to the boundary inside a convex
polytope and is at most the exact distance outside.  Exact distances come from
brute force over the hull's triangles (tests/geom_util.py)."""
import numpy as np
import pytest

from geom_util import signed_distance
from paper_2604_17538_b300 import scenes


@pytest.fixture(scope="module")
def piece():
    rng = np.random.default_rng(11)
    return scenes.hull_piece(rng.normal(0, 0.05, size=(64, 3)))


def _pts(rng, n, scale):
    return rng.normal(0, scale, size=(n, 3))


def test_hard_max_is_exact_distance_inside(oracle_lib, piece):
    V, P, _ = piece
    rng = np.random.default_rng(0)
    n_in = 0
    for x in _pts(rng, 200, 0.04):
        sd = signed_distance(x, V.astype(np.float64))
        if sd >= 0:
            continue
        n_in += 1
        m, _ = oracle_lib.sdf(P, x, 1e-12)
        # polytope planes from float32 storage: agreement to float32 rounding
        assert abs(m - sd) < 2e-7, (m, sd)
    assert n_in > 20


def test_hard_max_lower_bounds_distance_outside(oracle_lib, piece):
    V, P, _ = piece
    rng = np.random.default_rng(1)
    n_out = 0
    for x in _pts(rng, 200, 0.12):
        sd = signed_distance(x, V.astype(np.float64))
        if sd <= 0:
            continue
        n_out += 1
        m, _ = oracle_lib.sdf(P, x, 1e-12)
        assert m <= sd + 2e-7
        assert m > 0
    assert n_out > 50


def test_outside_along_face_normal_is_distance(oracle_lib, piece):
    """From a point inside a face, moving along the face normal, the closest
    point stays that face point, so the exact distance is the offset."""
    V, P, _ = piece
    P64 = P.astype(np.float64)
    hits = 0
    for k in range(len(P64)):
        n, h = P64[k, :3], P64[k, 3]
        on = np.abs(V.astype(np.float64) @ n + h) < 1e-6
        if on.sum() < 3:
            continue
        c = V[on].astype(np.float64).mean(0)
        for s in (0.001, 0.01):
            x = c + s * n
            sd = signed_distance(x, V.astype(np.float64))
            m, _ = oracle_lib.sdf(P, x, 1e-12)
            if abs(sd - s) < 1e-9:       # face point is the closest point
                assert abs(m - s) < 2e-7
                hits += 1
    assert hits > 10


def test_lse_bounds_and_monotone_limit(oracle_lib, piece):
    _, P, _ = piece
    F = len(P)
    rng = np.random.default_rng(2)
    for x in _pts(rng, 100, 0.08):
        m, _ = oracle_lib.sdf(P, x, 1e-12)
        prev = m
        for tau in (1e-6, 1e-4, 1e-3, 5e-3, 2e-2):
            phi, _ = oracle_lib.sdf(P, x, tau)
            assert m - 1e-12 <= phi <= m + tau * np.log(F) + 1e-12
            assert phi >= prev - 1e-12       # LSE is non-decreasing in tau
            prev = phi


def test_identical_and_single_planes(oracle_lib):
    plane = np.array([[0.6, 0.0, 0.8, -0.1]])
    x = np.array([0.3, -0.2, 0.5])
    v = 0.6 * 0.3 + 0.8 * 0.5 - 0.1
    phi, g = oracle_lib.sdf(plane, x, 5e-3)
    assert abs(phi - v) < 1e-15 and np.allclose(g, [0.6, 0.0, 0.8], atol=1e-15)
    for F in (2, 5, 17):
        phi, g = oracle_lib.sdf(np.repeat(plane, F, 0), x, 5e-3)
        assert abs(phi - (v + 5e-3 * np.log(F))) < 1e-14
        assert np.allclose(g, [0.6, 0.0, 0.8], atol=1e-14)


def test_gradient_is_derivative_and_1_lipschitz(oracle_lib, piece):
    _, P, _ = piece
    rng = np.random.default_rng(3)
    h = 1e-7
    for x in _pts(rng, 50, 0.08):
        phi, g = oracle_lib.sdf(P, x, 5e-3)
        fd = np.array([(oracle_lib.sdf(P, x + h * e, 5e-3)[0] - oracle_lib.sdf(P, x - h * e, 5e-3)[0]) / (2 * h)
                       for e in np.eye(3)])
        assert np.abs(fd - g).max() < 1e-6
        assert np.linalg.norm(g) <= 1.0 + 1e-6


def test_gradient_tends_to_face_normal(oracle_lib, piece):
    _, P, _ = piece
    P64 = P.astype(np.float64)
    rng = np.random.default_rng(4)
    for x in _pts(rng, 50, 0.08):
        vals = P64[:, :3] @ x + P64[:, 3]
        k = np.argsort(vals)
        if vals[k[-1]] - vals[k[-2]] < 1e-3:
            continue
        _, g = oracle_lib.sdf(P, x, 1e-5)
        assert np.abs(g - P64[k[-1], :3]).max() < 1e-6
