"""Pins of the oracle's tricubic spline SDF (Sec. 3.2) and of the contact
pipeline run on it (FLAG_SPLINE): the basis's own identities, interpolation at
the grid nodes, exact reproduction of linear fields, fourth-order convergence
to a smooth SDF, and the stacked-cube closed form of Sec. 5.2 with spline
SDFs.  The coefficients come from scenes.fit_spline (asset preparation); the
pins do not use the oracle to build what they compare against."""
import json
import os

import numpy as np
import pytest

from paper_2604_17538_b300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_basis_partition_support_and_continuity(oracle_lib):
    """sum_k u(t - k) = 6 for every t (the basis is 6 x the cubic B-spline),
    u vanishes on |t| >= 2, and u, u', u'' are continuous at |t| = 1 and 2."""
    u = oracle_lib.spline_u
    for t in np.linspace(-3.0, 3.0, 61) + 0.137:
        assert abs(sum(u(t - k) for k in range(-6, 7)) - 6.0) < 1e-12
    for t in (2.0, -2.0, 2.5, -3.1):
        assert u(t) == 0.0
    assert u(0.0) == 4.0 and u(1.0) == 1.0
    e = 1e-5
    for knot in (1.0, 2.0, -1.0):
        d1l = (u(knot) - u(knot - e)) / e
        d1r = (u(knot + e) - u(knot)) / e
        d2l = (u(knot) - 2 * u(knot - e) + u(knot - 2 * e)) / e**2
        d2r = (u(knot + 2 * e) - 2 * u(knot + e) + u(knot)) / e**2
        assert abs(d1l - d1r) < 1e-3 and abs(d2l - d2r) < 1e-2


def _one_piece_geom(field, lo, h, dims):
    """A one-piece geometry (a dummy tetrahedron) whose spline is fitted to
    ``field`` on the given grid."""
    tet = scenes.hull_piece(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) * 0.1)
    geom = scenes.geometry_from_bodies([[tet]])
    coef = scenes.fit_spline(field, np.asarray(lo, float), h, np.asarray(dims))
    geom.splines = scenes.SplineSet(np.array([[*lo, h]], np.float32),
                                    np.array([[*dims, 0]], np.int64), coef.astype(np.float32))
    return geom


def test_interpolates_the_fitted_values_at_the_nodes(oracle_lib):
    lo, h, dims = np.array([-0.3, -0.2, -0.25]), 0.0625, (8, 6, 7)

    def field(p):
        r = np.linalg.norm(p - [0.05, -0.02, 0.01], axis=1, keepdims=True)
        return np.concatenate([r - 0.15, np.sin(3 * p)], 1)
    geom = _one_piece_geom(field, lo, h, dims)
    # float32 coefficients: the interpolation holds to float32 rounding
    rng = np.random.default_rng(0)
    for _ in range(30):
        i = rng.integers(0, np.array(dims) + 1)
        x = lo + h * i
        phi, n = oracle_lib.spline_sdf(geom, 0, x)
        f = field(x[None])[0]
        assert abs(phi - f[0]) < 2e-6 and np.allclose(n, f[1:], atol=2e-6)


def test_reproduces_linear_fields_exactly(oracle_lib):
    """The natural end conditions hold for a linear field, so its spline is the
    field itself everywhere in the grid box; a constant normal likewise."""
    a, b = np.array([0.3, -0.7, 0.2]), 0.05
    lo, h, dims = np.array([-0.5, -0.5, -0.5]), 0.125, (8, 8, 8)
    # coefficients in float64 here (the field, not float32 storage, is pinned)
    geom = _one_piece_geom(lambda p: np.concatenate(
        [p @ a[:, None] + b, np.tile([0.1, 0.2, 0.3], (len(p), 1))], 1), lo, h, dims)
    geom.splines.coef = scenes.fit_spline(lambda p: np.concatenate(
        [p @ a[:, None] + b, np.tile([0.1, 0.2, 0.3], (len(p), 1))], 1), lo, h, np.array(dims))
    rng = np.random.default_rng(1)
    for x in rng.uniform(-0.5, 0.5, size=(100, 3)):
        phi, n = oracle_lib.spline_sdf(geom, 0, x)
        assert abs(phi - (a @ x + b)) < 1e-12
        assert np.allclose(n, [0.1, 0.2, 0.3], atol=1e-12)


def test_converges_to_a_smooth_sdf_at_fourth_order(oracle_lib):
    """A sphere's SDF |x - c| - r is smooth away from c: halving the voxel size
    cuts the interpolation error in the shell around the surface by about 16
    (cubic splines are fourth-order accurate)."""
    c, r = np.array([0.01, -0.02, 0.015]), 0.2
    rng = np.random.default_rng(2)
    d = rng.normal(size=(200, 3))
    pts = c + (r + rng.uniform(-0.05, 0.05, (200, 1))) * d / np.linalg.norm(d, axis=1, keepdims=True)
    errs = []
    for n in (8, 16, 32):
        lo, h = np.array([-0.4, -0.4, -0.4]), 0.8 / n

        def field(p):
            q = p - c
            nr = np.linalg.norm(q, axis=1, keepdims=True)
            return np.concatenate([nr - r, q / nr], 1)
        geom = _one_piece_geom(field, lo, h, (n, n, n))
        geom.splines.coef = scenes.fit_spline(field, lo, h, np.array((n, n, n)))
        errs.append(max(abs(oracle_lib.spline_sdf(geom, 0, x)[0] - (np.linalg.norm(x - c) - r))
                        for x in pts))
    assert errs[1] < errs[0] / 8 and errs[2] < errs[1] / 8, errs


def test_outside_the_grid_adds_the_distance_to_the_box(oracle_lib):
    a, b = np.array([0.0, 0.0, 1.0]), -0.1
    lo, h, dims = np.array([-0.25, -0.25, -0.25]), 0.0625, (8, 8, 8)
    field = lambda p: np.concatenate([p @ a[:, None] + b, np.tile(a, (len(p), 1))], 1)
    geom = _one_piece_geom(field, lo, h, dims)
    geom.splines.coef = scenes.fit_spline(field, lo, h, np.array(dims))
    for x in ([0.6, 0.1, 0.05], [-0.1, -0.9, 0.2], [0.4, 0.4, 0.4]):
        x = np.array(x)
        cpt = np.clip(x, -0.25, 0.25)
        phi, n = oracle_lib.spline_sdf(geom, 0, x)
        assert abs(phi - (a @ cpt + b + np.linalg.norm(x - cpt))) < 1e-12
        assert np.allclose(n, a, atol=1e-12)


def test_stacked_cubes_with_spline_sdfs_hard_limit(oracle_lib):
    """Sec. 5.2 stacked boxes with spline SDFs: A's SDF is the spline of the
    top face's half-space z - 0.5 (a linear field, so exact) with normal +z,
    B's the spline of its own box SDF.  The hand-derived hard limit of the
    golden file holds unchanged: B's group is its bottom face at depth -delta,
    A's group is empty."""
    with open(os.path.join(GOLDEN, "stacked_cubes_hard_limit.json")) as f:
        gold = json.load(f)
    for case in gold["cases"]:
        hb, delta = case["half_b"], case["delta"]
        A = [scenes.unit_cube_piece(0.5)]
        B = [scenes.unit_cube_piece(hb)]
        geom = scenes.geometry_from_bodies([A, B])
        lo_a, h_a, d_a = np.array([-0.6, -0.6, -0.6]), 0.075, np.array([16, 16, 16])
        ca = scenes.fit_spline(lambda p: np.concatenate(
            [p[:, 2:3] - 0.5, np.tile([0.0, 0.0, 1.0], (len(p), 1))], 1), lo_a, h_a, d_a)
        vb, fb, _ = B[0]
        lo_b, h_b, d_b, cb = scenes.piece_spline(vb, fb, voxels=16, margin=0.05)
        geom.splines = scenes.SplineSet(
            np.array([[*lo_a, h_a], [*lo_b, h_b]], np.float32),
            np.array([[*d_a, 0], [*d_b, len(ca)]], np.int64),
            np.concatenate([ca, cb]).astype(np.float64))
        I = np.eye(3)[None]
        sc = scenes.Scene(geom, np.zeros(1, np.int64), np.ones(1, np.int64),
                          scenes.pack_pose(I, np.zeros((1, 3))),
                          scenes.pack_pose(I, np.array([[0.0, 0.0, 0.5 + hb - delta]])))
        prm = oracle_lib.params(flags=oracle_lib.FLAG_SPLINE, **gold["params"])
        y = oracle_lib.forward(sc, prm)
        assert np.allclose(y[0], case["group_A"], atol=1e-9), y[0]
        assert np.allclose(y[1], case["group_B"], atol=1e-6), y[1]


def test_window_sum_equals_the_full_tensor_product_sum(oracle_lib):
    """The oracle evaluates each spline from the 64 coefficients whose basis
    functions reach the point; summing c_k u(t_x - (k_x - 1)) u(t_y - (k_y - 1))
    u(t_z - (k_z - 1)) over every coefficient of the grid (brute force, with
    the row layout of the coefficient table: z fastest) gives the same SDF
    value and normal at any point of the grid box, its faces and corners
    included -- so the window's cell index, its clamping at the last cell and
    the table's layout are those of the tensor-product definition of Sec. 3.2."""
    lo, h, dims = np.array([-0.2, -0.1, -0.15]), 0.05, np.array([5, 4, 6])

    def field(p):
        r = np.linalg.norm(p - [0.02, 0.01, -0.03], axis=1, keepdims=True)
        return np.concatenate([r - 0.08, np.cos(4 * p)], 1)
    geom = _one_piece_geom(field, lo, h, dims)
    coef = geom.splines.coef.astype(np.float64)
    u = np.vectorize(oracle_lib.spline_u)
    nx, ny, nz = dims + 3
    rng = np.random.default_rng(3)
    # the grid as the geometry stores it (float32)
    lo32, h32 = geom.splines.grid[0, :3].astype(np.float64), float(geom.splines.grid[0, 3])
    pts = list(lo32 + h32 * dims * rng.uniform(size=(40, 3)))
    pts += [lo32 + h32 * np.array(t, float)
            for t in ((0, 0, 0), dims, (dims[0], 0, dims[2]), dims // 2, (0, dims[1], 2.5))]
    for x in pts:
        t = (x - lo32) / h32
        # a point on a face may round to just outside the box: the extension
        # beyond it (the value at the nearest box point plus the distance)
        tc = np.clip(t, 0.0, dims)
        out = h32 * np.linalg.norm(t - tc)
        t = tc
        wx = u(t[0] - (np.arange(nx) - 1))
        wy = u(t[1] - (np.arange(ny) - 1))
        wz = u(t[2] - (np.arange(nz) - 1))
        w = (wx[:, None, None] * wy[None, :, None] * wz[None, None, :]).reshape(-1)
        ref = w @ coef[:nx * ny * nz]
        phi, n = oracle_lib.spline_sdf(geom, 0, x)
        assert out < 1e-12
        assert abs(phi - (ref[0] + out)) < 1e-12 and np.abs(n - ref[1:]).max() < 1e-12, (x, phi, ref)
