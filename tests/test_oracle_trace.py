"""Pins of the oracle's smooth operators (Sec. 2), sphere-traced edge contact
point (Sec. 4.2) and transition function (Sec. 4.3)."""
import numpy as np
import pytest

from geom_util import cyrus_beck
from paper_2604_17538_b300 import scenes


# ---------------------------------------------------------------- Sec. 2
def test_sigmoid_softplus_closed_values(oracle_lib):
    o = oracle_lib
    assert o.sigmoid(0.0) == 0.5
    for x in (-40.0, -3.0, -0.1, 0.2, 5.0, 700.0):
        assert abs(o.sigmoid(x) + o.sigmoid(-x) - 1.0) < 1e-15
    assert o.sigmoid(800.0) == 1.0 and 0.0 <= o.sigmoid(-800.0) < 1e-300
    tau = 5e-3
    assert abs(o.softplus(0.0, tau) - tau * np.log(2.0)) < 1e-18
    # relu limits and the softplus derivative = sigmoid(x / tau)
    assert abs(o.softplus(1.0, tau) - 1.0) < 1e-40 + 1e-15
    assert o.softplus(-1.0, tau) < 1e-80
    h = 1e-8
    for x in (-0.02, -0.004, 0.0, 0.003, 0.05):
        fd = (o.softplus(x + h, tau) - o.softplus(x - h, tau)) / (2 * h)
        assert abs(fd - o.sigmoid(x / tau)) < 1e-6


def test_softclip_properties(oracle_lib):
    o = oracle_lib
    tau, L = 5e-3, 0.3
    xs = np.linspace(-0.2, 0.5, 141)
    ys = np.array([o.softclip(x, 0.0, L, tau) for x in xs])
    assert np.all(ys >= 0.0) and np.all(ys <= L)
    near = (xs > -0.05) & (xs < L + 0.05)                  # strictly inside (0, L)
    assert np.all(ys[near] > 0.0) and np.all(ys[near] < L)
    assert np.all(np.diff(ys) >= 0) and np.all(np.diff(ys[near]) > 0)   # increasing
    assert abs(o.softclip(-1.0, 0.0, L, tau)) < 1e-30      # clips low
    assert abs(o.softclip(2.0, 0.0, L, tau) - L) < 1e-15   # clips high
    assert abs(o.softclip(0.15, 0.0, L, tau) - 0.15) < 1e-12
    # point symmetry about the middle of [lo, hi]
    for x in (-0.05, 0.0, 0.01, 0.1):
        assert abs(o.softclip(x, 0.0, L, tau) + o.softclip(L - x, 0.0, L, tau) - L) < 1e-15


# ---------------------------------------------------------------- Sec. 4.3
def test_transition_knots_and_c2(oracle_lib):
    o = oracle_lib
    dmax, eps = 0.01, 0.01
    for d in (-1.0, -0.05, 0.0, dmax - eps):
        assert o.transition(d, dmax, eps) == 1.0
    for d in (dmax, 0.02, 1.0):
        assert o.transition(d, dmax, eps) == 0.0
    assert abs(o.transition(dmax - eps / 2, dmax, eps) - 0.5) < 1e-15
    ds = np.linspace(-0.005, 0.015, 2001)
    f = np.array([o.transition(d, dmax, eps) for d in ds])
    assert np.all(np.diff(f) <= 0)                         # non-increasing
    h = 1e-7

    def d1(d):
        return (o.transition(d + h, dmax, eps) - o.transition(d - h, dmax, eps)) / (2 * h)

    def d2(d):
        return (o.transition(d + h, dmax, eps) - 2 * o.transition(d, dmax, eps)
                + o.transition(d - h, dmax, eps)) / h ** 2

    # f' vanishes quadratically and f'' linearly at both knots from inside the
    # band, and both are exactly zero outside it: f is C^2 across the knots
    for knot, inward in ((dmax - eps, 1), (dmax, -1)):
        a, b = knot + inward * 1e-3, knot + inward * 1e-4
        assert 0.008 < abs(d1(b) / d1(a)) < 0.014
        assert 0.08 < abs(d2(b) / d2(a)) < 0.15
        assert d1(knot - inward * 1e-4) == 0.0 and d2(knot - inward * 1e-4) == 0.0
    # f'' is bounded everywhere (C^2): max |f''| = 10 sqrt(3)/3 / eps^2
    f2 = np.diff(f, 2) / (ds[1] - ds[0]) ** 2
    assert np.abs(f2).max() < 10 * np.sqrt(3) / 3 / eps ** 2 * 1.01


# ---------------------------------------------------------------- Sec. 4.2
def _cube_planes(half=0.5):
    return scenes.unit_cube_piece(half)[1].astype(np.float64)


def test_both_corners_inside_gives_midpoint(oracle_lib):
    P = _cube_planes()
    rng = np.random.default_rng(5)
    for _ in range(20):
        a, b = rng.uniform(-0.35, 0.35, size=(2, 3))
        pe, al = oracle_lib.edge_point(P, a, b)
        assert np.abs(pe - 0.5 * (a + b)).max() < 1e-9


def test_ray_normal_to_face_converges_in_one_step(oracle_lib):
    P = _cube_planes()
    prm = oracle_lib.params(tau_sdf=1e-7, tau_trace=1e-7, tau_clip=1e-7, trace_iters=1)
    for h in (0.05, 0.2, 0.4):
        a = np.array([0.1, -0.2, 0.5 + h])     # above the top face
        b = np.array([0.1, -0.2, -0.3])        # inside
        pe, al = oracle_lib.edge_point(P, a, b, prm)
        assert abs(al[0] - h) < 1e-6           # traced corner lands on the face
        assert abs(al[1] - np.linalg.norm(b - a)) < 1e-6   # inside corner stays
        assert abs(pe[2] - 0.5 * (0.5 + (-0.3))) < 1e-6


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_chord_midpoint_limit_matches_cyrus_beck(oracle_lib, seed):
    rng = np.random.default_rng(100 + seed)
    V, P, _ = scenes.hull_piece(rng.normal(0, 0.05, size=(64, 3)))
    P = P.astype(np.float64)
    prm = oracle_lib.params(tau_sdf=1e-8, tau_trace=1e-8, tau_clip=1e-8, trace_iters=400)
    done = 0
    while done < 8:
        c = rng.normal(0, 0.01, 3)               # through the interior
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        a, b = c - 0.3 * d, c + 0.3 * d          # both corners outside
        iv = cyrus_beck(a, b, P)
        if iv is None or iv[0] <= 0 or iv[1] >= 1:
            continue
        mid = a + 0.5 * (iv[0] + iv[1]) * (b - a)
        pe, _ = oracle_lib.edge_point(P, a, b, prm)
        assert np.abs(pe - mid).max() < 2e-6, (pe, mid)
        done += 1


def test_traced_points_never_leave_the_edge(oracle_lib):
    rng = np.random.default_rng(7)
    V, P, _ = scenes.hull_piece(rng.normal(0, 0.05, size=(64, 3)))
    for _ in range(50):
        a, b = rng.normal(0, 0.15, size=(2, 3))
        pe, al = oracle_lib.edge_point(P, a, b)
        L = np.linalg.norm(b - a)
        t = (pe - a) @ (b - a) / L ** 2
        assert 0.0 < t < 1.0
        assert np.linalg.norm(np.cross(pe - a, b - a)) / L < 1e-12   # on the line
        assert 0.0 < al[2] < L + 1e-12 and 0.0 < al[3] < L + 1e-12


# ------------------------------------------- Sec. 4.2 at the default softness
def _soft_sdf(P, tau):
    from scipy.special import logsumexp
    return lambda x: tau * logsumexp((P[:, :3] @ x + P[:, 3]) / tau)


def test_trace_steps_follow_their_recurrence_at_default_softness(oracle_lib):
    """The oracle's traced corners after k = 0..3 steps (trace_iters = k) obey
    the sphere-trace recurrence of Sec. 4.2 with the soft gate of Sec. 2,
    alpha_{k+1} = alpha_k +/- sigmoid(phi_k / tau_trace) phi_k along the edge,
    with phi evaluated here by scipy's logsumexp of the plane values; and
    since phi is 1-Lipschitz and the gate below 1, no step crosses the surface:
    phi keeps the sign it has at the corner."""
    from scipy.special import expit
    rng = np.random.default_rng(11)
    V, P, _ = scenes.hull_piece(rng.normal(0, 0.05, size=(64, 3)))
    P = P.astype(np.float64)
    d = oracle_lib.DEFAULTS
    phi = _soft_sdf(P, d["tau_sdf"])
    checked = 0
    for _ in range(60):
        a, b = rng.normal(0, 0.12, size=(2, 3))
        L = np.linalg.norm(b - a)
        e = (b - a) / L
        al = [oracle_lib.edge_point(P, a, b, oracle_lib.params(trace_iters=k))[1] for k in range(4)]
        assert al[0][0] == 0.0 and abs(al[0][1] - L) < 1e-15
        for k in range(3):
            for c, sgn in ((0, 1.0), (1, -1.0)):        # corner I along +e, corner II along -e
                f = phi(a + al[k][c] * e)
                step = expit(f / d["tau_trace"]) * f
                assert abs(al[k + 1][c] - (al[k][c] + sgn * step)) < 1e-12
                f0 = phi(a + al[0][c] * e)
                f1 = phi(a + al[k + 1][c] * e)
                assert f1 == 0.0 or np.sign(f1) == np.sign(f0)
                checked += 1
    assert checked == 360


def test_trace_converges_to_the_soft_surface_at_default_softness(oracle_lib):
    """Many steps at the default softness: a corner outside the piece moves to
    the first zero of the soft SDF along its edge (a root found here by
    bracketing scipy's logsumexp SDF), for edges that cross the surface
    transversally."""
    from scipy.optimize import brentq
    rng = np.random.default_rng(12)
    V, P, _ = scenes.hull_piece(rng.normal(0, 0.05, size=(64, 3)))
    P = P.astype(np.float64)
    d = oracle_lib.DEFAULTS
    phi = _soft_sdf(P, d["tau_sdf"])
    prm = oracle_lib.params(trace_iters=400)
    done = 0
    while done < 10:
        c = rng.normal(0, 0.01, 3)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        a, b = c - 0.3 * u, c + 0.3 * u                  # both corners outside
        L = 0.6
        g = lambda t: phi(a + t * u)
        ts = np.linspace(0, L, 601)
        vals = np.array([g(t) for t in ts])
        if vals[0] <= 0 or vals[-1] <= 0 or vals.min() >= 0:
            continue
        i0 = np.argmax(vals < 0)                         # first sample inside
        i1 = len(ts) - 1 - np.argmax(vals[::-1] < 0)     # last sample inside
        t1 = brentq(g, ts[i0 - 1], ts[i0], xtol=1e-15)
        t2 = brentq(g, ts[i1], ts[i1 + 1], xtol=1e-15)
        h = 1e-7                                          # crossing slopes
        if min(abs(g(t1 + h) - g(t1 - h)), abs(g(t2 + h) - g(t2 - h))) / (2 * h) < 0.2:
            continue
        _, al = oracle_lib.edge_point(P, a, b, prm)
        assert abs(al[0] - t1) < 1e-9 and abs(al[1] - t2) < 1e-9, (al[:2], t1, t2)
        done += 1
