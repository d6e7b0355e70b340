"""FP64 CPU oracle (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the product path never does.  The
arithmetic lives in ``ccm_oracle.cpp`` (double precision, plain loops, forward-
mode dual numbers for exact derivatives); this file only builds it and
marshals numpy arrays through ctypes.

Parity status of each function (what pins it, see ``tests/test_oracle_*.py``):
  * ``body_sdf`` / FLAG_BODY_UNION -- LSE bounds against the pieces' SDFs,
                          finite differences, far-apart and single-piece limits,
                          rigid-motion invariance and body-swap symmetry, and
                          its definition evaluated with scipy's logsumexp.
  * FLAG_PROJECT       -- a single half-space and the stacked-cube face: the
                          projected points lie on the plane; on random hulls,
                          every projected point is p - phi n of its contact.
  * ``spline_u`` / ``spline_sdf`` / FLAG_SPLINE -- basis partition of unity
                          and support, interpolation at the nodes, exact
                          reproduction of linear fields, convergence to a
                          sphere's SDF, the stacked-cube closed form, and the
                          64-coefficient window against the brute-force sum
                          over every coefficient of the grid.
  * FLAG_UNGATED       -- separated bodies (every contact at d_max: uniform
                          weights, the mean of the contact points), a fully
                          immersed body (every f = 1: equal to the gated
                          blend), the tau_blend -> infinity mean and the
                          tau_blend -> 0 argmin over every contact.
  * ``sdf``            -- brute-force polytope distance, LSE bounds, tau -> 0 limit.
  * ``edge_point``     -- Cyrus-Beck chord midpoint (many iterations, small tau),
                          inside-edge midpoint, one-step convergence on a face;
                          at the default softness, every trace step against the
                          recurrence with scipy's logsumexp SDF (and no step
                          crossing the surface), and many steps converging to
                          the soft SDF's root along the edge.
  * ``transition``     -- knot values and C^2 continuity.
  * ``forward``        -- cube-on-cube closed form and hard limits, rigid-motion
                          invariance, body-swap symmetry, separation; on random
                          hulls in the hard limit, the deepest brute-force
                          contact (vertex plane maxima, edge chord midpoints).
  * ``gradient``/``hvp`` -- central finite differences in FP64, rigid-motion
                          null directions, Hessian symmetry.
  * ``pair_contacts`` / ``forward`` on random hulls at the default softness
                       -- every contact's SDF value and normal against scipy's
                          logsumexp / softmax of the plane values, vertex
                          contacts at their vertex, edge contacts strictly
                          inside their edge, the mollified depth against the
                          quintic smoothstep, each group against the softmax
                          average of its contacts.
  The paper prints no worked example or numeric table, so every pin is a
  definition evaluated independently, a limit, an invariant, brute force or
  finite differences; no function is left without one.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ccm_oracle.cpp")
_LIB = os.path.join(_HERE, "libccm_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (OpenMP) into ``oracle/libccm_oracle.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC", "-o", _LIB, _SRC]
        subprocess.run(cmd, check=True)
    return _LIB


class Params(C.Structure):
    _fields_ = [("tau_sdf", C.c_double), ("tau_trace", C.c_double), ("tau_clip", C.c_double),
                ("tau_blend", C.c_double), ("d_max", C.c_double), ("gate_width", C.c_double),
                ("trace_iters", C.c_int32), ("flags", C.c_int32)]


class _Geom(C.Structure):
    _fields_ = [("body_piece_off", C.c_void_p), ("piece_v_off", C.c_void_p),
                ("piece_f_off", C.c_void_p), ("piece_e_off", C.c_void_p),
                ("verts", C.c_void_p), ("planes", C.c_void_p), ("edges", C.c_void_p),
                ("spline_grid", C.c_void_p), ("spline_dims", C.c_void_p),
                ("spline_coef", C.c_void_p)]


DEFAULTS = dict(tau_sdf=5e-3, tau_trace=5e-3, tau_clip=5e-3, tau_blend=5e-3,
                d_max=0.01, gate_width=0.01, trace_iters=3, flags=0)

# forward variants (flags): the other body's SDF as the smooth union of its
# pieces (Sec. 3.1, Eq. soft_union); contact points projected onto the SDF's
# isosurface (Sec. 4.1)
FLAG_BODY_UNION = 2
FLAG_PROJECT = 4
# every SDF piece as its tricubic spline SDF with normal splines (Sec. 3.2);
# needs a geometry with splines (scenes.attach_splines)
FLAG_SPLINE = 8
# the literal "softmax on {d_c}" blend over every contact of a group, f = 0
# ones included (Sec. 4.4), for comparison with the gated blend
FLAG_UNGATED = 16

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P, I64, D, I = C.c_void_p, C.c_int64, C.c_double, C.c_int
        _lib.ccmo_forward.argtypes = [P, I64, P, P, P, P, P, P, P, I]
        _lib.ccmo_gradient.argtypes = [P, I64, P, P, P, P, P, P, P, P, P, P, I]
        _lib.ccmo_hvp.argtypes = [P, I64, P, P, P, P, P, P, P, P, P, P, P, P, I]
        _lib.ccmo_sdf.argtypes = [P, I, P, D, P]
        _lib.ccmo_sdf.restype = D
        _lib.ccmo_edge_point.argtypes = [P, I, P, P, P, P, P]
        for f in ("ccmo_transition",):
            getattr(_lib, f).argtypes = [D, D, D]
            getattr(_lib, f).restype = D
        _lib.ccmo_softclip.argtypes = [D, D, D, D]
        _lib.ccmo_softclip.restype = D
        _lib.ccmo_softplus.argtypes = [D, D]
        _lib.ccmo_softplus.restype = D
        _lib.ccmo_sigmoid.argtypes = [D]
        _lib.ccmo_sigmoid.restype = D
        _lib.ccmo_pair_contacts.argtypes = [P, I64, I64, P, P, P, P, I64]
        _lib.ccmo_pair_contacts.restype = I64
        _lib.ccmo_body_sdf.argtypes = [P, I64, P, D, P]
        _lib.ccmo_body_sdf.restype = D
        _lib.ccmo_spline_u.argtypes = [D]
        _lib.ccmo_spline_u.restype = D
        _lib.ccmo_spline_sdf.argtypes = [P, I64, P, P]
        _lib.ccmo_spline_sdf.restype = D
    return _lib


def params(**kw) -> Params:
    d = dict(DEFAULTS)
    d.update(kw)
    return Params(float(d["tau_sdf"]), float(d["tau_trace"]), float(d["tau_clip"]),
                  float(d["tau_blend"]), float(d["d_max"]), float(d["gate_width"]),
                  int(d["trace_iters"]), int(d["flags"]))


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class _Packed:
    """FP64 copies of a Geometry kept alive for the duration of a call."""

    def __init__(self, geom):
        self.arrs = [np.ascontiguousarray(geom.body_piece_off, np.int64),
                     np.ascontiguousarray(geom.piece_v_off, np.int64),
                     np.ascontiguousarray(geom.piece_f_off, np.int64),
                     np.ascontiguousarray(geom.piece_e_off, np.int64),
                     np.ascontiguousarray(geom.verts, np.float64),
                     np.ascontiguousarray(geom.planes, np.float64),
                     np.ascontiguousarray(geom.edges, np.int32)]
        sp = getattr(geom, "splines", None)
        if sp is not None:
            self.arrs += [np.ascontiguousarray(sp.grid, np.float64),
                          np.ascontiguousarray(sp.dims, np.int64),
                          np.ascontiguousarray(sp.coef, np.float64)]
        ptrs = [a.ctypes.data for a in self.arrs]
        self.s = _Geom(*(ptrs + [None] * (10 - len(ptrs))))

    def ref(self):
        return C.byref(self.s)


def _scene_args(scene):
    pa = np.ascontiguousarray(scene.pair_a, np.int64)
    pb = np.ascontiguousarray(scene.pair_b, np.int64)
    A = np.ascontiguousarray(scene.pose_a, np.float64)
    B = np.ascontiguousarray(scene.pose_b, np.float64)
    goff = scene.group_offsets()
    return pa, pb, A, B, goff


def forward(scene, prm=None, threads=0):
    """Group outputs y [G, 8] = (d, a, p, n) of every pair (Sec. 4.4)."""
    prm = prm or params()
    g = _Packed(scene.geom)
    pa, pb, A, B, goff = _scene_args(scene)
    y = np.zeros((int(goff[-1]), 8))
    lib().ccmo_forward(g.ref(), len(pa), _ptr(pa), _ptr(pb), _ptr(A), _ptr(B),
                       C.byref(prm), _ptr(goff), _ptr(y), threads)
    return y


def gradient(scene, ybar, prm=None, xi=None, threads=0):
    """(grad [n,12], y [G,8]) of L = <ybar, y> w.r.t. the twists
    (w_A, v_A, w_B, v_B), at Exp(xi) T."""
    prm = prm or params()
    g = _Packed(scene.geom)
    pa, pb, A, B, goff = _scene_args(scene)
    ybar = np.ascontiguousarray(ybar, np.float64)
    grad = np.zeros((len(pa), 12))
    y = np.zeros((int(goff[-1]), 8))
    xi_p = None
    if xi is not None:
        xi = np.ascontiguousarray(xi, np.float64)
        xi_p = _ptr(xi)
    lib().ccmo_gradient(g.ref(), len(pa), _ptr(pa), _ptr(pb), _ptr(A), _ptr(B), C.byref(prm),
                        _ptr(goff), _ptr(ybar), xi_p, _ptr(grad), _ptr(y), threads)
    return grad, y


def hvp(scene, ybar, u, prm=None, threads=0):
    """(grad [n,12], H u [n,12], J u [G,8], y [G,8]) in the twist chart at xi = 0."""
    prm = prm or params()
    g = _Packed(scene.geom)
    pa, pb, A, B, goff = _scene_args(scene)
    ybar = np.ascontiguousarray(ybar, np.float64)
    u = np.ascontiguousarray(u, np.float64)
    grad = np.zeros((len(pa), 12))
    hv = np.zeros((len(pa), 12))
    jv = np.zeros((int(goff[-1]), 8))
    y = np.zeros((int(goff[-1]), 8))
    lib().ccmo_hvp(g.ref(), len(pa), _ptr(pa), _ptr(pb), _ptr(A), _ptr(B), C.byref(prm),
                   _ptr(goff), _ptr(ybar), _ptr(u), _ptr(grad), _ptr(hv), _ptr(jv), _ptr(y),
                   threads)
    return grad, hv, jv, y


def sdf(planes, x, tau):
    """(phi, grad phi) of one piece at one point (Sec. 3, smooth intersection)."""
    planes = np.ascontiguousarray(planes, np.float64).reshape(-1, 4)
    x = np.ascontiguousarray(x, np.float64).reshape(3)
    g = np.zeros(3)
    phi = lib().ccmo_sdf(_ptr(planes), len(planes), _ptr(x), float(tau), _ptr(g))
    return phi, g


def edge_point(planes, vI, vII, prm=None):
    """(p^e, (alpha_I, alpha_II, clipped_I, clipped_II)) of one edge (Sec. 4.2)."""
    prm = prm or params()
    planes = np.ascontiguousarray(planes, np.float64).reshape(-1, 4)
    a = np.ascontiguousarray(vI, np.float64).reshape(3)
    b = np.ascontiguousarray(vII, np.float64).reshape(3)
    pe = np.zeros(3)
    al = np.zeros(4)
    lib().ccmo_edge_point(_ptr(planes), len(planes), _ptr(a), _ptr(b), C.byref(prm),
                          _ptr(pe), _ptr(al))
    return pe, al


def body_sdf(geom, body, x, tau):
    """(phi, grad phi) of the smooth union of body ``body``'s pieces at x
    (body frame; Sec. 3.1, Eq. soft_union)."""
    g = _Packed(geom)
    x = np.ascontiguousarray(x, np.float64).reshape(3)
    grad = np.zeros(3)
    phi = lib().ccmo_body_sdf(g.ref(), int(body), _ptr(x), float(tau), _ptr(grad))
    return phi, grad


def spline_u(t):
    """The paper's cubic spline basis u(t) (Sec. 3.2)."""
    return lib().ccmo_spline_u(float(t))


def spline_sdf(geom, piece, x):
    """(phi, n) of piece ``piece``'s tricubic spline SDF and normal splines at
    x (body frame; Sec. 3.2); ``geom`` must carry splines."""
    g = _Packed(geom)
    x = np.ascontiguousarray(x, np.float64).reshape(3)
    n = np.zeros(3)
    phi = lib().ccmo_spline_sdf(g.ref(), int(piece), _ptr(x), _ptr(n))
    return phi, n


def transition(d, d_max=0.01, eps=0.01):
    return lib().ccmo_transition(float(d), float(d_max), float(eps))


def softclip(x, lo, hi, tau):
    return lib().ccmo_softclip(float(x), float(lo), float(hi), float(tau))


def softplus(x, tau):
    return lib().ccmo_softplus(float(x), float(tau))


def sigmoid(x):
    return lib().ccmo_sigmoid(float(x))


def pair_contacts(scene, i=0, prm=None):
    """Every contact of pair ``i``: rows (group, phi, f, d_c, p_w(3), n_w(3))."""
    prm = prm or params()
    g = _Packed(scene.geom)
    A = np.ascontiguousarray(scene.pose_a[i], np.float64)
    B = np.ascontiguousarray(scene.pose_b[i], np.float64)
    bA, bB = int(scene.pair_a[i]), int(scene.pair_b[i])
    n = lib().ccmo_pair_contacts(g.ref(), bA, bB, _ptr(A), _ptr(B), C.byref(prm), None, 0)
    rows = np.zeros((n, 10))
    lib().ccmo_pair_contacts(g.ref(), bA, bB, _ptr(A), _ptr(B), C.byref(prm), _ptr(rows), n)
    return rows
