"""Seeded synthetic scenes: convex-decomposed bodies and rigid poses.

This module only *generates inputs*: meshes of convex pieces (vertices, face
planes, edges), body pairs and rigid poses.  It holds none of the contact
method's arithmetic (no smooth SDF, sphere trace, mollifier or blend); both the
CUDA path and the FP64 oracle consume what it returns.

Geometry conventions (Sec. 3, PSQ paragraph): every piece is a convex polytope
given by its hull vertices, its face planes ``(n, h)`` with ``n`` the unit
outward normal so that ``n.x + h`` is negative inside, and its edges as pairs of
piece-local vertex indices.  Poses are ``[n, 12]`` float32 rows: the row-major
rotation ``R`` (9 values) followed by the translation ``t`` (3 values); a pose
maps body-frame points to world points, ``x_w = R x + t``.

Workloads (all seeded):
  * ``cube_pair_scene``   -- unit cubes, one piece each, 64 poses with exact
                             box-box (15-axis SAT) penetration depth ~ U[0, 0.05].
  * ``hull_env_scene``    -- environments of two bodies with 8 pieces each; a
                             piece is the convex hull of 64 points N(c, 0.05^2),
                             c ~ N(0, 0.1^2) per axis; 70 % of the environments
                             penetrate by U[0, 0.02], 30 % are separated by a
                             max-plane gap U[0, 0.02].
  * ``uneven_scene``      -- pieces per body log-uniform in [1, 64], hull points
                             per piece log-uniform in [8, 512], same placement.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Geometry", "Scene", "SplineSet", "attach_splines", "fit_spline", "polytope_sdf", "unit_cube_piece", "hull_piece", "random_rotations",
    "geometry_from_bodies", "cube_pair_scene", "hull_env_scene", "uneven_scene",
    "log_uniform_int", "box_penetration_depth",
]


# ----------------------------------------------------------------------------
# containers
# ----------------------------------------------------------------------------
@dataclass
class Geometry:
    """A set of bodies; each body is a list of convex pieces (flat SoA arrays).

    ``body_piece_off[b] .. body_piece_off[b+1]`` are the pieces of body ``b``;
    ``piece_v_off``/``piece_f_off``/``piece_e_off`` index ``verts``/``planes``/
    ``edges`` the same way.  Edge indices are local to their piece.
    """
    body_piece_off: np.ndarray  # int64 [nb+1]
    piece_v_off: np.ndarray     # int64 [np+1]
    piece_f_off: np.ndarray     # int64 [np+1]
    piece_e_off: np.ndarray     # int64 [np+1]
    verts: np.ndarray           # float32 [V, 3]
    planes: np.ndarray          # float32 [F, 4]  (nx, ny, nz, h)
    edges: np.ndarray           # int32   [E, 2]  piece-local vertex indices
    splines: "SplineSet | None" = None   # optional tricubic spline SDF per piece

    @property
    def n_bodies(self) -> int:
        return len(self.body_piece_off) - 1

    @property
    def n_pieces(self) -> int:
        return len(self.piece_v_off) - 1

    def pieces_of(self, b: int) -> range:
        return range(int(self.body_piece_off[b]), int(self.body_piece_off[b + 1]))

    def piece(self, p: int):
        """(verts [V,3], planes [F,4], edges [E,2]) of piece ``p``."""
        v0, v1 = self.piece_v_off[p], self.piece_v_off[p + 1]
        f0, f1 = self.piece_f_off[p], self.piece_f_off[p + 1]
        e0, e1 = self.piece_e_off[p], self.piece_e_off[p + 1]
        return self.verts[v0:v1], self.planes[f0:f1], self.edges[e0:e1]

    def body_pieces(self, b: int):
        return [self.piece(p) for p in self.pieces_of(b)]

    def subset(self, bodies) -> "Geometry":
        """Geometry holding only ``bodies`` (in that order)."""
        return geometry_from_bodies([self.body_pieces(int(b)) for b in bodies])


@dataclass
class SplineSet:
    """Tricubic spline SDFs of a geometry's pieces (Sec. 3.2 representation).

    Piece p has a voxel grid with origin ``grid[p, :3]``, voxel size
    ``grid[p, 3]`` and ``dims[p, :3]`` voxels per axis; its coefficients are
    the rows ``coef[dims[p, 3] : dims[p, 3] + (nx+3)(ny+3)(nz+3)]`` in
    (x, y, z) order with z fastest, each row (phi, n_x, n_y, n_z): the SDF
    spline and the three normal splines.  Coefficient k of an axis belongs to
    grid node k - 1."""
    grid: np.ndarray            # float32 [P, 4]
    dims: np.ndarray            # int64   [P, 4]
    coef: np.ndarray            # float32 [rows, 4]


@dataclass
class Scene:
    """Body pairs with poses.  ``pair_a[i], pair_b[i]`` are body indices."""
    geom: Geometry
    pair_a: np.ndarray          # int64 [n]
    pair_b: np.ndarray          # int64 [n]
    pose_a: np.ndarray          # float32 [n, 12]
    pose_b: np.ndarray          # float32 [n, 12]
    meta: dict = field(default_factory=dict)

    @property
    def n_pairs(self) -> int:
        return len(self.pair_a)

    def group_offsets(self) -> np.ndarray:
        """int64 [n+1]: pair i owns groups [off[i], off[i+1]); the first
        N_A groups are the pieces of body A, then the N_B pieces of body B."""
        npb = np.diff(self.geom.body_piece_off)
        cnt = npb[self.pair_a] + npb[self.pair_b]
        return np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)

    def piece_pairs(self) -> int:
        npb = np.diff(self.geom.body_piece_off)
        return int(np.sum(npb[self.pair_a] * npb[self.pair_b]))

    def take(self, idx) -> "Scene":
        """Sub-scene of the pairs ``idx`` (geometry is shared, not copied)."""
        idx = np.asarray(idx, dtype=np.int64)
        return Scene(self.geom, self.pair_a[idx], self.pair_b[idx],
                     self.pose_a[idx].copy(), self.pose_b[idx].copy(), dict(self.meta))


def geometry_from_bodies(bodies) -> Geometry:
    """Pack ``bodies`` (list of list of (verts, planes, edges)) into SoA."""
    bpo = [0]
    pvo, pfo, peo = [0], [0], [0]
    V, F, E = [], [], []
    for pieces in bodies:
        for (v, f, e) in pieces:
            V.append(np.asarray(v, np.float32).reshape(-1, 3))
            F.append(np.asarray(f, np.float32).reshape(-1, 4))
            E.append(np.asarray(e, np.int32).reshape(-1, 2))
            pvo.append(pvo[-1] + len(V[-1]))
            pfo.append(pfo[-1] + len(F[-1]))
            peo.append(peo[-1] + len(E[-1]))
        bpo.append(bpo[-1] + len(pieces))
    return Geometry(
        np.asarray(bpo, np.int64), np.asarray(pvo, np.int64),
        np.asarray(pfo, np.int64), np.asarray(peo, np.int64),
        np.concatenate(V) if V else np.zeros((0, 3), np.float32),
        np.concatenate(F) if F else np.zeros((0, 4), np.float32),
        np.concatenate(E) if E else np.zeros((0, 2), np.int32))


# ----------------------------------------------------------------------------
# pieces
# ----------------------------------------------------------------------------
def unit_cube_piece(half=0.5, center=(0.0, 0.0, 0.0)):
    """Axis-aligned cube: 8 vertices, 6 face planes, 12 edges."""
    c = np.asarray(center, np.float64)
    verts = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)],
                     np.float64) * half + c
    planes = []
    for ax in range(3):
        for s in (-1.0, 1.0):
            n = np.zeros(3)
            n[ax] = s
            planes.append([*n, -(half + s * c[ax])])
    edges = []
    for i in range(8):
        for j in range(i + 1, 8):
            if np.sum(np.abs(verts[i] - verts[j]) > 1e-12) == 1:
                edges.append([i, j])
    return verts.astype(np.float32), np.asarray(planes, np.float32), np.asarray(edges, np.int32)


def hull_piece(points):
    """Convex hull of ``points`` [k,3] -> (verts, planes, edges).

    Uses Qhull through scipy (input preparation, not the method).  Facets are
    triangles; nearly identical facet planes (coplanar triangles) are merged
    so that each face plane appears once.
    """
    from scipy.spatial import ConvexHull

    pts = np.asarray(points, np.float64)
    hull = ConvexHull(pts)
    vid = np.asarray(hull.vertices)
    remap = -np.ones(len(pts), np.int64)
    remap[vid] = np.arange(len(vid))
    verts = pts[vid]
    eqs = hull.equations  # (n, offset): n.x + offset <= 0 inside, n unit outward
    same = np.abs(eqs[:, None, :] - eqs[None, :, :]).max(-1) < 1e-9
    first = ~np.tril(same, -1).any(1)          # keep the first of each coplanar set
    planes = eqs[first]
    tri = remap[hull.simplices]                                   # [T,3]
    pairs = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [0, 2]]])
    owner = np.tile(np.arange(len(tri)), 3)
    pairs.sort(axis=1)
    key = pairs[:, 0] * (len(verts) + 1) + pairs[:, 1]
    if len(planes) != len(eqs):
        # a segment shared by two coplanar triangles is a face diagonal, not an edge
        order = np.argsort(key, kind="stable")
        k, o = key[order], owner[order]
        dup = (k[1:] == k[:-1]) & (np.abs(eqs[o[1:]] - eqs[o[:-1]]).max(-1) < 1e-9)
        drop = set(k[1:][dup].tolist())
        keep = np.array([kk not in drop for kk in key])
        pairs, key = pairs[keep], key[keep]
    _, first = np.unique(key, return_index=True)
    edges = pairs[np.sort(first)]
    edges = edges[np.lexsort((edges[:, 1], edges[:, 0]))].astype(np.int32)
    return verts.astype(np.float32), np.asarray(planes, np.float32), edges


# ----------------------------------------------------------------------------
# spline SDFs of pieces (asset preparation: the values the paper's linear
# interpolation system is solved for; evaluating the spline is the method's)
# ----------------------------------------------------------------------------
def polytope_sdf(points, verts, planes):
    """Exact signed distance and its unit gradient of the convex polytope
    conv(verts) with face planes ``planes`` at ``points`` [m, 3] (float64):
    inside, the largest plane value and that plane's normal; outside, the
    distance to the nearest boundary point (over the hull's triangles) and
    the direction away from it."""
    from scipy.spatial import ConvexHull
    X = np.asarray(points, np.float64)
    V = np.asarray(verts, np.float64)
    P = np.asarray(planes, np.float64)
    vals = X @ P[:, :3].T + P[:, 3]
    k = np.argmax(vals, axis=1)
    phi = vals[np.arange(len(X)), k]
    nrm = P[k, :3].copy()
    out = phi > 0
    if out.any():
        Y = X[out]
        best = np.full(len(Y), np.inf)
        cp = np.zeros_like(Y)
        for tri in ConvexHull(V).simplices:
            q = _closest_on_triangles(Y, V[tri[0]], V[tri[1]], V[tri[2]])
            d = np.linalg.norm(Y - q, axis=1)
            better = d < best
            best[better] = d[better]
            cp[better] = q[better]
        phi[out] = best
        nrm[out] = (Y - cp) / best[:, None]
    return phi, nrm


def _closest_on_triangles(X, a, b, c):
    """Closest points of triangle abc to the points X [m, 3] (Voronoi regions
    of the vertices, edges and face, in the standard order)."""
    ab, ac = b - a, c - a
    ap = X - a
    d1, d2 = ap @ ab, ap @ ac
    bp = X - b
    d3, d4 = bp @ ab, bp @ ac
    cp = X - c
    d5, d6 = cp @ ab, cp @ ac
    va = d3 * d6 - d5 * d4
    vb = d5 * d2 - d1 * d6
    vc = d1 * d4 - d3 * d2
    den = np.where(va + vb + vc == 0, 1.0, va + vb + vc)
    v = vb / den
    w = vc / den
    res = a + v[:, None] * ab + w[:, None] * ac                       # face
    with np.errstate(divide="ignore", invalid="ignore"):
        t_ab = d1 / (d1 - d3)
        t_ac = d2 / (d2 - d6)
        t_bc = (d4 - d3) / ((d4 - d3) + (d5 - d6))
    e_ab = (vc <= 0) & (d1 >= 0) & (d3 <= 0)
    e_ac = (vb <= 0) & (d2 >= 0) & (d6 <= 0)
    e_bc = (va <= 0) & ((d4 - d3) >= 0) & ((d5 - d6) >= 0)
    # regions tested in the order a, b, ab, c, ac, bc (first match wins):
    # applied here from the last to the first
    res = np.where(e_bc[:, None], b + np.nan_to_num(t_bc)[:, None] * (c - b), res)
    res = np.where(e_ac[:, None], a + np.nan_to_num(t_ac)[:, None] * ac, res)
    res = np.where(((d6 >= 0) & (d5 <= d6))[:, None], c, res)
    res = np.where(e_ab[:, None], a + np.nan_to_num(t_ab)[:, None] * ab, res)
    res = np.where(((d3 >= 0) & (d4 <= d3))[:, None], b, res)
    res = np.where(((d1 <= 0) & (d2 <= 0))[:, None], a, res)
    return res


def spline_interp_matrix(n):
    """[n+3, n+1]: coefficients of the 1-D cubic spline through the values at
    the n + 1 nodes of n voxels (Sec. 3.2: c_k + 4 c_{k+1} + c_{k+2} = f_k,
    the paper's basis centred on the nodes), closed by a zero second
    derivative at both ends (c_0 - 2 c_1 + c_2 = 0 and the same at node n)."""
    A = np.zeros((n + 3, n + 3))
    A[0, 0:3] = [1.0, -2.0, 1.0]
    for i in range(n + 1):
        A[i + 1, i:i + 3] = [1.0, 4.0, 1.0]
    A[n + 2, n:n + 3] = [1.0, -2.0, 1.0]
    return np.linalg.inv(A)[:, 1:n + 2]


def fit_spline(field, origin, h, dims):
    """Coefficients [(nx+3)(ny+3)(nz+3), C] of the tricubic splines through
    ``field(points [m,3]) -> values [m, C]`` at the nodes of the grid
    (``dims`` voxels of size ``h`` from ``origin``), one axis at a time."""
    nx, ny, nz = (int(d) for d in dims)
    gx = origin[0] + h * np.arange(nx + 1)
    gy = origin[1] + h * np.arange(ny + 1)
    gz = origin[2] + h * np.arange(nz + 1)
    pts = np.stack(np.meshgrid(gx, gy, gz, indexing="ij"), -1).reshape(-1, 3)
    F = np.asarray(field(pts), np.float64).reshape(nx + 1, ny + 1, nz + 1, -1)
    C = np.einsum("ai,ijkc->ajkc", spline_interp_matrix(nx), F)
    C = np.einsum("bj,ajkc->abkc", spline_interp_matrix(ny), C)
    C = np.einsum("ck,abkq->abcq", spline_interp_matrix(nz), C)
    return C.reshape(-1, C.shape[-1])


def piece_spline(verts, planes, voxels=16, margin=0.03):
    """Grid (origin, h), voxel counts and [rows, 4] coefficients of one
    piece's spline SDF and normal splines, fitted to its exact polytope SDF
    on its bounding box grown by ``margin`` (cubic voxels, ``voxels`` along
    the longest side)."""
    V = np.asarray(verts, np.float64)
    lo, hi = V.min(0) - margin, V.max(0) + margin
    h = float((hi - lo).max()) / voxels
    dims = np.maximum(1, np.ceil((hi - lo) / h - 1e-9)).astype(np.int64)
    coef = fit_spline(lambda p: np.concatenate(
        [a.reshape(len(p), -1) for a in polytope_sdf(p, V, planes)], 1), lo, h, dims)
    return lo, h, dims, coef


def attach_splines(geom, voxels=16, margin=None):
    """``geom`` with a SplineSet of every piece (margin default: 2 voxel
    sizes' worth of the piece, at least 0.03)."""
    grid, dims, coefs, row = [], [], [], 0
    for p in range(geom.n_pieces):
        v, f, _ = geom.piece(p)
        ext = float((v.max(0) - v.min(0)).max())
        m = margin if margin is not None else max(0.03, 2.0 * ext / voxels)
        o, h, d, c = piece_spline(v, f, voxels, m)
        grid.append([*o, h])
        dims.append([*d, row])
        coefs.append(c)
        row += len(c)
    geom.splines = SplineSet(np.asarray(grid, np.float32), np.asarray(dims, np.int64),
                             np.concatenate(coefs).astype(np.float32))
    return geom


# ----------------------------------------------------------------------------
# poses
# ----------------------------------------------------------------------------
def random_rotations(rng, n):
    """Uniform rotations on SO(3) (Shoemake: normalised 4-D Gaussian quaternion)."""
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def random_unit_vectors(rng, n):
    u = rng.normal(size=(n, 3))
    return u / np.linalg.norm(u, axis=1, keepdims=True)


def pack_pose(R, t):
    """[n,3,3], [n,3] -> float32 [n,12]."""
    R = np.asarray(R, np.float64).reshape(-1, 9)
    t = np.asarray(t, np.float64).reshape(-1, 3)
    return np.concatenate([R, t], axis=1).astype(np.float32)


def unpack_pose(P):
    P = np.asarray(P, np.float64)
    return P[:, :9].reshape(-1, 3, 3), P[:, 9:12]


def log_uniform_int(rng, lo, hi, size):
    """Integers log-uniform in [lo, hi]: floor(exp(U(ln lo, ln(hi + 1))))."""
    x = np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi + 1), size=size))).astype(np.int64)
    return np.clip(x, lo, hi)


def _world_frame(rng, RA, tA, RB, tB):
    """Apply one common random rigid motion (offset in [-1,1]^3) per pair."""
    n = len(RA)
    Rw = random_rotations(rng, n)
    tw = rng.uniform(-1.0, 1.0, size=(n, 3))
    RA2 = Rw @ RA
    RB2 = Rw @ RB
    tA2 = np.einsum("nij,nj->ni", Rw, tA) + tw
    tB2 = np.einsum("nij,nj->ni", Rw, tB) + tw
    return RA2, tA2, RB2, tB2


# ----------------------------------------------------------------------------
# config: unit cube pair
# ----------------------------------------------------------------------------
def box_penetration_depth(RA, cA, eA, RB, cB, eB):
    """Exact penetration depth of two boxes by the separating-axis theorem
    over the 15 candidate axes (positive = overlap)."""
    axes = [RA[:, i] for i in range(3)] + [RB[:, j] for j in range(3)]
    for i in range(3):
        for j in range(3):
            c = np.cross(RA[:, i], RB[:, j])
            nc = np.linalg.norm(c)
            if nc > 1e-9:
                axes.append(c / nc)
    d = cB - cA
    best = np.inf
    for L in axes:
        rA = np.sum(eA * np.abs(RA.T @ L))
        rB = np.sum(eB * np.abs(RB.T @ L))
        best = min(best, rA + rB - abs(d @ L))
    return best


def cube_pair_scene(seed=1, n_poses=64, depth_range=(0.0, 0.05), half=0.5):
    """One pair of unit cubes under ``n_poses`` seeded relative poses.

    Rotation of B uniform on SO(3); B is translated along a uniform random
    direction until the exact (SAT) penetration depth equals delta ~ U(range),
    by bisection on the distance (monotone for centred symmetric pairs); a
    common random rigid motion is then applied to both bodies.
    """
    rng = np.random.default_rng(seed)
    geom = geometry_from_bodies([[unit_cube_piece(half)], [unit_cube_piece(half)]])
    RA = np.repeat(np.eye(3)[None], n_poses, 0)
    RB = random_rotations(rng, n_poses)
    u = random_unit_vectors(rng, n_poses)
    delta = rng.uniform(*depth_range, size=n_poses)
    e = np.full(3, half)
    tA = np.zeros((n_poses, 3))
    tB = np.zeros((n_poses, 3))
    for i in range(n_poses):
        lo, hi = 0.0, 4.0 * half * np.sqrt(3.0)
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            dep = box_penetration_depth(RA[i], np.zeros(3), e, RB[i], mid * u[i], e)
            if dep > delta[i]:
                lo = mid
            else:
                hi = mid
        tB[i] = 0.5 * (lo + hi) * u[i]
    RA, tA, RB, tB = _world_frame(rng, RA, tA, RB, tB)
    return Scene(geom, np.zeros(n_poses, np.int64), np.ones(n_poses, np.int64),
                 pack_pose(RA, tA), pack_pose(RB, tB),
                 {"workload": "cube pair", "depth": delta, "seed": seed})


# ----------------------------------------------------------------------------
# configs: hull environments
# ----------------------------------------------------------------------------
def _random_hull_body(rng, n_pieces, n_points, centre_sigma=0.1, point_sigma=0.05):
    pieces = []
    for k in range(n_pieces):
        c = rng.normal(0.0, centre_sigma, size=3)
        m = int(n_points[k]) if np.ndim(n_points) else int(n_points)
        pts = rng.normal(0.0, point_sigma, size=(m, 3)) + c
        pieces.append(hull_piece(pts))
    return pieces


def _pad_body(pieces):
    """Dense padded arrays of one body for the placement search."""
    P = len(pieces)
    Vm = max(len(p[0]) for p in pieces)
    Fm = max(len(p[1]) for p in pieces)
    V = np.zeros((P, Vm, 3))
    F = np.zeros((P, Fm, 4))
    F[:, :, 3] = -np.inf          # padded plane never binds (value -inf)
    for i, (v, f, _) in enumerate(pieces):
        V[i, :len(v)] = v
        V[i, len(v):] = v[0]      # padded vertex duplicates a real one
        F[i, :len(f)] = f
    return V, F


def _sup_contact_offset(VF, FS, RF, RS, u_w, target):
    """Largest s such that some vertex of body F, translated by s*u_w in world,
    lies at max-plane value <= -target inside some piece of body S.

    For a fixed (piece a, vertex v) the max-plane value along the ray is the
    convex piecewise-linear function max_k (c_k + s d_k); its sublevel set
    {<= -target} is an interval whose upper end is min over d_k > 0 of
    (-target - c_k)/d_k.  Returns -inf if no vertex ever reaches the level.
    """
    # vertices of F in S frame at s = 0, and the motion direction in S frame
    x0 = np.einsum("ij,pvj->pvi", RS.T @ RF, VF)           # [PF, V, 3]
    du = RS.T @ u_w                                          # [3]
    n = FS[..., :3]                                          # [PS, F, 3]
    h = FS[..., 3]
    c = np.einsum("afk,pvk->apvf", n, x0) + h[:, None, None, :]   # [PS,PF,V,F]
    d = np.einsum("afk,k->af", n, du)[:, None, None, :] * np.ones_like(c)
    lvl = -target
    with np.errstate(divide="ignore", invalid="ignore"):
        r = (lvl - c) / d
        hi = np.where(d > 0, r, np.inf).min(-1)
        lo = np.where(d < 0, r, -np.inf).max(-1)
        ok0 = np.where(d == 0, c <= lvl, True).all(-1)
    feas = ok0 & (lo <= hi) & np.isfinite(hi)
    if not feas.any():
        return -np.inf
    return hi[feas].max()


def _place_pair(rng_dir, bodyA, bodyB, RA, RB, target):
    """World translation of B (A at the origin) so that the deepest
    vertex-in-piece max-plane depth equals ``target`` (negative = gap)."""
    VA, FA = bodyA
    VB, FB = bodyB
    u = rng_dir
    sB = _sup_contact_offset(VB, FA, RB, RA, u, target)     # B's vertices in A
    sA = _sup_contact_offset(VA, FB, RA, RB, -u, target)    # A's vertices in B
    s = max(sB, sA)
    return s * u


def _make_env(args):
    """One environment from its own seed stream (independent of batching)."""
    seed, e, pieces, npts_spec, sep_frac, depth_range, gap_range = args
    rng = np.random.default_rng([seed, e])
    bodies = []
    for s in range(2):
        P = int(pieces[s])
        if npts_spec[0] == "fixed":
            npts = np.full(P, int(npts_spec[1]))
        else:
            npts = log_uniform_int(rng, npts_spec[1], npts_spec[2], size=P)
        bodies.append(_random_hull_body(rng, P, npts))
    RA = random_rotations(rng, 1)[0]
    RB = random_rotations(rng, 1)[0]
    u = random_unit_vectors(rng, 1)[0]
    separated = bool(rng.uniform() < sep_frac)
    target = -rng.uniform(*gap_range) if separated else rng.uniform(*depth_range)
    tB = _place_pair(u, _pad_body(bodies[0]), _pad_body(bodies[1]), RA, RB, target)
    RA2, tA2, RB2, tB2 = _world_frame(rng, RA[None], np.zeros((1, 3)), RB[None], tB[None])
    return bodies, RA2[0], tA2[0], RB2[0], tB2[0], target, separated


def _map_envs(jobs, workers):
    """Runs the per-environment jobs; ``workers`` None or 1 = serial, 0 = one
    spawned process per host core (at most 32).  A script that asks for worker
    processes must guard its entry point with ``if __name__ == "__main__"``,
    since spawned workers import the main module."""
    if workers == 0:
        import os
        workers = min(len(os.sched_getaffinity(0)), 32)
    if workers is None or workers <= 1 or len(jobs) < 64:
        return [_make_env(j) for j in jobs]
    import multiprocessing as mp
    # spawn: never fork a process that may already hold a CUDA context
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_make_env, jobs, chunksize=max(1, len(jobs) // (8 * workers)))


def hull_env_scene(seed=2, n_envs=4096, pieces_per_body=8, points_per_hull=64,
                   sep_frac=0.3, depth_range=(0.0, 0.02), gap_range=(0.0, 0.02),
                   workers=None):
    """``n_envs`` environments of two bodies with ``pieces_per_body`` pieces.

    Each piece is the hull of ``points_per_hull`` points N(c, 0.05^2), with the
    piece centre c ~ N(0, 0.1^2) per axis.  Bodies get uniform rotations; B is
    translated along a uniform direction so that the deepest vertex-in-piece
    max-plane depth is delta ~ U(depth_range) (70 %) or -g, g ~ U(gap_range)
    (30 %, separated); a common random rigid motion is applied to both.
    Every environment draws from its own seed stream ``(seed, env)``, so a
    scene does not depend on how many worker processes generated it.
    ``points_per_hull`` is an int or ``("log-uniform", lo, hi)``.
    """
    if np.ndim(pieces_per_body) == 0:
        pieces = np.full((n_envs, 2), int(pieces_per_body), np.int64)
    else:
        pieces = np.asarray(pieces_per_body, np.int64).reshape(n_envs, 2)
    spec = ("fixed", int(points_per_hull)) if np.ndim(points_per_hull) == 0 \
        else tuple(points_per_hull)
    jobs = [(seed, e, tuple(pieces[e]), spec, sep_frac, depth_range, gap_range)
            for e in range(n_envs)]
    res = _map_envs(jobs, workers)
    bodies = [b for r in res for b in r[0]]
    geom = geometry_from_bodies(bodies)
    RA = np.stack([r[1] for r in res])
    tA = np.stack([r[2] for r in res])
    RB = np.stack([r[3] for r in res])
    tB = np.stack([r[4] for r in res])
    pa = np.arange(0, 2 * n_envs, 2, dtype=np.int64)
    return Scene(geom, pa, pa + 1, pack_pose(RA, tA), pack_pose(RB, tB),
                 {"workload": "hull envs", "seed": seed,
                  "target_depth": np.array([r[5] for r in res]),
                  "separated": np.array([r[6] for r in res])})


def _sup_offset_pruned(bodyF, bodyS, RF, RS, u_w, target, shift_w=None):
    """_sup_contact_offset restricted to the piece pairs that can matter.

    For a vertex of piece f to reach max-plane level -target inside piece s,
    the vertex (within r_f of the centre c_f) must come within r_s +
    max(0, -target) of c_s, so along the ray its offset is at most
    (c_s - c_f).u + r_s + r_f + max(0, -target) (all in S's frame).  Piece
    pairs are visited by decreasing bound and the scan stops once the bound
    falls below the best offset found: the result equals the full search.
    ``shift_w`` (world) translates body F before the motion along u_w.
    """
    VF, FF, cF, rF = bodyF
    VS, FS, cS, rS = bodyS
    Rrel = RS.T @ RF
    du = RS.T @ u_w
    sh = np.zeros(3) if shift_w is None else RS.T @ shift_w
    cFs = cF @ Rrel.T + sh                 # feature piece centres in S frame (at s = 0)
    bound = (cS @ du)[:, None] - (cFs @ du)[None, :] + rS[:, None] + rF[None, :] + max(0.0, -target)
    order = np.argsort(-bound, axis=None)
    best = -np.inf
    lvl = -target
    for k in order:
        a, b = divmod(int(k), bound.shape[1])
        if bound[a, b] <= best:
            break
        x0 = VF[b] @ Rrel.T + sh                                # [V, 3]
        n = FS[a][:, :3]
        h = FS[a][:, 3]
        c = x0 @ n.T + h                                        # [V, F]
        d = np.broadcast_to(n @ du, c.shape)
        with np.errstate(divide="ignore", invalid="ignore"):
            r = (lvl - c) / d
            hi = np.where(d > 0, r, np.inf).min(-1)
            lo = np.where(d < 0, r, -np.inf).max(-1)
            ok0 = np.where(d == 0, c <= lvl, True).all(-1)
        feas = ok0 & (lo <= hi) & np.isfinite(hi)
        if feas.any():
            best = max(best, hi[feas].max())
    return best


def _body_arrays(pieces):
    """(vertices, planes, centres, radii) lists of one body for the placement."""
    V = [p[0].astype(np.float64) for p in pieces]
    F = [p[1].astype(np.float64) for p in pieces]
    c = np.array([v.mean(0) for v in V])
    r = np.array([np.linalg.norm(v - cc, axis=1).max() for v, cc in zip(V, c)])
    return V, F, c, r


def _make_pool_body(args):
    seed, k, P, lo, hi = args
    rng = np.random.default_rng([seed, 1 << 20, k])
    npts = log_uniform_int(rng, lo, hi, size=P)
    return _random_hull_body(rng, P, npts)


def _place_pool_pair(args):
    seed, i, bodyA, bodyB, sep_frac, depth_range, gap_range = args
    rng = np.random.default_rng([seed, 1 << 21, i])
    RA = random_rotations(rng, 1)[0]
    RB = random_rotations(rng, 1)[0]
    u = random_unit_vectors(rng, 1)[0]
    separated = bool(rng.uniform() < sep_frac)
    target = -rng.uniform(*gap_range) if separated else rng.uniform(*depth_range)
    sB = _sup_offset_pruned(bodyB, bodyA, RB, RA, u, target)      # B's vertices in A
    sA = _sup_offset_pruned(bodyA, bodyB, RA, RB, -u, target)     # A's vertices in B
    p = np.zeros(3)
    tries = 0
    while not np.isfinite(max(sA, sB)):
        # no vertex line along u meets the other body (small pieces far off
        # the line through the origin), or the target is deeper than any
        # piece can hold: shift B across u so that a random piece of each
        # body lies on one line, and halve a penetration target every four
        # tries
        if tries == 64:
            raise RuntimeError(f"pair {i}: no placement found")
        if tries % 4 == 3 and target > 0:
            target *= 0.5
        tries += 1
        a = int(rng.integers(0, len(bodyA[2])))
        b = int(rng.integers(0, len(bodyB[2])))
        delta = RA @ bodyA[2][a] - RB @ bodyB[2][b]
        p = delta - (delta @ u) * u
        sB = _sup_offset_pruned(bodyB, bodyA, RB, RA, u, target, p)
        sA = _sup_offset_pruned(bodyA, bodyB, RA, RB, -u, target, -p)
    tB = max(sA, sB) * u + p
    RA2, tA2, RB2, tB2 = _world_frame(rng, RA[None], np.zeros((1, 3)), RB[None], tB[None])
    return RA2[0], tA2[0], RB2[0], tB2[0], target, separated


def _pmap(fn, jobs, workers):
    if workers == 0:
        import os
        workers = min(len(os.sched_getaffinity(0)), 32)
    if workers is None or workers <= 1 or len(jobs) < 64:
        return [fn(j) for j in jobs]
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(fn, jobs, chunksize=max(1, len(jobs) // (8 * workers)))


def uneven_scene(seed=4, n_pairs=65536, max_pieces=64, min_points=8, max_points=512,
                 pool_bodies=8192, sep_frac=0.3, depth_range=(0.0, 0.02),
                 gap_range=(0.0, 0.02), workers=None):
    """Uneven batch: pieces per body log-uniform in [1, max_pieces], hull
    points per piece log-uniform in [min_points, max_points], the Gaussian
    hull generation and placement of ``hull_env_scene``.

    Bodies come from a seeded pool of ``pool_bodies`` distinct bodies (drawn
    with replacement for the two sides of every pair) so that generating
    65,536 pairs does not need ~2M convex hulls; every pair gets its own
    rotations, direction and target depth.  Returns a Scene whose geometry is
    the pool (pair_a / pair_b index into it)."""
    rng = np.random.default_rng(seed)
    pool_n = min(pool_bodies, 2 * n_pairs)
    pieces = log_uniform_int(rng, 1, max_pieces, size=pool_n)
    bodies = _pmap(_make_pool_body, [(seed, k, int(pieces[k]), min_points, max_points)
                                     for k in range(pool_n)], workers)
    arrays = [_body_arrays(b) for b in bodies]
    pa = rng.integers(0, pool_n, size=n_pairs)
    pb = rng.integers(0, pool_n, size=n_pairs)
    jobs = [(seed, i, arrays[pa[i]], arrays[pb[i]], sep_frac, depth_range, gap_range)
            for i in range(n_pairs)]
    res = _pmap(_place_pool_pair, jobs, workers)
    geom = geometry_from_bodies(bodies)
    RA = np.stack([r[0] for r in res])
    tA = np.stack([r[1] for r in res])
    RB = np.stack([r[2] for r in res])
    tB = np.stack([r[3] for r in res])
    return Scene(geom, pa.astype(np.int64), pb.astype(np.int64), pack_pose(RA, tA),
                 pack_pose(RB, tB),
                 {"workload": "uneven", "seed": seed, "pool_bodies": pool_n,
                  "target_depth": np.array([r[4] for r in res]),
                  "separated": np.array([r[5] for r in res])})
