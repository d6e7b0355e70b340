"""Independent brute-force geometry used to pin the oracle (tests only).

Nothing here calls the oracle or the CUDA path: exact polytope distances by
enumerating triangles, edges and vertices, and segment/polytope clipping by
the Cyrus-Beck method.
"""
import numpy as np
from scipy.spatial import ConvexHull


def closest_on_segment(x, a, b):
    d = b - a
    t = np.clip(np.dot(x - a, d) / np.dot(d, d), 0.0, 1.0)
    return a + t * d


def closest_on_triangle(x, a, b, c):
    """Closest point of triangle abc to x: plane projection if it falls inside
    (barycentric coordinates >= 0), else the closest point of the 3 sides."""
    n = np.cross(b - a, c - a)
    n = n / np.linalg.norm(n)
    q = x - np.dot(x - a, n) * n
    # barycentric coordinates of q
    v0, v1, v2 = b - a, c - a, q - a
    d00, d01, d11 = v0 @ v0, v0 @ v1, v1 @ v1
    d20, d21 = v2 @ v0, v2 @ v1
    den = d00 * d11 - d01 * d01
    v = (d11 * d20 - d01 * d21) / den
    w = (d00 * d21 - d01 * d20) / den
    u = 1.0 - v - w
    if u >= 0 and v >= 0 and w >= 0:
        return q
    cands = [closest_on_segment(x, a, b), closest_on_segment(x, b, c), closest_on_segment(x, a, c)]
    return min(cands, key=lambda p: np.linalg.norm(x - p))


def signed_distance(x, verts):
    """Exact signed distance of x to conv(verts) by brute force over all
    boundary triangles (negative inside)."""
    V = np.asarray(verts, np.float64)
    hull = ConvexHull(V)
    best = np.inf
    for tri in hull.simplices:
        p = closest_on_triangle(x, V[tri[0]], V[tri[1]], V[tri[2]])
        best = min(best, np.linalg.norm(x - p))
    inside = np.all(hull.equations[:, :3] @ x + hull.equations[:, 3] <= 0)
    return -best if inside else best


def cyrus_beck(p0, p1, planes):
    """Parameter interval [t_in, t_out] of the segment p0 + t (p1 - p0),
    t in [0, 1], inside the polytope {n.x + h <= 0}; None if it misses."""
    d = p1 - p0
    t_in, t_out = 0.0, 1.0
    for n0, n1, n2, h in planes:
        n = np.array([n0, n1, n2])
        num = -(n @ p0 + h)
        den = n @ d
        if abs(den) < 1e-15:
            if num < 0:
                return None
            continue
        t = num / den
        if den < 0:
            t_in = max(t_in, t)
        else:
            t_out = min(t_out, t)
    if t_in > t_out:
        return None
    return t_in, t_out


def rot(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K
