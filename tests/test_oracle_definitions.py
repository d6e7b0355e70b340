"""The oracle's contacts and blends on random hulls at the default softness,
checked against the definitions they follow, evaluated independently here:

  * the piece SDF (Sec. 3, Eq. smooth-intersection with half-space SDFs) is
    tau * logsumexp((n_k . x + h_k) / tau) over the piece's planes, computed
    with scipy's logsumexp; its gradient, the contact normal, is the softmax
    of the same values applied to the plane normals;
  * a vertex contact sits at the vertex; an edge contact (Sec. 4.2) sits
    strictly inside its edge, and its SDF value and normal are the SDF's at
    that point;
  * the mollified depth (Sec. 4.3) is f phi + (1 - f) d_max with f the
    quintic smoothstep of (d_max - phi) / eps clamped to [0, 1];
  * a group (Sec. 4.4) is the softmax average of its active contacts with
    weights f exp(-d_c / tau_blend), the normal renormalised.

Points are rebuilt from the float32 poses and vertices given to the oracle:
a feature's vertex goes to world frame (x_w = R_F v + t_F), into the SDF
body's frame (x = R_S^T (x_w - t_S)), and a contact found there back to
world frame (R_S x + t_S; the float32 rotations are orthonormal only to
rounding, so this round trip is not the identity).  What these checks leave to the oracle alone is where
the soft sphere trace puts an edge's point along the edge at the default
softness, which its limits pin (tests/test_oracle_trace.py)."""
import numpy as np
import pytest
from scipy.special import logsumexp, softmax

from paper_2604_17538_b300 import scenes

TAU, D_MAX, EPS = 5e-3, 0.01, 0.01


@pytest.fixture(scope="module")
def hulls():
    return scenes.hull_env_scene(seed=2, n_envs=6, workers=1)


def _sdf(planes, x):
    v = (planes[:, :3] @ x + planes[:, 3]) / TAU
    return TAU * logsumexp(v), softmax(v) @ planes[:, :3]


def _smoothstep(phi):
    s = np.clip((D_MAX - phi) / EPS, 0.0, 1.0)
    return s ** 3 * (10.0 - 15.0 * s + 6.0 * s * s)


def _pair_pieces(g, b):
    return range(int(g.body_piece_off[b]), int(g.body_piece_off[b + 1]))


def test_contacts_and_blends_follow_their_definitions(oracle_lib, hulls):
    sc, g = hulls, hulls.geom
    V = g.verts.astype(np.float64)
    P = g.planes.astype(np.float64)
    y = oracle_lib.forward(sc)
    off = sc.group_offsets()
    n_vert = n_edge = n_active = 0
    for i in range(sc.n_pairs):
        rows = oracle_lib.pair_contacts(sc, i)
        RA, tA = scenes.unpack_pose(sc.pose_a[i:i + 1])
        RB, tB = scenes.unpack_pose(sc.pose_b[i:i + 1])
        poses = ((RA[0], tA[0]), (RB[0], tB[0]))
        bodies = (int(sc.pair_a[i]), int(sc.pair_b[i]))
        k = 0          # running row index: the oracle's order of contacts
        group = 0
        for side in (0, 1):
            (RF, tF), (RS, tS) = poses[side], poses[1 - side]
            bF, bS = bodies[side], bodies[1 - side]
            for fp in _pair_pieces(g, bF):
                v0, v1 = int(g.piece_v_off[fp]), int(g.piece_v_off[fp + 1])
                e0, e1 = int(g.piece_e_off[fp]), int(g.piece_e_off[fp + 1])
                xw = V[v0:v1] @ RF.T + tF               # world frame
                xs = (xw - tS) @ RS                     # SDF body frame
                grp = []
                for s in _pair_pieces(g, bS):
                    pl = P[int(g.piece_f_off[s]):int(g.piece_f_off[s + 1])]
                    for j in range(v1 - v0):            # vertex contacts
                        r = rows[k]; k += 1
                        phi, n = _sdf(pl, xs[j])
                        assert r[0] == group
                        assert abs(r[1] - phi) < 1e-12
                        assert np.abs(r[4:7] - (RS @ xs[j] + tS)).max() < 1e-12
                        assert np.abs(r[7:10] - RS @ n).max() < 1e-10
                        n_vert += 1
                        grp.append(r)
                    for e in g.edges[e0:e1]:            # edge contacts
                        r = rows[k]; k += 1
                        a, b = xs[e[0]], xs[e[1]]
                        p = np.linalg.solve(RS, r[4:7] - tS)
                        L = np.linalg.norm(b - a)
                        t = (p - a) @ (b - a) / L
                        assert 0.0 < t < L
                        assert np.linalg.norm(p - a - t * (b - a) / L) < 1e-12
                        phi, n = _sdf(pl, p)
                        assert abs(r[1] - phi) < 1e-12
                        assert np.abs(r[7:10] - RS @ n).max() < 1e-10
                        n_edge += 1
                        grp.append(r)
                grp = np.array(grp)
                f = _smoothstep(grp[:, 1])
                assert np.abs(grp[:, 2] - f).max() < 1e-12
                assert np.abs(grp[:, 3] - (f * grp[:, 1] + (1 - f) * D_MAX)).max() < 1e-12
                yy = y[off[i] + group]
                act = grp[grp[:, 2] > 0]
                if len(act) == 0:
                    assert yy[0] == D_MAX and np.all(yy[1:] == 0)
                else:
                    w = act[:, 2] * np.exp(-(act[:, 3] - act[:, 3].min()) / TAU)
                    w /= w.sum()
                    nb = w @ act[:, 7:10]
                    assert abs(yy[0] - w @ act[:, 3]) < 1e-12
                    assert abs(yy[1] - w @ act[:, 2]) < 1e-12
                    assert np.abs(yy[2:5] - w @ act[:, 4:7]).max() < 1e-12
                    assert np.abs(yy[5:8] - nb / np.linalg.norm(nb)).max() < 1e-10
                    n_active += 1
                group += 1
        assert k == len(rows)
    assert n_vert > 1000 and n_edge > 1000 and n_active > 5
