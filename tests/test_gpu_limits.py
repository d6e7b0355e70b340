"""Size limits and the paths they select, against the oracle:

* a body of 300 pieces (more than the 256 SDF pieces a saved record marks per
  group): the reverse passes from the record fall back to one warp per work
  item with re-gating for SDF pieces 256 and up, then a per-pair reduction;
* large pieces (convex hulls of 300 points on a sphere: 300 vertices, ~600
  planes, ~900 edges per piece): budgets raised to the largest piece, one
  piece per chunk.
"""
import numpy as np
import pytest

from gpu_util import COND_FACTOR, GRAD_RTOL, compare, fp32_sensitivity, weight_slack
from paper_2604_17538_b300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_17538_b300 import api, build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _grid_body(nx, ny, half, pitch):
    return [scenes.unit_cube_piece(half, center=((i - nx / 2) * pitch, (j - ny / 2) * pitch, 0.0))
            for i in range(nx) for j in range(ny)]


def _check(oracle_lib, ctx, sc, seed):
    import torch
    from paper_2604_17538_b300 import api
    batch, pa, pb = api.scene_to_device(sc, ctx)
    rng = np.random.default_rng(seed)
    G = batch.n_groups
    ybar = rng.normal(size=(G, 8)).astype(np.float32)
    u = rng.normal(size=(sc.n_pairs, 12))
    u = (u / np.linalg.norm(u, axis=1, keepdims=True)).astype(np.float32)
    saved = batch.saved_buffer()
    y = batch.contacts(pa, pb, saved=saved)
    yb, ut = torch.from_numpy(ybar).cuda(), torch.from_numpy(u).cuda()
    g, _, _ = batch.backward(pa, pb, yb, saved=saved)
    g2, h, _ = batch.backward(pa, pb, yb, ut, want_jvp=True, saved=saved)
    torch.cuda.synchronize()
    compare(y.double().cpu().numpy(), oracle_lib.forward(sc), "y", a_slack=weight_slack(sc))
    go, ho, _, _ = oracle_lib.hvp(sc, ybar, u)
    kg, kh = fp32_sensitivity(oracle_lib, sc, ybar, u)
    for got, ref, k, name in ((g, go, kg, "gradient"), (g2, go, kg, "gradient (dual)"),
                              (h, ho, kh, "H u")):
        got = got.double().cpu().numpy()
        assert np.all(np.isfinite(got)), name
        err = np.abs(got - ref).max(1)
        tol = np.maximum(GRAD_RTOL, COND_FACTOR * k) * np.abs(ref).max(1) + 1e-6
        assert np.all(err <= tol), (name, float((err / (np.abs(ref).max(1) + 1e-30)).max()))
    assert np.abs(go).max() > 0
    batch.close()


def test_body_of_300_pieces_against_oracle(oracle_lib, ctx):
    # A: a 15 x 20 grid of small cubes; B: one cube resting on the grid at
    # depth 0.004, so contacts involve grid pieces beyond index 256
    grid = _grid_body(15, 20, 0.02, 0.05)
    big = [scenes.unit_cube_piece(0.3)]
    geom = scenes.geometry_from_bodies([grid, big])
    assert np.diff(geom.body_piece_off)[0] == 300
    R = scenes.random_rotations(np.random.default_rng(2), 3)
    poses_a, poses_b = [], []
    for k in range(3):
        tA = np.array([0.1 * k, -0.05 * k, 0.2])
        tB = tA + R[k] @ np.array([0.11 + 0.07 * k, 0.3 - 0.02 * k, 0.02 + 0.3 - 0.004])
        PA = scenes.pack_pose(R[k:k + 1], tA[None])[0]
        PB = scenes.pack_pose(R[k:k + 1], tB[None])[0]
        poses_a.append(PA)
        poses_b.append(PB)
    sc = scenes.Scene(geom, np.zeros(3, np.int64), np.ones(3, np.int64),
                      np.stack(poses_a).astype(np.float32), np.stack(poses_b).astype(np.float32))
    _check(oracle_lib, ctx, sc, 5)
    _host_step_equals_device_calls(ctx, sc)


def _host_step_equals_device_calls(ctx, sc):
    """ccm_contacts_step_host on a batch whose reverse passes cannot run per
    pair (so they stay in order on one stream) returns the device calls'
    results bitwise."""
    import torch
    from paper_2604_17538_b300 import api
    batch, pa, pb = api.scene_to_device(sc, ctx)
    rng = np.random.default_rng(21)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory()
    yb_h = pin(rng.normal(size=(batch.n_groups, 8)))
    u_h = pin(rng.normal(size=(batch.n_pairs, 12)))
    saved = batch.saved_buffer()
    y = batch.contacts(pa, pb, saved=saved)
    g, _, _ = batch.backward(pa, pb, yb_h.cuda(), saved=saved)
    _, h, j = batch.backward(pa, pb, yb_h.cuda(), u_h.cuda(), want_jvp=True, saved=saved)
    torch.cuda.synchronize()
    ref = [t.cpu().numpy() for t in (y, g, h, j)]
    out = batch.step_host(pin(sc.pose_a), pin(sc.pose_b), yb_h, u_h, want_jvp=True)
    torch.cuda.synchronize()
    for name, a, b in zip("yghj", out, ref):
        assert np.array_equal(a.numpy(), b), name
    batch.close()


def test_large_pieces_against_oracle(oracle_lib, ctx):
    rng = np.random.default_rng(7)
    bodies = []
    for _ in range(2):
        pieces = []
        for c in rng.normal(0, 0.1, size=(3, 3)):
            pts = c + 0.1 * scenes.random_unit_vectors(rng, 300)
            pieces.append(scenes.hull_piece(pts))
        bodies.append(pieces)
    geom = scenes.geometry_from_bodies(bodies)
    nv = np.diff(geom.piece_v_off)
    assert nv.min() == 300 and np.diff(geom.piece_f_off).min() > 500
    # four random relative poses with the bodies' centres 0.1 apart: overlapping pieces
    sc0 = scenes.Scene(geom, np.zeros(4, np.int64), np.ones(4, np.int64),
                       np.zeros((4, 12), np.float32), np.zeros((4, 12), np.float32))
    R = scenes.random_rotations(rng, 8)
    t = rng.normal(0, 0.02, size=(8, 3))
    sc0.pose_a = scenes.pack_pose(R[:4], t[:4]).astype(np.float32)
    sc0.pose_b = scenes.pack_pose(R[4:], t[4:] + np.array([0.0, 0.0, 0.1])).astype(np.float32)
    _check(oracle_lib, ctx, sc0, 9)
