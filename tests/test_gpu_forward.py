"""Parity of the CUDA forward path (through the C ABI) with the FP64 oracle."""
import numpy as np
import pytest

from gpu_util import compare, gpu_forward, oracle_params, weight_slack
from paper_2604_17538_b300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_17538_b300 import api, build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def cubes():
    return scenes.cube_pair_scene(seed=1)


@pytest.fixture(scope="module")
def hulls():
    # 96 environments of two 8-piece bodies: 1536 groups, i.e. several waves
    # of the 4-warp blocks and a ragged last block
    return scenes.hull_env_scene(seed=2, n_envs=96, workers=0)


def test_cube_pairs_match_oracle(oracle_lib, ctx, cubes):
    y = gpu_forward(cubes, ctx=ctx)
    ref = oracle_lib.forward(cubes)
    rep = compare(y, ref, "cube pairs", a_slack=weight_slack(cubes))
    print("cube pairs max err", rep)


def test_hull_envs_match_oracle(oracle_lib, ctx, hulls):
    y = gpu_forward(hulls, ctx=ctx)
    ref = oracle_lib.forward(hulls)
    rep = compare(y, ref, "hull envs", a_slack=weight_slack(hulls))
    print("hull envs max err", rep)
    assert (ref[:, 1] > 0).sum() > 50      # enough active groups to mean something


def test_culls_are_exact(ctx, hulls):
    """Evaluating every feature (no cull) gives the same blend to rounding."""
    y = gpu_forward(hulls, ctx=ctx)
    y_all = gpu_forward(hulls, params={"flags": 1}, ctx=ctx)
    compare(y, y_all, "cull vs no cull", a_slack=weight_slack(hulls))


@pytest.mark.parametrize("params", [
    {"trace_iters": 0}, {"trace_iters": 1}, {"trace_iters": 6},
    {"tau_sdf": 2e-3, "tau_blend": 1e-2, "d_max": 0.02, "gate_width": 0.015},
])
def test_other_constants(oracle_lib, ctx, hulls, params):
    sub = hulls.take(np.arange(24))
    y = gpu_forward(sub, params=params, ctx=ctx)
    ref = oracle_lib.forward(sub, oracle_params(params))
    compare(y, ref, f"params {params}", a_slack=weight_slack(sub, params))


def test_deterministic_and_batch_independent(ctx, hulls):
    y1 = gpu_forward(hulls, ctx=ctx)
    y2 = gpu_forward(hulls, ctx=ctx)
    assert np.array_equal(y1, y2)
    idx = np.array([5, 17, 60])
    alone = gpu_forward(hulls.take(idx), ctx=ctx)
    off = hulls.group_offsets()
    mix = np.concatenate([y1[off[i]:off[i + 1]] for i in idx])
    assert np.array_equal(alone, mix)


def _tetra(c, s=0.05):
    n = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float) / np.sqrt(3)
    return np.concatenate([n, (-(n @ c) - s)[:, None]], 1)


def test_degenerate_pieces(oracle_lib, ctx):
    """Single-vertex pieces without edges, single-piece bodies, and a pair
    separated far beyond d_max (empty groups)."""
    cube = scenes.unit_cube_piece(0.5)
    v = np.array([[0.1, -0.2, 0.497]])
    single = (v.astype(np.float32), _tetra(v[0]).astype(np.float32), np.zeros((0, 2), np.int32))
    # B's cube sits on A's cube (overlap 0.005), not coincident with it: two
    # coincident cubes blend opposite corner normals to a zero vector, where
    # the unit normal is undefined
    cube_b = scenes.unit_cube_piece(0.5, center=(0.3, 0.2, 0.995))
    geom = scenes.geometry_from_bodies([[cube], [single, cube_b], [cube]])
    R = scenes.random_rotations(np.random.default_rng(0), 3)
    t = np.array([[0.0, 0.0, 0.0], [0.3, 0.1, 0.2], [0.0, 0.0, 0.0]])
    pose = scenes.pack_pose(R, t)
    far = scenes.pack_pose(R, t + 10.0)
    shifted = scenes.pack_pose(R, t + [0.0, 0.3, 0.95])
    sc = scenes.Scene(geom, np.array([0, 0, 2], np.int64), np.array([1, 1, 0], np.int64),
                      np.stack([pose[0], pose[0], pose[2]]),
                      np.stack([pose[0], far[1], shifted[2]]))
    y = gpu_forward(sc, ctx=ctx)
    ref = oracle_lib.forward(sc)
    compare(y, ref, "degenerate", a_slack=weight_slack(sc))
    off = sc.group_offsets()
    assert np.all(y[off[1]:off[2], 0] == np.float32(0.01)) and np.all(y[off[1]:off[2], 1:] == 0)


def test_empty_batch(ctx):
    import torch
    from paper_2604_17538_b300 import api
    b = ctx.batch(np.zeros(0, np.uint64), np.zeros(0, np.uint64))
    pa = torch.zeros((0, 12), device="cuda")
    y = b.contacts(pa, pa)
    assert y.shape == (0, 8)
    b.close()


def test_bad_arguments_are_rejected(ctx):
    import torch
    from paper_2604_17538_b300 import abi
    with pytest.raises(abi.CcmError) as e:
        ctx.batch(np.array([12345], np.uint64), np.array([1], np.uint64))
    assert e.value.status == abi.CCM_ERR_INVALID
    sc = scenes.cube_pair_scene(seed=1, n_poses=2)
    from paper_2604_17538_b300 import api
    batch, pa, pb = api.scene_to_device(sc, ctx)
    with pytest.raises(abi.CcmError):
        batch.contacts(pa, pb, {"tau_sdf": 0.0})
    with pytest.raises(abi.CcmError):
        batch.contacts(pa, pb, {"trace_iters": 99})
    batch.close()
