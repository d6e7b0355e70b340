"""The tricubic spline-SDF forward (Sec. 3.2; CCM_FLAG_SPLINE) against the FP64
oracle, element by element with the parity bar of gpu_util: every convex piece
of the other body as its own spline SDF with normal splines, fitted to the
piece's exact polytope SDF (scenes.attach_splines)."""
import numpy as np
import pytest

from gpu_util import compare, weight_slack
from paper_2604_17538_b300 import scenes

pytestmark = pytest.mark.gpu

SPLINE, PROJECT = 8, 4


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_17538_b300 import api, build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def spline_scenes():
    cube = scenes.cube_pair_scene(seed=1, n_poses=24)
    scenes.attach_splines(cube.geom, voxels=12)
    hull = scenes.hull_env_scene(seed=2, n_envs=12, workers=0)
    scenes.attach_splines(hull.geom, voxels=12)
    return {"cube": cube, "hull": hull}


@pytest.mark.parametrize("name", ["cube", "hull"])
@pytest.mark.parametrize("flags", [SPLINE, SPLINE | PROJECT])
def test_spline_forward_matches_oracle(oracle_lib, ctx, spline_scenes, name, flags):
    import torch
    from paper_2604_17538_b300 import api
    sc = spline_scenes[name]
    handles = ctx.load_geometry(sc.geom)
    ctx.attach_splines(sc.geom, handles)
    batch = ctx.batch(handles[sc.pair_a], handles[sc.pair_b])
    pa = torch.from_numpy(np.ascontiguousarray(sc.pose_a, np.float32)).cuda()
    pb = torch.from_numpy(np.ascontiguousarray(sc.pose_b, np.float32)).cuda()
    y = batch.contacts(pa, pb, params={"flags": flags})
    torch.cuda.synchronize()
    ref = oracle_lib.forward(sc, oracle_lib.params(flags=flags))
    compare(y.double().cpu().numpy(), ref, f"spline {name} flags {flags}",
            a_slack=weight_slack(sc))
    assert np.any(ref[:, 1] > 0)
    # a different blend from the smooth-polytope SDF of the same pieces
    assert np.abs(ref - oracle_lib.forward(sc)).max() > 1e-6
    batch.close()


def test_spline_variant_needs_splines_and_is_forward_only(ctx, spline_scenes):
    import torch
    from paper_2604_17538_b300 import abi, api
    sc = scenes.hull_env_scene(seed=3, n_envs=2, workers=1)     # no splines attached
    batch, pa, pb = api.scene_to_device(sc, ctx)
    with pytest.raises(abi.CcmError) as e:
        batch.contacts(pa, pb, params={"flags": SPLINE})
    assert e.value.status == abi.CCM_ERR_INVALID and "spline" in str(e.value)
    yb = torch.zeros((batch.n_groups, 8), device="cuda")
    with pytest.raises(abi.CcmError) as e:
        batch.backward(pa, pb, yb, params={"flags": SPLINE})
    assert e.value.status == abi.CCM_ERR_INVALID
    batch.close()
