"""The voxel-grid broad phase (Sec. 4.3; ccm_build_voxel_grids and
CCM_FLAG_VOXEL_CULL): its culls are exact, so the outputs match those without
it (and the oracle) to float rounding while fewer plane evaluations run; and
pieces loaded after the grids were built are simply not culled by them."""
import numpy as np
import pytest

from gpu_util import compare, weight_slack
from paper_2604_17538_b300 import scenes

pytestmark = pytest.mark.gpu

VOXEL = 16


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_17538_b300 import api, build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("name", ["hull", "uneven"])
def test_voxel_culls_are_exact_and_save_plane_scans(oracle_lib, ctx, name):
    import torch
    from paper_2604_17538_b300 import api
    sc = (scenes.hull_env_scene(seed=2, n_envs=24, workers=0) if name == "hull"
          else scenes.uneven_scene(seed=4, n_pairs=64, pool_bodies=128, workers=0))
    batch, pa, pb = api.scene_to_device(sc, ctx)
    ctx.build_voxel_grids(8)
    c0 = torch.zeros(8, dtype=torch.int64, device="cuda")
    c1 = torch.zeros(8, dtype=torch.int64, device="cuda")
    y0 = batch.contacts(pa, pb, counters=c0).double().cpu().numpy()
    y1 = batch.contacts(pa, pb, params={"flags": VOXEL}, counters=c1).double().cpu().numpy()
    compare(y1, y0, f"{name} voxel cull vs plane culls", a_slack=weight_slack(sc))
    compare(y1, oracle_lib.forward(sc), f"{name} voxel cull vs oracle", a_slack=weight_slack(sc))
    c0, c1 = c0.cpu().numpy(), c1.cpu().numpy()
    assert c1[2] < c0[2], (c0, c1)             # fewer max-plane plane evaluations
    assert c1[6] == c0[6]                      # the same contacts of non-zero weight
    batch.close()


def test_pieces_loaded_after_the_grids_are_not_culled_by_them(ctx):
    import torch
    from paper_2604_17538_b300 import api
    a = scenes.hull_env_scene(seed=5, n_envs=4, workers=1)
    api.scene_to_device(a, ctx)
    ctx.build_voxel_grids(8)
    b = scenes.hull_env_scene(seed=6, n_envs=6, workers=1)      # loaded after the build
    batch, pa, pb = api.scene_to_device(b, ctx)
    y0 = batch.contacts(pa, pb).clone()
    y1 = batch.contacts(pa, pb, params={"flags": VOXEL})
    torch.cuda.synchronize()
    assert torch.equal(y0, y1)
    batch.close()
