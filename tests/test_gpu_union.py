"""The forward variants against the FP64 oracle: the body-level smooth-union
SDF (Sec. 3.1, Eq. soft_union; CCM_FLAG_BODY_UNION) and the isosurface
projection of contact points (Sec. 4.1; CCM_FLAG_PROJECT), element by element
with the parity bar of gpu_util, and the reverse passes refusing them."""
import numpy as np
import pytest

from gpu_util import compare, gpu_forward, weight_slack
from paper_2604_17538_b300 import scenes

pytestmark = pytest.mark.gpu

UNION, PROJECT = 2, 4


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_17538_b300 import api, build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def scenes_():
    return {"cube": scenes.cube_pair_scene(seed=1, n_poses=32),
            "hull": scenes.hull_env_scene(seed=2, n_envs=24, workers=0),
            "uneven": scenes.uneven_scene(seed=4, n_pairs=48, pool_bodies=96, workers=0)}


@pytest.mark.parametrize("name", ["cube", "hull", "uneven"])
@pytest.mark.parametrize("flags", [UNION, PROJECT, UNION | PROJECT])
def test_variant_matches_oracle(oracle_lib, ctx, scenes_, name, flags):
    sc = scenes_[name]
    y = gpu_forward(sc, params={"flags": flags}, ctx=ctx)
    ref = oracle_lib.forward(sc, oracle_lib.params(flags=flags))
    compare(y, ref, f"{name} flags {flags}", a_slack=weight_slack(sc))
    assert np.any(ref[:, 1] > 0)


def test_union_differs_from_the_per_piece_blend_on_multi_piece_bodies(oracle_lib, ctx, scenes_):
    """On single-piece bodies the union is the per-piece path; on 8-piece
    bodies it is a different (fewer-contact) blend, so the variant is really
    taken."""
    cube = scenes_["cube"]
    compare(gpu_forward(cube, params={"flags": UNION}, ctx=ctx), gpu_forward(cube, ctx=ctx),
            "union vs per piece, one piece", a_slack=weight_slack(cube))
    hull = scenes_["hull"]
    yu = gpu_forward(hull, params={"flags": UNION}, ctx=ctx)
    yp = gpu_forward(hull, ctx=ctx)
    assert np.abs(yu - yp).max() > 1e-4


def test_variants_are_forward_only(ctx, scenes_):
    import torch
    from paper_2604_17538_b300 import abi, api
    sc = scenes_["hull"].take(np.arange(4))
    batch, pa, pb = api.scene_to_device(sc, ctx)
    yb = torch.zeros((batch.n_groups, 8), device="cuda")
    for flags in (UNION, PROJECT):
        with pytest.raises(abi.CcmError) as e:
            batch.backward(pa, pb, yb, params={"flags": flags})
        assert e.value.status == abi.CCM_ERR_INVALID
        with pytest.raises(abi.CcmError) as e:
            batch.contacts(pa, pb, params={"flags": flags}, saved=batch.saved_buffer())
        assert e.value.status == abi.CCM_ERR_INVALID
    batch.close()
