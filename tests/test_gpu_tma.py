"""Staging of the SDF body's planes with bulk (TMA) copies completed on an
mbarrier: the staged data, hence every output, equals plain-load staging bit
for bit, and a wait that runs out is reported (CCM_ERR_TIMEOUT through
ccm_batch_check) instead of hanging: the test makes every wait run out by
giving it no polls, then checks that the batch recovers.  Both forwards
stage this way: the per-item kernel (the SDF body's planes per chunk) and the
flat stages (the gate's chunks of the SDF body, the feature stage's SDF
piece); each is run on its own."""
import numpy as np
import pytest

from paper_2604_17538_b300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_17538_b300 import api, build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("flat", [0, -1])
@pytest.mark.parametrize("name", ["hull", "uneven"])
def test_bulk_staging_equals_plain_loads(ctx, name, flat):
    import torch
    from paper_2604_17538_b300 import api
    sc = (scenes.hull_env_scene(seed=2, n_envs=24, workers=0) if name == "hull"
          else scenes.uneven_scene(seed=4, n_pairs=64, pool_bodies=128, workers=0))
    batch, pa, pb = api.scene_to_device(sc, ctx)
    batch.set_tuning(flat_forward=flat)
    if name == "uneven":                 # several staged chunks per SDF body
        batch.set_tuning(stage_planes=64, stage_verts=32)
    saved = batch.saved_buffer()
    y_tma = batch.contacts(pa, pb, saved=saved).clone()
    rec_tma = saved.clone()
    batch.check()
    batch.set_tuning(stage_tma=-1)
    y_ld = batch.contacts(pa, pb, saved=saved)
    torch.cuda.synchronize()
    assert torch.equal(y_tma, y_ld)
    assert torch.equal(rec_tma[:, :26], saved[:, :26])
    assert float(y_ld[:, 1].max()) > 0
    batch.close()


@pytest.mark.parametrize("flat", [0, -1])
def test_a_wait_that_runs_out_is_reported_and_the_batch_recovers(ctx, flat):
    import torch
    from paper_2604_17538_b300 import abi, api
    sc = scenes.hull_env_scene(seed=2, n_envs=8, workers=0)
    batch, pa, pb = api.scene_to_device(sc, ctx)
    batch.set_tuning(flat_forward=flat)
    y_ref = batch.contacts(pa, pb).clone()
    batch.check()
    batch.set_tuning(stage_wait=-1)      # no polls: every bulk-copy wait runs out
    batch.contacts(pa, pb)
    with pytest.raises(abi.CcmError) as e:
        batch.check()
    assert e.value.status == abi.CCM_ERR_TIMEOUT
    batch.check()                        # the flag was cleared
    batch.set_tuning(stage_wait=0)
    y = batch.contacts(pa, pb)
    batch.check()
    assert torch.equal(y, y_ref)
    batch.close()
