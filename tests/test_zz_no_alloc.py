"""The no-allocation reverse pass (ccm_contacts_backward_noalloc).

Callers that cannot obtain device memory for scratch (another framework owns
the memory pool, or allocation is forbidden after start-up) use a variant of
the reverse pass whose scratch is a fixed array inside the library.  Its
results must equal those of ccm_contacts_backward, call after call, although
every call reuses the same array.  This file is collected last so that a run
stopping at the first failure has run every other test before it.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2604_17538_b300 import scenes

pytestmark = pytest.mark.gpu


def _call_noalloc(batch, pa, pb, ybar, u=None):
    import torch
    from paper_2604_17538_b300 import abi, api
    n, G = batch.n_pairs, batch.n_groups
    grad = torch.empty((n, 12), device="cuda")
    hvp = torch.empty((n, 12), device="cuda") if u is not None else None
    jvp = torch.empty((G, 8), device="cuda") if u is not None else None
    prm = api._params(None)
    abi.check(abi.lib().ccm_contacts_backward_noalloc(
        batch.handle, abi.ptr(pa), abi.ptr(pb), C.byref(prm), abi.ptr(ybar), abi.ptr(u),
        abi.ptr(grad), abi.ptr(hvp), abi.ptr(jvp), abi.stream_of(pa)))
    return grad, hvp, jvp


def test_noalloc_backward_matches_the_workspace_version():
    """Bitwise equal to ccm_contacts_backward: each work item's slot is written
    by one warp and the pair sums run in index order in both.  Every call
    changes the poses and the cotangents, and the smaller scene runs after the
    larger one, so a slot that a call failed to rewrite would show up."""
    import torch
    from paper_2604_17538_b300 import api, build
    build.build()
    ctx = api.Context(0)
    rng = np.random.default_rng(5)
    for sc in (scenes.hull_env_scene(seed=2, n_envs=40, workers=0),
               scenes.cube_pair_scene(seed=1, n_poses=16)):
        batch, pa0, pb0 = api.scene_to_device(sc, ctx)
        for call in range(3):   # calls in a row share the fixed scratch
            # a small rigid nudge of B per call: new poses, same geometry
            pb = pb0.clone()
            pb[:, 9:12] += torch.from_numpy(
                rng.normal(scale=2e-3, size=(batch.n_pairs, 3)).astype(np.float32)).cuda()
            pa = pa0
            ybar = torch.from_numpy(rng.normal(size=(batch.n_groups, 8)).astype(np.float32)).cuda()
            u = rng.normal(size=(batch.n_pairs, 12))
            u = torch.from_numpy((u / np.linalg.norm(u, axis=1, keepdims=True)).astype(np.float32)).cuda()
            g_ref, _, _ = batch.backward(pa, pb, ybar)
            g2_ref, h_ref, j_ref = batch.backward(pa, pb, ybar, u, want_jvp=True)
            g, _, _ = _call_noalloc(batch, pa, pb, ybar)
            g2, h, j = _call_noalloc(batch, pa, pb, ybar, u)
            torch.cuda.synchronize()
            for got, ref, what in ((g, g_ref, "gradient"), (g2, g2_ref, "gradient (dual pass)"),
                                   (h, h_ref, "H u"), (j, j_ref, "J u")):
                assert bool(torch.isfinite(got).all()), (what, call)
                assert torch.equal(got, ref), (what, call, float((got - ref).abs().max()))
            assert float(g_ref.abs().max()) > 0.0   # the scene has contacts
        batch.close()
    ctx.close()


def test_noalloc_rejects_batches_beyond_its_scratch():
    from paper_2604_17538_b300 import abi, api, build
    import torch
    build.build()
    ctx = api.Context(0)
    geom = scenes.geometry_from_bodies([[scenes.unit_cube_piece(0.5)], [scenes.unit_cube_piece(0.5)]])
    handles = ctx.load_geometry(geom)
    n = 21846   # one pair more than 2^20 floats of 2 x 24-float slots hold
    batch = ctx.batch(np.full(n, handles[0]), np.full(n, handles[1]))
    pose = torch.zeros((n, 12), device="cuda")
    ybar = torch.zeros((batch.n_groups, 8), device="cuda")
    with pytest.raises(abi.CcmError) as e:
        _call_noalloc(batch, pose, pose, ybar)
    assert e.value.status == abi.CCM_ERR_INVALID and "fixed scratch" in str(e.value)
    batch.close()
    ctx.close()
