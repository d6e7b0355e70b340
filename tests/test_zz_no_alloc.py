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

from gpu_util import GRAD_RTOL
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


def _close(a, b, what):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    assert np.all(np.isfinite(a)), what
    err = np.abs(a - b).max(1)
    assert np.all(err <= GRAD_RTOL * np.abs(b).max(1) + 1e-6), (what, float(err.max()))


def test_noalloc_backward_matches_the_workspace_version():
    import torch
    from paper_2604_17538_b300 import api, build
    build.build()
    ctx = api.Context(0)
    rng = np.random.default_rng(5)
    for sc in (scenes.hull_env_scene(seed=2, n_envs=40, workers=0),
               scenes.cube_pair_scene(seed=1, n_poses=16)):
        batch, pa, pb = api.scene_to_device(sc, ctx)
        ybar = torch.from_numpy(rng.normal(size=(batch.n_groups, 8)).astype(np.float32)).cuda()
        u = rng.normal(size=(batch.n_pairs, 12))
        u = torch.from_numpy((u / np.linalg.norm(u, axis=1, keepdims=True)).astype(np.float32)).cuda()
        g_ref, _, _ = batch.backward(pa, pb, ybar)
        _, h_ref, j_ref = batch.backward(pa, pb, ybar, u, want_jvp=True)
        for _ in range(2):   # two calls in a row share the fixed scratch
            g, _, _ = _call_noalloc(batch, pa, pb, ybar)
            g2, h, j = _call_noalloc(batch, pa, pb, ybar, u)
            torch.cuda.synchronize()
            _close(g, g_ref, "gradient")
            _close(g2, g_ref, "gradient (dual pass)")
            _close(h, h_ref, "H u")
            _close(j, j_ref, "J u")
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
