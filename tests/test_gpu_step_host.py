"""ccm_contacts_step_host: one step from host buffers, with the copies
overlapped with the kernels on side streams, returns exactly what the device
calls (ccm_contacts_save, ccm_contacts_backward_saved with and without a
direction) return on the same data -- same kernels, same inputs -- in every
mode (forward only, + gradient, + H u / J u; with a direction the gradient is
that of the forward-over-reverse pass), across repeated calls whose buffers
are reused, and it rejects the mode errors."""
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


@pytest.fixture(scope="module")
def scene():
    return scenes.hull_env_scene(seed=2, n_envs=40, workers=0)


def _device_step(batch, pa, pb, yb, u):
    import torch
    saved = batch.saved_buffer()
    y = batch.contacts(pa, pb, saved=saved)
    g, _, _ = batch.backward(pa, pb, yb, saved=saved)
    g2, h, j = batch.backward(pa, pb, yb, u, want_jvp=True, saved=saved)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in (y, g, h, j, g2)]


def _host_inputs(sc, seed):
    import torch
    rng = np.random.default_rng(seed)
    G = int(sc.group_offsets()[-1])
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory()
    return (pin(sc.pose_a), pin(sc.pose_b), pin(rng.normal(size=(G, 8))),
            pin(rng.normal(size=(sc.n_pairs, 12))))


def test_step_host_equals_device_calls(ctx, scene):
    import torch
    from paper_2604_17538_b300 import api
    batch, _, _ = api.scene_to_device(scene, ctx)
    for seed, shift in ((0, 0.0), (1, 3e-3)):   # second call: other poses, reused buffers
        pa_h, pb_h, yb_h, u_h = _host_inputs(scene, seed)
        pa_h[:, 9:] += shift                      # move body A: other contacts
        ref = _device_step(batch, pa_h.cuda(), pb_h.cuda(), yb_h.cuda(), u_h.cuda())
        y, g, h, j = batch.step_host(pa_h, pb_h, yb_h, u_h, want_jvp=True)
        torch.cuda.synchronize()
        for name, a, b in zip("yghj", (y, g, h, j), (ref[0], ref[4], ref[2], ref[3])):
            assert np.array_equal(a.numpy(), b), (seed, name, np.abs(a.numpy() - b).max())
        assert np.isfinite(g.numpy()).all() and np.abs(g.numpy()).max() > 0


def test_step_host_on_an_overflowing_contact_list(ctx):
    """With a contact list too small for the cube contacts, the per-item
    forward and the per-pair reverse pass write the outputs, the gradient,
    H u and J u instead of the flat stages; the host step, whose copies wait
    on events around the passes, still returns exactly what the device calls
    return."""
    import torch
    from paper_2604_17538_b300 import api
    sc = scenes.cube_pair_scene(seed=1, n_poses=16)
    batch, _, _ = api.scene_to_device(sc, ctx)
    batch.set_tuning(flat_records=1)
    pa_h, pb_h, yb_h, u_h = _host_inputs(sc, 3)
    ref = _device_step(batch, pa_h.cuda(), pb_h.cuda(), yb_h.cuda(), u_h.cuda())
    y, g, h, j = batch.step_host(pa_h, pb_h, yb_h, u_h, want_jvp=True)
    torch.cuda.synchronize()
    for name, a, b in zip("yghj", (y, g, h, j), (ref[0], ref[4], ref[2], ref[3])):
        assert np.array_equal(a.numpy(), b), (name, np.abs(a.numpy() - b).max())
    assert np.abs(j.numpy()).max() > 0
    batch.close()


def test_step_host_modes(ctx, scene):
    import torch
    from paper_2604_17538_b300 import api
    batch, pa, pb = api.scene_to_device(scene, ctx)
    pa_h, pb_h, yb_h, u_h = _host_inputs(scene, 5)
    ref = _device_step(batch, pa_h.cuda(), pb_h.cuda(), yb_h.cuda(), u_h.cuda())
    y, g, h, j = batch.step_host(pa_h, pb_h)                    # forward only
    torch.cuda.synchronize()
    assert g is None and h is None and j is None
    assert np.array_equal(y.numpy(), ref[0])
    y, g, h, j = batch.step_host(pa_h, pb_h, yb_h)              # + gradient
    torch.cuda.synchronize()
    assert h is None and j is None
    assert np.array_equal(y.numpy(), ref[0]) and np.array_equal(g.numpy(), ref[1])
    y, g, h, j = batch.step_host(pa_h, pb_h, yb_h, u_h)         # + H u, no J u
    torch.cuda.synchronize()
    assert j is None and np.array_equal(h.numpy(), ref[2])


def test_step_host_rejects_bad_modes(ctx, scene):
    import ctypes as C
    from paper_2604_17538_b300 import abi, api
    batch, _, _ = api.scene_to_device(scene, ctx)
    pa_h, pb_h, yb_h, u_h = _host_inputs(scene, 7)
    y = np.empty((batch.n_groups, 8), np.float32)
    g = np.empty((batch.n_pairs, 12), np.float32)
    prm = api._params(None)
    L = abi.lib()
    p = abi.ptr
    # a direction without cotangents, cotangents without a gradient buffer,
    # a direction without an hvp buffer, no output buffer
    for args in ((p(pa_h), p(pb_h), C.byref(prm), None, p(u_h), y.ctypes.data, g.ctypes.data,
                  g.ctypes.data, None),
                 (p(pa_h), p(pb_h), C.byref(prm), p(yb_h), None, y.ctypes.data, None, None, None),
                 (p(pa_h), p(pb_h), C.byref(prm), p(yb_h), p(u_h), y.ctypes.data,
                  g.ctypes.data, None, None),
                 (p(pa_h), p(pb_h), C.byref(prm), None, None, None, None, None, None)):
        assert L.ccm_contacts_step_host(batch.handle, *args, None) == abi.CCM_ERR_INVALID
