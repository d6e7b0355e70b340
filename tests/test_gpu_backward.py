"""Parity of the hand-written adjoint (gradient), the forward-over-reverse
Hessian-vector product and the output tangents with the FP64 oracle, through
the C ABI and through torch.autograd (double backward)."""
import numpy as np
import pytest

from gpu_util import COND_FACTOR, GRAD_RTOL, MAX_WIDENED_SHARE, fp32_sensitivity, report_derivs
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
def cases():
    return {"cube": scenes.cube_pair_scene(seed=1),
            "hull": scenes.hull_env_scene(seed=2, n_envs=48, workers=0)}


def _inputs(sc, seed=0):
    rng = np.random.default_rng(seed)
    G = int(sc.group_offsets()[-1])
    ybar = rng.normal(size=(G, 8))
    u = rng.normal(size=(sc.n_pairs, 12))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    return ybar, u


def _per_pair_check(g, o, what, rtol=GRAD_RTOL, floor=1e-6):
    """||g - o||_inf <= rtol ||o||_inf per pair (rows); rtol may be per pair."""
    assert np.all(np.isfinite(g)), f"{what}: non-finite values"
    rt = np.broadcast_to(np.asarray(rtol, np.float64), (len(g),))
    report_derivs(g, o, what, widened=(rt > GRAD_RTOL).sum())
    err = np.abs(g - o).max(1)
    scale = np.abs(o).max(1)
    bad = err > rtol * scale + floor
    if bad.any():
        i = int(np.argmax(err - rtol * scale))
        raise AssertionError(f"{what}: {int(bad.sum())}/{len(g)} pairs over tolerance; worst "
                             f"pair {i}: err {err[i]:.3e} scale {scale[i]:.3e}\n gpu {g[i]}\n "
                             f"oracle {o[i]}")
    return float((err / np.maximum(scale, 1e-30)).max())


@pytest.mark.parametrize("name", ["cube", "hull"])
def test_gradient_hvp_jvp_match_oracle(oracle_lib, ctx, cases, name):
    import torch
    from paper_2604_17538_b300 import api
    sc = cases[name]
    ybar, u = _inputs(sc)
    batch, pa, pb = api.scene_to_device(sc, ctx)
    yb = torch.from_numpy(ybar.astype(np.float32)).cuda()
    ut = torch.from_numpy(u.astype(np.float32)).cuda()
    g, _, _ = batch.backward(pa, pb, yb)
    g2, hv, jv = batch.backward(pa, pb, yb, ut, want_jvp=True)
    torch.cuda.synchronize()
    # the oracle sees exactly the float32 values the GPU sees
    go, hvo, jvo, _ = oracle_lib.hvp(sc, ybar.astype(np.float32), u.astype(np.float32))
    # bar: 1e-3 relative, widened per pair only where the problem's one-ulp
    # float32 input sensitivity (times COND_FACTOR) exceeds it
    kg, kh = fp32_sensitivity(oracle_lib, sc, ybar.astype(np.float32), u.astype(np.float32))
    tol_g = np.maximum(GRAD_RTOL, COND_FACTOR * kg)
    tol_h = np.maximum(GRAD_RTOL, COND_FACTOR * kh)
    print(f"{name}: pairs with a widened bar: grad {int((tol_g > GRAD_RTOL).sum())}, "
          f"hvp {int((tol_h > GRAD_RTOL).sum())} of {sc.n_pairs}")
    # conditioning may widen the bar of a few ill-conditioned pairs, not of many
    assert (tol_g > GRAD_RTOL).mean() <= MAX_WIDENED_SHARE
    assert (tol_h > GRAD_RTOL).mean() <= MAX_WIDENED_SHARE
    rg = _per_pair_check(g.double().cpu().numpy(), go, f"{name} gradient", tol_g)
    _per_pair_check(g2.double().cpu().numpy(), go, f"{name} gradient (dual pass)", tol_g)
    rh = _per_pair_check(hv.double().cpu().numpy(), hvo, f"{name} H u", tol_h)
    off = sc.group_offsets()
    jvg = jv.double().cpu().numpy()
    assert np.all(np.isfinite(jvg))
    jmax = np.array([np.abs(jvg[off[i]:off[i + 1]] - jvo[off[i]:off[i + 1]]).max()
                     for i in range(sc.n_pairs)])
    jsc = np.array([np.abs(jvo[off[i]:off[i + 1]]).max() for i in range(sc.n_pairs)])
    assert np.all(jmax <= GRAD_RTOL * jsc + 1e-6), (jmax / (jsc + 1e-30)).max()
    print(f"{name}: max rel err grad {rg:.2e} hvp {rh:.2e}")
    assert np.abs(go).max() > 0 and np.abs(hvo).max() > 0
    # the same through the forward's saved record (ccm_contacts_save +
    # ccm_contacts_backward_saved): the passes visit only the directions the
    # forward found contacts in, against the same bars
    saved = batch.saved_buffer()
    y = batch.contacts(pa, pb, saved=saved)
    gs, _, _ = batch.backward(pa, pb, yb, saved=saved)
    gs2, hvs, jvs = batch.backward(pa, pb, yb, ut, want_jvp=True, saved=saved)
    torch.cuda.synchronize()
    _per_pair_check(gs.double().cpu().numpy(), go, f"{name} gradient (saved)", tol_g)
    _per_pair_check(gs2.double().cpu().numpy(), go, f"{name} gradient (dual, saved)", tol_g)
    _per_pair_check(hvs.double().cpu().numpy(), hvo, f"{name} H u (saved)", tol_h)
    jvs = jvs.double().cpu().numpy()
    jmax = np.array([np.abs(jvs[off[i]:off[i + 1]] - jvo[off[i]:off[i + 1]]).max()
                     for i in range(sc.n_pairs)])
    assert np.all(jmax <= GRAD_RTOL * jsc + 1e-6), (jmax / (jsc + 1e-30)).max()
    # record layout: U > 0 exactly for groups with a contact (a > 0), and such
    # a group has at least one hit bit (every SDF body here has < 256 pieces)
    rec = saved.cpu().numpy()
    yh = y.cpu().numpy()
    assert np.array_equal(rec[:, 1] > 0, yh[:, 1] > 0)
    hits = rec[:, 18:26].copy().view(np.uint32)
    assert np.all((hits != 0).any(1) == (yh[:, 1] > 0))
    # counted reverse passes give the same results, and the saved record
    # restricts them to fewer directions than a full re-gating
    for direction in (None, ut):
        c_full = torch.zeros(8, dtype=torch.int64, device="cuda")
        c_saved = torch.zeros(8, dtype=torch.int64, device="cuda")
        r_full = batch.backward(pa, pb, yb, direction, want_jvp=direction is not None,
                                counters=c_full)
        r_saved = batch.backward(pa, pb, yb, direction, want_jvp=direction is not None,
                                 saved=saved, counters=c_saved)
        torch.cuda.synchronize()
        ref_full = g if direction is None else hv
        ref_saved = gs if direction is None else hvs
        got_full = r_full[0] if direction is None else r_full[1]
        got_saved = r_saved[0] if direction is None else r_saved[1]
        assert torch.equal(got_full, ref_full) and torch.equal(got_saved, ref_saved)
        cf, cs = c_full.cpu().numpy(), c_saved.cpu().numpy()
        # with the record the passes run per contact from the forward's
        # contact list: no piece-pair gate, contacts with a live group among
        # those evaluated, and fewer plane evaluations than a full re-gating
        assert cf[3] > 0 and cs[3] == 0
        assert 0 < cs[1] <= cs[0] and cs[4] > 0 and cs[6] > 0
        assert cs[2:].sum() < cf[2:].sum()
    batch.close()


def test_separated_pairs_have_zero_derivatives(ctx):
    import torch
    from paper_2604_17538_b300 import api
    sc = scenes.hull_env_scene(seed=21, n_envs=4, workers=1)
    sc.pose_b[:, 9] += 5.0
    ybar, u = _inputs(sc)
    batch, pa, pb = api.scene_to_device(sc, ctx)
    yb = torch.from_numpy(ybar.astype(np.float32)).cuda()
    ut = torch.from_numpy(u.astype(np.float32)).cuda()
    g, hv, jv = batch.backward(pa, pb, yb, ut, want_jvp=True)
    assert torch.all(g == 0) and torch.all(hv == 0) and torch.all(jv == 0)
    batch.close()


def test_autograd_double_backward(oracle_lib, ctx, cases):
    import torch
    from paper_2604_17538_b300 import api, autograd
    sc = cases["hull"].take(np.arange(16))
    ybar, u = _inputs(sc, seed=3)
    batch, pa, pb = api.scene_to_device(sc, ctx)
    n = sc.n_pairs
    ta = torch.zeros((n, 6), device="cuda", requires_grad=True)
    tb = torch.zeros((n, 6), device="cuda", requires_grad=True)
    yb = torch.from_numpy(ybar.astype(np.float32)).cuda()
    ut = torch.from_numpy(u.astype(np.float32)).cuda()
    y = autograd.contacts(batch, pa, pb, ta, tb)
    L = (y * yb).sum()
    ga, gb = torch.autograd.grad(L, (ta, tb), create_graph=True)
    g = torch.cat([ga, gb], 1)
    ha, hb = torch.autograd.grad((g * ut).sum(), (ta, tb))
    h = torch.cat([ha, hb], 1)
    go, hvo, _, _ = oracle_lib.hvp(sc, ybar.astype(np.float32), u.astype(np.float32))
    kg, kh = fp32_sensitivity(oracle_lib, sc, ybar.astype(np.float32), u.astype(np.float32))
    _per_pair_check(g.detach().double().cpu().numpy(), go, "autograd gradient",
                    np.maximum(GRAD_RTOL, COND_FACTOR * kg))
    _per_pair_check(h.double().cpu().numpy(), hvo, "autograd H u",
                    np.maximum(GRAD_RTOL, COND_FACTOR * kh))
    batch.close()
