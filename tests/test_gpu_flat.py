"""The per-contact reverse passes that run from the forward's contact list
(ccm_contacts_save + ccm_contacts_backward_saved on a batch whose bodies have
at most 256 pieces).  Their parity with the oracle is checked wherever a test
uses the saved path (test_gpu_backward, test_gpu_fullsize, test_gpu_uneven,
test_gpu_step_host); here: agreement with the per-pair passes they replace,
the fallback to those passes when the list overflows, determinism, and
independence from the rest of the batch."""
import numpy as np
import pytest

from gpu_util import GRAD_RTOL, report_derivs
from paper_2604_17538_b300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_17538_b300 import api, build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _inputs(sc, seed=0):
    rng = np.random.default_rng(seed)
    G = int(sc.group_offsets()[-1])
    ybar = rng.normal(size=(G, 8)).astype(np.float32)
    u = rng.normal(size=(sc.n_pairs, 12))
    u = (u / np.linalg.norm(u, axis=1, keepdims=True)).astype(np.float32)
    return ybar, u


def _saved_step(ctx, sc, ybar, u, **tuning):
    """(y, grad, grad of the dual pass, H u, J u) of the saved path."""
    import torch
    from paper_2604_17538_b300 import api
    batch, pa, pb = api.scene_to_device(sc, ctx)
    if tuning:
        batch.set_tuning(**tuning)
    yb = torch.from_numpy(ybar).cuda()
    ut = torch.from_numpy(u).cuda()
    saved = batch.saved_buffer()
    y = batch.contacts(pa, pb, saved=saved)
    g, _, _ = batch.backward(pa, pb, yb, saved=saved)
    g2, h, j = batch.backward(pa, pb, yb, ut, want_jvp=True, saved=saved)
    torch.cuda.synchronize()
    out = [t.cpu().numpy() for t in (y, g, g2, h, j)]
    batch.close()
    return out


@pytest.mark.parametrize("name", ["cube", "hull"])
def test_contact_list_matches_the_per_pair_pass_and_falls_back_on_overflow(ctx, name):
    sc = (scenes.cube_pair_scene(seed=1, n_poses=16) if name == "cube"
          else scenes.hull_env_scene(seed=2, n_envs=24, workers=0))
    ybar, u = _inputs(sc)
    flat = _saved_step(ctx, sc, ybar, u)                        # default: the contact list
    pair = _saved_step(ctx, sc, ybar, u, flat_records=-1)       # no list: per-pair passes
    tiny = _saved_step(ctx, sc, ybar, u, flat_records=1)        # one record per group
    # the staged forward (with a list) and the per-item one (without) find the
    # same contacts and blend them in different orders
    from gpu_util import compare, weight_slack
    compare(flat[0].astype(np.float64), pair[0].astype(np.float64), f"{name} forward, list vs none",
            a_slack=weight_slack(sc))
    # a list that overflows leaves the per-item forward and the per-pair
    # passes to run: bitwise theirs
    if name == "cube":   # deep cube contacts: more than one contact per group
        for a, b in zip(tiny, pair):
            assert np.array_equal(a, b)
    # the per-contact passes agree with the per-pair ones to float rounding
    # (their blends fold the same contacts in another order)
    for k, what in ((1, "gradient"), (2, "gradient (dual pass)"), (3, "H u")):
        a, b = flat[k].astype(np.float64), pair[k].astype(np.float64)
        assert np.all(np.isfinite(a)), what
        report_derivs(a, b, f"{name} per-contact vs per-pair {what}")
        err = np.abs(a - b).max(1)
        assert np.all(err <= GRAD_RTOL * np.abs(b).max(1) + 1e-6), (what, float(err.max()))
    jf, jp = flat[4].astype(np.float64), pair[4].astype(np.float64)
    assert np.abs(jf - jp).max() <= GRAD_RTOL * np.abs(jp).max() + 1e-6
    assert np.abs(flat[3]).max() > 0


def test_contact_list_passes_are_deterministic_and_batch_independent(ctx):
    sc = scenes.hull_env_scene(seed=2, n_envs=40, workers=0)
    ybar, u = _inputs(sc, seed=4)
    a = _saved_step(ctx, sc, ybar, u)
    b = _saved_step(ctx, sc, ybar, u)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    idx = np.array([3, 17, 31])
    off = sc.group_offsets()
    rows = np.concatenate([np.arange(off[i], off[i + 1]) for i in idx])
    alone = _saved_step(ctx, sc.take(idx), ybar[rows], u[idx])
    assert np.array_equal(alone[1], a[1][idx]) and np.array_equal(alone[2], a[2][idx])
    assert np.array_equal(alone[3], a[3][idx]) and np.array_equal(alone[4], a[4][rows])
    assert np.abs(alone[3]).max() > 0


def test_a_record_of_an_earlier_forward_does_not_use_the_newer_list(ctx):
    """Two forwards keeping their records on one batch (as two autograd calls
    before one backward do): the contact list in the batch is the second
    one's, so a reverse pass given the first record must not use it -- it
    runs the per-pair passes from that record, bitwise those of a batch
    without a list."""
    import torch
    from paper_2604_17538_b300 import api
    sc = scenes.hull_env_scene(seed=2, n_envs=24, workers=0)
    ybar, u = _inputs(sc, seed=6)
    batch, pa, pb = api.scene_to_device(sc, ctx)
    plain, _, _ = api.scene_to_device(sc, ctx)
    plain.set_tuning(flat_records=-1)
    yb = torch.from_numpy(ybar).cuda()
    ut = torch.from_numpy(u).cuda()
    pb2 = pb.clone()
    pb2[:, 9] += 3e-3
    s1, s2 = batch.saved_buffer(), batch.saved_buffer()
    batch.contacts(pa, pb, saved=s1)
    batch.contacts(pa, pb2, saved=s2)         # the batch's list is now this forward's
    g1, _, _ = batch.backward(pa, pb, yb, saved=s1)
    _, h1, j1 = batch.backward(pa, pb, yb, ut, want_jvp=True, saved=s1)
    r1 = plain.saved_buffer()
    plain.contacts(pa, pb, saved=r1)
    g1r, _, _ = plain.backward(pa, pb, yb, saved=r1)
    _, h1r, j1r = plain.backward(pa, pb, yb, ut, want_jvp=True, saved=r1)
    torch.cuda.synchronize()
    # the same contacts (hit marks); the reverse passes from the first record
    # ran per pair, as on the batch without a list
    assert torch.equal(s1[:, 18:26], r1[:, 18:26])
    assert torch.equal(g1, g1r) and torch.equal(h1, h1r) and torch.equal(j1, j1r)
    assert float(h1.abs().max()) > 0
    batch.close()
    plain.close()


@pytest.mark.parametrize("name", ["cube", "hull", "uneven"])
def test_flat_forward_matches_the_per_item_forward(oracle_lib, ctx, name):
    """The staged forward (gate per direction, culls per live direction, one
    contact per thread, fold per group in a fixed order) finds the same
    contacts as the per-item kernel: the saved hit marks are equal bit for
    bit and the outputs agree to float rounding (the blends fold in another
    order); both match the oracle.  A contact list too small for the contacts
    makes it fall back to the per-item kernel: bitwise that kernel's outputs."""
    import torch
    from gpu_util import compare, weight_slack
    from paper_2604_17538_b300 import api
    sc = {"cube": lambda: scenes.cube_pair_scene(seed=1, n_poses=32),
          "hull": lambda: scenes.hull_env_scene(seed=2, n_envs=32, workers=0),
          "uneven": lambda: scenes.uneven_scene(seed=4, n_pairs=96, pool_bodies=160,
                                                workers=0)}[name]()
    out = {}
    for key, tuning in (("flat", {}), ("item", {"flat_forward": -1}),
                        ("tiny", {"flat_records": 1})):
        batch, pa, pb = api.scene_to_device(sc, ctx)
        if tuning:
            batch.set_tuning(**tuning)
        saved = batch.saved_buffer()
        y = batch.contacts(pa, pb, saved=saved)
        y2 = batch.contacts(pa, pb)
        torch.cuda.synchronize()
        out[key] = (y.cpu().numpy(), saved.cpu().numpy(), y2.cpu().numpy())
        batch.close()
    yf, sf, yf2 = out["flat"]
    yi, si, _ = out["item"]
    assert np.array_equal(yf, yf2)                       # with and without the record
    hf, hi = sf[:, 18:26].copy().view(np.uint32), si[:, 18:26].copy().view(np.uint32)
    assert np.array_equal(hf, hi)
    compare(yf.astype(np.float64), yi.astype(np.float64), f"{name} flat vs per-item forward",
            a_slack=weight_slack(sc))
    compare(yf.astype(np.float64), oracle_lib.forward(sc), f"{name} flat forward vs oracle",
            a_slack=weight_slack(sc))
    yt, st, _ = out["tiny"]
    if name == "cube":                                   # the list overflows
        assert np.array_equal(yt, yi) and np.array_equal(st[:, :26], si[:, :26])


def test_flat_forward_is_deterministic_and_batch_independent(ctx):
    import torch
    from paper_2604_17538_b300 import api
    sc = scenes.uneven_scene(seed=4, n_pairs=80, pool_bodies=120, workers=0)
    ys = []
    for idx in (np.arange(sc.n_pairs), np.arange(sc.n_pairs), np.array([5, 33, 70])):
        sub = sc.take(idx)
        batch, pa, pb = api.scene_to_device(sub, ctx)
        ys.append(batch.contacts(pa, pb).cpu().numpy())
        batch.close()
    assert np.array_equal(ys[0], ys[1])
    off = sc.group_offsets()
    rows = np.concatenate([np.arange(off[i], off[i + 1]) for i in (5, 33, 70)])
    assert np.array_equal(ys[2], ys[0][rows])


@pytest.mark.parametrize("name", ["cube", "hull"])
def test_chains_without_programmatic_dependent_launch_give_the_same_results(ctx, name):
    """Tuning pdl = -1 launches every stage (and the gated fallback kernels
    behind each chain) as an ordinary launch, the fallbacks' work counters
    reset by a memset: the same kernels in the same order, so every output of
    the forward and of both reverse passes is bitwise that of the default
    chained launches -- also when the contact list overflows (the cube scene
    with one record per group runs the fallbacks)."""
    sc = (scenes.cube_pair_scene(seed=1, n_poses=16) if name == "cube"
          else scenes.hull_env_scene(seed=2, n_envs=24, workers=0))
    ybar, u = _inputs(sc, seed=4)
    for extra in ({}, {"flat_records": 1}) if name == "cube" else ({},):
        on = _saved_step(ctx, sc, ybar, u, **extra)
        off = _saved_step(ctx, sc, ybar, u, pdl=-1, **extra)
        for a, b, what in zip(on, off, ("y", "gradient", "gradient (dual pass)", "H u", "J u")):
            assert np.array_equal(a, b), (name, extra, what, float(np.abs(a - b).max()))
        assert np.abs(on[3]).max() > 0
