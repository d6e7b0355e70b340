"""Uneven batches (pieces per body log-uniform in [1, 64], hull points
log-uniform in [8, 512]): forward, gradient and H u parity with the oracle,
and bit-identical results for a pair alone and inside the batch, and for a
CUDA-graph replay and the eager calls."""
import numpy as np
import pytest

from gpu_util import COND_FACTOR, GRAD_RTOL, compare, fp32_sensitivity, gpu_forward, weight_slack
from paper_2604_17538_b300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def uneven():
    return scenes.uneven_scene(seed=4, n_pairs=96, pool_bodies=96, workers=0)


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_17538_b300 import api, build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def test_uneven_forward_matches_oracle(oracle_lib, ctx, uneven):
    npb = np.diff(uneven.geom.body_piece_off)
    assert npb.max() >= 32 and npb.min() == 1          # heavy tail and single pieces
    y = gpu_forward(uneven, ctx=ctx)
    ref = oracle_lib.forward(uneven)
    print("uneven max err", compare(y, ref, "uneven", a_slack=weight_slack(uneven)))


def test_uneven_alone_equals_in_batch(ctx, uneven):
    y = gpu_forward(uneven, ctx=ctx)
    off = uneven.group_offsets()
    for i in (0, 7, 50):
        alone = gpu_forward(uneven.take([i]), ctx=ctx)
        assert np.array_equal(alone, y[off[i]:off[i + 1]])


def test_uneven_derivatives_match_oracle(oracle_lib, ctx, uneven):
    import torch
    from paper_2604_17538_b300 import api
    npb = np.diff(uneven.geom.body_piece_off)
    small = np.nonzero((npb[uneven.pair_a] * npb[uneven.pair_b]) <= 64)[0][:24]
    sc = uneven.take(small)
    rng = np.random.default_rng(1)
    G = int(sc.group_offsets()[-1])
    ybar = rng.normal(size=(G, 8)).astype(np.float32)
    u = rng.normal(size=(sc.n_pairs, 12))
    u = (u / np.linalg.norm(u, axis=1, keepdims=True)).astype(np.float32)
    batch, pa, pb = api.scene_to_device(sc, ctx)
    g, h, _ = batch.backward(pa, pb, torch.from_numpy(ybar).cuda(), torch.from_numpy(u).cuda())
    torch.cuda.synchronize()
    go, ho, _, _ = oracle_lib.hvp(sc, ybar, u)
    kg, kh = fp32_sensitivity(oracle_lib, sc, ybar, u)
    for got, ref, k, name in ((g, go, kg, "gradient"), (h, ho, kh, "H u")):
        got = got.double().cpu().numpy()
        assert np.all(np.isfinite(got))
        err = np.abs(got - ref).max(1)
        tol = np.maximum(GRAD_RTOL, COND_FACTOR * k) * np.abs(ref).max(1) + 1e-6
        assert np.all(err <= tol), (name, float((err / (np.abs(ref).max(1) + 1e-30)).max()))
    batch.close()


def test_work_item_size_and_budgets_change_only_rounding(ctx, uneven):
    """Any launch shape gives the same contacts and gradients up to float
    rounding order: items of 1, 3 or 32 feature pieces, small and large list
    budgets, 1 or 4 forward warps.  Items of one piece split every body into
    as many warp tasks as it has pieces, the most the reverse pass's per-pair
    slot reduction ever adds up."""
    import torch
    from paper_2604_17538_b300 import api
    batch, pa, pb = api.scene_to_device(uneven, ctx)
    rng = np.random.default_rng(2)
    ybar = torch.from_numpy(rng.normal(size=(batch.n_groups, 8)).astype(np.float32)).cuda()
    y0 = batch.contacts(pa, pb).double().cpu().numpy()
    g0, _, _ = batch.backward(pa, pb, ybar)
    g0 = g0.double().cpu().numpy()
    slack = weight_slack(uneven)
    for t in (dict(groups=1), dict(groups=3, item_v=64, item_e=128, item_vb=64, item_eb=128),
              dict(groups=16, stage_planes=64, stage_verts=32),
              dict(groups=16, groups_b=1), dict(groups=8, groups_b=16),
              dict(groups=32, item_v=1024, item_e=2048, item_vb=512, item_eb=1024, fwd_warps=1),
              dict(groups=8, fwd_warps=4)):
        batch.set_tuning(**t)
        assert batch.get_tuning()["groups"] == t["groups"]
        y = batch.contacts(pa, pb).double().cpu().numpy()
        compare(y, y0, f"tuning {t}", a_slack=slack)
        g, _, _ = batch.backward(pa, pb, ybar)
        g = g.double().cpu().numpy()
        assert np.all(np.isfinite(g))
        err = np.abs(g - g0).max(1)
        assert np.all(err <= GRAD_RTOL * np.abs(g0).max(1) + 1e-6), (t, float(err.max()))
    batch.close()


def test_autotune_times_the_saved_record_path(ctx, uneven):
    """The autotuner times the forward keeping its record and the per-pair
    reverse pass from it (the path a step runs), keeps a shape from its
    candidate lists, and that shape changes results only by rounding."""
    import torch
    from paper_2604_17538_b300 import api, tune
    batch, pa, pb = api.scene_to_device(uneven, ctx)
    rng = np.random.default_rng(6)
    ybar = torch.from_numpy(rng.normal(size=(batch.n_groups, 8)).astype(np.float32)).cuda()
    saved = batch.saved_buffer()
    y0 = batch.contacts(pa, pb, saved=saved).double().cpu().numpy()
    g0 = batch.backward(pa, pb, ybar, saved=saved)[0].double().cpu().numpy()
    tuning, log = tune.autotune(batch, pa, pb, ybar)
    for kind, cands in (("items", tune.GROUP_CANDIDATES), ("stage", tune.STAGE_CANDIDATES),
                        ("forward", tune.FWD_CANDIDATES), ("reverse", tune.BWD_CANDIDATES),
                        ("chunks", tune.CHUNK_CANDIDATES)):
        assert len(log[kind]) == len(cands)
        assert any(isinstance(t, float) for t in log[kind].values()), kind
    assert 1 <= len(log["joint"]) <= 4      # two staging budgets x two forward shapes
    assert any(isinstance(t, float) for t in log["joint"].values())
    assert dict(groups=tuning["groups"]) in tune.GROUP_CANDIDATES
    assert dict(item_vb=tuning["item_vb"], item_eb=tuning["item_eb"]) in tune.BWD_CANDIDATES
    y = batch.contacts(pa, pb, saved=saved).double().cpu().numpy()
    compare(y, y0, "autotuned", a_slack=weight_slack(uneven))
    g = batch.backward(pa, pb, ybar, saved=saved)[0].double().cpu().numpy()
    err = np.abs(g - g0).max(1)
    assert np.all(err <= GRAD_RTOL * np.abs(g0).max(1) + 1e-6), float(err.max())
    batch.close()


def test_graph_replay_equals_eager_calls(ctx, uneven):
    """The forward with its record, the gradient pass and the H u / J u pass
    captured once in a CUDA graph: every replay returns the eager calls'
    results bitwise (the work counters restart each replay), and a replay
    after the poses change in place returns the eager results at the new
    poses."""
    import torch
    from paper_2604_17538_b300 import api
    batch, pa, pb = api.scene_to_device(uneven, ctx)
    n, G = batch.n_pairs, batch.n_groups
    rng = np.random.default_rng(31)
    yb = torch.from_numpy(rng.normal(size=(G, 8)).astype(np.float32)).cuda()
    u = torch.from_numpy(rng.normal(size=(n, 12)).astype(np.float32)).cuda()
    saved = batch.saved_buffer()
    y = torch.empty((G, 8), device="cuda")
    g, g2, h = (torch.empty((n, 12), device="cuda") for _ in range(3))
    j = torch.empty((G, 8), device="cuda")

    def calls():
        batch.contacts(pa, pb, out=y, saved=saved)
        batch.backward(pa, pb, yb, out=(g, None, None), saved=saved)
        batch.backward(pa, pb, yb, u, want_jvp=True, out=(g2, h, j), saved=saved)

    def eager():
        calls()
        torch.cuda.synchronize()
        return [t.cpu().numpy().copy() for t in (y, g, g2, h, j)]

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):              # first calls (allocations) outside the capture
        for _ in range(2):
            calls()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    ref0 = eager()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        calls()
    for _ in range(3):
        for t in (y, g, g2, h, j):
            t.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        for name, a, b in zip(("y", "grad", "grad (dual)", "H u", "J u"), (y, g, g2, h, j), ref0):
            assert np.array_equal(a.cpu().numpy(), b), name

    pa_new = pa.clone()
    pa_new[:, 9:] += 2e-3                      # move every body A: other contacts
    pa.copy_(pa_new)
    ref1 = eager()
    for t in (y, g, g2, h, j):
        t.fill_(float("nan"))
    graph.replay()
    torch.cuda.synchronize()
    for name, a, b in zip(("y", "grad", "grad (dual)", "H u", "J u"), (y, g, g2, h, j), ref1):
        assert np.array_equal(a.cpu().numpy(), b), name
    assert not np.array_equal(ref0[0], ref1[0]) and not np.array_equal(ref0[3], ref1[3])
    batch.close()
