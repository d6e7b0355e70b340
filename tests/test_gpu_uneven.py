"""Uneven batches (pieces per body log-uniform in [1, 64], hull points
log-uniform in [8, 512]): forward, gradient and H u parity with the oracle,
and bit-identical results for a pair alone and inside the batch."""
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
