"""The autotuner's search on the host, with a fake batch whose timings come
from a cost table: each stage keeps the fastest candidate, and the joint
step over the staging budgets and the forward shape finds a pair that the
greedy order misses (the staging budgets are timed before the forward shape
that changes their ranking)."""
import pytest

from paper_2604_17538_b300 import tune

DEFAULT = dict(item_v=256, item_e=512, item_vb=256, item_eb=512, fwd_warps=2, groups=16,
               stage_planes=0, stage_verts=0, groups_b=4)


class FakeBatch:
    n_groups = 4

    def __init__(self):
        self.t = dict(DEFAULT)

    def set_tuning(self, **kw):
        assert set(kw) <= set(DEFAULT), kw
        self.t.update(kw)

    def get_tuning(self):
        return dict(self.t)

    def saved_buffer(self, device=None):
        return object()

    def contacts(self, *a, **k):
        return None

    def backward(self, *a, **k):
        return None


def cost(t):
    """ms of a step under shape t: staging (512, 256) wins at the default two
    warps per block, (256, 128) wins at four."""
    st = (t["stage_planes"], t["stage_verts"])
    ms = {(0, 0): 10.0, (512, 256): 8.0, (256, 128): 8.5, (128, 64): 9.0}[st]
    if t["fwd_warps"] == 4:
        ms -= 2.5 if st == (256, 128) else 1.0
    elif t["fwd_warps"] == 1:
        ms += 1.0
    ms += 0.01 * (t["item_v"] != 256)
    ms += {64: 0.3, 128: 0.2, 256: 0.1, 512: 0.2}[t["item_vb"]]
    ms += 0.01 * abs(t["groups_b"] - 4) + 0.01 * abs(t["groups"] - 16) / 4
    return ms


@pytest.fixture
def fake(monkeypatch):
    b = FakeBatch()
    monkeypatch.setattr(tune, "_time", lambda fn, reps=5: cost(b.t))
    return b


def test_joint_step_finds_what_the_greedy_order_misses(fake):
    import torch
    pose = torch.zeros((1, 12))
    tuning, log = tune.autotune(fake, pose, pose, torch.zeros((4, 8)))
    # (every timing includes the default reverse lists' 0.1 ms)
    # greedy alone: staging (512, 256) at two warps, then four warps -> 7.1 ms
    assert min(log["stage"].values()) == pytest.approx(8.1)
    assert min(log["forward"].values()) == pytest.approx(7.1)
    # crossed with the runner-up staging (256, 128): 6.1 ms
    assert len(log["joint"]) == 4
    assert min(log["joint"].values()) == pytest.approx(6.1)
    assert (tuning["stage_planes"], tuning["stage_verts"]) == (256, 128)
    assert tuning["fwd_warps"] == 4 and (tuning["item_v"], tuning["item_e"]) == (256, 512)
    assert (tuning["item_vb"], tuning["item_eb"]) == (256, 512)
    assert tuning["groups"] == 16 and tuning["groups_b"] == 4
    assert cost(tuning) == pytest.approx(6.1)


def test_failing_candidates_are_logged_and_skipped(fake, monkeypatch):
    import torch
    real_set = fake.set_tuning

    def picky(**kw):
        if kw.get("fwd_warps") == 4 and kw.get("item_v") == 512:
            raise RuntimeError("shape does not fit")
        real_set(**kw)
    monkeypatch.setattr(fake, "set_tuning", picky)
    pose = torch.zeros((1, 12))
    tuning, log = tune.autotune(fake, pose, pose, torch.zeros((4, 8)))
    errs = [c for c, t in log["forward"].items() if isinstance(t, str)]
    assert len(errs) == 1 and "512" in errs[0]
    assert tuning["fwd_warps"] == 4 and tuning["item_v"] != 512
