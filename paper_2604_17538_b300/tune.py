"""Autotuner of a batch's launch shape (``ccm_batch_set_tuning``).

Times the passes of a batch on its own poses and keeps the fastest shape; the
choice is written back into the batch.  First the work-item size (feature
pieces per warp task: small items balance uneven bodies over the warps, large
ones stage the SDF body's planes fewer times) and then the staging budgets
(planes and vertices held at once: smaller slices, more resident warps, more
chunks), each timed on forward + reverse pass together since both passes use
them; then the forward's list budgets and warps per block, which trade lane
utilisation (bigger lists of live piece pairs) against resident warps; then the
two fastest staging budgets crossed with the two fastest forward shapes, timed
together (both set the resident warps); then the reverse pass's list budgets
and its chunk size (fewer pieces per chunk keep a chunk's directions in one
list, which its adjoint sweep reuses).
"""
from __future__ import annotations

import itertools

FWD_CANDIDATES = [dict(item_v=v, item_e=e, fwd_warps=w)
                  for (v, e), w in itertools.product([(128, 256), (256, 512), (512, 1024)], [1, 2, 4])]
BWD_CANDIDATES = [dict(item_vb=v, item_eb=e) for v, e in [(64, 128), (128, 256), (256, 512), (512, 1024)]]
# feature pieces per chunk of the reverse pass (at most the work item's)
CHUNK_CANDIDATES = [dict(groups_b=g) for g in (2, 3, 4, 5, 8, 16)]
GROUP_CANDIDATES = [dict(groups=g) for g in (4, 8, 16, 32)]
# staging budgets (planes of an SDF-body chunk, vertices of a feature chunk):
# smaller slices keep more warps resident on bodies with many large pieces
STAGE_CANDIDATES = [dict(stage_planes=p, stage_verts=v)
                    for p, v in [(0, 0), (512, 256), (256, 128), (128, 64)]]


def _time(fn, reps=5):
    import torch
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    b.synchronize()
    return a.elapsed_time(b) / reps


def autotune(batch, pose_a, pose_b, ybar=None, direction=None, params=None, verbose=False,
             saved=True):
    """Picks the fastest forward shape, then the fastest reverse-pass shape
    (timed with a direction when one is given, i.e. on the dual kernel).
    ``saved`` (default): time the path a simulation step runs -- the forward
    keeping its record (``ccm_contacts_save``) and the reverse pass from it
    (``ccm_contacts_backward_saved``, per body pair); else the record-free
    calls.  The record does not depend on the shape, so one serves every
    reverse-pass candidate."""
    import torch
    log = {"items": {}, "stage": {}, "forward": {}, "joint": {}, "reverse": {}, "chunks": {}}
    if ybar is None:
        ybar = torch.ones((batch.n_groups, 8), device=pose_a.device)
    rec = batch.saved_buffer(pose_a.device) if saved else None

    def fwd():
        return batch.contacts(pose_a, pose_b, params, saved=rec)

    def bwd():
        return batch.backward(pose_a, pose_b, ybar, direction, params, saved=rec)
    gbest = None
    for cand in GROUP_CANDIDATES:
        try:
            batch.set_tuning(**cand)
            t = _time(lambda: (fwd(), bwd()))
        except Exception as ex:
            log["items"][str(cand)] = repr(ex)
            continue
        log["items"][str(cand)] = t
        if gbest is None or t < gbest[0]:
            gbest = (t, cand)
    batch.set_tuning(**gbest[1])
    stage_timed, fwd_timed = [], []
    sbest = None
    for cand in STAGE_CANDIDATES:
        try:
            batch.set_tuning(**cand)
            t = _time(lambda: (fwd(), bwd()))
        except Exception as ex:
            log["stage"][str(cand)] = repr(ex)
            continue
        log["stage"][str(cand)] = t
        stage_timed.append((t, cand))
        if sbest is None or t < sbest[0]:
            sbest = (t, cand)
    batch.set_tuning(**sbest[1])
    best = None
    for cand in FWD_CANDIDATES:
        try:
            batch.set_tuning(**cand)
            t = _time(fwd)
        except Exception as ex:   # a shape the device cannot hold
            log["forward"][str(cand)] = repr(ex)
            continue
        log["forward"][str(cand)] = t
        fwd_timed.append((t, cand))
        if best is None or t < best[0]:
            best = (t, cand)
    batch.set_tuning(**best[1])
    # the staging budgets and the forward's shape both set how many warps stay
    # resident, so the greedy picks are checked jointly: the two fastest of
    # each, crossed, timed on forward + reverse pass with more repetitions
    def top2(timed):
        return [c for _, c in sorted(timed, key=lambda x: x[0])[:2]]
    jbest = None
    for sc, fc in itertools.product(top2(stage_timed), top2(fwd_timed)):
        try:
            batch.set_tuning(**sc, **fc)
            t = _time(lambda: (fwd(), bwd()), reps=10)
        except Exception as ex:
            log["joint"][str((sc, fc))] = repr(ex)
            continue
        log["joint"][str((sc, fc))] = t
        if jbest is None or t < jbest[0]:
            jbest = (t, {**sc, **fc})
    if jbest is not None:
        batch.set_tuning(**jbest[1])
    if rec is not None:
        fwd()                     # the record of these poses for the reverse candidates
    bbest = None
    for cand in BWD_CANDIDATES:
        try:
            batch.set_tuning(**cand)
            t = _time(bwd)
        except Exception as ex:
            log["reverse"][str(cand)] = repr(ex)
            continue
        log["reverse"][str(cand)] = t
        if bbest is None or t < bbest[0]:
            bbest = (t, cand)
    batch.set_tuning(**bbest[1])
    cbest = None
    for cand in CHUNK_CANDIDATES:
        try:
            batch.set_tuning(**cand)
            t = _time(bwd)
        except Exception as ex:
            log["chunks"][str(cand)] = repr(ex)
            continue
        log["chunks"][str(cand)] = t
        if cbest is None or t < cbest[0]:
            cbest = (t, cand)
    batch.set_tuning(**cbest[1])
    if verbose:
        for k, v in log.items():
            for c, t in sorted(v.items(), key=lambda x: (isinstance(x[1], str), x[1])):
                print(f"{k:8s} {t if isinstance(t, str) else f'{t:8.3f} ms'}  {c}")
    return batch.get_tuning(), log
