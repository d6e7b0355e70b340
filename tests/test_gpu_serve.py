"""Serving loop (ccm_serve_start / ccm_submit / ccm_poll): served results equal
the batched entry points and the oracle, a request's results are bitwise the
same alone and in any mix of concurrent requests, queued requests are packed
into waves, and admission errors are reported."""
import numpy as np
import pytest

from gpu_util import GRAD_RTOL, compare, weight_slack
from paper_2604_17538_b300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def uneven():
    # geometry as in the uneven batch: pieces log-uniform in [1, 64], hull
    # points log-uniform in [8, 512]
    return scenes.uneven_scene(seed=9, n_pairs=160, pool_bodies=48, workers=0)


@pytest.fixture(scope="module")
def dev(uneven):
    """(ctx, handles, pose_a, pose_b) with the scene's geometry resident."""
    import torch
    from paper_2604_17538_b300 import api, build
    build.build()
    sc = uneven
    ctx = api.Context(0)
    handles = ctx.load_geometry(sc.geom)
    pa = torch.from_numpy(sc.pose_a.astype(np.float32)).cuda()
    pb = torch.from_numpy(sc.pose_b.astype(np.float32)).cuda()
    yield ctx, handles, pa, pb
    ctx.close()


def _requests(sc, rng, n_req, max_n=24):
    """(start, stop, with_grad) slices of the scene's pairs."""
    out = []
    for _ in range(n_req):
        n = int(scenes.log_uniform_int(rng, 1, max_n, size=1)[0])
        i0 = int(rng.integers(0, sc.n_pairs - n + 1))
        out.append((i0, i0 + n, bool(rng.uniform() < 0.5)))
    return out


def _ybar(sc, i0, i1, seed):
    import torch
    G = int(sc.group_offsets()[i1] - sc.group_offsets()[i0])
    r = np.random.default_rng([seed, i0, i1])
    return torch.from_numpy(r.normal(size=(G, 8)).astype(np.float32)).cuda()


def _submit(srv, sc, handles, pa, pb, req, seed=0):
    i0, i1, grad = req
    ybar = _ybar(sc, i0, i1, seed) if grad else None
    t, y, g = srv.submit(handles[sc.pair_a[i0:i1]], handles[sc.pair_b[i0:i1]],
                         pa[i0:i1], pb[i0:i1], ybar=ybar)
    return t, y, g, ybar


def _wait_all(srv, tickets):
    return [srv.wait(t, timeout_s=120.0) for t in tickets]


def test_served_results_match_batched_calls_and_oracle(dev, uneven, oracle_lib):
    import torch
    from paper_2604_17538_b300 import api
    ctx, handles, pa, pb = dev
    srv = api.Server(ctx, max_wave_pairs=256, max_wave_requests=32)
    try:
        rng = np.random.default_rng(3)
        reqs = _requests(uneven, rng, 40)
        subs = [_submit(srv, uneven, handles, pa, pb, r) for r in reqs]
        _wait_all(srv, [s[0] for s in subs])
        assert srv.stats()["served"] == len(reqs)
        slack = weight_slack(uneven)
        for (i0, i1, grad), (_, y, g, ybar) in zip(reqs, subs):
            batch = ctx.batch(handles[uneven.pair_a[i0:i1]], handles[uneven.pair_b[i0:i1]])
            yb = batch.contacts(pa[i0:i1].contiguous(), pb[i0:i1].contiguous())
            torch.cuda.synchronize()
            compare(y.double().cpu().numpy(), yb.double().cpu().numpy(), "served vs batched",
                    a_slack=slack)
            if grad:
                gb, _, _ = batch.backward(pa[i0:i1].contiguous(), pb[i0:i1].contiguous(), ybar)
                torch.cuda.synchronize()
                a = g.double().cpu().numpy()
                b = gb.double().cpu().numpy()
                assert np.all(np.isfinite(a))
                err = np.abs(a - b).max(1)
                assert np.all(err <= GRAD_RTOL * np.abs(b).max(1) + 1e-6), float(err.max())
            batch.close()
        # one served request against the FP64 oracle directly
        i0, i1, _ = reqs[0]
        ref = oracle_lib.forward(uneven.take(np.arange(i0, i1)))
        print("served vs oracle", compare(subs[0][1].double().cpu().numpy(), ref, "served",
                                          a_slack=slack))
    finally:
        srv.close()


def test_request_alone_equals_request_in_mix(dev, uneven):
    """Bitwise: the same request run alone, packed into one wave with others,
    and among free-running overlapping waves."""
    from paper_2604_17538_b300 import api
    ctx, handles, pa, pb = dev
    srv = api.Server(ctx, max_wave_pairs=1024, max_wave_requests=64)
    try:
        probe = [(10, 22, True), (100, 101, False), (40, 64, True)]
        alone = []
        for r in probe:
            t, y, g, _ = _submit(srv, uneven, handles, pa, pb, r, seed=1)
            srv.wait(t)
            alone.append((y.cpu().numpy().copy(), None if g is None else g.cpu().numpy().copy()))
        rng = np.random.default_rng(5)
        # (1) all in one wave, the probes at different offsets of it
        srv.hold(True)
        w0 = srv.stats()["waves"]
        others = [_submit(srv, uneven, handles, pa, pb, r) for r in _requests(uneven, rng, 12)]
        mixed = [_submit(srv, uneven, handles, pa, pb, r, seed=1) for r in probe]
        others += [_submit(srv, uneven, handles, pa, pb, r) for r in _requests(uneven, rng, 12)]
        srv.hold(False)
        _wait_all(srv, [s[0] for s in others + mixed])
        assert srv.stats()["waves"] == w0 + 1
        for (ya, ga), (_, y, g, _) in zip(alone, mixed):
            assert np.array_equal(ya, y.cpu().numpy())
            if ga is not None:
                assert np.array_equal(ga, g.cpu().numpy())
        # the completion queue retires what ccm_poll has not: nothing here
        assert srv.completed() == []
        # (2) free-running: requests join whichever wave forms next
        subs = []
        for k in range(60):
            subs.append(_submit(srv, uneven, handles, pa, pb, _requests(uneven, rng, 1)[0]))
            if k % 20 == 7:
                subs.append(("probe",) + _submit(srv, uneven, handles, pa, pb, probe[0], seed=1))
        _wait_all(srv, [s[1] if s[0] == "probe" else s[0] for s in subs])
        for s in subs:
            if s[0] == "probe":
                assert np.array_equal(alone[0][0], s[2].cpu().numpy())
                assert np.array_equal(alone[0][1], s[3].cpu().numpy())
    finally:
        srv.close()


def test_admission_and_ticket_errors(dev, uneven):
    import torch
    from paper_2604_17538_b300 import abi, api
    ctx, handles, pa, pb = dev
    srv = api.Server(ctx, max_wave_pairs=32, max_wave_requests=8, max_queued=4)
    try:
        srv.hold(True)
        subs = [_submit(srv, uneven, handles, pa, pb, (k, k + 2, False)) for k in range(4)]
        with pytest.raises(abi.CcmError) as e:        # the queue holds four
            _submit(srv, uneven, handles, pa, pb, (0, 2, False))
        assert e.value.status == abi.CCM_ERR_BUSY
        with pytest.raises(abi.CcmError) as e:        # larger than any wave
            _submit(srv, uneven, handles, pa, pb, (0, 33, False))
        assert e.value.status == abi.CCM_ERR_OOM
        bad = np.array([123456789], np.uint64)
        with pytest.raises(abi.CcmError) as e:
            srv.submit(bad, handles[:1], pa[:1], pb[:1])
        assert e.value.status == abi.CCM_ERR_INVALID
        assert srv.poll(subs[0][0]) == (False, None)  # queued, not run while held
        srv.hold(False)
        _wait_all(srv, [s[0] for s in subs])
        with pytest.raises(abi.CcmError) as e:        # retired
            srv.poll(subs[0][0])
        assert e.value.status == abi.CCM_ERR_UNKNOWN_TICKET
        with pytest.raises(abi.CcmError) as e:
            srv.poll(987654321)
        assert e.value.status == abi.CCM_ERR_UNKNOWN_TICKET
        with pytest.raises(abi.CcmError) as e:        # one loop per context
            api.Server(ctx)
        assert e.value.status == abi.CCM_ERR_INVALID
    finally:
        srv.close()
    torch.cuda.synchronize()


def test_budget_bounds_the_wave_buffers(uneven):
    from paper_2604_17538_b300 import abi, api
    small = api.Context(0, hbm_budget_bytes=1 << 20)
    try:
        handles = small.load_geometry(uneven.geom)
        with pytest.raises(abi.CcmError) as e:
            api.Server(small, max_wave_pairs=16384)
        assert e.value.status == abi.CCM_ERR_OOM
        srv = api.Server(small, max_wave_pairs=0, max_wave_requests=16)   # from the budget
        srv.close()
    finally:
        small.close()
    assert handles is not None


def test_completion_queue_reports_each_request_once(dev, uneven):
    from paper_2604_17538_b300 import abi, api
    ctx, handles, pa, pb = dev
    srv = api.Server(ctx, max_wave_pairs=256, max_wave_requests=16)
    try:
        rng = np.random.default_rng(8)
        subs = [_submit(srv, uneven, handles, pa, pb, r) for r in _requests(uneven, rng, 30)]
        tickets = {s[0] for s in subs}
        first = subs[0][0]
        srv.wait(first)                      # retired by ccm_poll: skipped below
        seen = {}
        import time
        t_end = time.perf_counter() + 60
        while len(seen) < len(tickets) - 1 and time.perf_counter() < t_end:
            for tk, lat in srv.completed(max_n=7):
                assert tk not in seen and tk in tickets and tk != first
                assert 0.0 <= lat < 60.0
                seen[tk] = lat
        assert len(seen) == len(tickets) - 1
        assert srv.completed() == []
        with pytest.raises(abi.CcmError) as e:   # retired by the completion queue
            srv.poll(next(iter(seen)))
        assert e.value.status == abi.CCM_ERR_UNKNOWN_TICKET
    finally:
        srv.close()


def test_stop_runs_queued_requests(dev, uneven):
    import torch
    from paper_2604_17538_b300 import api
    ctx, handles, pa, pb = dev
    srv = api.Server(ctx, max_wave_pairs=64, max_wave_requests=8)
    srv.hold(True)
    subs = [_submit(srv, uneven, handles, pa, pb, (8 * k, 8 * k + 8, k % 2 == 0))
            for k in range(6)]
    srv.close()                                    # drains through a released hold
    for k, (_, y, g, ybar) in enumerate(subs):
        batch = ctx.batch(handles[uneven.pair_a[8 * k:8 * k + 8]],
                          handles[uneven.pair_b[8 * k:8 * k + 8]])
        yb = batch.contacts(pa[8 * k:8 * k + 8].contiguous(), pb[8 * k:8 * k + 8].contiguous())
        torch.cuda.synchronize()
        compare(y.double().cpu().numpy(), yb.double().cpu().numpy(), "drained",
                a_slack=weight_slack(uneven))
        batch.close()


def test_replay_submits_on_schedule_and_matches_direct_submission(dev, uneven):
    """ccm_serve_replay (the native load generator): every request completes,
    none is submitted before its arrival, latency >= lag >= 0, and its results
    are bitwise those of the same requests submitted through ccm_submit."""
    import ctypes as C
    import torch
    from paper_2604_17538_b300 import abi, api
    ctx, handles, pa, pb = dev
    rng = np.random.default_rng(12)
    reqs = _requests(uneven, rng, 24)
    # reference: the same requests through ccm_submit, all queued before one wave
    srv = api.Server(ctx, max_wave_pairs=512, max_wave_requests=64)
    try:
        srv.hold(True)
        subs = [_submit(srv, uneven, handles, pa, pb, r, seed=4) for r in reqs]
        srv.hold(False)
        _wait_all(srv, [s[0] for s in subs])
    finally:
        srv.close()
    n = len(reqs)
    arr = np.cumsum(rng.exponential(2e-4, size=n))
    keep, table = [], (abi.ccm_request * n)()
    outs = []
    for k, (i0, i1, grad) in enumerate(reqs):
        A = np.ascontiguousarray(handles[uneven.pair_a[i0:i1]], np.uint64)
        B = np.ascontiguousarray(handles[uneven.pair_b[i0:i1]], np.uint64)
        G = int(uneven.group_offsets()[i1] - uneven.group_offsets()[i0])
        y = torch.empty((G, 8), device="cuda")
        g = torch.empty((i1 - i0, 12), device="cuda") if grad else None
        yb = _ybar(uneven, i0, i1, 4) if grad else None
        keep += [A, B, y, g, yb]
        outs.append((y, g))
        table[k] = abi.ccm_request(i1 - i0, A.ctypes.data, B.ctypes.data,
                                   pa[i0:i1].data_ptr(), pb[i0:i1].data_ptr(), y.data_ptr(),
                                   yb.data_ptr() if grad else None,
                                   g.data_ptr() if grad else None)
    lag, lat, el = np.full(n, -1.0), np.full(n, -1.0), C.c_double()
    srv = api.Server(ctx, max_wave_pairs=512, max_wave_requests=64)
    try:
        abi.check(abi.lib().ccm_serve_replay(ctx.handle, C.cast(table, C.c_void_p),
                                             arr.ctypes.data, n, lag.ctypes.data,
                                             lat.ctypes.data, C.byref(el)))
        assert srv.stats()["served"] == n
    finally:
        srv.close()
    torch.cuda.synchronize()
    assert np.all(lag >= 0.0) and np.all(lat >= lag) and np.all(lat < 60.0)
    assert el.value >= arr[-1] and el.value >= float((arr + lat).max()) - 1e-3
    # results are independent of the wave mix (bitwise)
    for (_, y0, g0, _), (y, g) in zip(subs, outs):
        assert torch.equal(y0, y)
        if g is not None:
            assert torch.equal(g0, g)
    # argument errors
    bad = np.array([1.0, 0.5])
    assert abi.lib().ccm_serve_replay(ctx.handle, C.cast(table, C.c_void_p), bad.ctypes.data,
                                      2, None, None, None) == abi.CCM_ERR_INVALID
