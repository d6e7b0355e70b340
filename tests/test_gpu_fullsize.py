"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times, on sampled outputs the oracle recomputes pair by pair:

* the 4096-environment step: 4096 pairs of two 8-piece bodies (seed 2), default
  launch shape, the forward keeping its record, then the gradient pass and the
  H u / J u pass running concurrently on two streams -- its derivatives also
  against central differences (h = 1e-4 and h/2, FP64, Richardson-combined)
  on the sampled environments not flagged near a transition knot;
* the uneven batch: 65,536 body pairs (seed 4), autotuned shape, forward and
  gradient from the record.

A seeded sample of pairs is taken out as a sub-scene (same geometry and
poses) for the oracle; over the whole launch every output must be finite and
every empty group exactly (d_max, 0, 0, 0)."""
import numpy as np
import pytest

from gpu_util import COND_FACTOR, GRAD_RTOL, compare, fp32_sensitivity, report_derivs, weight_slack
from paper_2604_17538_b300 import scenes

pytestmark = pytest.mark.gpu

D_MAX = 0.01   # the default d_max of ccm_default_params


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_17538_b300 import api, build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _rows(off, idx):
    return np.concatenate([np.arange(off[i], off[i + 1]) for i in idx])


def _check_whole(y):
    assert np.all(np.isfinite(y))
    empty = y[:, 1] == 0.0
    assert np.all(y[empty, 0] == np.float32(D_MAX)) and np.all(y[empty, 2:] == 0.0)


def _check_pairs(got, ref, tol, what):
    got = np.asarray(got, np.float64)
    assert np.all(np.isfinite(got)), what
    rt = np.broadcast_to(np.asarray(tol, np.float64), (len(got),))
    report_derivs(got, ref, what, widened=(rt > GRAD_RTOL).sum())
    err = np.abs(got - ref).max(1)
    scale = np.abs(ref).max(1)
    bad = err > tol * scale + 1e-6
    assert not bad.any(), (what, int(bad.sum()), float((err / (scale + 1e-30)).max()))


@pytest.fixture(scope="module")
def hull_step(ctx):
    """The 4096-environment scene and the bench step's outputs on it."""
    import torch
    from paper_2604_17538_b300 import api
    sc = scenes.hull_env_scene(seed=2, n_envs=4096, workers=0)
    batch, pa, pb = api.scene_to_device(sc, ctx)
    n, G = batch.n_pairs, batch.n_groups
    rng = np.random.default_rng(3)
    ybar = rng.normal(size=(G, 8)).astype(np.float32)
    u = rng.normal(size=(n, 12))
    u = (u / np.linalg.norm(u, axis=1, keepdims=True)).astype(np.float32)
    yb, ut = torch.from_numpy(ybar).cuda(), torch.from_numpy(u).cuda()
    # the bench step: record, then both reverse passes concurrently
    saved = batch.saved_buffer()
    g = torch.empty((n, 12), device="cuda")
    g2, h = torch.empty_like(g), torch.empty_like(g)
    j = torch.empty((G, 8), device="cuda")
    main, side = torch.cuda.current_stream(), torch.cuda.Stream()
    y = batch.contacts(pa, pb, saved=saved)
    side.wait_stream(main)
    with torch.cuda.stream(side):
        batch.backward(pa, pb, yb, saved=saved, out=(g, None, None))
    batch.backward(pa, pb, yb, ut, want_jvp=True, saved=saved, out=(g2, h, j))
    main.wait_stream(side)
    torch.cuda.synchronize()
    out = dict(sc=sc, ybar=ybar, u=u)
    out.update({k: t.double().cpu().numpy() for k, t in (("y", y), ("g", g), ("g2", g2),
                                                          ("h", h), ("j", j))})
    batch.close()
    return out


def test_hull_4096_step_sampled_against_oracle(oracle_lib, hull_step):
    sc, ybar, u = hull_step["sc"], hull_step["ybar"], hull_step["u"]
    y, g, g2, h, j = (hull_step[k] for k in ("y", "g", "g2", "h", "j"))
    n = sc.n_pairs
    _check_whole(y)
    assert np.all(np.isfinite(g)) and np.all(np.isfinite(h)) and np.all(np.isfinite(j))

    off = sc.group_offsets()
    idx = np.sort(np.random.default_rng(17).choice(n, 32, replace=False))
    sub = sc.take(idx)
    rows = _rows(off, idx)
    compare(y[rows], oracle_lib.forward(sub), "4096-env y (sampled)", a_slack=weight_slack(sub))
    yb_s, u_s = ybar[rows], u[idx]
    go, ho, jo, _ = oracle_lib.hvp(sub, yb_s, u_s)
    kg, kh = fp32_sensitivity(oracle_lib, sub, yb_s, u_s)
    tol_g = np.maximum(GRAD_RTOL, COND_FACTOR * kg)
    tol_h = np.maximum(GRAD_RTOL, COND_FACTOR * kh)
    _check_pairs(g[idx], go, tol_g, "gradient")
    _check_pairs(g2[idx], go, tol_g, "gradient (dual pass)")
    _check_pairs(h[idx], ho, tol_h, "H u")
    soff = sub.group_offsets()
    js = j[rows]
    for k in range(sub.n_pairs):
        a, b = soff[k], soff[k + 1]
        assert np.abs(js[a:b] - jo[a:b]).max() <= GRAD_RTOL * np.abs(jo[a:b]).max() + 1e-6, k
    assert np.abs(go).max() > 0 and np.abs(ho).max() > 0


def _exp_so3(w):
    """Rotation matrices Exp([w]x) of rotation vectors w [n,3] (Rodrigues)."""
    th = np.linalg.norm(w, axis=1)[:, None, None]
    K = np.zeros((len(w), 3, 3))
    K[:, 0, 1], K[:, 0, 2], K[:, 1, 2] = -w[:, 2], w[:, 1], -w[:, 0]
    K[:, 1, 0], K[:, 2, 0], K[:, 2, 1] = w[:, 2], -w[:, 1], w[:, 0]
    s = np.where(th > 0, np.sin(th) / np.where(th > 0, th, 1), 1.0)
    c = np.where(th > 0, (1 - np.cos(th)) / np.where(th > 0, th * th, 1), 0.5)
    return np.eye(3)[None] + s * K + c * (K @ K)


def _moved(sc, xi):
    """The scene with every pair moved to Exp(xi) T in the twist chart
    (R <- Exp([w]x) R, t <- t + v per body; xi = (w_A, v_A, w_B, v_B)), FP64 poses."""
    out = sc.take(np.arange(sc.n_pairs))
    for P, col in ((sc.pose_a, 0), (sc.pose_b, 6)):
        R, t = scenes.unpack_pose(P.astype(np.float64))
        R2 = _exp_so3(xi[:, col:col + 3]) @ R
        t2 = t + xi[:, col + 3:col + 6]
        Q = np.concatenate([R2.reshape(-1, 9), t2], axis=1)
        if col == 0:
            out.pose_a = Q
        else:
            out.pose_b = Q
    return out


def _knot_flags(oracle_lib, sub, hstep, d_max=D_MAX, eps=0.01):
    """Per pair: True where some contact's SDF value lies within 3 h (lever
    arm) of a knot of the transition (d_max - eps or d_max).  A step of h in
    the twist chart moves a contact's SDF by at most h times the lever arm
    (1 + the largest vertex norm + the distance between the bodies); within
    that of a knot the loss's third derivative jumps and a central difference
    of step h is not accurate to its own truncation order."""
    flags = np.zeros(sub.n_pairs, bool)
    vmax = float(np.linalg.norm(sub.geom.verts, axis=1).max())
    for i in range(sub.n_pairs):
        phi = oracle_lib.pair_contacts(sub, i)[:, 1]
        lever = 1.0 + vmax + float(np.linalg.norm(sub.pose_a[i, 9:] - sub.pose_b[i, 9:]))
        win = 3.0 * hstep * lever
        flags[i] = bool(np.any(np.abs(phi - (d_max - eps)) < win) or
                        np.any(np.abs(phi - d_max) < win))
    return flags


def test_hull_4096_derivatives_against_central_differences(oracle_lib, hull_step):
    """Gradient and H u of the bench step on 256 sampled environments against
    central differences in FP64 with the step the 4096-environment
    differentiation workload names, h = 1e-4, of L = <ybar, y> along each
    twist coordinate for the gradient, and of the fixed-chart gradient along
    +-h u for H u.  Environments with a contact within 3 h (lever arm) of a
    transition knot are flagged and left out.

    A central difference of step h is off by c h^2 + O(h^4): the mollifier's
    curvature makes c large enough that at h = 1e-4 a few environments sit
    above the 1e-3 bar on the truncation alone (the FP64 analytic gradient
    misses them the same way).  So the differences at h and h/2 are combined
    by Richardson extrapolation, (4 D(h/2) - D(h)) / 3, which cancels the h^2
    term; that is held to the parity bar with no allowance.  The plain h = 1e-4
    differences are held to the bar plus their own truncation estimate,
    |D(h) - D(h/2)| 4/3, measured per environment."""
    sc, ybar, u = hull_step["sc"], hull_step["ybar"], hull_step["u"]
    g, h = hull_step["g"], hull_step["h"]
    hstep = 1e-4
    idx0 = np.sort(np.random.default_rng(23).choice(sc.n_pairs, 256, replace=False))
    flags = _knot_flags(oracle_lib, sc.take(idx0), hstep)
    idx = idx0[~flags]
    assert len(idx) >= 64, int(flags.sum())
    sub = sc.take(idx)
    rows = _rows(sc.group_offsets(), idx)
    yb_s, u_s = ybar[rows].astype(np.float64), u[idx].astype(np.float64)
    soff = sub.group_offsets()

    def loss(s):
        y = oracle_lib.forward(s)
        return np.array([np.sum(y[soff[i]:soff[i + 1]] * yb_s[soff[i]:soff[i + 1]])
                         for i in range(s.n_pairs)])

    def differences(step):
        fd_g = np.zeros((sub.n_pairs, 12))
        for k in range(12):
            xi = np.zeros((sub.n_pairs, 12))
            xi[:, k] = step
            fd_g[:, k] = (loss(_moved(sub, xi)) - loss(_moved(sub, -xi))) / (2 * step)
        gp, _ = oracle_lib.gradient(sub, yb_s, xi=step * u_s)
        gm, _ = oracle_lib.gradient(sub, yb_s, xi=-step * u_s)
        return fd_g, (gp - gm) / (2 * step)
    g1, h1 = differences(hstep)
    g2, h2 = differences(hstep / 2)
    kg, kh = fp32_sensitivity(oracle_lib, sub, ybar[rows], u[idx])
    tol_g, tol_h = np.maximum(GRAD_RTOL, COND_FACTOR * kg), np.maximum(GRAD_RTOL, COND_FACTOR * kh)
    print(f"central differences at h = {hstep}: {int(flags.sum())} of {len(idx0)} "
          "environments flagged near a transition knot")
    _check_pairs(g[idx], (4 * g2 - g1) / 3, tol_g, "gradient vs FD (h=1e-4, Richardson)")
    _check_pairs(h[idx], (4 * h2 - h1) / 3, tol_h, "H u vs FD (h=1e-4, Richardson)")
    for got, d1, d2, tol, what in ((g[idx], g1, g2, tol_g, "gradient"), (h[idx], h1, h2, tol_h, "H u")):
        trunc = np.abs(d1 - d2).max(1) * 4 / 3
        err = np.abs(got - d1).max(1)
        scale = np.abs(d1).max(1)
        over = err > tol * scale + 1e-6
        print(f"{what} vs plain FD (h=1e-4): {int(over.sum())} of {len(idx)} environments above "
              f"the bar, largest truncation estimate "
              f"{float((trunc / np.maximum(scale, 1e-30)).max()):.2e} relative")
        assert np.all(err <= tol * scale + 1.5 * trunc + 1e-6), what
    assert np.abs(g1).max() > 0 and np.abs(h1).max() > 0


def test_uneven_65536_autotuned_sampled_against_oracle(oracle_lib, ctx):
    import torch
    from paper_2604_17538_b300 import api, tune
    sc = scenes.uneven_scene(seed=4, n_pairs=65536, workers=0)
    batch, pa, pb = api.scene_to_device(sc, ctx)
    n, G = batch.n_pairs, batch.n_groups
    ybar = np.random.default_rng(3).normal(size=(G, 8)).astype(np.float32)
    yb = torch.from_numpy(ybar).cuda()
    tune.autotune(batch, pa, pb, yb)
    saved = batch.saved_buffer()
    y = batch.contacts(pa, pb, saved=saved)
    g, _, _ = batch.backward(pa, pb, yb, saved=saved)
    torch.cuda.synchronize()
    y, g = y.double().cpu().numpy(), g.double().cpu().numpy()
    _check_whole(y)
    assert np.all(np.isfinite(g))

    off = sc.group_offsets()
    npb = np.diff(sc.geom.body_piece_off)
    pp = npb[sc.pair_a] * npb[sc.pair_b]
    rng = np.random.default_rng(19)
    # a sample across the range of sizes: pairs of up to 256 piece pairs, the
    # largest counts among them, and the 8 heaviest pairs of the launch (over
    # 1,024 piece pairs each), whose bodies span many staged chunks in the
    # autotuned shape
    light = np.nonzero(pp <= 256)[0]
    heavy = np.argsort(pp, kind="stable")[-8:]
    assert pp[heavy].min() > 1024
    idx = np.sort(np.concatenate([rng.choice(light, 20, replace=False),
                                  light[np.argsort(pp[light])[-4:]], heavy]))
    idx = np.unique(idx)
    sub = sc.take(idx)
    rows = _rows(off, idx)
    compare(y[rows], oracle_lib.forward(sub), "uneven y (sampled)", a_slack=weight_slack(sub))
    yb_s = ybar[rows]
    go, _ = oracle_lib.gradient(sub, yb_s)
    u0 = np.zeros((sub.n_pairs, 12), np.float32)
    kg, _ = fp32_sensitivity(oracle_lib, sub, yb_s, u0)
    _check_pairs(g[idx], go, np.maximum(GRAD_RTOL, COND_FACTOR * kg), "uneven gradient")
    batch.close()
