#!/usr/bin/env python3
"""Benchmark of the contact-manifold hot path on B300.

A step is one pass of the whole path over one batch of synthetic input:
forward contacts (gate, V-SDF / E-SDF narrow phase, blending), the reverse
pass (pose gradients) and the forward-over-reverse pass (Hessian-vector
products and output tangents) on 4096 environments of two 8-piece bodies
(262,144 piece pairs), with inputs resident in HBM.  The metric is piece-pair
contact queries per second.  ``--impl reference`` times the FP64 CPU oracle
on the same workload instead (a bounded sample per step).

Multi-GPU (torchrun): every rank runs its own 4096 environments (different
seed), weak scaling; the only collectives are a barrier and the max of the
timings -- there is no data-path exchange.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "piece-pair contact queries/sec fwd and fwd+bwd vs roofline; served p50/p99 latency"
UNIT = "piece-pair queries/s"
N_ENVS = 4096
PIECES = 8
POINTS = 64
WORKLOAD = ("4096 envs x 2 bodies x 8 hull pieces (64 pts); fwd + grad + HVP (the gradient "
            "as the primal part of the forward-over-reverse pass)")

# FLOP and SFU cost per plane evaluation of each kind (an FMA is 2 FLOP):
#   gate / max-plane: 3 FMA + max = 7;  value: 3 FMA + scale FMA + add = 9 + 1 ex2;
#   value + gradient: 9 + 3 FMA = 15 + 1 ex2;
#   value + gradient + Hessian-vector product: 15 + 5 (n.v) + 1 + 6 = 27 + 1 ex2;
#   dual-number versions (value + one tangent): gate 7, value 20, value+grad 32,
#   value+grad+Hv 59, each + 1 ex2.
COST = {"gate": 7, "val": 9, "grad": 15, "hv": 27, "dval": 20, "dgrad": 32, "dhv": 59}


def work_model(c, cv, ch):
    """Algorithmic FLOP and ex2 counts per launch from exact device counters:
    ``c`` of the forward, ``cv`` / ``ch`` of the reverse pass on float / on
    dual numbers (plane evaluations by kind and pass)."""
    gm = c["gatepass"] + c["maxpass"]
    eg, ev = c["eval_grad"], c["eval_val"]
    fwd = (COST["gate"] * gm + COST["grad"] * eg + COST["val"] * ev, eg + ev)

    def rev(k, dual):
        g, v, h = ("dgrad", "dval", "dhv") if dual else ("grad", "val", "hv")
        flop = (COST["gate"] * (k["gatepass"] + k["maxpass"]) + COST[g] * k["p1_grad"]
                + COST[v] * k["p1_val"] + COST[h] * k["p2_hv"] + COST[g] * k["p2_grad"])
        return flop, k["p1_grad"] + k["p1_val"] + k["p2_hv"] + k["p2_grad"]
    return {"forward": fwd, "vjp": rev(cv, False), "hvp": rev(ch, True)}


def kernel_source_hash():
    """sha256 of the contact kernels' device sources (the forward and reverse
    kernels and the headers they include, not the host-side runtime), to
    tell whether recorded ncu counters still apply."""
    import glob
    import hashlib
    d = os.path.join(ROOT, "paper_2604_17538_b300", "csrc")
    files = sorted(glob.glob(os.path.join(d, "*.cuh"))) + [
        os.path.join(d, f) for f in ("ccm_fwd.cu", "ccm_fwd.h", "ccm_bwd.cu", "ccm_bwd.h",
                                     "ccm_ffwd.cu", "ccm_ffwd.h", "ccm_flat.cu", "ccm_flat.h",
                                     "ccm_launch.h")]
    return hashlib.sha256(b"".join(open(f, "rb").read() for f in files)).hexdigest()


def derived_peaks(n_sm=148, clock_ghz=2.032, sfu_per_clk=32):
    """FP32: 128 FMA lanes per SM; SFU ex2: sfu_per_clk per SM (measured by
    the probe); both at the maximum SM clock."""
    return {"fp32_tflops": n_sm * 128 * 2 * clock_ghz / 1e3,
            "ex2_tops": n_sm * sfu_per_clk * clock_ghz / 1e3}


def alu_roofline(local, per, model, workload_key):
    """Roofline object of the dominant contact kernel: ``per`` = average
    launch duration (s) of each pass from CUDA events, ``model`` = the
    algorithmic (FLOP, ex2) of one launch of each pass (work_model).  The
    FP32 and ex2 peaks are derived from the SM count and the maximum clock,
    the ex2 rate per clock from the library's probe.  DRAM traffic per launch
    comes from profiles/traffic.json when a record there matches the kernel,
    the workload (``workload_key``) and the current kernel sources."""
    import ctypes as C
    import torch
    from paper_2604_17538_b300 import abi
    probe = {}
    try:
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        abi.check(abi.lib().ccm_peak_probe(local, C.byref(a), C.byref(b), C.byref(c)))
        probe = {"ffma_tflops": a.value, "ffma2_tflops": b.value, "ex2_tops": c.value}
    except Exception as ex:  # measurement aid only
        probe = {"error": str(ex)}
    props = torch.cuda.get_device_properties(local)
    sfu_per_clk = 32
    if "ex2_tops" in probe:
        # per-SM per-clock ex2 rate implied by the probe, rounded to the unit width
        r = probe["ex2_tops"] * 1e12 / (props.multi_processor_count * 2.032e9)
        sfu_per_clk = max(16, int(round(r / 16.0)) * 16)
    peaks = derived_peaks(props.multi_processor_count, 2.032, sfu_per_clk)
    dom = max(per, key=per.get)
    flop, ex2 = model[dom]
    fp32_ach = flop / per[dom] / 1e12
    ex2_ach = ex2 / per[dom] / 1e12
    fr_fp32 = fp32_ach / peaks["fp32_tflops"]
    fr_ex2 = ex2_ach / peaks["ex2_tops"]
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        # counters only count while the kernel sources are the ones captured
        for tr in json.load(open(tpath)):
            if (tr.get("kernel") == dom
                    and all(tr.get(k) == v for k, v in workload_key.items())
                    and tr.get("source_sha256") == kernel_source_hash()):
                traffic = tr.get("bytes_per_launch")
    return {"bound": "alu", "kernel": dom, "pipe": "fp32" if fr_fp32 >= fr_ex2 else "sfu_ex2",
            "achieved": fp32_ach, "peak": peaks["fp32_tflops"], "unit": "TFLOP/s",
            "frac": max(fr_fp32, fr_ex2), "frac_fp32": fr_fp32, "frac_ex2": fr_ex2,
            "ex2_achieved_tops": ex2_ach, "ex2_peak_tops": peaks["ex2_tops"],
            "ms_per_launch": 1e3 * per[dom],
            "peak_source": "derived: 148 SM x 128 FP32 lanes x 2 x 2.032 GHz; ex2: SM x "
                           f"{sfu_per_clk}/clk x 2.032 GHz (per-clock rate from the probe)",
            "probe": probe, "traffic": traffic, "flop_per_launch": flop,
            "ex2_per_launch": ex2}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.device_index = device_index
        self.proc = None
        self.path = os.path.join("/tmp", f"ccm_clocks_{os.getpid()}.csv")

    def _lines(self):
        try:
            with open(self.path) as f:
                return sum(1 for ln in f if ln.strip())
        except OSError:
            return 0

    def start(self):
        """Starts nvidia-smi and waits (at most 5 s) for its first sample, so
        that sampling is live when the timed region begins; samples taken
        before then are not reported."""
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device_index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t0 = time.perf_counter()
        while self._lines() == 0 and time.perf_counter() - t0 < 5.0:
            time.sleep(0.01)
        self.skip = self._lines()

    def extend(self, step, min_samples=3, max_s=3.0):
        """A timed region shorter than the sampling interval holds no sample:
        the same work then keeps running, untimed, until `min_samples` samples
        were taken since the timed region began (at most `max_s` seconds)."""
        import torch
        if self.proc is None:
            return
        self.extended = 0
        t0 = time.perf_counter()
        while self._lines() - self.skip < min_samples and time.perf_counter() - t0 < max_s:
            for _ in range(4):
                step()
            torch.cuda.synchronize()
            self.extended += 4

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = [ln for ln in open(self.path) if ln.strip()][getattr(self, "skip", 0):]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
               "reasons": sorted(reasons)}
        if getattr(self, "extended", 0):
            out["window"] = (f"timed loop, then {self.extended} untimed steps of the same work "
                             "until 3 samples (100 ms interval)")
        return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world):
    from paper_2604_17538_b300 import scenes, shard
    seed = shard.shard_seed(2, rank)
    sc = scenes.hull_env_scene(seed=seed, n_envs=args.envs, workers=0)

    import torch
    import torch.distributed as dist
    from paper_2604_17538_b300 import abi, api, build
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    ctx = api.Context(local)
    batch, pa, pb = api.scene_to_device(sc, ctx)
    n, G = batch.n_pairs, batch.n_groups
    rng = np.random.default_rng(3 + rank)
    ybar_h = rng.normal(size=(G, 8)).astype(np.float32)
    u_h = rng.normal(size=(n, 12))
    u_h = (u_h / np.linalg.norm(u_h, axis=1, keepdims=True)).astype(np.float32)
    ybar = torch.from_numpy(ybar_h).cuda()
    u = torch.from_numpy(u_h).cuda()
    piece_pairs = sc.piece_pairs()

    y = torch.empty((G, 8), device="cuda")
    saved = batch.saved_buffer()

    # exact work counters of the three passes (outside the timed region)
    cnt = torch.zeros(8, dtype=torch.int64, device="cuda")
    batch.contacts(pa, pb, counters=cnt)
    counters = dict(zip(abi.COUNTER_NAMES, cnt.cpu().tolist()))
    batch.contacts(pa, pb, out=y, saved=saved)
    cnt_v = torch.zeros(8, dtype=torch.int64, device="cuda")
    batch.backward(pa, pb, ybar, saved=saved, counters=cnt_v)
    cnt_h = torch.zeros(8, dtype=torch.int64, device="cuda")
    batch.backward(pa, pb, ybar, u, want_jvp=True, saved=saved, counters=cnt_h)
    counters_vjp = dict(zip(abi.BWD_COUNTER_NAMES, cnt_v.cpu().tolist()))
    counters_hvp = dict(zip(abi.BWD_COUNTER_NAMES, cnt_h.cpu().tolist()))
    model = work_model(counters, counters_vjp, counters_hvp)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    # one step: the forward keeping its record for the reverse passes (as the
    # autograd Function does), then the gradient pass and the H u / J u pass,
    # which both read only the record: they run concurrently, the gradient
    # pass on a side stream (every body here has <= 256 pieces, the per-pair
    # passes count their work on separate words)
    g_o, g2_o = (torch.empty((n, 12), device="cuda") for _ in range(2))
    h_o2, j_o2 = torch.empty((n, 12), device="cuda"), torch.empty((G, 8), device="cuda")

    def step(e_fwd=None):
        # the forward keeping its record and contact list, then one
        # forward-over-reverse pass: its primal part is the gradient, its
        # tangents H u and J u
        batch.contacts(pa, pb, out=y, saved=saved)
        if e_fwd is not None:
            e_fwd.record(stream)
        batch.backward(pa, pb, ybar, u, want_jvp=True, saved=saved, out=(g_o, h_o2, j_o2))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t_wall0 = time.perf_counter()
    n_launch0 = abi.kernel_launches()
    for k in range(args.steps):
        flush.zero_()                       # L2 (126 MB) flushed between steps, untimed
        e = evs[k]
        e[0].record(stream)
        step(e[1])
        e[2].record(stream)
    n_launches = abi.kernel_launches() - n_launch0
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    sampler.extend(step)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    t_fwd = sum(e[0].elapsed_time(e[1]) for e in evs) / 1e3
    t_step = sum(e[0].elapsed_time(e[2]) for e in evs) / 1e3

    # the passes one after the other on one stream, for the per-pass times
    # (breakdown and the dominant kernel's launch duration)
    evp = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        e = evp[k]
        e[0].record(stream)
        batch.contacts(pa, pb, out=y, saved=saved)
        e[1].record(stream)
        batch.backward(pa, pb, ybar, saved=saved, out=(g_o, None, None))
        e[2].record(stream)
        batch.backward(pa, pb, ybar, u, want_jvp=True, saved=saved, out=(g2_o, h_o2, j_o2))
        e[3].record(stream)
    torch.cuda.synchronize()
    t_fwd_seq = sum(e[0].elapsed_time(e[1]) for e in evp) / 1e3
    t_vjp = sum(e[1].elapsed_time(e[2]) for e in evp) / 1e3
    t_hvp = sum(e[2].elapsed_time(e[3]) for e in evp) / 1e3

    # end to end through the public API with host buffers: one
    # ccm_contacts_step_host call per step copies the step's inputs in from
    # pinned host memory, runs the three passes and copies every result back
    # (the cotangent and direction copies and the copies of y and of the
    # gradient overlap the kernels on side streams)
    pa_h = torch.from_numpy(sc.pose_a).pin_memory()
    pb_h = torch.from_numpy(sc.pose_b).pin_memory()
    yb_h = torch.from_numpy(ybar_h).pin_memory()
    uu_h = torch.from_numpy(u_h).pin_memory()
    y_o = torch.empty((G, 8)).pin_memory()
    g_o = torch.empty((n, 12)).pin_memory()
    h_o = torch.empty((n, 12)).pin_memory()
    j_o = torch.empty((G, 8)).pin_memory()
    h2d = sum(x.numel() * 4 for x in (pa_h, pb_h, yb_h, uu_h))
    d2h = sum(x.numel() * 4 for x in (y_o, g_o, h_o, j_o))

    def e2e_step():
        batch.step_host(pa_h, pb_h, yb_h, uu_h, want_jvp=True, out=(y_o, g_o, h_o, j_o),
                        stream=stream)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    t_e2e = 0.0
    for _ in range(args.steps):
        flush.zero_()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        e2e_step()
        a1.record(stream)
        a1.synchronize()
        t_e2e += a0.elapsed_time(a1) / 1e3

    # max over ranks of the times, sum over ranks of the work
    t_step, t_fwd, t_vjp, t_hvp, t_e2e = shard.reduce_max([t_step, t_fwd, t_vjp, t_hvp, t_e2e],
                                                          "cuda")
    (total_pp,) = shard.reduce_sum([piece_pairs], "cuda")
    K = args.steps

    out = None
    if rank == 0:
        per = {"forward": t_fwd / K, "vjp": t_vjp / K, "hvp": t_hvp / K}
        roof = alu_roofline(local, per, model, {"envs": args.envs})
        out = {
            "metric": METRIC, "value": total_pp * K / t_step, "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": 1e3 * t_step / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded convex-hull scenes)",
            "config": {"workload": WORKLOAD, "n_envs_per_gpu": args.envs, "pieces_per_body": PIECES,
                       "points_per_hull": POINTS, "piece_pairs_per_gpu": piece_pairs,
                       "l2": "flushed between timed steps (512 MiB write, untimed)",
                       "parallelism": f"independent shards x{world}"},
            "breakdown": {"fwd_qps": total_pp * K / t_fwd,
                          "fwd_bwd_qps": total_pp * K / (t_fwd + t_vjp),
                          "fwd_bwd_hvp_qps": total_pp * K / t_step,
                          "ms_forward": 1e3 * t_fwd / K,
                          "ms_reverse": 1e3 * (t_step - t_fwd) / K,
                          "ms_vjp": 1e3 * t_vjp / K, "ms_hvp": 1e3 * t_hvp / K,
                          "note": "the step's reverse pass is one forward-over-reverse pass "
                                  "(gradient as its primal part, H u and J u as its tangents; "
                                  "ms_reverse); ms_vjp / ms_hvp time the gradient-only pass "
                                  "and that pass alone in a second loop, and fwd_bwd_qps is "
                                  "forward + gradient-only pass"},
            "e2e": {"value": total_pp * K / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            # the library's own count of the kernels it launched in the
            # timed loop (the flat forward's stages and the per-item kernel
            # behind them, the reverse pass's stages and the per-pair kernel)
            "gpu_launches": n_launches,
            "roofline": roof,
            "work_counters": {"forward": counters, "vjp": counters_vjp, "hvp": counters_hvp},
            "clocks": clocks,
            "wall_s_timed_loop": t_wall,
        }
    return out, sc


# ---------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------
def oracle_sample_rate(sc, target_s=12.0, kind="hvp", what="environments"):
    """Times the oracle on a bounded seeded sample of the scene's pairs:
    kind "hvp" = forward, gradient and H u in one nested-dual pass, "grad" =
    the forward and the gradient, "fwd" = the forward alone; returns (qps,
    cores, sample, seconds)."""
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    rng = np.random.default_rng(7)
    order = rng.permutation(sc.n_pairs)

    def run(k):
        sub = sc.take(order[:k])
        G = int(sub.group_offsets()[-1])
        yb = np.random.default_rng(3).normal(size=(G, 8))
        u = np.random.default_rng(4).normal(size=(k, 12))
        t0 = time.perf_counter()
        if kind == "hvp":
            oracle.hvp(sub, yb, u, threads=cores)
        else:
            oracle.forward(sub, threads=cores)
            if kind == "grad":
                oracle.gradient(sub, yb, threads=cores)
        return time.perf_counter() - t0, sub.piece_pairs()

    k = min(16, sc.n_pairs)
    dt, pp = run(k)
    while dt < target_s / 4 and k < sc.n_pairs:
        k = min(sc.n_pairs, int(k * max(2.0, target_s / max(dt, 1e-3) / 2)))
        dt, pp = run(k)
    return pp / dt, cores, f"{k} of {sc.n_pairs} {what} ({pp} piece pairs), seeded", dt


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from paper_2604_17538_b300 import scenes
    sc = scenes.hull_env_scene(seed=2, n_envs=args.envs, workers=0)
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    rng = np.random.default_rng(7)
    k = min(args.ref_sample, sc.n_pairs)
    sub = sc.take(rng.permutation(sc.n_pairs)[:k])
    G = int(sub.group_offsets()[-1])
    yb = np.random.default_rng(3).normal(size=(G, 8))
    u = np.random.default_rng(4).normal(size=(k, 12))
    for _ in range(max(0, min(args.warmup, 1))):
        oracle.hvp(sub, yb, u, threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.hvp(sub, yb, u, threads=cores)
    dt = time.perf_counter() - t0
    qps = sub.piece_pairs() * args.steps / dt
    sample = f"{k} of {sc.n_pairs} environments per step ({sub.piece_pairs()} piece pairs), seeded"
    return {"impl": "reference", "metric": METRIC, "value": qps, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded convex-hull scenes)",
            "config": {"workload": WORKLOAD, "n_envs_per_gpu": args.envs, "pieces_per_body": PIECES,
                       "points_per_hull": POINTS},
            "cpu_baseline": {"value": qps, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": qps, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_uneven(args, rank, world):
    """Uneven batch: 65,536 body pairs, pieces per body log-uniform in [1, 64],
    hull points log-uniform in [8, 512]; autotuned shape (or the one --tuning
    gives); forward + gradient captured once in a CUDA graph and replayed."""
    from paper_2604_17538_b300 import scenes
    t0 = time.perf_counter()
    from paper_2604_17538_b300 import shard
    sc = scenes.uneven_scene(seed=shard.shard_seed(4, rank), n_pairs=args.pairs, workers=0)
    t_gen = time.perf_counter() - t0
    import torch
    from paper_2604_17538_b300 import abi, api, build, tune
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    ctx = api.Context(local)
    batch, pa, pb = api.scene_to_device(sc, ctx)
    n, G = batch.n_pairs, batch.n_groups
    rng = np.random.default_rng(3 + rank)
    ybar = torch.from_numpy(rng.normal(size=(G, 8)).astype(np.float32)).cuda()
    if args.tuning:
        # a fixed launch shape (for profiling without the autotuner's launches)
        batch.set_tuning(**{k: int(v) for k, v in (x.split("=") for x in args.tuning.split(","))})
        tuning = batch.get_tuning()
    else:
        tuning, _ = tune.autotune(batch, pa, pb, ybar)
    y = torch.empty((G, 8), device="cuda")
    grad = torch.empty((n, 12), device="cuda")
    saved = batch.saved_buffer()
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):            # warm-up outside the capture
        for _ in range(args.warmup):
            batch.contacts(pa, pb, out=y, saved=saved)
            batch.backward(pa, pb, ybar, out=(grad, None, None), saved=saved)
    torch.cuda.current_stream().wait_stream(stream)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    n_launch0 = abi.kernel_launches()
    with torch.cuda.graph(graph):
        batch.contacts(pa, pb, out=y, saved=saved)
        batch.backward(pa, pb, ybar, out=(grad, None, None), saved=saved)
    graph_kernels = abi.kernel_launches() - n_launch0
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t = 0.0
    cur = torch.cuda.current_stream()
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(cur)
        graph.replay()
        b.record(cur)
        b.synchronize()
        t += a.elapsed_time(b) / 1e3
    sampler.extend(graph.replay)
    clocks = sampler.stop()

    # per-kernel times for the roofline: the same two calls eagerly, with an
    # event between them, L2 flushed before each step (a second loop, not
    # part of the headline value)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(cur)
        batch.contacts(pa, pb, out=y, saved=saved)
        ev[k][1].record(cur)
        batch.backward(pa, pb, ybar, out=(grad, None, None), saved=saved)
        ev[k][2].record(cur)
    torch.cuda.synchronize()
    t_fwd = sum(e[0].elapsed_time(e[1]) for e in ev) / 1e3
    t_vjp = sum(e[1].elapsed_time(e[2]) for e in ev) / 1e3
    # exact work counters of both passes (after the timed loops)
    cnt = torch.zeros(8, dtype=torch.int64, device="cuda")
    batch.contacts(pa, pb, counters=cnt)
    # a fresh record and contact list for the counted reverse pass (the counted
    # forward keeps none), so that it counts the per-contact pass the step runs
    batch.contacts(pa, pb, out=y, saved=saved)
    cnt_v = torch.zeros(8, dtype=torch.int64, device="cuda")
    batch.backward(pa, pb, ybar, saved=saved, counters=cnt_v)
    counters = dict(zip(abi.COUNTER_NAMES, cnt.cpu().tolist()))
    counters_vjp = dict(zip(abi.BWD_COUNTER_NAMES, cnt_v.cpu().tolist()))
    model = work_model(counters, counters_vjp, counters_vjp)
    t_fwd, t_vjp = shard.reduce_max([t_fwd, t_vjp], "cuda")
    pp_all, t, _ = shard.job_rate(sc.piece_pairs(), t, "cuda")
    if rank != 0:
        return None, sc
    K = args.steps
    roof = alu_roofline(local, {"forward": t_fwd / K, "vjp": t_vjp / K},
                        {"forward": model["forward"], "vjp": model["vjp"]},
                        {"pairs": args.pairs,   # DRAM bytes depend on the staging shape
                         "tuning": ",".join(f"{k}={v}" for k, v in tuning.items())})
    npb = np.diff(sc.geom.body_piece_off)
    return {
        "metric": METRIC, "value": pp_all * args.steps / t, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded convex-hull scenes)",
        "config": {"workload": f"uneven batch: {args.pairs} body pairs drawn from a pool of "
                               f"{sc.geom.n_bodies} distinct bodies ({sc.geom.n_pieces} pieces), "
                               "pieces/body log-U[1,64], hull points log-U[8,512]; fwd + grad in "
                               "one CUDA graph", "piece_pairs_per_gpu": sc.piece_pairs(),
                   "bodies": sc.geom.n_bodies, "pieces": sc.geom.n_pieces,
                   "pieces_per_body_mean": float(npb[sc.pair_a].mean()),
                   "l2": "flushed between timed steps (512 MiB write, untimed)",
                   "tuning": tuning, "generation_s": t_gen},
        "breakdown": {"ms_forward": 1e3 * t_fwd / K, "ms_vjp": 1e3 * t_vjp / K,
                      "note": "eager calls timed in a second loop; the headline replays "
                              "both in one CUDA graph"},
        # per step: the forward keeping its record and the per-pair gradient
        # pass from it (bodies of more than 256 pieces would add the
        # per-work-item reduction kernel)
        # kernels of the captured graph (the library's own count at capture)
        # times the replays
        "gpu_launches": graph_kernels * args.steps, "roofline": roof,
        "work_counters": {"forward": counters, "vjp": counters_vjp}, "clocks": clocks,
    }, sc


# ---------------------------------------------------------------------------
# serving loop: Poisson arrivals, continuous batching vs per-request launches
# ---------------------------------------------------------------------------
SERVE_BUDGET = 256 << 20   # HBM budget of the serving context (wave buffers)


SERVE_LOADS = (0.1, 0.3, 0.6, 0.9, 1.2)   # offered rates, x the served saturation rate


def _serve_requests(sc, rng, n_req, rate):
    """Arrival times (s), pair slices and kinds of ``n_req`` requests: Poisson
    arrivals at ``rate`` per second (all at t = 0 for rate None), 1-256
    environments (body pairs) drawn log-uniformly, half of them forward only,
    half forward + gradient."""
    from paper_2604_17538_b300 import scenes
    arr = (np.zeros(n_req) if rate is None
           else np.cumsum(rng.exponential(1.0 / rate, size=n_req)))
    size = scenes.log_uniform_int(rng, 1, 256, size=n_req)
    start = np.array([rng.integers(0, sc.n_pairs - k + 1) for k in size])
    grad = rng.uniform(size=n_req) < 0.5
    return arr, start, start + size, grad


def _pct(x, q):
    return float(np.percentile(np.asarray(x), q)) * 1e3 if len(x) else None


def run_serve(args, rank, world, n_req=10000, rates=None):
    """Serving sweep.  First the saturation rate of the continuous-batching
    loop (every request queued at t = 0), then, for offered rates of
    SERVE_LOADS x that rate (or the rates given), ``n_req`` requests with
    Poisson arrivals through the loop (ccm_submit / ccm_poll) and the same
    requests as plain per-request launches (ccm_contacts [+
    ccm_contacts_backward] on a batch planned in advance, one stream,
    launched at arrival).  Reports p50 / p99 latency (arrival to completion)
    and throughput."""
    import ctypes as C
    import torch
    from paper_2604_17538_b300 import abi, api, build, scenes
    t0 = time.perf_counter()
    sc = scenes.uneven_scene(seed=11 + 1000 * rank, n_pairs=args.serve_pairs,
                             pool_bodies=min(8192, 2 * args.serve_pairs), workers=0)
    t_gen = time.perf_counter() - t0
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    ctx = api.Context(local, hbm_budget_bytes=SERVE_BUDGET)
    handles = ctx.load_geometry(sc.geom)
    pa = torch.from_numpy(sc.pose_a.astype(np.float32)).cuda()
    pb = torch.from_numpy(sc.pose_b.astype(np.float32)).cuda()
    off = sc.group_offsets()
    npb = np.diff(sc.geom.body_piece_off)
    pp_pair = (npb[sc.pair_a] * npb[sc.pair_b]).astype(np.int64)
    pp_cum = np.concatenate([[0], np.cumsum(pp_pair)])
    ybar_all = torch.from_numpy(np.random.default_rng(5).normal(
        size=(int(off[-1]), 8)).astype(np.float32)).cuda()
    L = abi.lib()
    h = ctx.handle

    def prepare(seed, rate):
        """Requests as an array of C structs (replayed by the native load
        generator) and their per-request launch arguments; outputs
        preallocated as slices."""
        rng = np.random.default_rng(seed)
        arr, i0, i1, grad = _serve_requests(sc, rng, n_req, rate)
        A = [handles[sc.pair_a[a:b]] for a, b in zip(i0, i1)]
        B = [handles[sc.pair_b[a:b]] for a, b in zip(i0, i1)]
        qp = int(sum(pp_cum[b] - pp_cum[a] for a, b in zip(i0, i1)))
        G_req = np.array([off[b] - off[a] for a, b in zip(i0, i1)])
        goff = np.concatenate([[0], np.cumsum(G_req)])
        poff = np.concatenate([[0], np.cumsum(i1 - i0)])
        y_all = torch.empty((int(goff[-1]), 8), device="cuda")
        g_all = torch.empty((int(poff[-1]), 12), device="cuda")
        yb = [ybar_all[off[a]:off[b]] if g else None for a, b, g in zip(i0, i1, grad)]
        ys = [y_all[goff[k]:goff[k + 1]] for k in range(n_req)]
        gs = [g_all[poff[k]:poff[k + 1]] for k in range(n_req)]
        keep, reqs = [y_all, g_all], (abi.ccm_request * n_req)()
        for k in range(n_req):
            Ak = np.ascontiguousarray(A[k], np.uint64)
            Bk = np.ascontiguousarray(B[k], np.uint64)
            keep += [Ak, Bk]
            reqs[k] = abi.ccm_request(
                int(i1[k] - i0[k]), Ak.ctypes.data, Bk.ctypes.data, pa[i0[k]:i1[k]].data_ptr(),
                pb[i0[k]:i1[k]].data_ptr(), ys[k].data_ptr(),
                yb[k].data_ptr() if grad[k] else None, gs[k].data_ptr() if grad[k] else None)
        calls = [(pa[i0[k]:i1[k]].data_ptr(), pb[i0[k]:i1[k]].data_ptr(), ys[k].data_ptr(),
                  yb[k].data_ptr() if grad[k] else None, gs[k].data_ptr() if grad[k] else None)
                 for k in range(n_req)]
        return {"arr": arr, "A": A, "B": B, "qp": qp, "reqs": reqs, "calls": calls, "keep": keep,
                "i0": i0, "i1": i1}

    def served(P):
        """Continuous batching: the native load generator (ccm_serve_replay)
        submits each request at its arrival time and drains completions."""
        arr = np.ascontiguousarray(P["arr"], np.float64)
        srv = api.Server(ctx, max_wave_pairs=0, max_wave_requests=1024)
        torch.cuda.synchronize()
        lat, lag = np.zeros(n_req), np.zeros(n_req)
        el = C.c_double()
        abi.check(L.ccm_serve_replay(h, C.cast(P["reqs"], C.c_void_p), arr.ctypes.data, n_req,
                                     lag.ctypes.data, lat.ctypes.data, C.byref(el)))
        t_srv = el.value
        st = srv.stats()
        srv.close()
        return {"p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99),
                # the loop's own share: submission to completion (the
                # generator's lag behind the schedule taken out)
                "loop_p50_ms": _pct(lat - lag, 50), "loop_p99_ms": _pct(lat - lag, 99),
                "qps": P["qp"] / t_srv, "req_s": n_req / t_srv, "waves": st["waves"],
                "mean_wave_pairs": st["wave_pairs"] / max(1, st["waves"]),
                "wave_gpu_ms_mean": 1e3 * st["gpu_s"] / max(1, st["waves"]),
                "wave_form_ms_mean": 1e3 * st["form_s"] / max(1, st["waves"]),
                "client_lag_p99_ms": _pct(lag, 99)}

    def per_request(P):
        """Plain per-request launches, in arrival order on one stream."""
        arr = P["arr"]
        # one small batch per request; the per-item kernels (no contact list),
        # so that thousands of planned batches do not each hold list buffers
        batches = []
        for k in range(n_req):
            b = ctx.batch(P["A"][k], P["B"][k])
            b.set_tuning(flat_records=-1)
            batches.append(b)
        prm = C.byref(api._params(None))
        stream = torch.cuda.current_stream()
        sh = stream.cuda_stream
        fwd, bwd = L.ccm_contacts, L.ccm_contacts_backward
        evs = [torch.cuda.Event() for _ in range(n_req)]
        torch.cuda.synchronize()
        lat, lag = np.zeros(n_req), np.zeros(n_req)
        fifo = []
        tb = time.perf_counter()
        k = j = 0
        while j < n_req:
            now = time.perf_counter() - tb
            while k < n_req and arr[k] <= now:
                bh = batches[k].handle
                p_a, p_b, py, pyb, pg = P["calls"][k]
                abi.check(fwd(bh, p_a, p_b, prm, py, sh))
                if pyb is not None:
                    abi.check(bwd(bh, p_a, p_b, prm, pyb, None, pg, None, None, sh))
                evs[k].record(stream)
                lag[k] = time.perf_counter() - tb - arr[k]
                fifo.append(k)
                k += 1
            while j < len(fifo) and evs[fifo[j]].query():
                kk = fifo[j]
                lat[kk] = time.perf_counter() - tb - arr[kk]
                j += 1
        t_plain = time.perf_counter() - tb
        for bt in batches:
            bt.close()
        return {"p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99),
                "loop_p50_ms": _pct(lat - lag, 50), "loop_p99_ms": _pct(lat - lag, 99),
                "qps": P["qp"] / t_plain, "req_s": n_req / t_plain,
                "client_lag_p99_ms": _pct(lag, 99)}

    def plain_batched(P, reps=5):
        """The same request mix as plain batched launches on the same GPU:
        the forward-only requests' pairs as one batch (ccm_contacts), the
        forward + gradient requests' pairs as another (ccm_contacts_save and
        ccm_contacts_backward_saved), back to back on one stream, as if every
        request had arrived at once and been planned together."""
        cat = lambda xs: np.concatenate(xs) if xs else np.zeros(0, np.uint64)
        kinds = [c[3] is not None for c in P["calls"]]
        out = {}
        runs = []
        for want_grad in (False, True):
            ks = [k for k in range(n_req) if kinds[k] == want_grad]
            if not ks:
                continue
            A, B = cat([P["A"][k] for k in ks]), cat([P["B"][k] for k in ks])
            rows = np.concatenate([np.arange(P["i0"][k], P["i1"][k]) for k in ks])
            bt = ctx.batch(A, B)
            ra = torch.from_numpy(rows).cuda()
            p_a, p_b = pa[ra].contiguous(), pb[ra].contiguous()
            yy = torch.empty((bt.n_groups, 8), device="cuda")
            if want_grad:
                gro = torch.cat([ybar_all[off[P["i0"][k]]:off[P["i1"][k]]] for k in ks])
                rec = bt.saved_buffer()
                gg = torch.empty((bt.n_pairs, 12), device="cuda")
                runs.append(lambda bt=bt, p_a=p_a, p_b=p_b, yy=yy, rec=rec, gro=gro, gg=gg: (
                    bt.contacts(p_a, p_b, out=yy, saved=rec),
                    bt.backward(p_a, p_b, gro, saved=rec, out=(gg, None, None))))
            else:
                runs.append(lambda bt=bt, p_a=p_a, p_b=p_b, yy=yy: bt.contacts(p_a, p_b, out=yy))
            out.setdefault("batches", []).append(bt)
        for _ in range(3):
            for r in runs:
                r()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            for r in runs:
                r()
        b.record()
        b.synchronize()
        t = a.elapsed_time(b) / 1e3 / reps
        for bt in out["batches"]:
            bt.close()
        return {"ms": 1e3 * t, "qps": P["qp"] / t, "req_s": n_req / t,
                "note": "all requests at once: forward-only pairs in one batch, forward + "
                        "gradient pairs in another, planned in advance (not timed), launched "
                        "back to back; device time (CUDA events), mean of 5"}

    sat = served(prepare([rank, 99], None))
    if rates is None and args.serve_rates != "auto":
        rates = [float(r) for r in args.serve_rates.split(",")]
    loads = None
    if rates is None:
        loads = list(SERVE_LOADS)
        rates = [f * sat["req_s"] for f in loads]
    results = []

    def run_rate(ri, rate, load):
        P = prepare([rank, ri], rate)
        row = {"rate_req_s": rate, "requests": n_req, "piece_pairs": P["qp"]}
        if load is not None:
            row["load"] = load
        row["served"] = served(P)
        row["per_request_launch"] = per_request(P)
        results.append(row)
        return P
    for ri, rate in enumerate(rates):
        P = run_rate(ri, rate, loads[ri] if loads is not None else None)
    if loads is not None:
        # past the burst estimate: raise the offered rate until the loop
        # serves less than it is offered, so that the sweep reaches saturation
        f = loads[-1]
        while (results[-1]["served"]["req_s"] >= 0.95 * results[-1]["rate_req_s"]
               and f < 4.0):
            f *= 1.5
            P = run_rate(len(results), f * sat["req_s"], round(f, 3))
    top = max(results, key=lambda r: r["served"]["req_s"])
    plain = plain_batched(P)
    extra = {}
    if not args.no_cpu_baseline:
        # the oracle on the same pool's pairs, forward alone and forward +
        # gradient, combined for the 50/50 request mix
        qf, cores, sf, tf = oracle_sample_rate(sc, target_s=4.0, kind="fwd", what="body pairs")
        qg, _, sg, tg = oracle_sample_rate(sc, target_s=4.0, kind="grad", what="body pairs")
        extra["cpu_baseline"] = {
            "value": 1.0 / (0.5 / qf + 0.5 / qg), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"forward: {sf}, {tf:.1f} s; forward + gradient: {sg}, {tg:.1f} s; "
                      "rate of the 50/50 mix of the two"}
    return {**extra, "geometry": f"uneven pool: {sc.n_pairs} placed pairs over "
                        f"{len(npb)} bodies, pieces/body log-U[1,64], hull points log-U[8,512]",
            "requests": "Poisson arrivals; 1-256 envs log-uniform; 50/50 fwd vs fwd+grad",
            "hbm_budget_bytes": SERVE_BUDGET, "generation_s": t_gen,
            "saturation": {"requests": n_req, "arrivals": "all at t = 0",
                           "req_s": sat["req_s"], "qps": sat["qps"],
                           "mean_wave_pairs": sat["mean_wave_pairs"]},
            "served_max": {"req_s": top["served"]["req_s"], "qps": top["served"]["qps"],
                           "at_rate_req_s": top["rate_req_s"]},
            "plain_batched": plain,
            "latency": "arrival to completion as seen by the host (ms)", "sweep": results}


def run_broadphase(args):
    """Broad phase against d_max, shaped like the paper's Sec. 5.4 sweep: one
    pair of 8-piece hull bodies, B translated along x through a batch of
    offsets spanning overlap to separation, the forward timed at several
    d_max with (a) the exact plane culls, (b) those plus the voxel grids
    (Sec. 4.3) and (c) no culls at all (every feature through the narrow
    phase), with the plane-evaluation counters of each."""
    import torch
    from paper_2604_17538_b300 import abi, api, build, scenes
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    base = scenes.hull_env_scene(seed=9, n_envs=1, workers=0)
    V = base.geom.verts
    ext = float((V.max(0) - V.min(0)).max())
    n = args.bp_pairs
    shift = np.linspace(0.1 * ext, 0.9 * ext, n)
    pose_b = np.repeat(base.pose_b, n, axis=0).copy()
    pose_b[:, 9] = base.pose_a[0, 9] + shift
    sc = scenes.Scene(base.geom, np.zeros(n, np.int64), np.ones(n, np.int64),
                      np.repeat(base.pose_a, n, axis=0), pose_b)
    ctx = api.Context(local)
    batch, pa, pb = api.scene_to_device(sc, ctx)
    ctx.build_voxel_grids(args.bp_voxels)
    rows = []
    for d_max in (0.0, 0.01, 0.02, 0.05, 0.1):
        row = {"d_max": d_max}
        for name, flags in (("plane_culls", 0), ("plane_and_voxel_culls", 16), ("no_culls", 1)):
            prm = {"d_max": d_max, "flags": flags}
            cnt = torch.zeros(8, dtype=torch.int64, device="cuda")
            batch.contacts(pa, pb, params=prm, counters=cnt)
            for _ in range(3):
                batch.contacts(pa, pb, params=prm)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(args.steps):
                batch.contacts(pa, pb, params=prm)
            b.record()
            b.synchronize()
            row[name] = {"ms": a.elapsed_time(b) / args.steps,
                         "counters": dict(zip(abi.COUNTER_NAMES, cnt.cpu().tolist()))}
        rows.append(row)
    batch.check()
    return {"workload": f"{n} translations of one pair of 8-piece hull bodies along x, "
                        f"0.1-0.9 x the scene's extent ({ext:.3f})",
            "voxels": args.bp_voxels, "sweep": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--envs", type=int, default=N_ENVS)
    ap.add_argument("--ref-sample", type=int, default=24)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="hull", choices=["hull", "uneven", "serve",
                                                            "broadphase"])
    ap.add_argument("--bp-pairs", type=int, default=4096)
    ap.add_argument("--bp-voxels", type=int, default=8)
    ap.add_argument("--pairs", type=int, default=65536)
    ap.add_argument("--tuning", default="",
                    help="uneven workload: a fixed launch shape (key=value,... of "
                         "ccm_tuning fields) instead of autotuning it")
    ap.add_argument("--serve-pairs", type=int, default=8192)
    ap.add_argument("--serve-rates", default="auto",
                    help="offered rates (req/s, comma-separated) or 'auto': "
                         "0.1-1.2 x the measured saturation rate")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-uneven", action="store_true",
                    help="skip the uneven-batch line of the default run")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))

    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if args.workload == "broadphase":
        if rank == 0:
            print(json.dumps({"metric": METRIC, "unit": "ms per forward", "broadphase":
                              run_broadphase(args)}))
        return
    if args.workload == "uneven":
        out, sc = run_uneven(args, rank, world)
        if rank == 0:
            print(json.dumps(out))
        return
    if args.workload == "serve":
        if rank == 0:
            sv = run_serve(args, rank, world, n_req=args.serve_requests)
            top = sv["sweep"][-1]
            print(json.dumps({
                "metric": METRIC, "value": top["served"]["qps"], "unit": UNIT, "n_gpus": 1,
                "steps": len(sv["sweep"]), "warmup": 0, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded convex-hull scenes)",
                "config": {"workload": "serving loop at the highest swept rate"}, "serving": sv}))
        return
    out, sc = run_ours(args, rank, world)
    if not args.no_uneven:
        # the uneven batch (65,536 pairs, forward + gradient, autotuned shape,
        # one CUDA graph) as its own line inside the default run
        un, usc = run_uneven(args, rank, world)
        if rank == 0:
            if not args.no_cpu_baseline:
                qps, cores, sample, dt = oracle_sample_rate(usc, target_s=8.0, kind="grad",
                                                            what="body pairs")
                un["cpu_baseline"] = {"value": qps, "unit": UNIT, "cores": cores,
                                      "kind": "oracle",
                                      "sample": sample + f"; fwd + grad, {dt:.1f} s"}
            out["uneven"] = {k: un[k] for k in ("value", "unit", "ms_per_step", "config",
                                                "breakdown", "gpu_launches", "roofline",
                                                "work_counters", "clocks", "cpu_baseline")
                             if k in un}
        del usc
    if rank == 0 and not args.no_serve:
        out["serving"] = run_serve(args, rank, world, n_req=args.serve_requests)
    if rank == 0:
        if not args.no_cpu_baseline:
            qps, cores, sample, dt = oracle_sample_rate(sc)
            out["cpu_baseline"] = {"value": qps, "unit": UNIT, "cores": cores, "kind": "oracle",
                                   "sample": sample + f"; fwd + grad + H u, {dt:.1f} s"}
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
