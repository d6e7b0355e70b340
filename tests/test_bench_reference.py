"""bench.py's reference arm (the FP64 oracle timed on the host cores) prints
one JSON line with the keys the benchmark contract names, on a small
sample, without a GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--envs", "16", "--ref-sample", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 2 and d["n_gpus"] == 1
    assert d["unit"] == "piece-pair queries/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert "3 of 16 environments" in cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_under_two_ranks_prints_once():
    """Launched as the multi-GPU run is (torchrun, two ranks): rank 0 alone
    times the oracle and prints; the other rank exits 0 without work."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                        "--master-port", str(port), "bench.py", "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "1", "--envs", "16",
                        "--ref-sample", "2"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_oracle_sample_rates_of_each_kind():
    """The oracle timing behind the CPU baselines (the 4096-environment step,
    the uneven batch and the serving mix): a bounded seeded sample for every
    kind of pass, a positive rate, and a sample description that names it."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    from paper_2604_17538_b300 import scenes
    sc = scenes.uneven_scene(seed=3, n_pairs=40, max_pieces=3, max_points=24, pool_bodies=12,
                             workers=1)
    for kind in ("fwd", "grad", "hvp"):
        qps, cores, sample, dt = bench.oracle_sample_rate(sc, target_s=0.2, kind=kind,
                                                          what="body pairs")
        assert qps > 0 and cores >= 1 and dt > 0
        assert "of 40 body pairs" in sample and "piece pairs" in sample
