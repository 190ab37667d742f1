"""The multi-rank host path of bench.py on CPU: two gloo ranks, no GPU.

Every rank runs its own copy of the workload (replicas, weak scaling); the
timed region is the slowest rank's, and the whole-job value counts every
rank's node-updates.  The reference arm runs on rank 0 only.
"""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_WORKER = r"""
import os, sys, json
sys.path.insert(0, os.environ["BENCH_ROOT"])
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world, local = bench.dist_env()
seconds = 1.0 + rank                      # rank 1 is the slow one
slowest = bench.max_over_ranks(dist, seconds, "cpu")
value = bench.whole_job_value(1000, 50, 3, world, slowest)
print(json.dumps({"rank": rank, "world": world, "slowest": slowest, "value": value}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _spawn(code, world, extra_env=None, timeout=120):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), BENCH_ROOT=ROOT)
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, cwd=ROOT))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=timeout)
        except subprocess.TimeoutExpired:
            p.kill()
            o, e = p.communicate()
        outs.append((p.returncode, o, e))
    return outs


def test_two_gloo_ranks_take_the_slowest_time_and_count_every_rank():
    pytest.importorskip("torch")
    import json
    outs = _spawn(_WORKER, 2)
    for rc, o, e in outs:
        assert rc == 0, e
    lines = [json.loads(o.strip().splitlines()[-1]) for _, o, _ in outs]
    for d in lines:
        assert d["world"] == 2
        assert d["slowest"] == 2.0                      # max over ranks, on every rank
        assert d["value"] == 1000 * 50 * 3 * 2 / 2.0    # both ranks' node-updates / slowest time


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 1.25, "cpu") == 1.25
    assert bench.whole_job_value(10, 5, 2, 1, 0.5) == 200.0
    assert bench.launches_per_run(50, True) == 53      # fill + 50 steps + 2 conversions
    assert bench.launches_per_run(20, False) == 21


def test_reference_arm_runs_on_rank_zero_only():
    # rank 1 of a two-rank reference run exits at once, printing nothing
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "C1",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120,
                       cwd=ROOT)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_error_vs_oracle_scales_by_each_problems_initial_max():
    """bench.error_vs_oracle: absolute max and RMS over all nodes; the
    relative figure divides each problem's error by its own max |V^0|."""
    import bench

    class P:
        def __init__(self, n, scale):
            self.mesh = type("M", (), {"n_nodes": n})()
            self.v0 = np.full(n, scale)

    probs = [P(3, 2.0), P(2, 0.5)]
    want = [np.zeros(3), np.zeros(2)]
    got = np.array([0.0, 1e-3, 0.0, 0.0, 2e-3])
    e = bench.error_vs_oracle(probs, got, want)
    assert e["max_abs"] == 2e-3
    assert abs(e["l2_rms"] - np.sqrt((1e-6 + 4e-6) / 5)) < 1e-15
    assert abs(e["max_rel_to_max_v0"] - 4e-3) < 1e-15
