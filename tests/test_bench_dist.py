"""The multi-rank path of bench.py on CPU: two gloo ranks (no GPU).

bench.py under torchrun runs one replica per rank (each solves its own
instances, no data-path collective); the job's time is the slowest rank's
and its throughput counts every rank's solves. These tests run that
aggregation with world_size 2, and check that the reference arm prints on
rank 0 only.
"""

import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.0 + 2.0 * rank)          # rank 1 is the slow one
        out[rank] = (t, bench.job_rate(10, world, t))
    finally:
        tdist.destroy_process_group()


def test_max_over_ranks_and_job_rate_two_gloo_ranks():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for rank in (0, 1):
        t, rate = out[rank]
        assert t == 3.0                       # every rank sees the slowest time
        assert rate == pytest.approx(20 / 3.0)  # 10 solves on each of 2 ranks


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.job_rate(4, 1, 2.0) == 2.0


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--n", "256", "--s", "64"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert p.returncode == 0
    assert p.stdout.strip() == ""


def test_reference_arm_line_on_rank_zero():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--n", "256", "--s", "64", "--ref-sample-iters", "1"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    line = json.loads(p.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    # a complete oracle solve was timed, and the steps' own time is reported
    assert line["cpu_baseline"]["complete_solve_s"] > 0 and line["cpu_baseline"]["complete_solve_iters"] > 0
    assert line["ms_per_step"] > 0


def test_oracle_baselines_of_the_other_configs():
    """The cpu_baseline leg's oracle timings beside the headline one: the
    n = 1024 outlier system solved to 1e-10 with every BLAS thread and with
    one (child processes), and the oracle's Hutchinson estimate on a given
    matrix with the probes the GPU draws (the trace estimator's mean is the
    trace; checked on a small diagonal matrix, where every probe gives it)."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    r = bench.oracle_config0_timing()
    assert "error" not in r, r
    for k in ("all_threads", "one_thread"):
        assert r[k]["converged"] and r[k]["iters"] > 0 and r[k]["solves_per_s"] > 0
    d = np.linspace(1.0, 2.0, 300).astype(np.float32)
    h = bench.oracle_hutchinson_timing(np.diag(d), bench.SEED)
    assert "error" not in h, h
    assert abs(h["estimate"] - float(d.astype(np.float64).sum())) <= 1e-9 * d.sum()
    assert h["std_err"] <= 1e-9 * d.sum() and h["estimates_per_s"] > 0
