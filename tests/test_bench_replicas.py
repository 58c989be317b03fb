"""Host logic of bench.py's multi-GPU path (independent replicas, one per rank),
run as two gloo ranks on CPU: the timed region is the maximum over ranks, the
value counts every rank's solves, every replica draws its own input, and the
reference arm does its work on rank 0 only."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, v = bench.aggregate_timing(100.0 + 50.0 * rank, world, 5, dist, device="cpu")
        q.put((rank, t, v))
    finally:
        dist.destroy_process_group()


def test_aggregate_timing_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, v in got:
        assert t == 150.0                       # max over ranks
        assert abs(v - 2 * 5 / 0.150) < 1e-9     # both ranks' solves over the longest region


def test_single_rank_aggregate_and_replica_inputs():
    import bench
    import workloads as W
    assert bench.aggregate_timing(200.0, 1, 4) == (200.0, 4 / 0.2)
    a = W.klein_3p1(n=8, nt=4, seed=bench.replica_seed(0))
    b = W.klein_3p1(n=8, nt=4, seed=bench.replica_seed(1))
    assert a.extra["p0"] != b.extra["p0"] and not np.allclose(a.psi0, b.psi0)
    assert bench.headline_workload(0).extra["seed"] == 1


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import argparse
    import bench
    args = argparse.Namespace(steps=1, warmup=0, gpus=2)
    assert bench.run_reference(args, 1) is None
    assert capsys.readouterr().out == ""
