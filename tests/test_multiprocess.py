"""The replicas path on CPU (gloo, two ranks): each replica draws disjoint evaluation
queries, the job's time is the slowest replica's, the job's value counts every replica's
queries, and only rank 0 runs the reference arm."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    from paper_2310_06822_gb300 import inputs as I
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank
    slowest = bench.max_over_ranks(ms, dist, world)
    q = I.sample_queries(I.RAY3, bench.rank_seed(bench.SEED_QUERY, rank), 64)
    out[rank] = (slowest, q.tobytes())
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_on_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 15.0
    assert out[0][1] != out[1][1]  # disjoint evaluation queries per replica
    import bench
    assert bench.job_value(1000, world, 15.0) == 2 * 1000 / 0.015
    assert bench.max_over_ranks(7.0, None, 1) == 7.0


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    bench.reference_arm(argparse.Namespace(steps=1, warmup=0, gpus=2))
    assert capsys.readouterr().out == ""
