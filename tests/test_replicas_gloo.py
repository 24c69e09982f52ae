"""The multi-process (replicas) path of bench.py on CPU: two gloo ranks with
different step times and unit counts; every rank must report the slowest
rank's time and the units of all ranks over it, and the reference arm must
run on rank 0 only."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms, value = bench.replica_reduce(10.0 + 5.0 * rank, 1000.0 * (rank + 1), ws, "cpu")
    env = bench.dist_env()
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, value, env))


def test_replica_reduce_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, env in out:
        assert ms == 15.0                                   # the slower rank's step time
        assert value == pytest.approx(3000.0 / 0.015)       # all ranks' units over it
        assert env == (2, rank, rank)


def test_replica_reduce_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.replica_reduce(20.0, 500.0, 1, "cpu")
    assert ms == 20.0 and value == pytest.approx(25000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:
        config = 2
        scale = 1.0

    assert bench.run_reference(Args()) is None              # returns before any work or output
