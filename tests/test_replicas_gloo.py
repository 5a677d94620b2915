"""The N > 1 path of bench.py on the host: two gloo ranks on the CPU.

The path does not shard (one state vector per GPU), so N GPUs run N independent replicas;
the only collectives are the barrier around the timed region and the aggregation of the
result (sum of units over ranks, max of times).  These tests run that host logic with
world_size 2 and check the aggregate, and that the reference arm prints on rank 0 only."""
import io
import os
import socket
import contextlib

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    units, sec = bench.aggregate(float(10 * (rank + 1)), float(rank + 2), world)
    bench.barrier(world)
    out[rank] = (units, sec, bench.dist_env())
    dist.destroy_process_group()


def test_two_replicas_aggregate():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        units, sec, env = res[rank]
        assert units == 30.0            # sum over ranks
        assert sec == 3.0               # the slowest rank's time
        assert env == (world, rank, rank)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(type("A", (), {"warmup": 3, "steps": 1, "workload": "L24_mixed"})())
    assert buf.getvalue() == ""   # rank 1 returns before any oracle work


def test_single_rank_aggregate_is_identity():
    import bench
    assert bench.aggregate(5.0, 2.0, 1) == (5.0, 2.0)
