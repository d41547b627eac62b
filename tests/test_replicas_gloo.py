"""Multi-GPU runs are independent replicas of the workload (the path does not
shard: a Lanczos recursion is sequential).  The host side of that path -- the
whole-job rate over the slowest rank -- on two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, local_ms, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        rate, total = bench.replica_rate(local_ms[rank], 3, 100, world, bench.torch_group_max())
        out[rank] = (rate, total)
    finally:
        dist.destroy_process_group()


def test_replica_rate_two_ranks():
    world = 2
    local_ms = [800.0, 1000.0]          # rank 1 is the slowest
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, local_ms, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    rate, total = res[0]
    assert total == 1000.0
    assert rate == pytest.approx(world * 3 * 100 / 1.0)


def test_replica_rate_single_rank():
    import bench
    rate, total = bench.replica_rate(500.0, 2, 100, 1, lambda x: x)
    assert total == 500.0 and rate == pytest.approx(400.0)


def test_reference_arm_other_ranks_exit(monkeypatch):
    """Under torchrun only rank 0 times the oracle; the other ranks exit 0."""
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(gpus=2, steps=1, warmup=0)
    assert bench.run_reference(args) == 0
