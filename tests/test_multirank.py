"""Replicas across ranks (CPU, gloo, world size 2): the benchmark's only collective is
the MAX over rank times; whole-job throughput counts every rank's units."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_info()
    ms = 100.0 + 50.0 * r  # rank 1 is the slower replica
    value, total = bench.job_throughput(ms, 1000, w)
    out[r] = (value, total)
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        value, total = res[r]
        assert total == 150.0
        assert abs(value - world * 1000 / 0.150) < 1e-9


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    value, total = bench.job_throughput(200.0, 500, 1)
    assert total == 200.0 and abs(value - 2500.0) < 1e-12


def test_replica_inputs_differ_by_rank():
    """Each rank draws its own seeded system (seed 1 + rank): replicas, not shards."""
    from paper_2209_04015_b300.synthetic import make_config
    a, _ = make_config("c1", seed=1)
    b, _ = make_config("c1", seed=2)
    assert not (a.h1 == b.h1).all()
