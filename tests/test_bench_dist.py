"""The multi-rank host logic of bench.py (replicas: barrier, max over ranks,
whole-job value) with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        got = bench.all_max([1.0 + rank, 10.0 - rank], world)
        out[rank] = (got, bench.replica_value(100.0, got[0], world))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_sum_the_units():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        got, value = res[rank]
        assert got == [2.0, 10.0]              # max over ranks, element-wise
        assert value == pytest.approx(100.0 * 2 / 2.0)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.all_max([3.0, 4.0], 1) == [3.0, 4.0]
    assert bench.replica_value(10.0, 2.0, 1) == 5.0
