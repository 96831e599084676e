"""The multi-GPU path of bench.py is replicas only: every rank advances its
own copy, and the reported time is the maximum over ranks.  This runs that
aggregation with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank
    total = bench.max_over_ranks(ms, world, device="cpu")
    value = bench.replica_throughput(cells=1000, steps=50, world=world, ms=total)
    out[rank] = (total, value)
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(2, port, out), nprocs=2, start_method="spawn")
    assert out[0] == out[1]
    total, value = out[0]
    assert total == 15.0                                    # the slowest rank decides
    assert value == pytest.approx(1000 * 50 * 2 / 15e-3 / 1e6)
