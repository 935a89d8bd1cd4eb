"""The multi-GPU mode is replicas only (the solve does not shard): each rank
solves its own right-hand sides, the job time is the max over ranks and the
reported value is time / (right-hand sides of all ranks).  Checked here with
two CPU ranks over gloo."""
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
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    elapsed = [120.0, 150.0][rank]  # rank 1 is the slow one
    tmax, value = bench.replica_time(elapsed, steps=5)
    out[rank] = (tmax, value)
    dist.destroy_process_group()


def test_replica_time_two_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        tmax, value = out[r]
        assert tmax == 150.0
        assert value == pytest.approx(150.0 / (5 * 2))


def test_replica_time_single_process():
    import bench

    assert bench.replica_time(80.0, steps=4) == (80.0, 20.0)
