"""The multi-GPU path is replicas only: every rank solves its own copy of the
workload and the bench reports the longest rank's time and the operator
applications of all ranks.  Checked here with two gloo ranks on the CPU."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 17.25][rank]
    ops = [300, 304][rank]
    out[rank] = bench.replicas_aggregate(ms, ops, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [1, 2])
def test_replicas_aggregate(world):
    if world == 1:
        import bench

        assert bench.replicas_aggregate(12.5, 300, None, "cpu") == (12.5, 300)
        return
    import socket

    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as sk:  # a port that is free now
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        assert out[0] == (17.25, 604) and out[1] == (17.25, 604)
