"""The multi-process path of bench.py on CPU: world size 2 over gloo, one replica per rank,
the reported time is the maximum over ranks (no collective on the data path)."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    val = bench.aggregate_max(10.0 + 5.0 * rank, world)
    out[rank] = val
    dist.barrier()
    dist.destroy_process_group()


def test_replica_time_is_max_over_ranks():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1] == 15.0


def test_single_process_aggregate_is_identity():
    import bench
    assert bench.aggregate_max(3.5, 1) == 3.5
