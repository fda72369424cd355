"""The multi-GPU path is replicas (no data exchange on the hot path): each
rank solves its own copy and the benchmark takes the slowest rank's time and
the dofs of all ranks.  The rank logic is checked here with two gloo ranks on
CPU."""
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
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def reduce_max(v):
        t = torch.tensor([v])
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    value, t_max = bench.replica_value(1000, 1, world, 100.0 + 50.0 * rank, reduce_max)
    out[rank] = (value, t_max)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_uses_slowest_rank():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == (2000 / 0.15, 150.0)
