"""Multi-process path of bench.py (replicas: the sign-function path has no
exchange step): world size 2 on the gloo backend, CPU only."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, port, out):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    ms_local = 100.0 * (rank + 1)  # rank 1 is the slower replica
    ms, value = bench.replica_throughput(ms_local, 40, 2, "cpu")
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_replica_throughput_uses_slowest_rank():
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        ms, value = res[r]
        assert ms == 200.0
        assert abs(value - 2 * 40 / 0.2) < 1e-9
