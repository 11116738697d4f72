"""The multi-GPU benchmark path runs independent replicas: each rank times its
own copy of the workload and the job's throughput is all ranks' work divided
by the slowest rank's time.  This checks that host logic with two gloo ranks
on the CPU (no GPU, no data-path collective)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    local_ms = [40.0, 50.0][rank]                 # rank 1 is the slower replica
    ms, per_s = bench.replica_throughput(local_ms, 1000.0, world)
    dist.barrier()
    q.put((rank, ms, per_s))
    dist.destroy_process_group()


def test_two_gloo_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, per_s in res:
        assert ms == 50.0                          # max over ranks
        assert per_s == pytest.approx(2 * 1000.0 / 0.050)   # both ranks' units / slowest time


def test_single_rank_is_plain_ratio():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    ms, per_s = bench.replica_throughput(20.0, 500.0, 1)
    assert ms == 20.0 and per_s == pytest.approx(500.0 / 0.020)
